// Fixed-point BF16 digit operands for the exact-accumulation split GEMM
// (tt_tcgen05z.cu; Ozaki scheme, see tt_ozaki.cu for the arithmetic).
//
// A digit row holds K values v_k as four BF16 levels a0..a3 with
// v_k ~ 2^(e - 1054) (a0 2^24 + a1 2^16 + a2 2^8 + a3), e the largest biased
// FP64 exponent of the row, and e itself as an int16 next to the levels.
//  * digit_copy_kernel: FP64 rows (any row / element stride) -> digit rows
//    padded for TMA; one CTA per group of 32 rows of an item; a warp per row
//    when elements are contiguous, else lanes along the rows (coalesced
//    reads) and warps along K with the row exponent combined in shared
//    memory.
//  * gather_digits_kernel: the W-gather of the exact path: sums of two-float
//    (hi, lo) S1 outputs times MPO coefficients in two-float arithmetic
//    (TwoProd by FMA, TwoSum), then digits of every output row segment by
//    exact FP32 steps; two adjacent columns per lane, narrow rows packed
//    several to a warp.
// All arithmetic is FP32 / integer: GB300's FP64 pipe runs at ~1/64 of FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_kernels.h"

namespace tt {

namespace {

__device__ __forceinline__ int slot_of(Ref r) { return (int)(r >> 56); }
__device__ __forceinline__ long long off_of(Ref r) { return (long long)(r & 0x00FFFFFFFFFFFFFFull); }

__device__ __forceinline__ int dexp(double v) {
  return (int)((static_cast<unsigned long long>(__double_as_longlong(v)) >> 52) & 0x7FF);
}
// biased FP64 exponent of a float (0 for zero / subnormal)
__device__ __forceinline__ int fexp(float v) {
  const int e = (__float_as_int(v) >> 23) & 0xFF;
  return e == 0 ? 0 : e + 896;
}

// BF16 of a small integer held in an int (exact: |a| <= 256)
__device__ __forceinline__ __nv_bfloat16 bf16_of_int(int a) {
  return __ushort_as_bfloat16((unsigned short)(__float_as_uint((float)a) >> 16));
}

// balanced base-256 digits of the integer F (|F| <= 2^32) into 4 levels
__device__ __forceinline__ void put_digits(long long F, __nv_bfloat16* d, long long lo) {
  const int a0 = (int)((F + (1ll << 23)) >> 24);
  const int r0 = (int)(F - ((long long)a0 << 24));  // |r0| <= 2^23
  const int a1 = (r0 + (1 << 15)) >> 16;
  const int r1 = r0 - (a1 << 16);
  const int a2 = (r1 + (1 << 7)) >> 8;
  const int a3 = r1 - (a2 << 8);
  d[0] = bf16_of_int(a0);
  d[lo] = bf16_of_int(a1);
  d[2 * lo] = bf16_of_int(a2);
  d[3 * lo] = bf16_of_int(a3);
}

// F = round(v 2^(1054 - emax)) from the exponent and mantissa fields of v
__device__ __forceinline__ long long fixed_of_double(double v, int emax) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0) return 0;
  const int sh = 21 + emax - E;
  if (sh >= 64) return 0;
  const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  long long F = (long long)((M + (1ull << (sh - 1))) >> sh);
  return (bits >> 63) ? -F : F;
}

// 2^x for -126 <= x <= 127 from the exponent field
__device__ __forceinline__ float p2f(int x) { return __int_as_float((x + 127) << 23); }

constexpr int DT = 256;

// One CTA per (item, group of 32 digit rows): grid (items, max row groups).
__global__ void __launch_bounds__(DT) digit_copy_kernel(const DItem* __restrict__ items, Bases bs) {
  const DItem it = items[blockIdx.x];
  const int r0 = blockIdx.y * 32;
  if (r0 >= it.rows) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* src = reinterpret_cast<const double*>(sel_base(bs, slot_of(it.src))) + off_of(it.src);
  __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(sel_base(bs, slot_of(it.dst))) + off_of(it.dst);
  short* ex = reinterpret_cast<short*>(sel_base(bs, slot_of(it.e))) + off_of(it.e);
  const long long lo = sel_lo(bs, slot_of(it.dst));
  if (it.s_k == 1) {
    // contiguous rows: each warp takes 4 of the 32 rows, lanes along K
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + warp * 4 + q;
      if (r >= it.rows) break;
      const double* sp = src + (long long)r * it.s_r;
      int m = 0;
      for (int k = lane; k < it.cols; k += 32) m = max(m, dexp(sp[k]));
      m = __reduce_max_sync(0xffffffffu, m);
      for (int k = lane; k < it.cols; k += 32)
        put_digits(fixed_of_double(sp[k], m), dst + (long long)r * it.dst_rs + k, lo);
      if (lane == 0) ex[(long long)r * it.e_rs] = (short)m;
    }
  } else {
    // strided rows (a transposed block): lanes along the 32 rows (coalesced
    // reads along the source row), warps split K, the row exponent combined
    // in shared memory
    __shared__ int emax_s[32];
    if (threadIdx.x < 32) emax_s[threadIdx.x] = 0;
    __syncthreads();
    const int r = r0 + lane;
    const bool in = r < it.rows;
    const double* sp = src + (long long)r * it.s_r;
    int m = 0;
    if (in)
      for (int k = warp; k < it.cols; k += DT / 32) m = max(m, dexp(sp[(long long)k * it.s_k]));
    if (in) atomicMax(&emax_s[lane], m);
    __syncthreads();
    const int e = emax_s[lane];
    if (in) {
      for (int k = warp; k < it.cols; k += DT / 32)
        put_digits(fixed_of_double(sp[(long long)k * it.s_k], e), dst + (long long)r * it.dst_rs + k, lo);
      if (warp == 0) ex[(long long)r * it.e_rs] = (short)e;
    }
  }
}

// two-float c (hi, lo) += coef * (xh + xl), coef split into (ch, cl)
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ch, float cl, float xh, float xl) {
  const float p = ch * xh;
  const float pe = fmaf(ch, xh, -p) + (ch * xl + cl * xh);
  const float s = sh + p;
  const float bp = s - sh;
  const float ap = s - bp;
  sl += ((sh - ap) + (p - bp)) + pe;
  sh = s;
}

constexpr int GMAXC = 256;  // longest digit row (segment) of the exact path
constexpr int GMAXK = 64;   // most MPO coefficients of one item (split in shared memory)

// Balanced base-256 digits of round(S + Sl) (a normalised two-float value,
// |Sl| <= ulp(S) / 2, |S| < 2^31, scaled so that the row's bound is 2^31), in
// FP32 arithmetic only: every step is exact, the roundings are those of rintf.  Returned as the BF16 bit
// patterns (the digits are integers of magnitude <= 256, so their FP32 and
// BF16 forms agree in the upper 16 bits).
__device__ __forceinline__ void digits_of_pair(float S, float Sl, uint32_t* d) {
  const float R = rintf(S);
  const float f = (S - R) + Sl;
  const float a0 = rintf(R * 5.9604644775390625e-08f);   // R / 2^24
  const float rem = (R - a0 * 16777216.f) + rintf(f);    // |rem| < 2^24
  const float a1 = rintf(rem * 1.52587890625e-05f);      // rem / 2^16
  const float r1 = rem - a1 * 65536.f;
  const float a2 = rintf(r1 * 0.00390625f);              // r1 / 2^8
  const float a3 = r1 - a2 * 256.f;
  d[0] = __float_as_uint(a0);
  d[1] = __float_as_uint(a1);
  d[2] = __float_as_uint(a2);
  d[3] = __float_as_uint(a3);
}

// One CTA per item.  Each row is taken by a group of G lanes (G the smallest
// power of two with 2 G >= cols, at most 32), two adjacent columns per lane,
// so that 32 / G rows share a warp when the item is narrow; the row exponent
// is a max-reduction inside the group.
__global__ void __launch_bounds__(DT) gather_digits_kernel(const GItem* __restrict__ items,
                                                           const GContrib* __restrict__ cs, Bases bs) {
  const GItem it = items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int lg = 0;
  while ((1 << lg) < 32 && 2 * (1 << lg) < it.cols) ++lg;
  const int G = 1 << lg, rpw = 32 >> lg;
  const int sub = lane >> lg, gl = lane & (G - 1);
  uint32_t* dst = reinterpret_cast<uint32_t*>(reinterpret_cast<__nv_bfloat16*>(sel_base(bs, slot_of(it.dst))) +
                                              off_of(it.dst));
  short* ex = reinterpret_cast<short*>(sel_base(bs, slot_of(it.e))) + off_of(it.e);
  const long long lo2 = sel_lo(bs, slot_of(it.dst)) / 2;  // level stride in BF16 pairs
  constexpr int PP = GMAXC / 64;                          // column pairs per lane at G = 32
  // the item's MPO coefficients as float pairs, split once per CTA (FP64
  // arithmetic runs at ~1/64 of FP32 on GB300)
  __shared__ float2 cf[GMAXK];
  // the host rejects items with more terms; the clamp keeps the table in bounds
  const int nk = min(it.c1 - it.c0, GMAXK);
  for (int k = threadIdx.x; k < nk; k += DT) {
    const double v = cs[it.c0 + k].coef;
    const float ch = (float)v;
    cf[k] = make_float2(ch, (float)(v - (double)ch));
  }
  __syncthreads();
  for (int r0 = warp * rpw; r0 < it.rows; r0 += (DT / 32) * rpw) {
    const int r = r0 + sub;
    const bool rin = r < it.rows;
    float h[2 * PP], l[2 * PP];
#pragma unroll
    for (int i = 0; i < 2 * PP; ++i) { h[i] = 0.f; l[i] = 0.f; }
    for (int k = it.c0; k < it.c0 + nk; ++k) {
      const GContrib cb = cs[k];
      const float ch = cf[k - it.c0].x, cl = cf[k - it.c0].y;
      const float2* s = reinterpret_cast<const float2*>(sel_base(bs, slot_of(cb.src))) + off_of(cb.src) +
                        (long long)r * cb.src_rs;
      const bool al16 = (reinterpret_cast<uintptr_t>(s) & 15) == 0;
#pragma unroll
      for (int i = 0; i < PP; ++i) {
        const int c = 2 * (gl + G * i);
        if (rin && c < it.cols) {
          float4 v;
          if (al16 && c + 1 < it.cols) {
            v = *reinterpret_cast<const float4*>(s + c);
          } else {
            const float2 v0 = s[c];
            const float2 v1 = c + 1 < it.cols ? s[c + 1] : make_float2(0.f, 0.f);
            v = make_float4(v0.x, v0.y, v1.x, v1.y);
          }
          df_fma(h[2 * i], l[2 * i], ch, cl, v.x, v.y);
          df_fma(h[2 * i + 1], l[2 * i + 1], ch, cl, v.z, v.w);
        }
      }
    }
    // renormalise every pair (TwoSum of h and l): after cancellation l may be
    // as large as h, and the digits below are taken from h and l separately
#pragma unroll
    for (int i = 0; i < 2 * PP; ++i) {
      const float sv = h[i] + l[i];
      const float bp = sv - h[i];
      l[i] = (h[i] - (sv - bp)) + (l[i] - bp);
      h[i] = sv;
    }
    int m = 0;
#pragma unroll
    for (int i = 0; i < PP; ++i) {
      const int c = 2 * (gl + G * i);
      if (c < it.cols) m = max(m, fexp(h[2 * i]));
      if (c + 1 < it.cols) m = max(m, fexp(h[2 * i + 1]));
    }
    for (int o = G >> 1; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    // one exponent above the largest: |h + l| < 2^(m - 1023), so the scaled
    // values stay below 2^31 also after rounding
    if (m) m = m + 1;
    // scale 2^(1054 - m) as two exact power-of-two factors in the FP32 range
    const int sh = m ? 1054 - m : 0, sa = sh / 2, sb = sh - sa;
    const float fa = p2f(sa), fb = p2f(sb);
    if (rin) {
      uint32_t* drow = dst + ((long long)r * it.dst_rs >> 1);
#pragma unroll
      for (int i = 0; i < PP; ++i) {
        const int c = 2 * (gl + G * i);
        if (c < it.cols) {
          uint32_t d0[4], d1[4] = {0u, 0u, 0u, 0u};
          digits_of_pair((h[2 * i] * fa) * fb, (l[2 * i] * fa) * fb, d0);
          if (c + 1 < it.cols) digits_of_pair((h[2 * i + 1] * fa) * fb, (l[2 * i + 1] * fa) * fb, d1);
#pragma unroll
          for (int lv = 0; lv < 4; ++lv) drow[lv * lo2 + (c >> 1)] = __byte_perm(d0[lv], d1[lv], 0x7632);
        }
      }
      if (gl == 0) ex[(long long)r * it.e_rs] = (short)m;
    }
  }
}

}  // namespace

cudaError_t launch_digit_copy(const DevDigit& d, const Bases& b, cudaStream_t s) {
  if (d.nitems == 0) return cudaSuccess;
  digit_copy_kernel<<<dim3(d.nitems, d.maxgroups > 0 ? d.maxgroups : 1), DT, 0, s>>>(d.items, b);
  return cudaGetLastError();
}

cudaError_t launch_gather_digits(const DevGather& g, const Bases& b, cudaStream_t s) {
  if (g.nitems == 0) return cudaSuccess;
  gather_digits_kernel<<<g.nitems, DT, 0, s>>>(g.items, g.contribs, b);
  return cudaGetLastError();
}

int gather_digits_max_cols() { return GMAXC; }
int gather_digits_max_contribs() { return GMAXK; }

}  // namespace tt
