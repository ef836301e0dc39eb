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
//    (TwoProd by FMA, TwoSum), then digits of every output row segment.
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

// balanced base-256 digits of the integer F (|F| <= 2^32) into 4 levels
__device__ __forceinline__ void put_digits(long long F, __nv_bfloat16* d, long long lo) {
  const long long a0 = (F + (1ll << 23)) >> 24;
  const long long r0 = F - a0 * (1ll << 24);
  const long long a1 = (r0 + (1ll << 15)) >> 16;
  const long long r1 = r0 - a1 * (1ll << 16);
  const long long a2 = (r1 + (1ll << 7)) >> 8;
  const long long a3 = r1 - a2 * (1ll << 8);
  d[0] = __float2bfloat16_rn((float)a0);
  d[lo] = __float2bfloat16_rn((float)a1);
  d[2 * lo] = __float2bfloat16_rn((float)a2);
  d[3 * lo] = __float2bfloat16_rn((float)a3);
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

// F = round((hi + lo) 2^(1054 - emax)) for a two-float value, |hi + lo| < 2^(emax - 1022)
__device__ __forceinline__ long long fixed_of_pair(float hi, float lo, int emax) {
  if (emax == 0) return 0;
  const int sh = 1054 - emax;  // scale exponent, |hi| 2^sh < 2^32; two exact power-of-2 factors in range
  const int sa = sh / 2, sb = sh - sa;
  const float fa = p2f(sa), fb = p2f(sb);
  const float S = (hi * fa) * fb, Sl = (lo * fa) * fb;
  const float R = rintf(S);
  const float f = (S - R) + Sl;
  return (long long)R + (long long)rintf(f);
}

constexpr int DT = 256;

// One CTA per (item, group of 32 digit rows): grid (items, max row groups).
__global__ void __launch_bounds__(DT) digit_copy_kernel(const DItem* __restrict__ items, Bases bs) {
  const DItem it = items[blockIdx.x];
  const int r0 = blockIdx.y * 32;
  if (r0 >= it.rows) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* src = reinterpret_cast<const double*>(bs.p[slot_of(it.src)]) + off_of(it.src);
  __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(bs.p[slot_of(it.dst)]) + off_of(it.dst);
  short* ex = reinterpret_cast<short*>(bs.p[slot_of(it.e)]) + off_of(it.e);
  const long long lo = bs.lo[slot_of(it.dst)];
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

__global__ void __launch_bounds__(DT) gather_digits_kernel(const GItem* __restrict__ items,
                                                           const GContrib* __restrict__ cs, Bases bs) {
  const GItem it = items[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(bs.p[slot_of(it.dst)]) + off_of(it.dst);
  short* ex = reinterpret_cast<short*>(bs.p[slot_of(it.e)]) + off_of(it.e);
  const long long lo = bs.lo[slot_of(it.dst)];
  constexpr int PER = GMAXC / 32;
  for (int r = warp; r < it.rows; r += DT / 32) {
    float h[PER], l[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) { h[i] = 0.f; l[i] = 0.f; }
    for (int k = it.c0; k < it.c1; ++k) {
      const GContrib cb = cs[k];
      const float ch = (float)cb.coef, cl = (float)(cb.coef - (double)ch);
      const float2* s = reinterpret_cast<const float2*>(bs.p[slot_of(cb.src)]) + off_of(cb.src) + (long long)r * cb.src_rs;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int c = lane + 32 * i;
        if (c < it.cols) {
          const float2 v = s[c];
          df_fma(h[i], l[i], ch, cl, v.x, v.y);
        }
      }
    }
    int m = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i)
      if (lane + 32 * i < it.cols) m = max(m, fexp(h[i] + l[i]));
    m = __reduce_max_sync(0xffffffffu, m);
    // one exponent above the largest: |h + l| < 2^(m - 1022) also after rounding
    if (m) m = m + 1;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int c = lane + 32 * i;
      if (c < it.cols) put_digits(fixed_of_pair(h[i], l[i], m), dst + (long long)r * it.dst_rs + c, lo);
    }
    if (lane == 0) ex[(long long)r * it.e_rs] = (short)m;
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

}  // namespace tt
