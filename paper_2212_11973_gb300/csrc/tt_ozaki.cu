// Exact-accumulation split GEMM on the tensor cores for FP64 operands
// (Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59 (2012); here with fixed-point
// slices, as in the integer variants of that scheme).
//
// The grouped, segmented GEMM of the plans (C_g = sum over segments of
// A_seg B_seg, any transposition of A and B) reads FP64 operands directly.
// Per 32-wide K tile every row of the A tile and every column of the B tile is
// cut into four fixed-point digits relative to the largest binary exponent in
// that row (column) of the tile: v ~ 2^(e - 1054) F with the integer
// F = round(v 2^(1054 - e)), |F| <= 2^32, written as balanced base-256 digits
// F = a0 2^24 + a1 2^16 + a2 2^8 + a3, |a_s| <= 256.  The digits are exact in
// BF16, so every tensor-core product a_s b_t (|.| <= 2^16) is exact and a sum
// of at most 4 x 32 of them (< 2^24) is exact in the FP32 accumulator: the
// K tile's contribution of the digit pairs with s + t = d is an exact integer
// D_d.  The pairs with s + t <= 3 are kept (10 of 16); the tile contributes
// sum_d D_d 2^(eA + eB - 2060 - 8 d), which is added to a two-float (hi, lo)
// accumulator with TwoSum (Knuth, TAOCP vol. 2, 4.2.2) for d = 0, 1 and plain
// additions into lo for d = 2, 3.  Error: the digit truncation (<= 2^-33 of
// the row / column bound) and the dropped pairs, about 2^-32 of
// sum_k max_row |a| max_col |b| per K tile, against ~2^-24 for split-BF16
// with FP32 accumulation; no error grows with the number of K tiles beyond
// the two-float accumulation (~2^-48).
//
// The slicing is done on the fly from the FP64 operands in integer
// arithmetic (exponent and mantissa fields), because GB300's FP64 pipe runs at
// about 1/64 of its FP32 rate.  One CTA per 64 x 64 output tile, 16 warps of
// 16 x 16, mma.sync m16n8k16 (BF16 in, FP32 accumulate).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_kernels.h"

namespace tt {

namespace {

constexpr int OBM = 64, OBN = 64, OBK = 32, OPAD = 8, ODIG = 4;
constexpr int OT = 512;              // threads per CTA
constexpr int OEL = OBM * OBK / OT;  // tile elements per thread (4)

__device__ __forceinline__ int slot_of(Ref r) { return (int)(r >> 56); }
__device__ __forceinline__ long long off_of(Ref r) { return (long long)(r & 0x00FFFFFFFFFFFFFFull); }

__device__ __forceinline__ int biased_exp(double v) {
  return (int)((static_cast<unsigned long long>(__double_as_longlong(v)) >> 52) & 0x7FF);
}

// Balanced base-256 digits of F = round(v 2^(1054 - emax)) (emax: the largest
// biased exponent of the row, so |v| < 2^(emax - 1022) and |F| <= 2^32).
// Zero and subnormal v give F = 0.
__device__ __forceinline__ void fixed_digits(double v, int emax, __nv_bfloat16* d0, long long stride) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int E = (int)((bits >> 52) & 0x7FF);
  long long F = 0;
  if (E != 0) {
    const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 21 + emax - E;  // >= 21
    if (sh < 64) {
      F = (long long)((M + (1ull << (sh - 1))) >> sh);
      if (bits >> 63) F = -F;
    }
  }
  const long long a0 = (F + (1ll << 23)) >> 24;  // floor division (arithmetic shift)
  const long long r0 = F - a0 * (1ll << 24);     // [-2^23, 2^23)
  const long long a1 = (r0 + (1ll << 15)) >> 16;
  const long long r1 = r0 - a1 * (1ll << 16);    // [-2^15, 2^15)
  const long long a2 = (r1 + (1ll << 7)) >> 8;
  const long long a3 = r1 - a2 * (1ll << 8);     // [-128, 128)
  d0[0] = __float2bfloat16_rn((float)a0);
  d0[stride] = __float2bfloat16_rn((float)a1);
  d0[2 * stride] = __float2bfloat16_rn((float)a2);
  d0[3 * stride] = __float2bfloat16_rn((float)a3);
}

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (x - bp);
  hi = s;
}

// 2^x as a float for -126 <= x <= 127, else 0 (contributions below the FP32
// normal range are dropped; they are < 2^-126 in absolute value)
__device__ __forceinline__ float pow2f(int x) {
  return (x >= -126 && x <= 127) ? __int_as_float((x + 127) << 23) : 0.f;
}

// Element i (0..OEL-1) of thread tid in a 64 x 32 (rows x K) tile, coalesced for
// either storage order: kmajor (element (r, k) at r * ld + k) or not (at
// k * ld + r).
__device__ __forceinline__ int tile_row(bool kmajor, int tid, int i) { return kmajor ? (tid >> 5) + 16 * i : (tid & 63); }
__device__ __forceinline__ int tile_k(bool kmajor, int tid, int i) { return kmajor ? (tid & 31) : (tid >> 6) + 8 * i; }

__device__ __forceinline__ void load_tile(const double* __restrict__ P, long long ld, bool kmajor, int r0, int rmax,
                                          int k0, int kmax, int tid, double* v) {
#pragma unroll
  for (int i = 0; i < OEL; ++i) {
    const int gr = r0 + tile_row(kmajor, tid, i), gk = k0 + tile_k(kmajor, tid, i);
    v[i] = (gr < rmax && gk < kmax) ? (kmajor ? P[(long long)gr * ld + gk] : P[(long long)gk * ld + gr]) : 0.0;
  }
}

// Largest biased exponent per row of the tile into e[] (zeroed before).
__device__ __forceinline__ void row_exponents(const double* v, bool kmajor, int tid, int* e) {
  if (kmajor) {  // a warp holds one row per i: reduce over the lanes
#pragma unroll
    for (int i = 0; i < OEL; ++i) {
      const int m = __reduce_max_sync(0xffffffffu, biased_exp(v[i]));
      if ((tid & 31) == 0) atomicMax(&e[tile_row(true, tid, i)], m);
    }
  } else {  // a thread holds OEL K values of one row
    int m = 0;
#pragma unroll
    for (int i = 0; i < OEL; ++i) m = max(m, biased_exp(v[i]));
    atomicMax(&e[tile_row(false, tid, 0)], m);
  }
}

__global__ void __launch_bounds__(OT) gemm_oz_kernel(const GGroup* __restrict__ groups, const GSeg* __restrict__ segs,
                                                      const GTile* __restrict__ tiles, Bases bs) {
  __shared__ __align__(16) __nv_bfloat16 As[ODIG][OBM][OBK + OPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[ODIG][OBN][OBK + OPAD];
  __shared__ int eA[OBM], eB[OBN];
  const GTile tl = tiles[blockIdx.x];
  const GGroup g = groups[tl.g];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 16, wn = (warp & 3) * 16;
  const int gid = lane >> 2, tig = lane & 3;
  constexpr long long DS = (long long)OBM * (OBK + OPAD);  // digit stride in As / Bs

  float acc[ODIG][2][4], hi[2][4], lo[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      hi[j][r] = 0.f;
      lo[j][r] = 0.f;
#pragma unroll
      for (int d = 0; d < ODIG; ++d) acc[d][j][r] = 0.f;
    }

  for (int si = g.seg0; si < g.seg1; ++si) {
    const GSeg sg = segs[si];
    const double* A = reinterpret_cast<const double*>(sel_base(bs, slot_of(sg.A))) + off_of(sg.A);
    const double* B = reinterpret_cast<const double*>(sel_base(bs, slot_of(sg.B))) + off_of(sg.B);
    for (int k0 = 0; k0 < sg.K; k0 += OBK) {
      double va[OEL], vb[OEL];
      const bool ka = sg.tA == 0, kb = sg.tB == 1;
      // A logical M x K: stored M x K (tA = 0, K contiguous) or K x M (tA = 1);
      // B logical N x K: stored N x K (tB = 1) or K x N (tB = 0)
      load_tile(A, sg.lda, ka, tl.m0, g.M, k0, sg.K, tid, va);
      load_tile(B, sg.ldb, kb, tl.n0, g.N, k0, sg.K, tid, vb);
      if (tid < OBM) eA[tid] = 0;
      else if (tid < OBM + OBN) eB[tid - OBM] = 0;
      __syncthreads();
      row_exponents(va, ka, tid, eA);
      row_exponents(vb, kb, tid, eB);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < OEL; ++i) {
        const int ra = tile_row(ka, tid, i), rb = tile_row(kb, tid, i);
        fixed_digits(va[i], eA[ra], &As[0][ra][tile_k(ka, tid, i)], DS);
        fixed_digits(vb[i], eB[rb], &Bs[0][rb][tile_k(kb, tid, i)], DS);
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < OBK; ks += 16) {
        uint32_t af[ODIG][4];
#pragma unroll
        for (int s = 0; s < ODIG; ++s) {
          const int r0 = wm + gid;
          af[s][0] = *reinterpret_cast<const uint32_t*>(&As[s][r0][ks + 2 * tig]);
          af[s][1] = *reinterpret_cast<const uint32_t*>(&As[s][r0 + 8][ks + 2 * tig]);
          af[s][2] = *reinterpret_cast<const uint32_t*>(&As[s][r0][ks + 8 + 2 * tig]);
          af[s][3] = *reinterpret_cast<const uint32_t*>(&As[s][r0 + 8][ks + 8 + 2 * tig]);
        }
#pragma unroll
        for (int t = 0; t < ODIG; ++t) {
          uint32_t bf[2][2];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int c0 = wn + 8 * j + gid;
            bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[t][c0][ks + 2 * tig]);
            bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[t][c0][ks + 8 + 2 * tig]);
          }
#pragma unroll
          for (int s = 0; s + t < ODIG; ++s)
#pragma unroll
            for (int j = 0; j < 2; ++j) mma16816(acc[s + t][j], af[s], bf[j]);
        }
      }
      // fold this K tile: D_d 2^(eA + eB - 2060 - 8 d) into (hi, lo)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int m = wm + gid + ((r >= 2) ? 8 : 0);
          const int n = wn + 8 * j + 2 * tig + (r & 1);
          const int x = eA[m] + eB[n] - 2060;
          two_sum_into(hi[j][r], lo[j][r], acc[0][j][r] * pow2f(x));
          two_sum_into(hi[j][r], lo[j][r], acc[1][j][r] * pow2f(x - 8));
          lo[j][r] += acc[2][j][r] * pow2f(x - 16) + acc[3][j][r] * pow2f(x - 24);
#pragma unroll
          for (int d = 0; d < ODIG; ++d) acc[d][j][r] = 0.f;
        }
      __syncthreads();
    }
  }
  const bool accum = g.flags & 1;
  const bool out_f32 = g.flags & 2;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gm = tl.m0 + wm + gid + ((r >= 2) ? 8 : 0);
      const int gn = tl.n0 + wn + 8 * j + 2 * tig + (r & 1);
      if (gm >= g.M || gn >= g.N) continue;
      const long long o = (long long)gm * g.ldc + gn;
      const double v = (double)hi[j][r] + (double)lo[j][r];
      if (out_f32) {
        float* C = reinterpret_cast<float*>(sel_base(bs, slot_of(g.C))) + off_of(g.C) + o;
        *C = accum ? *C + (float)v : (float)v;
      } else {
        double* C = reinterpret_cast<double*>(sel_base(bs, slot_of(g.C))) + off_of(g.C) + o;
        *C = accum ? *C + v : v;
      }
    }
}

}  // namespace

cudaError_t launch_gemm_oz(const DevGemm& g, const Bases& b, cudaStream_t s) {
  if (g.ntiles64 == 0) return cudaSuccess;
  gemm_oz_kernel<<<g.ntiles64, OT, 0, s>>>(g.groups, g.segs, g.tiles64, b);
  return cudaGetLastError();
}

}  // namespace tt
