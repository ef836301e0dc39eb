// Device kernels of the tanTRG hot path (sm_103a).
//
//  * grouped, segmented GEMM (FP64 FMA; split-BF16 x3 on the tensor cores):
//    every contraction of the H_eff apply (Supplement, Fig. "Lanczos": L_i A_i,
//    then H_i, then R_i), the bond apply (Fig. "optimalB"(d)), the environment
//    updates and the absorb step is a list of groups C_g = sum_seg A_seg B_seg;
//  * W gather: applies the sparse MPO tensor between the two GEMM stages;
//  * Lanczos vector kernels in FP64 (Supplement, "Lanczos-based exponential
//    method"), with deterministic two-stage reductions;
//  * the small Krylov exponential exp(t T) e_1 by scaling and squaring of a
//    Taylor polynomial (Moler & Van Loan);
//  * Householder QR (FP64) of the per-sector gauge matrices.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "tt_kernels.h"

namespace tt {

namespace {

__device__ __forceinline__ int slot_of(Ref r) { return (int)(r >> 56); }
__device__ __forceinline__ long long off_of(Ref r) { return (long long)(r & 0x00FFFFFFFFFFFFFFull); }

template <typename T>
__device__ __forceinline__ T* rptr(const Bases& b, Ref r) {
  return reinterpret_cast<T*>(sel_base(b, slot_of(r))) + off_of(r);
}

constexpr int NBLK = 304;  // 2 x 152 SMs for the vector reductions
constexpr int VT = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// FP64 grouped GEMM: one 64 x 64 output tile per CTA, 256 threads, 4 x 4 per
// thread, K staged through shared memory in chunks of 16.
// ---------------------------------------------------------------------------
constexpr int FBM = 64, FBN = 64, FBK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GGroup* __restrict__ groups,
                                                       const GSeg* __restrict__ segs,
                                                       const GTile* __restrict__ tiles, Bases bs) {
  __shared__ double As[FBK][FBM + 1];
  __shared__ double Bs[FBK][FBN + 1];
  const GTile tl = tiles[blockIdx.x];
  const GGroup g = groups[tl.g];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;  // 16 x 16 threads, each 4 x 4 outputs
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int si = g.seg0; si < g.seg1; ++si) {
    const GSeg sg = segs[si];
    const double* A = rptr<const double>(bs, sg.A);
    const double* B = rptr<const double>(bs, sg.B);
    for (int k0 = 0; k0 < sg.K; k0 += FBK) {
      // load A tile: FBM x FBK logical (m, k)
      for (int e = tid; e < FBM * FBK; e += 256) {
        int mm, kk;
        if (sg.tA) { mm = e % FBM; kk = e / FBM; } else { kk = e % FBK; mm = e / FBK; }
        int gm = tl.m0 + mm, gk = k0 + kk;
        double v = 0.0;
        if (gm < g.M && gk < sg.K)
          v = sg.tA ? A[(long long)gk * sg.lda + gm] : A[(long long)gm * sg.lda + gk];
        As[kk][mm] = v;
      }
      for (int e = tid; e < FBN * FBK; e += 256) {
        int nn, kk;
        if (sg.tB) { kk = e % FBK; nn = e / FBK; } else { nn = e % FBN; kk = e / FBN; }
        int gn = tl.n0 + nn, gk = k0 + kk;
        double v = 0.0;
        if (gn < g.N && gk < sg.K)
          v = sg.tB ? B[(long long)gn * sg.ldb + gk] : B[(long long)gk * sg.ldb + gn];
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < FBK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  double* C = rptr<double>(bs, g.C);
  const bool accum = g.flags & 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = tl.m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = tl.n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      double* c = C + (long long)gm * g.ldc + gn;
      *c = accum ? *c + acc[i][j] : acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// The same grouped GEMM in double-float arithmetic on the FP32 pipe (GB300
// issues ~2 FP64 FMA per clock per SM against 128 FP32): FP64 operands split
// into float pairs (hi, lo) as they are staged, every product by the FMA
// TwoProduct with the cross terms, every sum by TwoSum into an unnormalised
// (hi, lo) accumulator (Dekker; Knuth TAOCP vol. 2, 4.2.2): ~2^-46 relative
// per operation, K 2^-46 of sum |a| |b| per output.  Output FP64.  Used by the
// mixed modes' CholeskyQR Gram and apply GEMMs.
// ---------------------------------------------------------------------------
// v = hi + lo: hi the top 24 significant bits of v (truncated), lo the other
// 29 rounded to 24 (error <= 2^-47 |v|), by integer operations on the FP64 bit
// pattern (no FP64 arithmetic); zero for zero and FP64 subnormals, FP64
// conversions for |v| outside [2^-97, 2^127]
__device__ __forceinline__ float2 df_split(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return make_float2(0.f, 0.f);
  if (e < 926 || e > 1150) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
  }
  const unsigned sg = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sg | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  // low 29 mantissa bits times 2^(e - 1075) = (ml 2^-29) 2^(e - 1046), e - 1046 >= -120
  const float lo = ((float)(unsigned)(b & 0x1FFFFFFFull) * 1.862645149230957e-09f) *
                   __uint_as_float((unsigned)(e - 1046 + 127) << 23);
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sg));
}

__global__ void __launch_bounds__(256) gemm_df_kernel(const GGroup* __restrict__ groups, const GSeg* __restrict__ segs,
                                                      const GTile* __restrict__ tiles, Bases bs) {
  __shared__ float2 As[FBK][FBM + 1];
  __shared__ float2 Bs[FBK][FBN + 1];
  const GTile tl = tiles[blockIdx.x];
  const GGroup g = groups[tl.g];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  float ah_[4][4], al_[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { ah_[i][j] = 0.f; al_[i][j] = 0.f; }

  for (int si = g.seg0; si < g.seg1; ++si) {
    const GSeg sg = segs[si];
    const double* A = rptr<const double>(bs, sg.A);
    const double* B = rptr<const double>(bs, sg.B);
    for (int k0 = 0; k0 < sg.K; k0 += FBK) {
      for (int e = tid; e < FBM * FBK; e += 256) {
        int mm, kk;
        if (sg.tA) { mm = e % FBM; kk = e / FBM; } else { kk = e % FBK; mm = e / FBK; }
        const int gm = tl.m0 + mm, gk = k0 + kk;
        double v = 0.0;
        if (gm < g.M && gk < sg.K) v = sg.tA ? A[(long long)gk * sg.lda + gm] : A[(long long)gm * sg.lda + gk];
        As[kk][mm] = df_split(v);
      }
      for (int e = tid; e < FBN * FBK; e += 256) {
        int nn, kk;
        if (sg.tB) { kk = e % FBK; nn = e / FBK; } else { nn = e % FBN; kk = e / FBN; }
        const int gn = tl.n0 + nn, gk = k0 + kk;
        double v = 0.0;
        if (gn < g.N && gk < sg.K) v = sg.tB ? B[(long long)gn * sg.ldb + gk] : B[(long long)gk * sg.ldb + gn];
        Bs[kk][nn] = df_split(v);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < FBK; ++kk) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float p = a[i].x * b[j].x;
            float e = fmaf(a[i].x, b[j].x, -p);
            e = fmaf(a[i].x, b[j].y, e);
            e = fmaf(a[i].y, b[j].x, e);
            const float s = ah_[i][j] + p;
            const float bp = s - ah_[i][j];
            al_[i][j] += ((ah_[i][j] - (s - bp)) + (p - bp)) + e;
            ah_[i][j] = s;
          }
      }
      __syncthreads();
    }
  }
  double* C = rptr<double>(bs, g.C);
  const bool accum = g.flags & 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = tl.m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = tl.n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      double* c = C + (long long)gm * g.ldc + gn;
      const double v = (double)ah_[i][j] + (double)al_[i][j];
      *c = accum ? *c + v : v;
    }
  }
}

// ---------------------------------------------------------------------------
// Split-BF16 grouped GEMM on the tensor cores (mma.sync m16n8k16, FP32
// accumulation).  Operands are stored as NS bf16 levels x = x0 + x1 (+ x2),
// level l at element offset l * lo[slot]; the products with l_A + l_B < NS are
// summed: NS = 2 -> 3 products (~2^-16 relative), NS = 3 -> 6 products
// (~2^-24).  The leading product x0*y0 and the smaller ones accumulate in
// separate FP32 registers; every 32-wide K chunk the leading one is folded
// into a two-float (hi, lo) sum with TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
// the small one is added to lo, so the accumulation error does not grow with
// K.  64 x 64 tile per CTA, 4 warps of 32 x 32.  Output FP64 or FP32 (flags
// bit1).
// ---------------------------------------------------------------------------
constexpr int HBM = 64, HBN = 64, HBK = 32, HPAD = 8;

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (x - bp);
  hi = s;
}

template <int NS>
__global__ void __launch_bounds__(128) gemm_bf16_split_kernel(const GGroup* __restrict__ groups,
                                                              const GSeg* __restrict__ segs,
                                                              const GTile* __restrict__ tiles, Bases bs) {
  __shared__ __align__(16) __nv_bfloat16 As[NS][HBM][HBK + HPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[NS][HBN][HBK + HPAD];
  const GTile tl = tiles[blockIdx.x];
  const GGroup g = groups[tl.g];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4], accs[2][4][4], hi[2][4][4], lo[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) { acc[i][j][r] = 0.f; accs[i][j][r] = 0.f; hi[i][j][r] = 0.f; lo[i][j][r] = 0.f; }

  for (int si = g.seg0; si < g.seg1; ++si) {
    const GSeg sg = segs[si];
    const __nv_bfloat16* A0 = rptr<const __nv_bfloat16>(bs, sg.A);
    const __nv_bfloat16* B0 = rptr<const __nv_bfloat16>(bs, sg.B);
    const long long loA = sel_lo(bs, slot_of(sg.A)), loB = sel_lo(bs, slot_of(sg.B));
    for (int k0 = 0; k0 < sg.K; k0 += HBK) {
      for (int e = tid; e < HBM * HBK; e += 128) {
        int mm, kk;
        if (sg.tA) { mm = e % HBM; kk = e / HBM; } else { kk = e % HBK; mm = e / HBK; }
        const int gm = tl.m0 + mm, gk = k0 + kk;
        const bool in = gm < g.M && gk < sg.K;
        const long long o = sg.tA ? (long long)gk * sg.lda + gm : (long long)gm * sg.lda + gk;
#pragma unroll
        for (int l = 0; l < NS; ++l) As[l][mm][kk] = in ? A0[l * loA + o] : __float2bfloat16(0.f);
      }
      for (int e = tid; e < HBN * HBK; e += 128) {
        int nn, kk;
        if (sg.tB) { kk = e % HBK; nn = e / HBK; } else { nn = e % HBN; kk = e / HBN; }
        const int gn = tl.n0 + nn, gk = k0 + kk;
        const bool in = gn < g.N && gk < sg.K;
        const long long o = sg.tB ? (long long)gn * sg.ldb + gk : (long long)gk * sg.ldb + gn;
#pragma unroll
        for (int l = 0; l < NS; ++l) Bs[l][nn][kk] = in ? B0[l * loB + o] : __float2bfloat16(0.f);
      }
      __syncthreads();
#pragma unroll
      for (int pass = 0; pass < (NS == 2 ? 3 : 6); ++pass) {
        // (la, lb): NS=2: (0,0) (0,1) (1,0); NS=3 adds (0,2) (1,1) (2,0); small products first
        const int order = (NS == 2 ? 2 : 5) - pass;
        const int la = (order == 2 || order == 4) ? 1 : (order == 5 ? 2 : 0);
        const int lb = (order == 1 || order == 4) ? 1 : (order == 3 ? 2 : 0);
#pragma unroll
        for (int ks = 0; ks < HBK; ks += 16) {
          uint32_t af[2][4], bf[4][2];
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int r0 = wm + 16 * i + gid;
            af[i][0] = *reinterpret_cast<const uint32_t*>(&As[la][r0][ks + 2 * tig]);
            af[i][1] = *reinterpret_cast<const uint32_t*>(&As[la][r0 + 8][ks + 2 * tig]);
            af[i][2] = *reinterpret_cast<const uint32_t*>(&As[la][r0][ks + 8 + 2 * tig]);
            af[i][3] = *reinterpret_cast<const uint32_t*>(&As[la][r0 + 8][ks + 8 + 2 * tig]);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c0 = wn + 8 * j + gid;
            bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[lb][c0][ks + 2 * tig]);
            bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[lb][c0][ks + 8 + 2 * tig]);
          }
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_bf16_16816(order == 0 ? acc[i][j] : accs[i][j], af[i], bf[j]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            two_sum_acc(hi[i][j][r], lo[i][j][r], acc[i][j][r]);
            lo[i][j][r] += accs[i][j][r];
            acc[i][j][r] = 0.f;
            accs[i][j][r] = 0.f;
          }
    }
  }
  const bool accum = g.flags & 1;
  const bool out_f32 = g.flags & 2;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int gm = tl.m0 + wm + 16 * i + gid + ((r >= 2) ? 8 : 0);
        const int gn = tl.n0 + wn + 8 * j + 2 * tig + (r & 1);
        if (gm >= g.M || gn >= g.N) continue;
        const long long o = (long long)gm * g.ldc + gn;
        const double v = (double)hi[i][j][r] + (double)lo[i][j][r];
        if (out_f32) {
          float* C = rptr<float>(bs, g.C) + o;
          *C = accum ? *C + (float)v : (float)v;
        } else {
          double* C = rptr<double>(bs, g.C) + o;
          *C = accum ? *C + v : v;
        }
      }
}

// ---------------------------------------------------------------------------
// W gather: dst[r, c] = sum_k coef_k src_k[r, c]  (one CTA per item, rows
// strided over the 8 warps, columns over the lanes).  FP64 in, FP64 out for
// the FP64 path.  Mixed path: the sources are the FP32 outputs of S1, so the
// sum and the split into bf16 levels run in FP32 (GB300 has about 1/64 of
// its FP32 rate in FP64); each level's remainder is exact in FP32.
// ---------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void store_split_f32(__nv_bfloat16* p, long long lo, float v) {
#pragma unroll
  for (int l = 0; l < NS; ++l) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    p[l * lo] = h;
    v -= __bfloat162float(h);
  }
}
// FP64 value: the first level is rounded from the double and its remainder
// (|r| <= 2^-9 |x|) is rounded to FP32 once, so the levels carry the value to
// about 2^-25 relative with two FP64 operations per element.
template <int NS>
__device__ __forceinline__ void store_split_f64(__nv_bfloat16* p, long long lo, double x) {
  const __nv_bfloat16 h0 = __double2bfloat16(x);
  p[0] = h0;
  store_split_f32<NS - 1>(p + lo, lo, __double2float_rn(x - (double)__bfloat162float(h0)));
}

template <int IN, int OUT>
__global__ void __launch_bounds__(256) gather_kernel(const GItem* __restrict__ items,
                                                     const GContrib* __restrict__ cs, Bases bs) {
  const GItem it = items[blockIdx.x];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < it.rows; r += 8)
    for (int c = tx; c < it.cols; c += 32) {
      const long long d = (long long)r * it.dst_rs + c;
      if constexpr (IN == 0) {
        double acc = 0.0;
        for (int k = it.c0; k < it.c1; ++k) {
          const GContrib cb = cs[k];
          acc = fma(cb.coef, rptr<const double>(bs, cb.src)[(long long)r * cb.src_rs + c], acc);
        }
        if constexpr (OUT == 0) rptr<double>(bs, it.dst)[d] = acc;
        else if constexpr (OUT == 1) rptr<float>(bs, it.dst)[d] = (float)acc;
        else store_split_f64<OUT>(rptr<__nv_bfloat16>(bs, it.dst) + d, sel_lo(bs, slot_of(it.dst)), acc);
      } else {
        float acc = 0.f;
        for (int k = it.c0; k < it.c1; ++k) {
          const GContrib cb = cs[k];
          acc = fmaf((float)cb.coef, rptr<const float>(bs, cb.src)[(long long)r * cb.src_rs + c], acc);
        }
        if constexpr (OUT == 0) rptr<double>(bs, it.dst)[d] = (double)acc;
        else if constexpr (OUT == 1) rptr<float>(bs, it.dst)[d] = acc;
        else store_split_f32<OUT>(rptr<__nv_bfloat16>(bs, it.dst) + d, sel_lo(bs, slot_of(it.dst)), acc);
      }
    }
}

// Strided 2-D copies, one item = rows x cols elements with arbitrary row and
// column strides on both sides.  The item is cut into 32 x 32 tiles; the
// CTAs of grid row blockIdx.x share item blockIdx.x's tiles (stride
// gridDim.y).  A tile goes through shared memory so that both the load and
// the store run along whichever side has unit stride (a transposing copy is
// coalesced on both ends).  NS = 0: FP64 -> FP64; NS = 2, 3: FP64 -> split
// bf16 levels at dst + l * lo[slot(dst)].
template <int NS>
__global__ void __launch_bounds__(256) tile_copy_kernel(const CItem* __restrict__ items, Bases bs) {
  __shared__ double tile[32][33];
  const CItem it = items[blockIdx.x];
  const double* src = rptr<const double>(bs, it.src);
  const int tcr = (it.rows + 31) >> 5, tcc = (it.cols + 31) >> 5;
  const int ntiles = tcr * tcc;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const bool src_rmaj = it.src_cs == 1 || it.src_rs != 1;   // src contiguous along c
  const bool dst_rmaj = it.dst_cs == 1 || it.dst_rs != 1;
  for (int t = blockIdx.y; t < ntiles; t += gridDim.y) {
    const int r0 = (t / tcc) << 5, c0 = (t % tcc) << 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = ty + 8 * k;  // slow index within the tile
      const int r = src_rmaj ? r0 + a : r0 + tx, c = src_rmaj ? c0 + tx : c0 + a;
      if (r < it.rows && c < it.cols) {
        const double v = src[(long long)r * it.src_rs + (long long)c * it.src_cs];
        if (src_rmaj) tile[a][tx] = v;
        else tile[tx][a] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = ty + 8 * k;
      const int lr = dst_rmaj ? a : tx, lc = dst_rmaj ? tx : a;
      const int r = r0 + lr, c = c0 + lc;
      if (r < it.rows && c < it.cols) {
        const long long o = (long long)r * it.dst_rs + (long long)c * it.dst_cs;
        const double v = tile[lr][lc];
        if constexpr (NS == 0) rptr<double>(bs, it.dst)[o] = v;
        else store_split_f64<NS>(rptr<__nv_bfloat16>(bs, it.dst) + o, sel_lo(bs, slot_of(it.dst)), v);
      }
    }
    __syncthreads();
  }
}

static dim3 copy_grid(const DevCopy& c) {
  // enough CTAs per item for about four tiles each, at most 256 per item
  const int y = std::max(1, std::min(256, (c.maxtiles + 3) / 4));
  return dim3((unsigned)c.nitems, (unsigned)y);
}

// x (FP64, n) -> ns bf16 levels out[l * n + i], x ~ sum_l out[l].
__global__ void split_bf16_kernel(const double* __restrict__ x, long long n, int ns, __nv_bfloat16* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (ns == 2) store_split_f64<2>(out + i, n, x[i]);
    else store_split_f64<3>(out + i, n, x[i]);
  }
}


// ---------------------------------------------------------------------------
// Lanczos vector kernels
// ---------------------------------------------------------------------------
// partial[blk * 17 + j] = sum over this block's chunk of Q_j . w   (j < nv)
template <int MAXV>
__global__ void __launch_bounds__(VT) multidot_kernel(const double* __restrict__ Q, long long ldq, int j0, int nv,
                                                      const double* __restrict__ w, long long n,
                                                      double* __restrict__ partial) {
  double acc[MAXV];
#pragma unroll
  for (int j = 0; j < MAXV; ++j) acc[j] = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    double wi = w[i];
#pragma unroll
    for (int j = 0; j < MAXV; ++j)
      if (j < nv) acc[j] = fma(Q[(long long)(j0 + j) * ldq + i], wi, acc[j]);
  }
  __shared__ double red[VT / 32][MAXV];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < MAXV; ++j) {
    double v = warp_sum(acc[j]);
    if (lane == 0) red[wp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int q = 0; q < VT / 32; ++q) s += red[q][threadIdx.x];
    partial[blockIdx.x * 17 + threadIdx.x] = s;
  }
}

__global__ void sumsq_kernel(const double* __restrict__ v, long long n, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
    acc = fma(v[i], v[i], acc);
  __shared__ double red[VT / 32];
  double s = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < VT / 32; ++q) t += red[q];
    partial[blockIdx.x * 17] = t;
  }
}

// out[j] = sum_b partial[b * 17 + j] in a fixed order (deterministic)
__device__ void finalize_sums(const double* partial, int nblk, int nv, double* out) {
  // called by one warp
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < nv; ++j) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partial[b * 17 + j];
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
  }
}

__global__ void norm_init_finalize(const double* partial, int nblk, KrylovState* ks) {
  __shared__ double s;
  finalize_sums(partial, nblk, 1, &s);
  __syncwarp();
  if (threadIdx.x == 0) {
    double nb = sqrt(s);
    ks->nb = nb;
    ks->hscale = 0.0;
    ks->resid = 0.0;
    ks->kdim = 0;
    ks->broken = 0;
    ks->bad = !isfinite(nb) ? 1 : 0;
    for (int j = 0; j < 17; ++j) { ks->alpha[j] = 0; ks->beta[j] = 0; ks->h[j] = 0; ks->c[j] = 0; }
  }
}

__global__ void scale_kernel(const double* __restrict__ v, long long n, const double* __restrict__ denom,
                             const int* __restrict__ dead, double* __restrict__ out) {
  const double d = *denom;
  const bool z = (dead && *dead) || d == 0.0;
  const double inv = z ? 0.0 : 1.0 / d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = v[i] * inv;
}

__global__ void alpha_finalize(const double* partial, int nblk, int k, KrylovState* ks) {
  __shared__ double s;
  finalize_sums(partial, nblk, 1, &s);
  __syncwarp();
  if (threadIdx.x == 0 && !ks->broken) ks->alpha[k] = s;
}

__global__ void three_term_kernel(const double* __restrict__ Q, long long ldq, int k, double* __restrict__ w,
                                  long long n, const KrylovState* __restrict__ ks) {
  const double a = ks->alpha[k];
  const double b = (k > 0) ? ks->beta[k - 1] : 0.0;
  const double* qk = Q + (long long)k * ldq;
  const double* qp = Q + (long long)(k > 0 ? k - 1 : 0) * ldq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = w[i] - a * qk[i];
    if (k > 0) v -= b * qp[i];
    w[i] = v;
  }
}

__global__ void h_finalize(const double* partial, int nblk, int nv, KrylovState* ks) {
  finalize_sums(partial, nblk, nv, ks->h);
}

// w -= sum_j h_j Q_j ; optional partial ||w||^2
__global__ void __launch_bounds__(VT) axpy_multi_kernel(const double* __restrict__ Q, long long ldq, int nv,
                                                        const KrylovState* __restrict__ ks, double* __restrict__ w,
                                                        long long n, double* __restrict__ partial) {
  __shared__ double h[17];
  if (threadIdx.x < 17) h[threadIdx.x] = ks->h[threadIdx.x];
  __syncthreads();
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    double v = w[i];
    for (int j = 0; j < nv; ++j) v -= h[j] * Q[(long long)j * ldq + i];
    w[i] = v;
    acc = fma(v, v, acc);
  }
  if (partial) {
    __shared__ double red[VT / 32];
    double s = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < VT / 32; ++q) t += red[q];
      partial[blockIdx.x * 17] = t;
    }
  }
}

// beta_k = ||w||; breakdown test of the oracle; stores beta (or 0 if broken).
__global__ void beta_finalize(const double* partial, int nblk, int k, int K, double tol, KrylovState* ks) {
  __shared__ double s;
  finalize_sums(partial, nblk, 1, &s);
  __syncwarp();
  if (threadIdx.x != 0) return;
  if (ks->broken) {
    ks->beta[k] = 0.0;
    return;
  }
  double b = sqrt(s);
  if (!isfinite(b) || !isfinite(ks->alpha[k])) ks->bad = 1;
  double hs = fmax(ks->hscale, fabs(ks->alpha[k]) + b);
  ks->hscale = hs;
  ks->kdim = k + 1;
  if (k == K - 1) {
    ks->beta[k] = b;  // residual norm, not part of T
    return;
  }
  if (b <= tol * hs) {
    ks->broken = 1;
    ks->beta[k] = 0.0;
    return;
  }
  ks->beta[k] = b;
}

// c = exp(t T) e_1 for the kdim x kdim tridiagonal T, by scaling and squaring
// with a degree-18 Taylor polynomial (Moler & Van Loan, "Nineteen dubious
// ways", method 3): M = t T / 2^s with ||M||_1 <= 1/4, E = sum_k M^k / k!
// (Horner), then E <- E^2 s times.  One thread per matrix entry (kdim <= 16).
__global__ void __launch_bounds__(256) krylov_exp_kernel(KrylovState* ks, double t, int K) {
  __shared__ double M[16][16], E[16][16], P[16][16];
  __shared__ int m_s, s_s;
  const int tid = threadIdx.x, i = tid / 16, j = tid % 16;
  if (tid == 0) {
    const int m = ks->kdim;
    double nrm = 0.0;  // ||t T||_1 (T symmetric tridiagonal)
    for (int c = 0; c < m; ++c) {
      double col = fabs(ks->alpha[c]);
      if (c > 0) col += fabs(ks->beta[c - 1]);
      if (c + 1 < m) col += fabs(ks->beta[c]);
      nrm = fmax(nrm, fabs(t) * col);
    }
    int sq = 0;
    while (nrm > 0.25 && sq < 60) { nrm *= 0.5; ++sq; }
    m_s = m;
    s_s = sq;
  }
  __syncthreads();
  const int m = m_s, sq = s_s;
  const double scale = ldexp(t, -sq);
  double mij = 0.0;
  if (i < m && j < m) {
    if (i == j) mij = ks->alpha[i];
    else if (j == i + 1) mij = ks->beta[i];
    else if (i == j + 1) mij = ks->beta[j];
    mij *= scale;
  }
  M[i][j] = mij;
  E[i][j] = (i == j && i < m) ? 1.0 : 0.0;  // Horner: E = I + M/18, then E = I + M E / k
  __syncthreads();
  for (int k = 18; k >= 1; --k) {
    double acc = 0.0;
    for (int q = 0; q < m; ++q) acc = fma(M[i][q], E[q][j], acc);
    __syncthreads();
    E[i][j] = (i < m && j < m) ? ((i == j ? 1.0 : 0.0) + acc / (double)k) : 0.0;
    __syncthreads();
  }
  for (int r = 0; r < sq; ++r) {
    double acc = 0.0;
    for (int q = 0; q < m; ++q) acc = fma(E[i][q], E[q][j], acc);
    P[i][j] = acc;
    __syncthreads();
    E[i][j] = P[i][j];
    __syncthreads();
  }
  if (tid < 17) ks->c[tid] = (tid < m) ? E[tid][0] : 0.0;
  if (tid == 0) ks->resid = (!ks->broken && m == K) ? ks->nb * ks->beta[K - 1] * fabs(E[K - 1][0]) : 0.0;
}

__global__ void __launch_bounds__(VT) combine_kernel(const double* __restrict__ Q, long long ldq,
                                                     const KrylovState* __restrict__ ks, double* __restrict__ y,
                                                     long long n, double* __restrict__ partial) {
  __shared__ double c[17];
  __shared__ int m;
  if (threadIdx.x < 17) c[threadIdx.x] = ks->c[threadIdx.x] * ks->nb;
  if (threadIdx.x == 0) m = ks->kdim;
  __syncthreads();
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) v = fma(c[j], Q[(long long)j * ldq + i], v);
    y[i] = v;
    acc = fma(v, v, acc);
  }
  __shared__ double red[VT / 32];
  double s = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < VT / 32; ++q) t += red[q];
    partial[blockIdx.x * 17] = t;
  }
}

__global__ void nrm_finalize(const double* partial, int nblk, KrylovState* ks, RhoScalars* rs) {
  __shared__ double s;
  finalize_sums(partial, nblk, 1, &s);
  __syncwarp();
  if (threadIdx.x != 0) return;
  double nrm = sqrt(s);
  ks->nrm = nrm;
  if (!isfinite(nrm) || nrm == 0.0 || ks->bad) {
    rs->bad = 1;
    return;
  }
  rs->logscale += log(nrm);
  rs->resid_max = fmax(rs->resid_max, ks->resid);
}

// ---------------------------------------------------------------------------
// Householder QR, one CTA per column-major matrix (ld = m).
// ---------------------------------------------------------------------------
constexpr int QRT = 256;
constexpr int QR_MAXN = 2048;

__device__ __forceinline__ void qr_one(const QrJob J, double* __restrict__ ws);

__global__ void __launch_bounds__(QRT) qr_kernel(const QrJob* __restrict__ jobs, double* __restrict__ ws,
                                                 const int* __restrict__ only, int* __restrict__ nrun) {
  if (only && !only[blockIdx.x]) return;  // masked launch: fallback sectors only
  if (nrun && threadIdx.x == 0) atomicAdd(nrun, 1);
  qr_one(jobs[blockIdx.x], ws);
}

// one matrix whose job record travels as a kernel argument (no device copy of it)
__global__ void __launch_bounds__(QRT) qr_byval_kernel(const QrJob J, double* __restrict__ ws) { qr_one(J, ws); }

__device__ __forceinline__ void qr_one(const QrJob J, double* __restrict__ ws) {
  const int m = J.m, n = J.n;
  double* A = ws + J.a;
  double* Qm = ws + J.q;
  double* R = ws + J.r;
  __shared__ double tau_s[QR_MAXN];
  __shared__ double red[QRT / 32];
  __shared__ double bcast;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = QRT / 32;
  const int kmax = m < n ? m : n;
  for (int k = 0; k < kmax; ++k) {
    double* col = A + (long long)k * m;
    double s = 0.0;
    for (int i = k + 1 + threadIdx.x; i < m; i += QRT) s = fma(col[i], col[i], s);
    s = warp_sum(s);
    if (lane == 0) red[wp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < nw; ++q) t += red[q];
      double alpha = col[k];
      double tau = 0.0, scale = 0.0;
      if (t > 0.0) {
        double beta = -copysign(sqrt(alpha * alpha + t), alpha);
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
        col[k] = beta;
      }
      tau_s[k] = tau;
      bcast = scale;
    }
    __syncthreads();
    const double scale = bcast;
    if (tau_s[k] != 0.0)
      for (int i = k + 1 + threadIdx.x; i < m; i += QRT) col[i] *= scale;
    __syncthreads();
    const double tau = tau_s[k];
    if (tau != 0.0) {
      for (int j = k + 1 + wp; j < n; j += nw) {
        double* cj = A + (long long)j * m;
        double w = 0.0;
        for (int i = k + 1 + lane; i < m; i += 32) w = fma(col[i], cj[i], w);
        w = warp_sum(w) + cj[k];
        w *= tau;
        if (lane == 0) cj[k] -= w;
        for (int i = k + 1 + lane; i < m; i += 32) cj[i] = fma(-w, col[i], cj[i]);
      }
    }
    __syncthreads();
  }
  // R (n x n, column-major)
  for (long long e = threadIdx.x; e < (long long)n * n; e += QRT) {
    int i = (int)(e % n), j = (int)(e / n);
    R[e] = (i <= j && i < m) ? A[(long long)j * m + i] : 0.0;
  }
  // Q = H_0 ... H_{kmax-1} [I_n ; 0]   (columns j >= m stay zero)
  for (long long e = threadIdx.x; e < (long long)m * n; e += QRT) {
    int i = (int)(e % m), j = (int)(e / m);
    Qm[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = kmax - 1; k >= 0; --k) {
    const double tau = tau_s[k];
    if (tau == 0.0) continue;
    const double* v = A + (long long)k * m;
    for (int j = k + wp; j < n; j += nw) {
      double* qj = Qm + (long long)j * m;
      double w = 0.0;
      for (int i = k + 1 + lane; i < m; i += 32) w = fma(v[i], qj[i], w);
      w = warp_sum(w) + qj[k];
      w *= tau;
      if (lane == 0) qj[k] -= w;
      for (int i = k + 1 + lane; i < m; i += 32) qj[i] = fma(-w, v[i], qj[i]);
    }
    __syncthreads();
  }
  // sign convention diag(R) >= 0
  for (int k = wp; k < n; k += nw) {
    double d = (R[(long long)k * n + k] < 0.0) ? -1.0 : 1.0;
    __syncwarp();
    if (d < 0) {
      for (int i = lane; i < m; i += 32) Qm[(long long)k * m + i] = -Qm[(long long)k * m + i];
      for (int j = k + lane; j < n; j += 32) R[(long long)j * n + k] = -R[(long long)j * n + k];
    }
  }
}

// Cholesky G = R^T R (R upper; G the sum of the job's partial Gram matrices,
// row-major n x n at ws + g) and R^-1, one CTA per job.  Optional diagonal
// shift s = 11 (m n + n (n + 1)) u tr(G) (shifted CholeskyQR, Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa 2020).  A non-positive or non-finite pivot
// marks fail[sec] and leaves the job to the Householder fallback.
//
// The upper triangle is packed row by row (row i holds columns i..n-1) in
// shared memory, or for n > CHOL_SMEM_MAXN in the job's workspace scratch,
// factorised in place (right-looking: pivot row scaled, then every trailing
// row updated, a warp per row, lanes along the columns), R written out, then
// inverted in place, also right-looking: rows k = n-1 .. 0 of R^-1 are
// finalised in turn (row k divided by R(k, k)) and every row above takes its
// rank-1 update, R^-1(i, c) -= R(i, k) R^-1(k, c) (back substitution of
// R X = I, with R(i, k) read just before its slot becomes R^-1(i, k)).  Every
// step is parallel over a whole trailing block.
//
// Element arithmetic: FP64, or double-float (a pair of floats, the error-free
// TwoSum / FMA TwoProduct transformations of Dekker and Knuth; ~2^-46
// relative), which runs on the FP32 pipe: GB300 executes ~2 FP64 FMA per clock
// per SM against 128 FP32, and one CTA factorises one sector.
constexpr int CHOL_SMEM_MAXN = 230;
constexpr int CHOL_T = 512;

__device__ __forceinline__ int pk(int i, int j, int n) { return i * n - (i * (i - 1)) / 2 + (j - i); }

struct CholF64 {
  using T = double;
  static constexpr double u = 1.1102230246251565e-16;  // unit roundoff 2^-53
  static __device__ __forceinline__ T of(double x) { return x; }
  static __device__ __forceinline__ double dbl(T a) { return a; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T add(T a, double v) { return a + v; }
  // |a - target| (a test against a threshold)
  static __device__ __forceinline__ double dev(T a, double target) { return fabs(a - target); }
  // a - b c
  static __device__ __forceinline__ T fnms(T a, T b, T c) { return fma(-b, c, a); }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
};

// FP64 value of a normal float by integer operations (exponent rebias and
// mantissa shift); zero for zero and float subnormals
__device__ __forceinline__ double dbl_of_float(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

struct CholDF {
  using T = float2;  // value x + y, |y| <= ulp(x) / 2
  // unit roundoff of the double-float Gram (gemm_df_kernel) and factor
  static constexpr double u = 1.4210854715202004e-14;  // 2^-46
  static __device__ __forceinline__ T of(double v) { return df_split(v); }
  // one FP64 addition (the conversions are integer operations)
  static __device__ __forceinline__ double dbl(T a) { return dbl_of_float(a.x) + dbl_of_float(a.y); }
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ T two_sum(float s, float t) {
    const float h = s + t;
    const float bp = h - s;
    return make_float2(h, (s - (h - bp)) + (t - bp));
  }
  static __device__ __forceinline__ T add(T a, double v) {
    const float2 b = df_split(v);
    const float s = a.x + b.x;
    const float bp = s - a.x;
    const float t = ((a.x - (s - bp)) + (b.x - bp)) + (a.y + b.y);
    return two_sum(s, t);
  }
  static __device__ __forceinline__ double dev(T a, double target) {
    return (double)fabsf((a.x - (float)target) + a.y);
  }
  static __device__ __forceinline__ T fnms(T a, T b, T c) {
    const float p = b.x * c.x;
    float e = fmaf(b.x, c.x, -p);  // b.x c.x = p + e exactly
    e = fmaf(b.x, c.y, e);
    e = fmaf(b.y, c.x, e);
    const float s = a.x - p;       // a.x - p = s + t exactly
    const float bp = s - a.x;
    float t = (a.x - (s - bp)) + (-p - bp);
    t += a.y - e;
    return two_sum(s, t);
  }
  static __device__ __forceinline__ T mul(T a, T b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return two_sum(p, e);
  }
};

template <class A>
__global__ void __launch_bounds__(CHOL_T, 1) chol_inv_smem_kernel(const CholJob* __restrict__ jobs, double* __restrict__ ws,
                                                               int* __restrict__ fail) {
  using T = typename A::T;
  extern __shared__ __align__(16) unsigned char chol_raw[];
  const CholJob J = jobs[blockIdx.x];
  const int n = J.n;
  // the packed triangle: shared memory, or the job's workspace scratch (L2
  // resident) for the sectors too large for it
  T* sm = n <= CHOL_SMEM_MAXN ? reinterpret_cast<T*>(chol_raw) : reinterpret_cast<T*>(ws + J.pk);
  if (J.shift == 3) {
    if (threadIdx.x == 0) fail[J.sec] = 1;
    return;
  }
  if (fail[J.sec]) return;
  double* G = ws + J.g;
  double* R = ws + J.r;
  double* Ri = ws + J.ri;
  const long long nn = (long long)n * n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  __shared__ double red[CHOL_T / 32];
  __shared__ T piv_t, ipiv_t;  // the current pivot and its reciprocal
  __shared__ int bad;
  // G = sum of the partial Gram matrices, upper triangle into shared memory
  for (int i = warp; i < n; i += nw)
    for (int j = i + lane; j < n; j += 32) {
      const long long e = (long long)i * n + j;
      T acc = A::of(G[e]);
      for (int s = 1; s < J.parts; ++s) acc = A::add(acc, G[s * nn + e]);
      sm[pk(i, j, n)] = acc;
    }
  __syncthreads();
  if (J.shift == 2) {
    // last pass: G = I + E; first-order factor when n max|E| <= 1e-8, else a
    // full factorisation; far from I (> 1e-3): Householder fallback
    double mx = 0.0;
    for (int i = warp; i < n; i += nw)
      for (int j = i + lane; j < n; j += 32) {
        const double dev = A::dev(sm[pk(i, j, n)], i == j ? 1.0 : 0.0);
        mx = (dev <= mx) ? mx : (dev == dev ? dev : 1e300);
      }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    double all = 0.0;
    for (int q = 0; q < nw; ++q) all = fmax(all, red[q]);
    if (!(all <= 1e-3)) {
      if (tid == 0) fail[J.sec] = 1;
      return;
    }
    if ((double)n * all <= 1e-8) {
      for (int i = warp; i < n; i += nw)
        for (int j = lane; j < n; j += 32) {
          const long long e = (long long)i * n + j;
          if (j < i) {
            R[e] = 0.0;
            Ri[e] = 0.0;
          } else if (j == i) {
            const double h = 0.5 * (A::dbl(sm[pk(i, i, n)]) - 1.0);
            R[e] = 1.0 + h;
            Ri[e] = 1.0 - h;
          } else {
            const double g = A::dbl(sm[pk(i, j, n)]);
            R[e] = g;
            Ri[e] = -g;
          }
        }
      return;
    }
  }
  if (tid == 0) {
    bad = 0;
    if (J.shift == 1) {
      // shift s = 11 (m n + n (n + 1)) u ||X||^2 with ||X||^2 <= tr(G), u the
      // unit roundoff of the arithmetic that formed G and factorises it
      double tr = 0.0;
      for (int i = 0; i < n; ++i) tr += A::dbl(sm[pk(i, i, n)]);
      const double sft = 11.0 * ((double)J.m * n + (double)n * (n + 1)) * A::u * tr;
      for (int i = 0; i < n; ++i) sm[pk(i, i, n)] = A::of(A::dbl(sm[pk(i, i, n)]) + sft);
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double d = A::dbl(sm[pk(k, k, n)]);
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        fail[J.sec] = 1;
      }
      const double p = bad ? 1.0 : sqrt(d);
      piv_t = A::of(p);
      ipiv_t = A::of(1.0 / p);
    }
    __syncthreads();
    if (bad) return;
    for (int j = k + tid; j < n; j += blockDim.x) sm[pk(k, j, n)] = j == k ? piv_t : A::mul(sm[pk(k, j, n)], ipiv_t);
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += nw) {
      const T rki = sm[pk(k, i, n)];
      for (int j = i + lane; j < n; j += 32) sm[pk(i, j, n)] = A::fnms(sm[pk(i, j, n)], rki, sm[pk(k, j, n)]);
    }
    __syncthreads();
  }
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) R[(long long)i * n + j] = (j >= i) ? A::dbl(sm[pk(i, j, n)]) : 0.0;
  // in-place inverse, rows from the bottom
  for (int k = n - 1; k >= 0; --k) {
    __syncthreads();
    if (tid == 0) ipiv_t = A::of(1.0 / A::dbl(sm[pk(k, k, n)]));
    __syncthreads();
    for (int c = k + tid; c < n; c += blockDim.x) sm[pk(k, c, n)] = c == k ? ipiv_t : A::mul(sm[pk(k, c, n)], ipiv_t);
    __syncthreads();
    for (int i = warp; i < k; i += nw) {
      const T rik = sm[pk(i, k, n)];
      __syncwarp();
      for (int c = k + lane; c < n; c += 32)
        sm[pk(i, c, n)] = A::fnms(c == k ? A::zero() : sm[pk(i, c, n)], rik, sm[pk(k, c, n)]);
    }
  }
  __syncthreads();
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) Ri[(long long)i * n + j] = (j >= i) ? A::dbl(sm[pk(i, j, n)]) : 0.0;
}

__global__ void dot_finalize(const double* partial, int nblk, double* out) {
  __shared__ double s;
  finalize_sums(partial, nblk, 1, &s);
  __syncwarp();
  if (threadIdx.x == 0) *out = s;
}

__global__ void __launch_bounds__(VT) dot_kernel(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                                 double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
    acc = fma(x[i], y[i], acc);
  __shared__ double red[VT / 32];
  double s = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < VT / 32; ++q) t += red[q];
    partial[blockIdx.x * 17] = t;
  }
}

// Local observables at one site: partial[b*2 + {0,1}] = sum over block b of
// A[a, pair, c] T[a, pair, c] w{n,d}(pair)  (T = EL A, right environment = 1).
__global__ void __launch_bounds__(256) local_obs_kernel(const ObsItem* __restrict__ items, const double* __restrict__ A,
                                                        const double* __restrict__ T, double* __restrict__ partial) {
  const ObsItem it = items[blockIdx.x];
  double sn = 0.0, sd = 0.0;
  const long long total = (long long)it.dl * it.m * it.dr;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int pr = (int)((e / it.dr) % it.m);
    const double v = A[it.off + e] * T[it.off + e];
    sn = fma(v, it.wn[pr], sn);
    sd = fma(v, it.wd[pr], sd);
  }
  __shared__ double red[2][8];
  sn = warp_sum(sn);
  sd = warp_sum(sd);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sn; red[1][threadIdx.x >> 5] = sd; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int q = 0; q < 8; ++q) { a += red[0][q]; b += red[1][q]; }
    partial[blockIdx.x * 2] = a;
    partial[blockIdx.x * 2 + 1] = b;
  }
}

__global__ void local_obs_finalize(const double* __restrict__ partial, int n, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0, b = 0;
  for (int i = 0; i < n; ++i) { a += partial[2 * i]; b += partial[2 * i + 1]; }
  out[0] += a;
  out[1] += b;
}

// rows of a column-major m x k matrix (ld) scaled by s[row]  /  columns scaled by s[col]
__global__ void scale_rc_kernel(double* __restrict__ a, long long ld, int rows, int cols, const double* __restrict__ s,
                                int by_col) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e % rows), c = (int)(e / rows);
    a[r + c * ld] *= by_col ? s[c] : s[r];
  }
}

inline int grid_for(long long n) {
  long long g = (n + VT - 1) / VT;
  if (g > NBLK) g = NBLK;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
int lanczos_nblk() { return NBLK; }

cudaError_t launch_gemm_f64(const DevGemm& g, const Bases& b, cudaStream_t s) {
  if (g.ntiles64 == 0) return cudaSuccess;
  gemm_f64_kernel<<<g.ntiles64, 256, 0, s>>>(g.groups, g.segs, g.tiles64, b);
  return cudaGetLastError();
}

cudaError_t launch_gemm_df(const DevGemm& g, const Bases& b, cudaStream_t s) {
  if (g.ntiles64 == 0) return cudaSuccess;
  gemm_df_kernel<<<g.ntiles64, 256, 0, s>>>(g.groups, g.segs, g.tiles64, b);
  return cudaGetLastError();
}

cudaError_t launch_gemm_bf16(const DevGemm& g, const Bases& b, int nsplit, cudaStream_t s) {
  if (g.ntiles64 == 0) return cudaSuccess;
  if (nsplit == 2) gemm_bf16_split_kernel<2><<<g.ntiles64, 128, 0, s>>>(g.groups, g.segs, g.tiles64, b);
  else if (nsplit == 3) gemm_bf16_split_kernel<3><<<g.ntiles64, 128, 0, s>>>(g.groups, g.segs, g.tiles64, b);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_gather(const DevGather& g, const Bases& b, int in_type, int out_type, cudaStream_t s) {
  if (g.nitems == 0) return cudaSuccess;
  if (in_type == 0 && out_type == 0) gather_kernel<0, 0><<<g.nitems, 256, 0, s>>>(g.items, g.contribs, b);
  else if (in_type == 1 && out_type == 2) gather_kernel<1, 2><<<g.nitems, 256, 0, s>>>(g.items, g.contribs, b);
  else if (in_type == 1 && out_type == 3) gather_kernel<1, 3><<<g.nitems, 256, 0, s>>>(g.items, g.contribs, b);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_copy(const DevCopy& c, const Bases& b, cudaStream_t s) {
  if (c.nitems == 0) return cudaSuccess;
  tile_copy_kernel<0><<<copy_grid(c), 256, 0, s>>>(c.items, b);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16(const double* x, int64_t n, int nsplit, void* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  split_bf16_kernel<<<grid_for(n) * 2, VT, 0, s>>>(x, n, nsplit, reinterpret_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) { return cudaMemsetAsync(p, 0, bytes, s); }

cudaError_t launch_split_copy(const DevCopy& c, const Bases& b, int nsplit, cudaStream_t s) {
  if (c.nitems == 0) return cudaSuccess;
  if (nsplit == 2) tile_copy_kernel<2><<<copy_grid(c), 256, 0, s>>>(c.items, b);
  else if (nsplit == 3) tile_copy_kernel<3><<<copy_grid(c), 256, 0, s>>>(c.items, b);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t k_norm_init(const double* v, int64_t n, double* partial, KrylovState* ks, double* q0, cudaStream_t s) {
  int g = grid_for(n);
  sumsq_kernel<<<g, VT, 0, s>>>(v, n, partial);
  norm_init_finalize<<<1, 32, 0, s>>>(partial, g, ks);
  scale_kernel<<<g, VT, 0, s>>>(v, n, &ks->nb, nullptr, q0);
  return cudaGetLastError();
}

cudaError_t k_dots_alpha(const double* Q, int64_t ldq, int k, const double* w, int64_t n, double* partial,
                         KrylovState* ks, cudaStream_t s) {
  int g = grid_for(n);
  multidot_kernel<1><<<g, VT, 0, s>>>(Q, ldq, k, 1, w, n, partial);
  alpha_finalize<<<1, 32, 0, s>>>(partial, g, k, ks);
  return cudaGetLastError();
}

cudaError_t k_three_term(const double* Q, int64_t ldq, int k, double* w, int64_t n, KrylovState* ks, cudaStream_t s) {
  three_term_kernel<<<grid_for(n), VT, 0, s>>>(Q, ldq, k, w, n, ks);
  return cudaGetLastError();
}

cudaError_t k_cgs_pass(const double* Q, int64_t ldq, int k, double* w, int64_t n, double* partial, KrylovState* ks,
                       int last, double tol, int K, double* qnext, cudaStream_t s) {
  int g = grid_for(n);
  int nv = k + 1;
  if (nv <= 4) multidot_kernel<4><<<g, VT, 0, s>>>(Q, ldq, 0, nv, w, n, partial);
  else if (nv <= 8) multidot_kernel<8><<<g, VT, 0, s>>>(Q, ldq, 0, nv, w, n, partial);
  else multidot_kernel<17><<<g, VT, 0, s>>>(Q, ldq, 0, nv, w, n, partial);
  h_finalize<<<1, 32, 0, s>>>(partial, g, nv, ks);
  axpy_multi_kernel<<<g, VT, 0, s>>>(Q, ldq, nv, ks, w, n, last ? partial : nullptr);
  if (last) {
    beta_finalize<<<1, 32, 0, s>>>(partial, g, k, K, tol, ks);
    if (k < K - 1) scale_kernel<<<g, VT, 0, s>>>(w, n, &ks->beta[k], &ks->broken, qnext);
  }
  return cudaGetLastError();
}

cudaError_t k_krylov_exp(KrylovState* ks, double t, int K, cudaStream_t s) {
  krylov_exp_kernel<<<1, 256, 0, s>>>(ks, t, K);
  return cudaGetLastError();
}

cudaError_t k_combine(const double* Q, int64_t ldq, const KrylovState* ks, double* y, int64_t n, double* partial,
                      KrylovState* ksw, cudaStream_t s) {
  (void)ksw;
  combine_kernel<<<grid_for(n), VT, 0, s>>>(Q, ldq, ks, y, n, partial);
  return cudaGetLastError();
}

cudaError_t k_dot_plain(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t s) {
  int g = grid_for(n);
  dot_kernel<<<g, VT, 0, s>>>(x, y, n, partial);
  dot_finalize<<<1, 32, 0, s>>>(partial, g, out);
  return cudaGetLastError();
}

cudaError_t launch_local_obs(const ObsItem* items, int nitems, const double* A, const double* T, double* partial,
                             double* out, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  local_obs_kernel<<<nitems, 256, 0, s>>>(items, A, T, partial);
  local_obs_finalize<<<1, 32, 0, s>>>(partial, nitems, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_rc(double* a, long long ld, int rows, int cols, const double* sv, int by_col, cudaStream_t s) {
  long long total = (long long)rows * cols;
  if (total == 0) return cudaSuccess;
  scale_rc_kernel<<<grid_for(total), VT, 0, s>>>(a, ld, rows, cols, sv, by_col);
  return cudaGetLastError();
}

cudaError_t launch_qr(const QrJob* jobs, int njobs, double* ws, cudaStream_t s) {
  if (njobs == 0) return cudaSuccess;
  qr_kernel<<<njobs, QRT, 0, s>>>(jobs, ws, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_qr_job(const QrJob& job, double* ws, cudaStream_t s) {
  qr_byval_kernel<<<1, QRT, 0, s>>>(job, ws);
  return cudaGetLastError();
}

cudaError_t launch_qr_masked(const QrJob* jobs, int njobs, double* ws, const int* only, int* nrun, cudaStream_t s) {
  if (njobs == 0) return cudaSuccess;
  qr_kernel<<<njobs, QRT, 0, s>>>(jobs, ws, only, nrun);
  return cudaGetLastError();
}

cudaError_t launch_chol_inv(const CholJob* jobs, int njobs, double* ws, int* fail, cudaStream_t s, int maxn, bool df) {
  if (njobs == 0) return cudaSuccess;
  const int ns = maxn < CHOL_SMEM_MAXN ? maxn : CHOL_SMEM_MAXN;
  const size_t smem = ((size_t)ns * (ns + 1) / 2) * 8;
  const int smax = (int)(((size_t)CHOL_SMEM_MAXN * (CHOL_SMEM_MAXN + 1) / 2) * 8);
  // once per process (thread-safe static initialisation): the largest size
  static const cudaError_t e1 =
      cudaFuncSetAttribute(chol_inv_smem_kernel<CholF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  static const cudaError_t e2 =
      cudaFuncSetAttribute(chol_inv_smem_kernel<CholDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e1 != cudaSuccess) return e1;
  if (e2 != cudaSuccess) return e2;
  if (df) chol_inv_smem_kernel<CholDF><<<njobs, CHOL_T, smem, s>>>(jobs, ws, fail);
  else chol_inv_smem_kernel<CholF64><<<njobs, CHOL_T, smem, s>>>(jobs, ws, fail);
  return cudaGetLastError();
}

__global__ void plain_nrm_finalize(const double* partial, int nblk, KrylovState* ks, RhoScalars* rs) {
  __shared__ double s;
  finalize_sums(partial, nblk, 1, &s);
  __syncwarp();
  if (threadIdx.x != 0) return;
  double nrm = sqrt(s);
  ks->nrm = nrm;
  if (!isfinite(nrm) || nrm == 0.0) {
    rs->bad = 1;
    return;
  }
  rs->logscale += log(nrm);
}

cudaError_t k_normalise_inplace(double* v, int64_t n, double* partial, KrylovState* ks, RhoScalars* rs, cudaStream_t s) {
  int g = grid_for(n);
  sumsq_kernel<<<g, VT, 0, s>>>(v, n, partial);
  plain_nrm_finalize<<<1, 32, 0, s>>>(partial, g, ks, rs);
  scale_kernel<<<g, VT, 0, s>>>(v, n, &ks->nrm, nullptr, v);
  return cudaGetLastError();
}

// Normalisation after the Krylov combination: finalize ||y|| then y /= ||y||.
cudaError_t k_finish_normalise(double* y, int64_t n, double* partial, KrylovState* ks, RhoScalars* rs,
                               cudaStream_t s) {
  int g = grid_for(n);
  nrm_finalize<<<1, 32, 0, s>>>(partial, g, ks, rs);
  scale_kernel<<<g, VT, 0, s>>>(y, n, &ks->nrm, nullptr, y);
  return cudaGetLastError();
}

}  // namespace tt
