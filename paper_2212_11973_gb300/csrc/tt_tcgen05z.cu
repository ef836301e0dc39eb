// Exact-accumulation split GEMM on the 5th-generation tensor cores (sm_103a).
//
// Operands are fixed-point BF16 digits (Ozaki scheme with one exponent per
// operand row and GEMM segment; see tt_ozaki.cu for the arithmetic): a row
// with largest biased exponent e holds v ~ 2^(e - 1054) F, F = a0 2^24 +
// a1 2^16 + a2 2^8 + a3, |a_s| <= 256, the four digit levels stored like
// split-BF16 levels (K-major, rows padded to 8, level l at l * lo[slot]) and
// the int16 exponents per row next to them.  Every tensor-core product of
// two digits is exact and, for a segment of K <= 256, every sum of the digit
// pairs with s + t = d is an integer below 2^24, exact in the FP32 TMEM
// accumulator.  The kernel keeps the ten pairs with s + t <= 3 in four TMEM
// accumulators D_0..D_3 and, once per segment, the epilogue warps add
// sum_d D_d 2^(eA + eB - 2060 - 8 d) to a two-float (hi, lo) sum in
// registers (TwoSum for d = 0, 1): ~2^-32 of the rows' bounds, with no
// rounding that grows with K.
//
// Structure as gemm_tcp_kernel (tt_tcgen05p.cu): persistent, one CTA per SM,
// 128 x 64 output tiles; warp 0 streams the digit tiles (A 4 x 16 KB, B 4 x
// 8 KB per 64-wide K chunk) into two shared-memory stages, warp 1 issues the
// MMAs of a segment into one of two TMEM buffers (4 accumulators x 64
// columns each), warps 2-9 fold a finished buffer while the next segment's
// MMAs run in the other (two warps per TMEM lane quarter, 32 columns each,
// so that every SM sub-partition has two folding warps), and write each
// finished tile as FP64 or as a two-float pair (flags bit 1) through a
// per-warp, XOR-swizzled shared-memory staging buffer (coalesced 128-byte
// row stores, no cross-warp barrier).  Waits are bounded as in the other
// tcgen05 kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_kernels.h"
#include "tt_tc_ptx.h"

namespace tt {

namespace {

using namespace tcx;

constexpr int ZBM = 128, ZBN = 64, ZBK = 64, ZDIG = 4, ZPAIRS = 10;
constexpr int ZA_BYTES = ZBM * ZBK * 2;  // 16 KB per digit level
constexpr int ZB_BYTES = ZBN * ZBK * 2;  // 8 KB per digit level
constexpr int ZSTAGE_BYTES = ZDIG * (ZA_BYTES + ZB_BYTES);
constexpr int ZSTAGES = 2;
constexpr uint32_t ZTMEM_COLS = 512;
constexpr int ZEPI = 8;  // epilogue warps
constexpr int ZTHREADS = 64 + 32 * ZEPI;
constexpr int ZMAXK = 256;  // longest segment whose digit sums stay exact
// epilogue staging, after the two TMA stages: per epilogue warp 32 rows x 16
// columns of 8-byte outputs, column c of row r at word r * 16 + (c ^ (r & 15))
constexpr int ZSTG_WARP = 32 * 16;
constexpr int ZSTG_BYTES = ZEPI * ZSTG_WARP * 8;

__device__ __forceinline__ void mbar_arrive_z(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool wait_z(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_f,
                                       int* err) {
  if (mbar_test_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_f) return false;
    if (budget <= 0 || (long long)(globaltimer() - t0) > budget) {
      *abort_f = 1;
      if (err) atomicExch(err, 1);
      return false;
    }
  }
}

// 16 TMEM columns of this warp's lane quarter, not yet waited for: the caller
// issues tmem_wait_ld16() with one set of registers and tmem_dep16() with
// every other set before reading them (the registers pass through those asm
// statements, so no use is scheduled before the wait)
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_dep16(uint32_t* r) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

__device__ __forceinline__ void two_sum_z(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float ap = s - bp;
  lo += (hi - ap) + (x - bp);
  hi = s;
}

// digit pair p -> (s, t): d = s + t ascending, the first pair of each d at
// p = 0, 1, 3, 6
__device__ __forceinline__ void pair_of(int p, int& s, int& t) {
  const int d = (p >= 1) + (p >= 3) + (p >= 6);
  s = p - d * (d + 1) / 2;
  t = d - s;
}

// PAIR: every group of the launch writes two-float pairs (flags bit 1), else
// FP64 (accumulating with flags bit 0); one kernel per output form keeps the
// FP64 conversions out of the pair kernel entirely
template <bool PAIR>
__global__ void __launch_bounds__(ZTHREADS, 1) gemm_tcz_kernel(const GGroup* __restrict__ groups,
                                                               const GSeg* __restrict__ segs,
                                                               const GTile* __restrict__ tiles, int ntiles,
                                                               const CUtensorMap* __restrict__ maps, Bases bs,
                                                               int* __restrict__ err, long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[ZSTAGES], empty_bar[ZSTAGES], accf[2], acce[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s, issued_s, consumed_s, last_commit_s, last_accf_s;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  volatile int* abort_f = &abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(ZTMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < ZSTAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], ZEPI);
    }
    abort_s = 0;
    issued_s = 0;
    consumed_s = 0;
    last_commit_s = -1;
    last_accf_s = -1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int it = 0, fenced = -1;
      for (int t = blockIdx.x; t < ntiles && !*abort_f; t += gridDim.x) {
        const GTile tl = tiles[t];
        const GGroup g = groups[tl.g];
        for (int si = g.seg0; si < g.seg1 && !*abort_f; ++si) {
          const int K = segs[si].K;
          const CUtensorMap* ma = maps + 3 * si;
          const CUtensorMap* mb = maps + 3 * si + 2;
          if (fenced != si) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(ma))
                         : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mb))
                         : "memory");
            fenced = si;
          }
          for (int k0 = 0; k0 < K; k0 += ZBK) {
            const int s = it % ZSTAGES;
            if (!wait_z(&empty_bar[s], ((it / ZSTAGES) & 1) ^ 1, wait_ns, abort_f, err)) break;
            uint8_t* st = smem + s * ZSTAGE_BYTES;
            mbar_expect_tx(&full_bar[s], ZSTAGE_BYTES);
#pragma unroll
            for (int l = 0; l < ZDIG; ++l) tma_load_3d(st + l * ZA_BYTES, ma, k0, tl.m0, l, &full_bar[s]);
#pragma unroll
            for (int l = 0; l < ZDIG; ++l)
              tma_load_3d(st + ZDIG * ZA_BYTES + l * ZB_BYTES, mb, k0, tl.n0, l, &full_bar[s]);
            ++it;
            issued_s = it;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one fold unit per segment ----------------
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ZBN >> 3) << 17) | ((uint32_t)(ZBM >> 4) << 24);
      int it = 0, fg = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const GTile tl = tiles[t];
        const GGroup g = groups[tl.g];
        for (int si = g.seg0; si < g.seg1 && ok; ++si) {
          const int nch = (segs[si].K + ZBK - 1) / ZBK;
          const int b = fg & 1;
          ok = wait_z(&acce[b], ((fg >> 1) & 1) ^ 1, wait_ns, abort_f, err);
          if (!ok) break;
          fence_after();
          const uint32_t tb = tmem + 256 * b;
          for (int c = 0; c < nch; ++c) {
            const int s = it % ZSTAGES;
            ok = wait_z(&full_bar[s], (it / ZSTAGES) & 1, wait_ns, abort_f, err);
            if (!ok) break;
            consumed_s = it + 1;
            fence_after();
            const uint32_t sa = smem_u32(smem + s * ZSTAGE_BYTES);
#pragma unroll
            for (int p = 0; p < ZPAIRS; ++p) {
              int ls, lt;
              pair_of(p, ls, lt);
              const bool first = (p == 0 || p == 1 || p == 3 || p == 6);
              const uint32_t aa = sa + ls * ZA_BYTES, ba = sa + ZDIG * ZA_BYTES + lt * ZB_BYTES;
              const uint32_t dst = tb + 64 * (ls + lt);
#pragma unroll
              for (int kk = 0; kk < ZBK / 16; ++kk) {
                const uint32_t acc = (c > 0 || kk > 0 || !first) ? 1u : 0u;
                umma_f16(dst, make_desc(aa + kk * 32), make_desc(ba + kk * 32), idesc, acc);
              }
            }
            umma_commit(&empty_bar[s]);
            last_commit_s = it;
            ++it;
          }
          if (!ok) break;
          umma_commit(&accf[b]);
          last_accf_s = fg;
          ++fg;
        }
      }
    }
  } else {
    // ---------------- epilogue: fold per segment, write per tile ----------------
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (the quarter its SM sub-
    // partition may access) and folds columns 32 h .. 32 h + 31 of them
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    uint64_t* stg = reinterpret_cast<uint64_t*>(smem + ZSTAGES * ZSTAGE_BYTES) + (warp - 2) * ZSTG_WARP;
    int fg = 0;
    bool ok = true;
    float hi[32], lo[32];
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const GTile tl = tiles[t];
      const GGroup g = groups[tl.g];
      const int row = tl.m0 + 32 * q + lane;
      const int col_l = tl.n0 + 32 * h + lane;  // the column whose exponent this lane loads
#pragma unroll
      for (int i = 0; i < 32; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
      for (int si = g.seg0; si < g.seg1; ++si) {
        const GSeg sg = segs[si];
        const int b = fg & 1;
        ok = __all_sync(0xffffffffu, wait_z(&accf[b], (fg >> 1) & 1, wait_ns, abort_f, err));
        if (!ok) break;
        fence_after();
        // the scale of D_0 at (row, column) is 2^(eA + eB - 2060): as a biased
        // FP32 exponent xa + eB, clamped to [0, 254] (0: below the normal
        // range, dropped like the digits below it)
        const short* eAp = reinterpret_cast<const short*>(sel_base(bs, slot_of(sg.eA))) + off_of(sg.eA);
        const short* eBp = reinterpret_cast<const short*>(sel_base(bs, slot_of(sg.eB))) + off_of(sg.eB);
        const int ea = row < g.M ? (int)eAp[(long long)row * sg.eas] : 0;
        const int eb = col_l < g.N ? (int)eBp[(long long)col_l * sg.ebs] : 0;
        const int xa = ea - 2060 + 127;
        const uint32_t tb = tmem + 256 * b + lane_off + 32 * h;
        const bool first = si == g.seg0;
#pragma unroll
        for (int cb = 0; cb < 32; cb += 16) {
          uint32_t dv[ZDIG][16];
#pragma unroll
          for (int d = 0; d < ZDIG; ++d) tmem_ld16_nw(tb + 64 * d + cb, dv[d]);
          tmem_wait_ld16(dv[0]);
#pragma unroll
          for (int d = 1; d < ZDIG; ++d) tmem_dep16(dv[d]);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int xe = xa + __shfl_sync(0xffffffffu, eb, cb + i);
            const float sc = __int_as_float(min(max(xe, 0), 254) << 23);
            // D_0 + D_1 2^-8 as an exact pair (sv, ev) (TwoSum), D_2 2^-16 and
            // D_3 2^-24 into ev, then the pair scaled by the power of two sc
            const float d0 = __uint_as_float(dv[0][i]);
            const float p1 = __uint_as_float(dv[1][i]) * 0.00390625f;
            const float sv = d0 + p1;
            const float bp = sv - d0;
            float ev = (d0 - (sv - bp)) + (p1 - bp);
            ev = fmaf(__uint_as_float(dv[2][i]), 1.52587890625e-05f, ev);
            ev = fmaf(__uint_as_float(dv[3][i]), 5.9604644775390625e-08f, ev);
            const float s2 = sv * sc, e2 = ev * sc;
            if (first) {
              hi[cb + i] = s2;
              lo[cb + i] = e2;
            } else {
              two_sum_z(hi[cb + i], lo[cb + i], s2);
              lo[cb + i] += e2;
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_z(&acce[b]);
        ++fg;
      }
      if (!ok) break;
      // the finished 32 x 32 block, 16 columns at a time through this warp's
      // staging buffer: one row per lane on the way in, 16 lanes per row (128
      // contiguous bytes) on the way out
      const bool accum = g.flags & 1;
      const int c_l = lane & 15;
      uint64_t* const Cb = reinterpret_cast<uint64_t*>(sel_base(bs, slot_of(g.C))) + off_of(g.C);
#pragma unroll
      for (int cb = 0; cb < 32; cb += 16) {
        if (PAIR) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            stg[lane * 16 + (i ^ (lane & 15))] =
                ((uint64_t)__float_as_uint(lo[cb + i]) << 32) | (uint64_t)__float_as_uint(hi[cb + i]);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            stg[lane * 16 + (i ^ (lane & 15))] =
                (uint64_t)__double_as_longlong((double)hi[cb + i] + (double)lo[cb + i]);
        }
        __syncwarp();
        const int col = tl.n0 + 32 * h + cb + c_l;
        for (int rr = lane >> 4; rr < 32; rr += 2) {
          const int grow = tl.m0 + 32 * q + rr;
          if (grow < g.M && col < g.N) {
            const long long o = (long long)grow * g.ldc + col;
            const uint64_t bits = stg[rr * 16 + (c_l ^ (rr & 15))];
            if (PAIR || !accum) {
              Cb[o] = bits;
            } else {
              double* Cp = reinterpret_cast<double*>(Cb + o);
              *Cp += __longlong_as_double((long long)bits);
            }
          }
        }
        __syncwarp();
      }
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (abort_s && tid == 0) {
    for (int c = consumed_s; c < issued_s; ++c) mbar_wait(&full_bar[c % ZSTAGES], (c / ZSTAGES) & 1, DRAIN_NS);
    if (last_commit_s >= 0) mbar_wait(&empty_bar[last_commit_s % ZSTAGES], (last_commit_s / ZSTAGES) & 1, DRAIN_NS);
    if (last_accf_s >= 0) mbar_wait(&accf[last_accf_s & 1], (last_accf_s >> 1) & 1, DRAIN_NS);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ZTMEM_COLS) : "memory");
}

int sm_count_z() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 148;
    }
    return v;
  }();
  return n;
}

}  // namespace

int tcz_max_k() { return ZMAXK; }
size_t tcz_smem_bytes() { return (size_t)ZSTAGES * ZSTAGE_BYTES + ZSTG_BYTES + 1024; }

cudaError_t launch_gemm_tcz(const GGroup* groups, const GSeg* segs, const GTile* tiles, int ntiles, const void* maps,
                            const Bases& b, int* err, long long wait_ns, bool pair, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const size_t smem = tcz_smem_bytes();
  static const cudaError_t e1 =
      cudaFuncSetAttribute(gemm_tcz_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  static const cudaError_t e2 =
      cudaFuncSetAttribute(gemm_tcz_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e1 != cudaSuccess) return e1;
  if (e2 != cudaSuccess) return e2;
  const int grid = ntiles < sm_count_z() ? ntiles : sm_count_z();
  if (pair)
    gemm_tcz_kernel<true><<<grid, ZTHREADS, smem, s>>>(groups, segs, tiles, ntiles, (const CUtensorMap*)maps, b, err,
                                                       wait_ns);
  else
    gemm_tcz_kernel<false><<<grid, ZTHREADS, smem, s>>>(groups, segs, tiles, ntiles, (const CUtensorMap*)maps, b, err,
                                                        wait_ns);
  return cudaGetLastError();
}

}  // namespace tt
