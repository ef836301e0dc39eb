// Persistent, warp-specialised split-BF16 grouped GEMM on the 5th-generation
// tensor cores (sm_103a): the same arithmetic as gemm_tc_kernel
// (tt_tcgen05.cu: NS bf16 levels per operand, the level products l_A + l_B <
// NS, the leading product in one TMEM accumulator and the smaller ones in a
// second, folded every two 64-wide K chunks into a two-float TwoSum sum), laid
// out for throughput:
//
//  * one CTA per SM walks the 128 x 64 output tiles blockIdx.x, blockIdx.x +
//    gridDim.x, ... so TMEM allocation and barrier set-up happen once;
//  * warp 0 (one lane) streams the A (128 x 64 K) and B (64 x 64 K) level
//    tiles by TMA into a ring of STAGES shared-memory stages, running ahead
//    across fold groups and tiles;
//  * warp 1 (one lane) issues tcgen05.mma (M = 128, N = 64, K = 16) into one
//    of two TMEM accumulator buffers per fold group and commits each stage
//    back to the producer and each buffer to the epilogue;
//  * warps 2-5 fold a finished buffer into the two-float sum (TMEM, hi and lo)
//    while the MMAs of the next fold group run in the other buffer, and write
//    every finished tile's hi + lo (FP32 or FP64, optionally accumulated).
//
// TMEM (512 columns): buffer b at [128 b, 128 b + 128) (leading product,
// smaller products), hi [256, 320), lo [320, 384).  Every wait is bounded by
// wait_ns; a role whose wait runs out raises a shared abort flag that the
// other roles' waits observe, the CTA records the error, drains its own TMA
// copies and MMAs (fixed budget), frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_kernels.h"
#include "tt_tc_ptx.h"

namespace tt {

namespace {

using namespace tcx;

constexpr int PBM = 128, PBN = 64, PBK = 64;
constexpr int PA_BYTES = PBM * PBK * 2;  // 16 KB per level
constexpr int PB_BYTES = PBN * PBK * 2;  // 8 KB per level
constexpr int PFOLD = 2;
constexpr uint32_t PTMEM_COLS = 512;
constexpr int PTHREADS = 192;

template <int NS>
struct PCfg {
  static constexpr int STAGES = NS == 3 ? 3 : 4;
  static constexpr int STAGE_BYTES = NS * (PA_BYTES + PB_BYTES);
  static constexpr int NPROD = NS == 2 ? 3 : 6;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait that also gives up when another role raised the abort flag
__device__ __forceinline__ bool wait_ab(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_f,
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

__device__ __forceinline__ int tile_chunks(const GGroup& g, const GSeg* segs) {
  int t = 0;
  for (int si = g.seg0; si < g.seg1; ++si) t += (segs[si].K + PBK - 1) / PBK;
  return t;
}

template <int NS>
__global__ void __launch_bounds__(PTHREADS, 1) gemm_tcp_kernel(const GGroup* __restrict__ groups,
                                                               const GSeg* __restrict__ segs,
                                                               const GTile* __restrict__ tiles, int ntiles,
                                                               const CUtensorMap* __restrict__ maps, Bases bs,
                                                               int* __restrict__ err, long long wait_ns) {
  using C = PCfg<NS>;
  constexpr int S = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], accf[2], acce[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s, issued_s, consumed_s, last_commit_s, last_accf_s;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  volatile int* abort_f = &abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(PTMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);  // one arrive per epilogue warp
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
    // ---------------- producer: TMA ring ----------------
    if (lane == 0) {
      int it = 0, fenced = -1;
      for (int t = blockIdx.x; t < ntiles && !*abort_f; t += gridDim.x) {
        const GTile tl = tiles[t];
        const GGroup g = groups[tl.g];
        for (int si = g.seg0; si < g.seg1 && !*abort_f; ++si) {
          const int K = segs[si].K;
          const CUtensorMap* ma = maps + 3 * si;
          const CUtensorMap* mb = maps + 3 * si + 2;
          if (fenced != si) {  // tensor maps written by a host copy: acquire before first use
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(ma))
                         : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mb))
                         : "memory");
            fenced = si;
          }
          for (int k0 = 0; k0 < K; k0 += PBK) {
            const int s = it % S;
            if (!wait_ab(&empty_bar[s], ((it / S) & 1) ^ 1, wait_ns, abort_f, err)) break;
            uint8_t* st = smem + s * C::STAGE_BYTES;
            mbar_expect_tx(&full_bar[s], C::STAGE_BYTES);
#pragma unroll
            for (int l = 0; l < NS; ++l) tma_load_3d(st + l * PA_BYTES, ma, k0, tl.m0, l, &full_bar[s]);
#pragma unroll
            for (int l = 0; l < NS; ++l) tma_load_3d(st + NS * PA_BYTES + l * PB_BYTES, mb, k0, tl.n0, l, &full_bar[s]);
            ++it;
            issued_s = it;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PBN >> 3) << 17) | ((uint32_t)(PBM >> 4) << 24);
      int it = 0, fg = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const GTile tl = tiles[t];
        const GGroup g = groups[tl.g];
        const int T = tile_chunks(g, segs);
        for (int b0 = 0; b0 < T && ok; b0 += PFOLD) {
          const int b = fg & 1;
          ok = wait_ab(&acce[b], ((fg >> 1) & 1) ^ 1, wait_ns, abort_f, err);
          if (!ok) break;
          fence_after();
          const uint32_t t_acc = tmem + 128 * b, t_acc2 = t_acc + 64;
          const int b1 = min(T, b0 + PFOLD);
          for (int c = b0; c < b1; ++c) {
            const int s = it % S;
            ok = wait_ab(&full_bar[s], (it / S) & 1, wait_ns, abort_f, err);
            if (!ok) break;
            consumed_s = it + 1;
            fence_after();
            const uint32_t sa = smem_u32(smem + s * C::STAGE_BYTES);
#pragma unroll
            for (int p = 0; p < C::NPROD; ++p) {
              const int la = (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0);
              const int lb = (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0);
              const uint32_t aa = sa + la * PA_BYTES, ba = sa + NS * PA_BYTES + lb * PB_BYTES;
#pragma unroll
              for (int kk = 0; kk < PBK / 16; ++kk) {
                const uint32_t acc = (c > b0 || p > 1 || kk > 0) ? 1u : 0u;
                umma_f16(p == 0 ? t_acc : t_acc2, make_desc(aa + kk * 32), make_desc(ba + kk * 32), idesc, acc);
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
    // ---------------- epilogue: warps 2..5 ----------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const uint32_t t_hi = tmem + 256, t_lo = tmem + 320;
    int fg = 0;
    bool ok = true;
    float v[32], u[32], h[32], w[32];
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const GTile tl = tiles[t];
      const GGroup g = groups[tl.g];
      const int T = tile_chunks(g, segs);
      int folds = 0;
      for (int b0 = 0; b0 < T; b0 += PFOLD) {
        const int b = fg & 1;
        ok = __all_sync(0xffffffffu, wait_ab(&accf[b], (fg >> 1) & 1, wait_ns, abort_f, err));
        if (!ok) break;  // warp-uniform: the TMEM loads below are warp-collective
        fence_after();
        const uint32_t t_acc = tmem + 128 * b, t_acc2 = t_acc + 64;
#pragma unroll 1
        for (int cb = 0; cb < PBN; cb += 32) {
          tmem_ld32(t_acc + lane_off + cb, v);
          tmem_ld32(t_acc2 + lane_off + cb, u);
          if (folds == 0) {
            tmem_st32(t_hi + lane_off + cb, v);
            tmem_st32(t_lo + lane_off + cb, u);
          } else {
            tmem_ld32(t_hi + lane_off + cb, h);
            tmem_ld32(t_lo + lane_off + cb, w);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const float s = h[i] + v[i];
              const float bp = s - h[i];
              const float ap = s - bp;
              w[i] += ((h[i] - ap) + (v[i] - bp)) + u[i];
              h[i] = s;
            }
            tmem_st32(t_hi + lane_off + cb, h);
            tmem_st32(t_lo + lane_off + cb, w);
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
        ++folds;
        ++fg;
      }
      if (!ok) break;
      // the finished tile: row = TMEM lane, 32 consecutive columns per load
      const bool accum = g.flags & 1, out_f32 = g.flags & 2;
      const int row = tl.m0 + 32 * q + lane;
#pragma unroll 1
      for (int cb = 0; cb < PBN; cb += 32) {
        if (folds > 0) {
          tmem_ld32(t_hi + lane_off + cb, h);
          tmem_ld32(t_lo + lane_off + cb, w);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) { h[i] = 0.f; w[i] = 0.f; }
        }
        if (row < g.M) {
          const long long o = (long long)row * g.ldc + tl.n0 + cb;
          const int ncol = min(32, g.N - tl.n0 - cb);
          if (out_f32) {
            float* Cp = reinterpret_cast<float*>(sel_base(bs, slot_of(g.C))) + off_of(g.C) + o;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < ncol) Cp[i] = accum ? Cp[i] + (h[i] + w[i]) : (h[i] + w[i]);
          } else {
            double* Cp = reinterpret_cast<double*>(sel_base(bs, slot_of(g.C))) + off_of(g.C) + o;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < ncol) {
                const double val = (double)h[i] + (double)w[i];
                Cp[i] = accum ? Cp[i] + val : val;
              }
          }
        }
      }
      fence_before();  // the next tile's first fold overwrites hi / lo after these loads
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (abort_s && tid == 0) {
    // drain what this CTA still has in flight: TMA chunks issued but not
    // consumed (each the newest phase of its stage barrier), the MMAs up to
    // the last stage commit, the last accumulator commit
    for (int c = consumed_s; c < issued_s; ++c) mbar_wait(&full_bar[c % S], (c / S) & 1, DRAIN_NS);
    if (last_commit_s >= 0) mbar_wait(&empty_bar[last_commit_s % S], (last_commit_s / S) & 1, DRAIN_NS);
    if (last_accf_s >= 0) mbar_wait(&accf[last_accf_s & 1], (last_accf_s >> 1) & 1, DRAIN_NS);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PTMEM_COLS) : "memory");
}

int sm_count() {
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

size_t tcp_smem_bytes(int nsplit) {
  return nsplit == 3 ? (size_t)PCfg<3>::STAGES * PCfg<3>::STAGE_BYTES + 1024
                     : (size_t)PCfg<2>::STAGES * PCfg<2>::STAGE_BYTES + 1024;
}

cudaError_t launch_gemm_tcp(const GGroup* groups, const GSeg* segs, const GTile* tiles, int ntiles, const void* maps,
                            const Bases& b, int nsplit, int* err, long long wait_ns, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const size_t smem = tcp_smem_bytes(nsplit);
  const int grid = ntiles < sm_count() ? ntiles : sm_count();
  if (nsplit == 2) {
    static const cudaError_t e =
        cudaFuncSetAttribute(gemm_tcp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tcp_kernel<2><<<grid, PTHREADS, smem, s>>>(groups, segs, tiles, ntiles, (const CUtensorMap*)maps, b, err,
                                                    wait_ns);
  } else if (nsplit == 3) {
    static const cudaError_t e =
        cudaFuncSetAttribute(gemm_tcp_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tcp_kernel<3><<<grid, PTHREADS, smem, s>>>(groups, segs, tiles, ntiles, (const CUtensorMap*)maps, b, err,
                                                    wait_ns);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tt
