// Split-BF16 grouped GEMM on the 5th-generation tensor cores (sm_103a).
//
// One CTA computes a 128 x 128 output tile of one group: for every segment of
// the group and every 64-wide K chunk, TMA loads the NS bf16 levels of the A
// tile (128 rows x 64 K) and of the B tile (128 rows x 64 K, K-major) into
// 128B-swizzled shared memory, one elected thread issues tcgen05.mma
// (kind::f16, bf16 x bf16 -> f32, M = 128, N = 128, K = 16) for the level
// products l_A + l_B < NS, the leading product into one TMEM accumulator and
// the smaller ones into a second; every FOLD chunks all 128 threads read both
// back (tcgen05.ld) and add them into a two-float (hi, lo) sum kept in TMEM
// (TwoSum, Knuth TAOCP 4.2.2), so the FP32 accumulation error does not grow
// with K.  The epilogue stages hi + lo through shared memory and writes FP32
// or FP64 rows coalesced.  Two shared-memory stages overlap the TMA of chunk c+1 with the
// MMAs of chunk c.  Every mbarrier wait is bounded by a time budget (ns, a
// kernel argument, measured on %globaltimer).  Thread 0 alone waits on the
// copy, MMA and accumulator barriers and broadcasts an abort through shared
// memory, so all threads leave the main loop together.  On abort the CTA
// records an error code, waits (with a fixed drain budget) for the at most two
// TMA chunks still in flight and for its last MMA commit, frees its TMEM and
// returns.
//
// Both operands must be K-major (A stored M x K, B stored N x K, K contiguous)
// with leading dimensions and offsets that are multiples of 8 elements; the
// host checks this before choosing the kernel.  maps holds three tensor maps
// per segment: A (box 64 K x 128 rows), B (64 x 128), B (64 x 64).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_kernels.h"
#include "tt_tc_ptx.h"

namespace tt {

namespace {

using namespace tcx;

constexpr int TBM = 128, TBN = 128, TBK = 64;
constexpr int TILE_BYTES = TBM * TBK * 2;  // 16 KB per level and operand
constexpr int FOLD = 2;                    // chunks per TMEM fold
// TMEM columns: the leading level product hi*hi accumulates in [0,128), the
// five (x6) or two (x3) smaller products in [128,256); the running two-float
// sum of the folds is hi [256,384), lo [384,512).  Keeping the small products
// out of the main accumulator means the FP32 roundings of the tensor-core
// accumulation act on the dominant term only 4 times per 64-long K chunk
// instead of 4 * (number of products) times.
constexpr uint32_t TMEM_COLS = 512;

template <int NS>
__global__ void __launch_bounds__(128, 1) gemm_tc_kernel(const GGroup* __restrict__ groups,
                                                         const GSeg* __restrict__ segs,
                                                         const GTile* __restrict__ tiles,
                                                         const CUtensorMap* __restrict__ maps, Bases bs,
                                                         int* __restrict__ err, long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[2], empty_bar[2], acc_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  constexpr int NPROD = NS == 2 ? 3 : 6;
  constexpr int STAGE_BYTES = 2 * NS * TILE_BYTES;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  const int tid = threadIdx.x, warp = tid >> 5;
  const GTile tl = tiles[blockIdx.x];
  const GGroup g = groups[tl.g];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&full_bar[0], 1);
    mbar_init(&full_bar[1], 1);
    mbar_init(&empty_bar[0], 1);
    mbar_init(&empty_bar[1], 1);
    mbar_init(&acc_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_s;
  const uint32_t t_acc = tmem, t_acc2 = tmem + TBN, t_hi = tmem + 2 * TBN, t_lo = tmem + 3 * TBN;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

  // instruction descriptor: D f32, A/B bf16, both K-major, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);

  // chunk bookkeeping (thread 0 walks the segments)
  int total = 0;
  for (int si = g.seg0; si < g.seg1; ++si) total += (segs[si].K + TBK - 1) / TBK;

  int cur_seg = g.seg0, cur_k = 0, fenced_seg = -1;  // producer cursor
  auto issue_tma = [&](int c) {
    // advance cursor to chunk c (chunks are issued in order)
    while (cur_seg < g.seg1 && cur_k >= segs[cur_seg].K) { ++cur_seg; cur_k = 0; }
    const int s = c & 1;
    uint8_t* st = smem + s * STAGE_BYTES;
    const CUtensorMap* ma = maps + 3 * cur_seg;
    const CUtensorMap* mb = maps + 3 * cur_seg + 1;
    if (fenced_seg != cur_seg) {  // tensor maps written by a host copy: acquire before first use
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(ma)) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mb)) : "memory");
      fenced_seg = cur_seg;
    }
    mbar_expect_tx(&full_bar[s], STAGE_BYTES);
#pragma unroll
    for (int l = 0; l < NS; ++l) tma_load_3d(st + l * TILE_BYTES, ma, cur_k, tl.m0, l, &full_bar[s]);
#pragma unroll
    for (int l = 0; l < NS; ++l) tma_load_3d(st + (NS + l) * TILE_BYTES, mb, cur_k, tl.n0, l, &full_bar[s]);
    cur_k += TBK;
  };

  // Thread 0's bookkeeping for a clean abort: chunks [consumed, issued) may
  // still have TMA copies in flight; last_commit is the last chunk whose MMAs
  // were committed to its empty barrier (they complete in issue order, so that
  // commit covers every earlier MMA); acc_pending marks an accumulator commit
  // whose wait did not succeed.
  int issued = 0, consumed = 0, last_commit = -1;
  bool acc_pending = false;
  int folds = 0;
  bool ok = true;
  float v[32], u[32], h[32], w[32];
  for (int b0 = 0; b0 < total; b0 += FOLD) {
    const int b1 = min(total, b0 + FOLD);
    if (tid == 0) {
      for (int c = b0; c < b1 && ok; ++c) {
        if (issued == c) { issue_tma(c); ++issued; }
        if (c + 1 < total && issued == c + 1) {
          // stage (c+1)&1 was last read by the MMAs of chunk c-1
          if (c + 1 >= 2) ok = mbar_wait(&empty_bar[(c + 1) & 1], ((c - 1) >> 1) & 1, wait_ns);
          if (ok) { issue_tma(c + 1); ++issued; }
        }
        if (!ok) break;
        const int s = c & 1;
        ok = mbar_wait(&full_bar[s], (c >> 1) & 1, wait_ns);
        if (!ok) break;
        consumed = c + 1;
        fence_after();
        const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
        for (int p = 0; p < NPROD; ++p) {
          const int la = (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0);
          const int lb = (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0);
          const uint32_t aa = sa + la * TILE_BYTES, ba = sa + (NS + lb) * TILE_BYTES;
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            const uint32_t acc = (c > b0 || p > 1 || kk > 0) ? 1u : 0u;
            umma_f16(p == 0 ? t_acc : t_acc2, make_desc(aa + kk * 32), make_desc(ba + kk * 32), idesc, acc);
          }
        }
        umma_commit(&empty_bar[s]);
        last_commit = c;
      }
      if (ok) {
        umma_commit(&acc_bar);
        acc_pending = true;
        ok = mbar_wait(&acc_bar, folds & 1, wait_ns);
        if (ok) acc_pending = false;
      }
      abort_s = ok ? 0 : 1;
    }
    __syncthreads();
    if (abort_s) break;
    fence_after();
#pragma unroll 1
    for (int cb = 0; cb < TBN; cb += 32) {
      // main part: TwoSum into (hi, lo); small products: added to lo
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
    ++folds;
    fence_before();
    __syncthreads();
    fence_after();
  }

  if (abort_s) {
    // drain what this CTA still has in flight, then give up: the TMA chunks
    // not yet consumed (at most two, each the newest phase of its barrier),
    // the MMAs up to the last commit, and an unconsumed accumulator commit
    if (tid == 0) {
      if (err) atomicExch(err, 1);
      for (int c = consumed; c < issued; ++c) mbar_wait(&full_bar[c & 1], (c >> 1) & 1, DRAIN_NS);
      if (last_commit >= 0) mbar_wait(&empty_bar[last_commit & 1], (last_commit >> 1) & 1, DRAIN_NS);
      if (acc_pending) mbar_wait(&acc_bar, folds & 1, DRAIN_NS);
    }
    __syncthreads();
  } else {
    // epilogue: TMEM lane = tile row = tid.  Each 32-column slice goes through
    // shared memory (the idle stage buffers) so that a warp stores 32
    // consecutive columns of one row per instruction.
    const bool accum = g.flags & 1, out_f32 = g.flags & 2;
    float* stg = reinterpret_cast<float*>(smem);     // [128][33]
    double* stgd = reinterpret_cast<double*>(smem);  // [128][33]
    const int lane = tid & 31;
#pragma unroll 1
    for (int cb = 0; cb < TBN; cb += 32) {
      if (folds > 0) {
        tmem_ld32(t_hi + lane_off + cb, h);
        tmem_ld32(t_lo + lane_off + cb, w);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) { h[i] = 0.f; w[i] = 0.f; }
      }
      if (out_f32) {
#pragma unroll
        for (int i = 0; i < 32; ++i) stg[tid * 33 + i] = h[i] + w[i];
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) stgd[tid * 33 + i] = (double)h[i] + (double)w[i];
      }
      __syncthreads();
      const int col = tl.n0 + cb + lane;
      for (int rr = warp; rr < TBM; rr += 4) {
        const int row = tl.m0 + rr;
        if (row < g.M && col < g.N) {
          const long long o = (long long)row * g.ldc + col;
          if (out_f32) {
            float* C = reinterpret_cast<float*>(sel_base(bs, slot_of(g.C))) + off_of(g.C) + o;
            const float val = stg[rr * 33 + lane];
            *C = accum ? *C + val : val;
          } else {
            double* C = reinterpret_cast<double*>(sel_base(bs, slot_of(g.C))) + off_of(g.C) + o;
            const double val = stgd[rr * 33 + lane];
            *C = accum ? *C + val : val;
          }
        }
      }
      __syncthreads();
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

size_t tc_smem_bytes(int nsplit) { return (size_t)2 * 2 * nsplit * TILE_BYTES + 1024; }

cudaError_t launch_gemm_tc(const GGroup* groups, const GSeg* segs, const GTile* tiles128, int ntiles,
                           const void* maps, const Bases& b, int nsplit, int* err, long long wait_ns, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const size_t smem = tc_smem_bytes(nsplit);
  if (nsplit == 2) {
    // once per process (thread-safe static initialisation)
    static const cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tc_kernel<2><<<ntiles, 128, smem, s>>>(groups, segs, tiles128, (const CUtensorMap*)maps, b, err, wait_ns);
  } else if (nsplit == 3) {
    // once per process (thread-safe static initialisation)
    static const cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tc_kernel<3><<<ntiles, 128, smem, s>>>(groups, segs, tiles128, (const CUtensorMap*)maps, b, err, wait_ns);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tt
