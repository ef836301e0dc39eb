// Launch wrappers of the device kernels (tt_kernels.cu).  Every wrapper is
// asynchronous on the given stream and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_core.h"

namespace tt {

// Slot table passed by value to the plan-driven kernels: base pointer of each
// slot and, for split-BF16 buffers, the element offset of the "lo" half.
struct Bases {
  void* p[8];
  long long lo[8];
};

#ifdef __CUDACC__
// bs.p[slot] by selects: indexing the by-value kernel argument with a
// run-time slot would copy the array to local memory first
__device__ __forceinline__ void* sel_base(const Bases& bs, int slot) {
  void* p = bs.p[0];
#pragma unroll
  for (int k = 1; k < 8; ++k)
    if (slot == k) p = bs.p[k];
  return p;
}
__device__ __forceinline__ long long sel_lo(const Bases& bs, int slot) {
  long long v = bs.lo[0];
#pragma unroll
  for (int k = 1; k < 8; ++k)
    if (slot == k) v = bs.lo[k];
  return v;
}
#endif

// Device copies of a plan.
struct DevGemm {
  GGroup* groups = nullptr;
  GSeg* segs = nullptr;
  GTile* tiles64 = nullptr;   // 64 x 64 output tiles
  int ngroups = 0, nsegs = 0, ntiles64 = 0;
  double flops = 0;
};
struct DevGather {
  GItem* items = nullptr;
  GContrib* contribs = nullptr;
  int nitems = 0;
  double elems = 0;
};
struct DevCopy {
  CItem* items = nullptr;
  int nitems = 0;
  int maxtiles = 0;  // largest item, in 32 x 32 tiles
};
struct DevDigit {
  DItem* items = nullptr;
  int nitems = 0;
  int maxgroups = 0;  // largest item, in groups of 32 digit rows
};

// Device-side Krylov bookkeeping of one Lanczos exponential.
struct KrylovState {
  double alpha[17];
  double beta[17];
  double h[17];
  double c[17];
  double nb;        // ||v||
  double hscale;    // max(|alpha_j| + beta_j)
  double resid;     // ||v|| beta_K |c_K|
  double nrm;       // norm of the result (before normalisation)
  int kdim;         // Krylov dimension in use
  int broken;       // breakdown seen
  int bad;          // NaN / Inf seen
  int pad;
};

// Global accumulators of a state (device).
struct RhoScalars {
  double logscale;
  double resid_max;
  int bad;
  int pad;
};

cudaError_t launch_gemm_f64(const DevGemm& g, const Bases& b, cudaStream_t s);
// The same in double-float arithmetic on the FP32 pipe (~2^-46 per operation).
cudaError_t launch_gemm_df(const DevGemm& g, const Bases& b, cudaStream_t s);
// Exact-accumulation split GEMM (tt_ozaki.cu): FP64 operands of the FP64
// plans, four fixed-point BF16 digits per K tile, ~2^-32 normwise.
cudaError_t launch_gemm_oz(const DevGemm& g, const Bases& b, cudaStream_t s);
// nsplit = 2 (3 products) or 3 (6 products); operand level l at offset l * lo[slot]
cudaError_t launch_gemm_bf16(const DevGemm& g, const Bases& b, int nsplit, cudaStream_t s);
// in_type / out_type: 0 = double, 1 = float, 2 / 3 = split bf16 with that many levels
cudaError_t launch_gather(const DevGather& g, const Bases& b, int in_type, int out_type, cudaStream_t s);
cudaError_t launch_copy(const DevCopy& c, const Bases& b, cudaStream_t s);
cudaError_t launch_split_bf16(const double* x, int64_t n, int nsplit, void* out /* bf16[nsplit*n] */, cudaStream_t s);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);
// strided FP64 -> split-bf16 copy (levels at dst + l * lo[slot(dst)])
cudaError_t launch_split_copy(const DevCopy& c, const Bases& b, int nsplit, cudaStream_t s);
// tcgen05 grouped GEMM (tt_tcgen05.cu): K-major A and B, 128 x 128 tiles,
// maps = 3 CUtensorMap per segment in global memory: A (box 64 K x 128 rows),
// B (64 x 128), B (64 x 64).
size_t tc_smem_bytes(int nsplit);
// Persistent warp-specialised variant (tt_tcgen05p.cu): 128 x 64 tiles, one
// CTA per SM, TMA ring / MMA warp / fold-and-epilogue warps, the same
// arithmetic and maps.
size_t tcp_smem_bytes(int nsplit);
cudaError_t launch_gemm_tcp(const GGroup* groups, const GSeg* segs, const GTile* tiles128x64, int ntiles,
                            const void* maps, const Bases& b, int nsplit, int* err, long long wait_ns, cudaStream_t s);
// Exact-accumulation split GEMM on tcgen05 (tt_tcgen05z.cu): digit operands
// (4 levels + int16 row exponents, GSeg.eA / eB), persistent 128 x 64 tiles,
// the same maps; segments of K <= tcz_max_k(); output FP64 or two-float pairs
// (flags bit 1, the same in every group of a launch: pair).
int tcz_max_k();
size_t tcz_smem_bytes();
cudaError_t launch_gemm_tcz(const GGroup* groups, const GSeg* segs, const GTile* tiles128x64, int ntiles,
                            const void* maps, const Bases& b, int* err, long long wait_ns, bool pair, cudaStream_t s);
// Digit producers (tt_digits.cu): FP64 rows -> digit rows; the W-gather of
// the exact path (two-float S1 outputs -> digit rows of T2, rows up to
// gather_digits_max_cols() long, at most gather_digits_max_contribs() MPO
// terms per item).
cudaError_t launch_digit_copy(const DevDigit& d, const Bases& b, cudaStream_t s);
cudaError_t launch_gather_digits(const DevGather& g, const Bases& b, cudaStream_t s);
int gather_digits_max_cols();
int gather_digits_max_contribs();
// err: set to 1 by a CTA whose bounded wait (budget wait_ns) ran out.
cudaError_t launch_gemm_tc(const GGroup* groups, const GSeg* segs, const GTile* tiles128, int ntiles,
                           const void* maps, const Bases& b, int nsplit, int* err, long long wait_ns, cudaStream_t s);

// Lanczos exponential steps on flat FP64 vectors of length n.  Q holds the
// Krylov basis with leading dimension ldq.  `partial` is scratch of
// nblk * 17 doubles.
int lanczos_nblk();
cudaError_t k_norm_init(const double* v, int64_t n, double* partial, KrylovState* ks, double* q0, cudaStream_t s);
cudaError_t k_dots_alpha(const double* Q, int64_t ldq, int k, const double* w, int64_t n, double* partial,
                         KrylovState* ks, cudaStream_t s);
cudaError_t k_three_term(const double* Q, int64_t ldq, int k, double* w, int64_t n, KrylovState* ks, cudaStream_t s);
cudaError_t k_cgs_pass(const double* Q, int64_t ldq, int k, double* w, int64_t n, double* partial, KrylovState* ks,
                       int last, double breakdown_tol, int K, double* qnext, cudaStream_t s);
cudaError_t k_krylov_exp(KrylovState* ks, double t, int K, cudaStream_t s);
cudaError_t k_combine(const double* Q, int64_t ldq, const KrylovState* ks, double* y, int64_t n, double* partial,
                      KrylovState* ksw, cudaStream_t s);
// after k_combine (same n): finalize ||y||, logscale += ln ||y||, y /= ||y||
cudaError_t k_finish_normalise(double* y, int64_t n, double* partial, KrylovState* ks, RhoScalars* rs, cudaStream_t s);

// v /= ||v||, logscale += ln ||v|| (rs->bad set on zero / non-finite norm)
cudaError_t k_normalise_inplace(double* v, int64_t n, double* partial, KrylovState* ks, RhoScalars* rs, cudaStream_t s);

// Householder QR of a batch of column-major matrices in workspace `ws`.
cudaError_t launch_qr(const QrJob* jobs, int njobs, double* ws, cudaStream_t s);
// one job passed by value (the record is a kernel argument, not device memory)
cudaError_t launch_qr_job(const QrJob& job, double* ws, cudaStream_t s);
// the same, only for the jobs whose only[job] != 0
// Householder QR of the jobs whose flag in `only` is set; *nrun (if not null)
// counts the sectors factorised.
cudaError_t launch_qr_masked(const QrJob* jobs, int njobs, double* ws, const int* only, int* nrun, cudaStream_t s);
// Cholesky + triangular inverse per job (shifted on request); fail[sec] set on
// a non-positive pivot.
// maxn: the largest n of the jobs (shared-memory variant up to 230); df: that
// variant in double-float arithmetic (~2^-46) instead of FP64.
cudaError_t launch_chol_inv(const CholJob* jobs, int njobs, double* ws, int* fail, cudaStream_t s, int maxn = 0,
                            bool df = false);
// Sign fix diag(R) >= 0 done inside launch_qr.

// Per-block item of the local measurement (d = 4 local space, <= 4 pairs).
struct ObsItem {
  long long off;
  int dl, m, dr, pad;
  double wn[4], wd[4];
};
// out[0] += sum A T w_n ; out[1] += sum A T w_d  (partial: 2 * nitems doubles)
cudaError_t launch_local_obs(const ObsItem* items, int nitems, const double* A, const double* T, double* partial,
                             double* out, cudaStream_t s);
// column-major a (ld): by_col ? a[:, c] *= s[c] : a[r, :] *= s[r]
cudaError_t launch_scale_rc(double* a, long long ld, int rows, int cols, const double* sv, int by_col, cudaStream_t s);

// *out = x . y (deterministic two-stage reduction)
cudaError_t k_dot_plain(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t s);

}  // namespace tt
