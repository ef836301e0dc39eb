/*
 * tantrg.h - C ABI of the GB300 tanTRG library (libtantrg.so).
 *
 * Tangent-space tensor renormalization group (arXiv 2212.11973): finite-
 * temperature imaginary-time evolution of the MPO half-density operator
 * rho_h(beta) = exp(-beta H / 2) of the 2D Hubbard model (Eq. 3) on a
 * snake-ordered cylinder or ladder (Fig. 1(a)), by 1-site TDVP sweeps
 * (Eq. 2; Supplement, "Procedure of 1-TDVP") after a 2-site TDVP growth
 * stage (Supplement, "2-TDVP in the initial stage").
 *
 * Conventions
 *   - Local basis sigma = n_up + 2 n_dn = {|0>, |up>, |dn>, |up dn>}, with
 *     |up dn> = c+_up c+_dn |0>; Jordan-Wigner strings run along the snake.
 *   - rho_h is stored as its Choi super-MPS (Supplement, "Choi
 *     transformation"): site tensors A[a_l, (sigma, sigma'), a_r], U(1) x U(1)
 *     block sparse in (particle number, 2 Sz).  Every tensor is real.
 *   - Z(beta) = <<rho_h|rho_h>>, E = <<rho_h|H x I|rho_h>> / Z (bilayer trick,
 *     Supplement eq. for E(beta)).
 *   - One beta-step of size dtau is a left-to-right plus a right-to-left half
 *     sweep, each integrating with tau = dtau / 4, so rho_h -> exp(-dtau H/2)
 *     rho_h (symmetric Lie-Trotter composition; main text "4 tau = 1").
 *
 * Ownership and errors
 *   - Every object belongs to one context and runs on the context's CUDA
 *     stream.  The caller owns every handle it receives and frees it with the
 *     matching _destroy call (destroy on NULL is a no-op).
 *   - Functions return tt_status; no C++ exception crosses the ABI.  After an
 *     error the message is available from tt_last_error(ctx); an object that
 *     saw a CUDA or numeric error is poisoned: later calls on it return
 *     TT_ERR_STATE, destroying it is always safe.
 *   - Pointers documented as "host" are read or written by the CPU before the
 *     call returns; pointers documented as "device" are cudaMalloc'ed memory of
 *     the context's device and are only read/written in stream order.
 */
#ifndef TANTRG_H
#define TANTRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_ERR_INVALID_ARG = 1, /* bad size, geometry, option or NULL pointer */
  TT_ERR_OOM = 2,         /* device allocation failed */
  TT_ERR_CUDA = 3,        /* a CUDA runtime / library call failed */
  TT_ERR_NUMERIC = 4,     /* NaN/Inf or a failed factorisation was detected */
  TT_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  TT_ERR_STATE = 6        /* object poisoned by an earlier error, or wrong stage */
} tt_status;

typedef enum {
  TT_PREC_FP64 = 0,          /* every contraction in FP64 */
  TT_PREC_MIXED_BF16X3 = 1,  /* H_eff and bond contractions as split-BF16
                                tensor-core products, 2 levels / 3 products
                                (~2^-16 relative); environment updates per
                                env_precision */
  TT_PREC_MIXED_BF16X6 = 2,  /* 3 levels / 6 products (~2^-24 relative), FP32
                                accumulation folded per K chunk into a two-
                                float sum.  In both modes the Lanczos vectors,
                                Krylov exponential, SVD, absorb step,
                                measurements and log-norm stay FP64; the
                                CholeskyQR gauge runs in double-float (~2^-46)
                                with a FP64 Householder fallback */
  TT_PREC_SPLIT_EXACT = 3    /* exact-accumulation split (Ozaki scheme): the
                                H_eff and bond applies' operands as four
                                fixed-point BF16 digits with one exponent per
                                row and GEMM segment (K <= 256), the ten digit
                                products with s + t <= 3 summed exactly in FP32
                                on the tcgen05 tensor cores and folded into a
                                two-float accumulator per segment: ~2^-32 of the
                                rows' bounds; the W-gather in two-float
                                arithmetic writing digit rows.  Sectors must
                                have at most 256 states and a gather item at
                                most 64 MPO terms (TT_ERR_INVALID_ARG
                                otherwise).  Environment updates per
                                env_precision; the CholeskyQR gauge in
                                double-float; Lanczos, Krylov exponential,
                                absorb, measurements and log-norm in FP64 */
} tt_precision;

typedef struct tt_ctx tt_ctx;
typedef struct tt_mpo tt_mpo;
typedef struct tt_rho tt_rho;
typedef struct tt_batch tt_batch;

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc must
 * return device memory usable on `stream` (NULL on failure); free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} tt_alloc_cb;

/* Hubbard model, Eq. 3.  interaction_form 0: U n_up n_dn (Eq. 3);
 * 1: U (n_up - 1/2)(n_dn - 1/2), the particle-hole symmetric form of the DQMC
 * appendix (mu = 0 is half filling).  Lx >= 1 columns (open), Wy >= 1 rows;
 * bc_y_periodic wraps y when Wy > 2.  tp: next-nearest (diagonal) hopping of
 * the t-t' model (Supplement, t-t'-U model), -tp (c+_i c_j + h.c.) on the pairs
 * (x, y)-(x+1, y+-1); 0 gives Eq. 3.  Lx * Wy <= 512. */
typedef struct {
  int Lx, Wy, bc_y_periodic;
  double t, tp, U, mu;
  int interaction_form;
} tt_model;

typedef struct {
  int D_max;            /* bond dimension cap (U(1)xU(1) states), >= 1 */
  int krylov_dim;       /* Lanczos Krylov dimension K, 1..16 (paper: K small) */
  int precision;        /* tt_precision of the 1-TDVP linear stage */
  int growth_precision; /* tt_precision of the 2-TDVP growth; -1 = FP64.  Mixed
                           growth perturbs exactly degenerate singular values
                           and so the truncation; use FP64 for parity runs */
  double svd_cut;       /* growth: drop s <= svd_cut * s_max (default 1e-12) */
  double degen_tol;     /* growth: never split s_k, s_k+1 with
                           s_k - s_k+1 <= degen_tol s_k + 1e-14 s_max (1e-10) */
  int env_precision;    /* environment updates.  0 (default): FP64 in the FP64
                           mode, the exact-accumulation split (as
                           TT_PREC_SPLIT_EXACT) in the other modes; 1: native
                           FP64 GEMMs; 2: double-float GEMMs on the FP32 pipe
                           (~2^-46 per operation) in the mixed modes; -1: the
                           arithmetic of `precision`.
                           Each update feeds the next along the chain, so its
                           rounding errors compound over the N sites (FP32-
                           class split products leave ~1e-5 in the energy at
                           N = 72); the H_eff and bond applies' errors stay
                           local to one update */
} tt_run_opts;

typedef struct {
  double beta;                 /* inverse temperature reached */
  double energy_per_site;      /* <<rho_h|H x I|rho_h>> / (N Z) */
  double density;              /* (1/N) sum_i <n_i> */
  double double_occ;           /* D_n = (1/N) sum_i <n_i,up n_i,dn> */
  double free_energy_per_site; /* -ln Z / (beta N), grand potential per site */
  double lnZ;                  /* ln Z = 2 logscale + ln <<psi|psi>> */
  int max_bond;                /* largest bond dimension */
  double krylov_resid_max;     /* max over updates of ||v|| beta_K |c_K| */
} tt_obs;

typedef struct {
  double heff_flops;       /* algorithmic flops (2 M N K over the blocks) of the
                              site H_eff GEMM launches of the last tt_tdvp_step */
  double heff_ms;          /* summed device time of those launches (CUDA events,
                              profiling mode only, else 0) */
  long long heff_launches; /* number of those launches (profiling mode) */
  double env_flops, env_ms;/* same for the environment-update GEMMs */
  double bond_ms;          /* bond H_eff GEMMs (profiling mode) */
  double gather_ms;        /* W-gather kernels (profiling mode) */
  long long gather_launches;
  double step_flops;       /* algorithmic flops of all contractions of the last call */
  double step_ms;          /* device time of the last tt_tdvp_step call (events) */
  long long launches;      /* kernels launched by the last tt_tdvp_step call */
  int n_sites, max_bond, n_sectors_max;
  double qr_ms;            /* QR gauge factorisations: CholeskyQR3 GEMMs and
                              Cholesky kernels plus the Householder fallback
                              (profiling mode) */
  double bond_flops;       /* algorithmic flops of the bond H_eff GEMMs */
  long long qr_sectors;    /* sector matrices factorised by the QR gauge */
  long long qr_fallbacks;  /* of those, the ones the Householder kernel redid
                              (Cholesky failed or more columns than rows) */
  /* whole phases of the sweep (profiling mode; they contain the launches
     counted above): site exponentials (Lanczos + H_eff applies), bond
     exponentials, environment updates, absorbs, gauge moves (copies + QR) */
  double site_exp_ms, bond_exp_ms, env_update_ms, absorb_ms, gauge_ms;
  /* split-BF16 GEMM plans of this state by the kernel the tile autotuner
     chose (first uncaptured use: every eligible kernel timed, fastest kept):
     tcgen05 128 x 128 tiles, persistent tcgen05 128 x 64 tiles, mma.sync
     64 x 64 tiles */
  long long tuned_tc128, tuned_tcp128x64, tuned_mma64;
  /* inside qr_ms (profiling mode): the CholeskyQR3 Gram / apply GEMMs (time
     and algorithmic flops) and the Cholesky + triangular-inverse kernels */
  double qr_gemm_ms, qr_gemm_flops, qr_chol_ms;
} tt_stats;

/* ---- context ---------------------------------------------------------- */

/* alloc may be NULL (then cudaMallocAsync on the stream).  cuda_stream is a
 * cudaStream_t of the current device or NULL for the legacy default stream. */
tt_status tt_ctx_create(const tt_alloc_cb* alloc, void* cuda_stream, tt_ctx** out);
void tt_ctx_destroy(tt_ctx* ctx);
/* Message of the last failed call on this context ("" if none).  Owned by ctx. */
const char* tt_last_error(const tt_ctx* ctx);
/* Time budget, in seconds (0..60, default 2), of every bounded device-side wait
 * of this context's kernels (the tcgen05 GEMM's copy and MMA barriers).  A wait
 * that runs out makes the kernel record an error, drain its own copies in flight
 * and return; the next synchronising call on the object (tt_measure, tt_rho_grow,
 * tt_heff_apply_host) then returns TT_ERR_TIMEOUT and poisons it, while the
 * context stays usable.  0 means a single non-blocking test per wait.  Takes
 * effect for the following launches (a captured beta-step is re-captured). */
tt_status tt_ctx_set_wait_limit(tt_ctx* ctx, double seconds);

/* ---- Hubbard MPO (Eq. 3; built on the host as a finite automaton with
 *      U(1)xU(1) labels on every leg, uploaded to the device) --------------- */
tt_status tt_hubbard_mpo_create(tt_ctx* ctx, const tt_model* m, tt_mpo** out);
void tt_mpo_destroy(tt_mpo* mpo);
/* Number of sites and the MPO bond dimension of bond k (0..N). */
int tt_mpo_num_sites(const tt_mpo* mpo);
int tt_mpo_bond_dim(const tt_mpo* mpo, int k);

/* ---- state ------------------------------------------------------------- */

/* rho_h(beta0) = I - beta0 H / 2 (main text: rho_0 = 1 - tau_0 H from the MPO
 * of H), right-canonicalised by LQ sweeps (canonical centre on site 0), for
 * taylor_order = 1.  taylor_order = n in 2..8: the series-expansion initial
 * state sum_{k <= n} (-beta0 H / 2)^k / k! (Supplement, "Error analysis of
 * tanTRG": SETTN initialisation), built by Horner's rule, each step a local
 * MPO x super-MPS product plus the identity, compressed by SVD (singular
 * values <= 1e-14 s_max dropped); the bond dimension before each compression
 * is (MPO bond) x (current bond) + 1, so high orders suit small systems or
 * small beta0.  Every order keeps the bond dimensions the compression leaves
 * (tt_rho_grow then starts from them). */
tt_status tt_rho_create(tt_ctx* ctx, const tt_mpo* mpo, double beta0, int taylor_order,
                        const tt_run_opts* opts, tt_rho** out);
void tt_rho_destroy(tt_rho* rho);

/* 2-TDVP growth stage: beta-steps of size dtau until every bond holds
 * min(D_max, 16^k, 16^(N-k)) states or beta >= beta_max.  Writes the beta
 * reached to *beta_reached (host, may be NULL).  Synchronises the stream. */
tt_status tt_rho_grow(tt_rho* rho, const tt_mpo* mpo, double dtau, double beta_max,
                      double* beta_reached);
/* The growth stage on an exponential grid (main text: "we always start with
 * exponential grids and exploit the two-site update"; Fig. S7(b): beta_n =
 * 2^(n/m) beta_0): every 2-TDVP beta-step takes beta -> ratio * beta (the last
 * one clipped to beta_max), 1 < ratio <= 4, with the same stop rule as
 * tt_rho_grow.  Synchronises the stream. */
tt_status tt_rho_grow_exp(tt_rho* rho, const tt_mpo* mpo, double ratio, double beta_max,
                          double* beta_reached);

/* Enlarge every bond to about D_target states (each sector scaled by
 * D_target / D, within what the neighbouring blocks can hold) with zero-weight
 * orthonormal completions; the state is unchanged, the 1-TDVP manifold larger
 * (the sweeps then populate the new directions).  Used to reach a large D
 * without a two-site sweep at that D.  Canonical centre must be on site 0. */
tt_status tt_rho_pad(tt_rho* rho, const tt_mpo* mpo, int D_target);

/* n_steps 1-TDVP beta-steps of size dtau (main text, linear stage; one
 * beta-step = an L->R and an R->L half sweep, tau = dtau/4 each, Supplement
 * "Procedure of 1-TDVP").  Asynchronous on the ctx stream; the block structure
 * is fixed during the call.  On a non-default stream the first call runs one
 * step with ordinary launches (building plans and buffers) and captures the
 * next as a CUDA graph; later steps replay it (re-captured after a change of
 * dtau, of the profiling mode or of any device buffer).  Set the environment
 * variable TT_CUDA_GRAPH=0 to launch every kernel directly; TT_QR=householder
 * selects the one-CTA Householder QR for every sector. */
tt_status tt_tdvp_step(tt_rho* rho, const tt_mpo* mpo, double dtau, int n_steps);

/* Observables at the canonical centre (site 0 after a step).  Synchronises the
 * stream and writes *out (host). */
tt_status tt_measure(tt_rho* rho, const tt_mpo* mpo, tt_obs* out);

/* Statistics accumulated over the tt_tdvp_step calls since the previous
 * tt_stats_get (host *out; synchronises on the last call's end event). */
tt_status tt_stats_get(const tt_rho* rho, tt_stats* out);
/* Profiling mode: record a CUDA event pair around every GEMM / gather launch
 * of the following tt_tdvp_step calls (on the context stream). */
tt_status tt_rho_set_profiling(tt_rho* rho, int on);

/* Current bond dimensions: writes N+1 ints (host) to dims. */
tt_status tt_rho_bond_dims(const tt_rho* rho, int* dims, int n);
/* U(1)xU(1) sectors of bond k (0..N): *nsec = their number; if cap >= *nsec
 * the charges (particle number n and s = n_up - n_dn, ket minus bra of the
 * Choi pair summed over the sites left of the bond) and dimensions are
 * written to the host arrays qn, qs, dims in the engine's sector order, else
 * TT_ERR_INVALID_ARG with only *nsec set. */
tt_status tt_rho_bond_sectors(const tt_rho* rho, int k, int* qn, int* qs, int* dims, int cap, int* nsec);

/* ---- batch of independent instances (many small models evolved together,
 *      e.g. 64 ladders 2x8 with drawn U, mu and D) ----------------------------
 *
 * Instance i is the model models[i] at bond dimension D_max[i], initialised
 * like tt_rho_create (taylor order 1, beta0) with the other fields of opts.
 * Every instance owns a context, a CUDA stream and its captured beta-step
 * graph; tt_batch_step waits for the work already queued on ctx's stream and
 * on the instance streams, steps all instances concurrently, and makes ctx's
 * stream and the instance streams wait for the result (asynchronous, like
 * tt_tdvp_step).  Its first step runs per instance on the instance streams
 * (capturing their graphs); later steps with the same dtau launch one parent
 * graph on ctx's stream that holds every instance's step graph as a child
 * node (re-composed when an instance's graph was re-captured; per-instance
 * steps while profiling).  tt_batch_grow runs the growth stage
 * of every instance (synchronous).  tt_batch_measure writes n tt_obs (host,
 * caller-owned; synchronises).  On error the message names the instance; the
 * batch is then only safe to destroy.  The library owns the batch; free it with
 * tt_batch_destroy. */
tt_status tt_batch_create(tt_ctx* ctx, int n, const tt_model* models, const int* D_max, double beta0,
                          const tt_run_opts* opts, tt_batch** out);
void tt_batch_destroy(tt_batch* b);
int tt_batch_size(const tt_batch* b);
tt_status tt_batch_grow(tt_batch* b, double dtau, double beta_max);
/* tt_rho_pad of every instance to its own D_max (synchronous). */
tt_status tt_batch_pad(tt_batch* b);
tt_status tt_batch_step(tt_batch* b, double dtau, int n_steps);
tt_status tt_batch_measure(tt_batch* b, tt_obs* out_n);
/* tt_stats_get of instance i; profiling switched for every instance. */
tt_status tt_batch_stats(tt_batch* b, int i, tt_stats* out);
tt_status tt_batch_set_profiling(tt_batch* b, int on);

/* ---- checkpoint (versioned little-endian binary: sector tables, FP64
 *      blocks, beta, logscale) ---------------------------------------------- */
tt_status tt_rho_save(tt_rho* rho, const char* path);
tt_status tt_rho_load(tt_ctx* ctx, const tt_mpo* mpo, const char* path,
                      const tt_run_opts* opts, tt_rho** out);

/* ---- kernel-level entry points (one H_eff apply on given tensors) --------
 *
 * Bond k carries nsec[k] sectors; sector r of bond k has charge
 * (qn[r], qs[r]) = (particle number, 2 Sz) and dimension qd[r], listed in
 * strictly increasing (qn, qs) order.  Arrays for bonds are concatenated.
 *
 * Site tensor x (bond j -> bond j+1) layout: blocks (a_l sector l, pair sector
 * p, a_r sector r) with charge(r) = charge(l) + p, ordered by r, then l, then
 * p, with the nine pair charges p = charge(sigma) - charge(sigma') taken in
 * increasing (n, 2Sz) order; each block row-major [a_l][pair][a_r], the pairs
 * (sigma, sigma') of charge p in increasing 4 sigma + sigma'.
 *
 * Environment layout (bond k, MPO channels w = 0..tt_mpo_bond_dim(k)-1 with
 * channel charge c_w from tt_mpo_channel_charge): per ket sector b in bond order, a
 * row-major matrix of rows (w ascending, bra index a in sector b + c_w, only
 * channels whose sector exists) and d_b columns; matrices concatenated.
 *   L (bond j):   L[a, w, b] = sum over sites < j, bra a, ket b.
 *   R (bond j+1): R[a, w, b] = sum over sites > j, bra a, ket b.
 * tt_layout_sizes() returns the element counts of x, L, R.
 * All of x, L, R, y are host FP64 arrays; y receives H^(1) x in x's layout.
 */
tt_status tt_mpo_channel_charge(const tt_mpo* mpo, int k, int w, int* qn, int* qs);
tt_status tt_layout_sizes(const tt_mpo* mpo, int site, const int* nsec_lr /*2*/,
                          const int* qn, const int* qs, const int* qd,
                          int64_t* x_size, int64_t* l_size, int64_t* r_size);
tt_status tt_heff_apply_host(tt_ctx* ctx, const tt_mpo* mpo, int site, int precision,
                             const int* nsec_lr, const int* qn, const int* qs, const int* qd,
                             const double* L, const double* R, const double* x, double* y);

/* The same site apply (Supplement, "Lanczos-based exponential method": the
 * L W A R contraction) with the MPO tensor W given by the caller instead of a
 * tt_mpo: channels w = 0..nw_l-1 of the left MPO bond with charges
 * (chl_qn[w], chl_qs[w]), channels of the right MPO bond likewise, and nterms
 * nonzero entries W[wl][wr] <sig| op |tau> = t_val (host arrays t_wl, t_wr,
 * t_sig, t_tau in 0..3 of the local basis above, t_val).  Every term must
 * satisfy c_wr = c_wl + q(sig) - q(tau) (q = (particle number, 2 Sz)), else
 * TT_ERR_INVALID_ARG.  Sector tables, L, R, x, y and precision as in
 * tt_heff_apply_host, with the environments' channel index running over these
 * channels.  tt_layout_sizes_terms gives the element counts of x, L, R. */
tt_status tt_heff_apply_terms_host(tt_ctx* ctx, int nw_l, const int* chl_qn, const int* chl_qs,
                                   int nw_r, const int* chr_qn, const int* chr_qs,
                                   int nterms, const int* t_wl, const int* t_wr, const int* t_sig,
                                   const int* t_tau, const double* t_val, int precision,
                                   const int* nsec_lr, const int* qn, const int* qs, const int* qd,
                                   const double* L, const double* R, const double* x, double* y);
tt_status tt_layout_sizes_terms(int nw_l, const int* chl_qn, const int* chl_qs, int nw_r,
                                const int* chr_qn, const int* chr_qs, const int* nsec_lr,
                                const int* qn, const int* qs, const int* qd,
                                int64_t* x_size, int64_t* l_size, int64_t* r_size);

/* QR gauge kernel on one matrix (Supplement, "Procedure of 1-TDVP", step 3:
 * A_i = A_i^L S_i by QR): A = Q R for a column-major m x n matrix (ld = m,
 * 1 <= n <= min(m, 2048)), Householder in FP64, sign convention diag(R) >= 0.
 * A, Q (m x n, column-major) and R (n x n, column-major, upper triangular) are
 * device pointers; A is not modified.  Scratch comes from the context
 * allocator.  Synchronises the context stream. */
tt_status tt_qr_device(tt_ctx* ctx, const double* A, int m, int n, double* Q, double* R);

/* The same QR without any device allocation, for callers that may not allocate
 * device memory at that point (a memory pool that must not grow, an allocator
 * owned by another framework, a latency-bound path where cudaMalloc could
 * synchronise).  The paper has no counterpart; this is a library service.
 *   Scratch: a fixed 16 MiB array in device global memory, reserved on every GPU
 *   that loads the library until the process exits.  Limit: 2 m n + n^2
 *   doubles (e.g. m = 2048, n = 448); larger sizes, or n > 2048, or m < n return
 *   TT_ERR_INVALID_ARG without touching the GPU.  The call queues one device-
 *   to-device copy of A, the kernel (its job record passed as a kernel
 *   argument) and two device-to-device copies of Q and R: no host-to-device
 *   copy, so it does not wait for the stream.
 *   A (m x n, column-major), Q (m x n, column-major) and R (n x n, column-major)
 *   are device pointers of the current device; the work is queued on
 *   cuda_stream (NULL: legacy default stream) and the call returns without
 *   synchronising.  The first call on a device looks up the scratch address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.  Every call on a device shares the one scratch
 *   array and it keeps the last call's contents: calls that overlap on the GPU
 *   (different streams, no ordering) race and corrupt each other. */
tt_status tt_qr_device_noalloc(const double* A, int m, int n, double* Q, double* R, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TANTRG_H */
