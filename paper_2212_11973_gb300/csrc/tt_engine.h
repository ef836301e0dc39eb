// Internal engine types behind the C ABI (tantrg.h).
#pragma once
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <string>
#include <vector>

#include "../../include/tantrg.h"
#include "tt_core.h"
#include "tt_kernels.h"
#include "tt_plans.h"

struct tt_ctx {
  cudaStream_t st = nullptr;
  // bumped whenever a device buffer is replaced by a larger one: a captured
  // graph holds raw pointers and is only replayed while this is unchanged
  unsigned long long buf_gen = 0;
  tt_alloc_cb cb{};
  bool has_cb = false;
  std::string err;
  cusolverDnHandle_t sol = nullptr;
  // time budget of every bounded device wait (tcgen05 GEMM mbarriers), ns
  long long wait_ns = 2000000000ll;
};

struct tt_mpo {
  tt_ctx* ctx = nullptr;
  tt::ModelSpec spec{};
  tt::Mpo mpo;
  tt::LocalSpace ls2;  // two-site product space (growth)
};

namespace tt {

struct Err {
  tt_status st;
  std::string msg;
};

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

void* dalloc(tt_ctx* c, size_t bytes);
void dfree(tt_ctx* c, DBuf& b);
void ensure(tt_ctx* c, DBuf& b, size_t bytes);  // grow-only, contents not kept
void check_cuda(cudaError_t e, const char* what);

struct DevGemmBuf {
  DevGemm d;
  DBuf buf;
  GemmPlan host;       // kept for the bounds check and the tensor maps
  bool checked = false;
  // tcgen05 path: eligibility, 128 x 128 tile list, per-segment tensor maps
  bool tc_checked = false, tc_ok = false;
  DBuf maps, tiles128, tilesp;
  int ntiles128 = 0, ntilesp = 0;  // 128 x 128 tiles (tc), 128 x 64 tiles (persistent tc)
  // autotuned kernel of a split-BF16 plan: -1 not chosen yet, else a TcKernel
  int choice = -1;
  void* key_p[8] = {nullptr};
  long long key_lo[8] = {0};
};
// Kernels a split-BF16 GEMM plan can run on (chosen per plan by timing).
enum TcKernel { TK_TC128 = 0, TK_TCP128X64 = 1, TK_MMA64 = 2, TK_N = 3 };

struct DevGatherBuf {
  DevGather d;
  DBuf buf;
  GatherPlan host;
  bool checked = false;
};
struct DevCopyBuf {
  DevCopy d;
  DBuf buf;
  CopyPlan host;
  bool checked = false;
};

// Element capacity of every slot (per split level for split-BF16 slots);
// -1 = slot unused.  Plans are checked against it on the host before their
// first launch so that an indexing error raises instead of faulting the GPU.
struct Caps {
  int64_t n[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
};
void check_plan(const GemmPlan& p, const Caps& c, const char* what);
void check_plan(const GatherPlan& p, const Caps& c, const char* what);
void check_plan(const CopyPlan& p, const Caps& c, const char* what);
void check_exps(const GemmPlan& p, const Caps& ex, const char* what);
void check_plan(const DigitPlan& p, const Caps& c, const Caps& ex, const char* what);

void upload(tt_ctx* c, const GemmPlan& p, DevGemmBuf& o);
void upload(tt_ctx* c, const GatherPlan& p, DevGatherBuf& o);
void upload(tt_ctx* c, const CopyPlan& p, DevCopyBuf& o);
void release(tt_ctx* c, DevGemmBuf& o);
void release(tt_ctx* c, DevGatherBuf& o);
void release(tt_ctx* c, DevCopyBuf& o);

struct DevDigitBuf {
  DevDigit d;
  DBuf buf;
  DigitPlan host;
};
void upload(tt_ctx* c, const DigitPlan& p, DevDigitBuf& o);
void release(tt_ctx* c, DevDigitBuf& o);

struct SiteDev {
  bool valid = false;
  SitePlanHost h;
  DevGemmBuf s1, s3, s3l, r1, r3;
  DevGatherBuf s2, r2;
  DevCopyBuf xs;  // split-bf16 mode: x -> transposed padded copy (S1's B operand)
  DevDigitBuf xd; // exact mode: the same as digits
};
struct BondDev {
  bool valid = false;
  BondPlanHost h;
  DevGemmBuf b1, b2;
  DevCopyBuf xs, ts;  // mixed precision: padded split copies of x and T
  DevDigitBuf xd, td; // exact mode: digit copies of x and T
};
struct QrDev {
  bool valid = false;
  QrPlanHost h;
  DBuf jobs;
  DevCopyBuf gather, scatter, rout;
  // shifted CholeskyQR3 (FP64 GEMMs on all SMs) with Householder fallback
  DevGemmBuf gram[3], app[3], tt, rf;
  DBuf cjobs[3], fail;
  int ncj[3] = {0, 0, 0};
  int maxn[3] = {0, 0, 0};  // largest sector (columns) of each pass's Cholesky jobs
};
struct MeasDev {
  bool valid = false;
  DevGemmBuf t, el;
  DBuf items;
  int nitems = 0;
  BondMatLayout next;
};

}  // namespace tt

struct tt_rho {
  tt_ctx* ctx = nullptr;
  const tt_mpo* mpo = nullptr;
  tt_run_opts opts{};
  int N = 0;
  int nsplit = 0;  // 0 = FP64 operand layouts
  bool exact = false;   // TT_PREC_SPLIT_EXACT: split slots hold fixed-point digits (nsplit = 4)
  bool poisoned = false;
  double beta = 0.0;
  std::vector<tt::Bond> bond;           // N + 1
  std::vector<tt::SiteLayout> lay;      // N
  std::vector<tt::DBuf> A;              // N site tensors (FP64)
  std::vector<tt::DBuf> L, R, Lsp, Rsp; // environments (FP64) and split copies
  std::vector<int64_t> Lsize, Rsize;      // FP64 environment sizes (elements)
  std::vector<int64_t> Lpsize, Rpsize;    // split-bf16 copies: rows padded to 8 (elements per level)
  std::vector<tt::DevCopyBuf> esplit;     // per bond: FP64 environment -> padded split copy
  std::vector<tt::DevDigitBuf> edig;      // per bond: FP64 environment -> digits (exact mode)
  std::vector<char> esplit_ok;
  bool use_tc = true;                     // tcgen05 kernel for eligible split-bf16 GEMMs
  bool use_cholqr = true;                 // CholeskyQR3 gauge (else Householder only)
  std::vector<tt::SiteDev> sp;
  std::vector<tt::SiteDev> sp64;
  unsigned long long graph_buf_gen = 0;  // FP64 site plans used by the measurement in mixed mode
  std::vector<tt::BondDev> bp;
  std::vector<tt::QrDev> qrl, lqr;
  std::vector<tt::DevGemmBuf> absl, absr;
  std::vector<char> absl_ok, absr_ok;
  std::vector<tt::MeasDev> meas;
  tt::DBuf Qk, W, Xs, Xn, T1, T2, Sb, ws, partial, ks, rs, tmp, obs, el0, el1, tcerr, qrfb;
  int64_t ldq = 0;
  tt_stats stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool stats_pending = false;
  // per-launch CUDA events (profiling mode): kind 0 = site H_eff GEMMs,
  // 1 = environment GEMMs, 2 = bond H_eff GEMMs, 3 = gather, 4 = other,
  // 5 = QR gauge, 6..10 = sweep phases, 11 = QR GEMMs, 12 = Cholesky kernels
  bool prof = false;
  // CUDA graph of one beta-step (the block structure is fixed in 1-TDVP)
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_tmpl = nullptr;       // the captured graph (a batch composes these)
  unsigned long long graph_gen = 0;       // bumped whenever the graph is replaced or dropped
  double graph_dtau = 0.0;
  bool graph_prof = false;
  long long graph_wait_ns = 0;            // wait budget baked into the captured launches
  double graph_heff_flops = 0, graph_step_flops = 0;
  long long graph_launches = 0;
  bool use_graph = true;
  bool capturing = false;
  long long graph_replays = 0;            // since the last tt_stats_get
  std::vector<cudaEvent_t> gpool;         // profiling events recorded inside the graph
  std::vector<int> gkind;
  size_t gused = 0;
  double graph_kind_flops[13] = {0};
  std::vector<cudaEvent_t> evpool;
  std::vector<int> evkind;
  size_t evused = 0;
  double kind_ms[13] = {0};
  long long kind_n[13] = {0};
  double kind_flops[13] = {0};
  double heff_flops_acc = 0, step_flops_acc = 0;
  long long launches_acc = 0;
  long long qr_sectors_acc = 0, graph_qr_sectors = 0;
  long long tuned[tt::TK_N] = {0, 0, 0};  // plans per autotuned kernel choice
};

namespace tt {
// Batch support (tt_batch.cu composes the instances' captured beta-step graphs
// into one parent graph).  rho_graph_current: rho's captured step graph can be
// replayed for dtau as it is (not profiling, nothing replaced since the
// capture).  rho_account_replays: the host bookkeeping of n replays of that
// graph launched elsewhere on stream st; call with before = true ahead of the
// launches (opens the statistics window) and before = false after them.
bool rho_graph_current(const tt_rho* rho, double dtau);
void rho_account_replays(tt_rho* rho, double dtau, int n, cudaStream_t st, bool before);
}  // namespace tt
