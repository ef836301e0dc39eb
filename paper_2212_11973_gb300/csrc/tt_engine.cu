// tanTRG engine: state management, Lanczos driver, 1-TDVP sweeps, 2-TDVP
// growth, measurements and the C ABI of include/tantrg.h.
//
// Algorithm (Supplement, "Procedure of 1-TDVP"): left-to-right, for each site
// i: A_i <- exp(-tau H1) A_i (Lanczos); A_i = A_i^L S_i (QR); build L_{i+1};
// S_i <- exp(+tau H0) S_i (Lanczos); A_{i+1} <- S_i A_{i+1}; no bond step after
// the last site; then the mirror sweep right-to-left.  Growth ("2-TDVP in the
// initial stage"): two-site exponentials, SVD truncation, backward one-site
// steps.  All numerics run on the GPU; the host only compiles plans and, in the
// untimed growth stage, chooses the truncation from the singular values.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>

#include <cudaTypedefs.h>

#include "tt_engine.h"

using namespace tt;

namespace tt {

static const double BREAKDOWN_TOL = 1e-13;
static const double DEGEN_ABS = 1e-14;

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw Err{TT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}
#define CK(x) check_cuda((x), #x)

void* dalloc(tt_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->has_cb) {
    p = c->cb.alloc(bytes, (void*)c->st, c->cb.user);
    if (!p) throw Err{TT_ERR_OOM, "allocator callback returned NULL for " + std::to_string(bytes) + " bytes"};
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, c->st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Err{TT_ERR_OOM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e)};
    }
  }
  return p;
}

void dfree(tt_ctx* c, DBuf& b) {
  if (!b.p) return;
  if (c->has_cb) c->cb.free(b.p, b.bytes, (void*)c->st, c->cb.user);
  else cudaFreeAsync(b.p, c->st);
  b.p = nullptr;
  b.bytes = 0;
}

void ensure(tt_ctx* c, DBuf& b, size_t bytes) {
  if (bytes <= b.bytes && b.p) return;
  if (b.p) ++c->buf_gen;
  dfree(c, b);
  size_t want = std::max<size_t>(bytes, 256);
  b.p = dalloc(c, want);
  b.bytes = want;
}

template <class T>
static size_t align_up(size_t x) {
  return (x + 255) / 256 * 256 + 0 * sizeof(T);
}

void upload(tt_ctx* c, const GemmPlan& p, DevGemmBuf& o) {
  std::vector<GTile> tiles;
  std::vector<std::pair<double, int>> order;
  for (size_t g = 0; g < p.groups.size(); ++g) {
    double k = 0;
    for (int s = p.groups[g].seg0; s < p.groups[g].seg1; ++s) k += p.segs[s].K;
    order.push_back({-k, (int)g});
  }
  std::stable_sort(order.begin(), order.end());
  for (auto& og : order) {
    const GGroup& g = p.groups[og.second];
    for (int m0 = 0; m0 < g.M; m0 += 64)
      for (int n0 = 0; n0 < g.N; n0 += 64) tiles.push_back(GTile{og.second, m0, n0, 0});
  }
  size_t bg = align_up<GGroup>(p.groups.size() * sizeof(GGroup));
  size_t bsg = align_up<GSeg>(p.segs.size() * sizeof(GSeg));
  size_t bt = align_up<GTile>(tiles.size() * sizeof(GTile));
  ensure(c, o.buf, bg + bsg + bt);
  char* base = (char*)o.buf.p;
  if (!p.groups.empty()) CK(cudaMemcpyAsync(base, p.groups.data(), p.groups.size() * sizeof(GGroup), cudaMemcpyHostToDevice, c->st));
  if (!p.segs.empty()) CK(cudaMemcpyAsync(base + bg, p.segs.data(), p.segs.size() * sizeof(GSeg), cudaMemcpyHostToDevice, c->st));
  if (!tiles.empty()) CK(cudaMemcpyAsync(base + bg + bsg, tiles.data(), tiles.size() * sizeof(GTile), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  o.d.groups = (GGroup*)base;
  o.d.segs = (GSeg*)(base + bg);
  o.d.tiles64 = (GTile*)(base + bg + bsg);
  o.d.ngroups = (int)p.groups.size();
  o.d.nsegs = (int)p.segs.size();
  o.d.ntiles64 = (int)tiles.size();
  o.d.flops = p.flops;
  o.host = p;
  o.checked = false;
  o.tc_checked = o.tc_ok = false;
  o.ntiles128 = o.ntilesp = 0;
  o.choice = -1;
  for (int i = 0; i < 8; ++i) { o.key_p[i] = nullptr; o.key_lo[i] = 0; }
}

void upload(tt_ctx* c, const GatherPlan& p, DevGatherBuf& o) {
  size_t bi = align_up<GItem>(p.items.size() * sizeof(GItem));
  size_t bc = align_up<GContrib>(p.contribs.size() * sizeof(GContrib));
  ensure(c, o.buf, bi + bc);
  char* base = (char*)o.buf.p;
  if (!p.items.empty()) CK(cudaMemcpyAsync(base, p.items.data(), p.items.size() * sizeof(GItem), cudaMemcpyHostToDevice, c->st));
  if (!p.contribs.empty()) CK(cudaMemcpyAsync(base + bi, p.contribs.data(), p.contribs.size() * sizeof(GContrib), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  o.d.items = (GItem*)base;
  o.d.contribs = (GContrib*)(base + bi);
  o.d.nitems = (int)p.items.size();
  o.d.elems = p.elems;
  o.host = p;
  o.checked = false;
}

void upload(tt_ctx* c, const CopyPlan& p, DevCopyBuf& o) {
  ensure(c, o.buf, p.items.size() * sizeof(CItem));
  if (!p.items.empty()) CK(cudaMemcpyAsync(o.buf.p, p.items.data(), p.items.size() * sizeof(CItem), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  o.d.items = (CItem*)o.buf.p;
  o.d.nitems = (int)p.items.size();
  o.d.maxtiles = 0;
  for (const CItem& it : p.items)
    o.d.maxtiles = std::max<int64_t>(o.d.maxtiles, (int64_t)((it.rows + 31) / 32) * ((it.cols + 31) / 32));
  o.host = p;
  o.checked = false;
}

void release(tt_ctx* c, DevGemmBuf& o) {
  dfree(c, o.buf);
  dfree(c, o.maps);
  dfree(c, o.tiles128);
  dfree(c, o.tilesp);
  o.d = DevGemm();
  o.host = GemmPlan();
  o.checked = o.tc_checked = o.tc_ok = false;
  o.ntiles128 = o.ntilesp = 0;
  o.choice = -1;
  for (int i = 0; i < 8; ++i) { o.key_p[i] = nullptr; o.key_lo[i] = 0; }
}
void release(tt_ctx* c, DevGatherBuf& o) { dfree(c, o.buf); o.d = DevGather(); o.host = GatherPlan(); o.checked = false; }
void release(tt_ctx* c, DevCopyBuf& o) { dfree(c, o.buf); o.d = DevCopy(); o.host = CopyPlan(); o.checked = false; }

void upload(tt_ctx* c, const DigitPlan& p, DevDigitBuf& o) {
  ensure(c, o.buf, p.items.size() * sizeof(DItem) + 16);
  if (!p.items.empty())
    CK(cudaMemcpyAsync(o.buf.p, p.items.data(), p.items.size() * sizeof(DItem), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  o.d.items = (DItem*)o.buf.p;
  o.d.nitems = (int)p.items.size();
  o.d.maxgroups = 0;
  for (const DItem& it : p.items) o.d.maxgroups = std::max(o.d.maxgroups, (it.rows + 31) / 32);
  o.host = p;
}
void release(tt_ctx* c, DevDigitBuf& o) { dfree(c, o.buf); o.d = DevDigit(); o.host = DigitPlan(); }

static void check_ref(Ref r, int64_t last, const Caps& c, const char* what, const char* op) {
  int slot = (int)(r >> 56);
  int64_t off = (int64_t)(r & 0x00FFFFFFFFFFFFFFull);
  if (slot < 0 || slot > 7 || c.n[slot] < 0 || off < 0 || last < off || last >= c.n[slot])
    throw Err{TT_ERR_STATE, std::string("plan bounds check failed (") + what + ", " + op + "): slot " +
                                std::to_string(slot) + " offset " + std::to_string(off) + " last " + std::to_string(last) +
                                " capacity " + std::to_string(slot >= 0 && slot < 8 ? c.n[slot] : -2)};
}

void check_plan(const GemmPlan& p, const Caps& c, const char* what) {
  for (const GGroup& g : p.groups) {
    if (g.M <= 0 || g.N <= 0) continue;
    if (g.ldc < g.N) throw Err{TT_ERR_STATE, std::string("bad ldc in ") + what};
    int64_t off = (int64_t)(g.C & 0x00FFFFFFFFFFFFFFull);
    check_ref(g.C, off + (int64_t)(g.M - 1) * g.ldc + g.N - 1, c, what, "C");
    for (int si = g.seg0; si < g.seg1; ++si) {
      const GSeg& s = p.segs[si];
      if (s.K <= 0) continue;
      int64_t ao = (int64_t)(s.A & 0x00FFFFFFFFFFFFFFull), bo = (int64_t)(s.B & 0x00FFFFFFFFFFFFFFull);
      int64_t alast = s.tA ? ao + (int64_t)(s.K - 1) * s.lda + g.M - 1 : ao + (int64_t)(g.M - 1) * s.lda + s.K - 1;
      int64_t blast = s.tB ? bo + (int64_t)(g.N - 1) * s.ldb + s.K - 1 : bo + (int64_t)(s.K - 1) * s.ldb + g.N - 1;
      if ((s.tA ? s.lda < g.M : s.lda < s.K) || (s.tB ? s.ldb < s.K : s.ldb < g.N))
        throw Err{TT_ERR_STATE, std::string("bad leading dimension in ") + what};
      check_ref(s.A, alast, c, what, "A");
      check_ref(s.B, blast, c, what, "B");
    }
  }
}

// digit exponents of a GEMM plan: ex = capacity per slot of the exponent
// region (which starts after the four levels, i.e. at 4 * level size)
void check_exps(const GemmPlan& p, const Caps& ex, const char* what) {
  for (const GGroup& g : p.groups) {
    if (g.M <= 0 || g.N <= 0) continue;
    for (int si = g.seg0; si < g.seg1; ++si) {
      const GSeg& s = p.segs[si];
      if (s.K <= 0) continue;
      if (s.eas <= 0 || s.ebs <= 0) throw Err{TT_ERR_STATE, std::string("missing digit exponents in ") + what};
      const int64_t ao = (int64_t)(s.eA & 0x00FFFFFFFFFFFFFFull), bo = (int64_t)(s.eB & 0x00FFFFFFFFFFFFFFull);
      check_ref(s.eA, ao + (int64_t)(g.M - 1) * s.eas, ex, what, "exponents of A");
      check_ref(s.eB, bo + (int64_t)(g.N - 1) * s.ebs, ex, what, "exponents of B");
    }
  }
}

void check_plan(const DigitPlan& p, const Caps& c, const Caps& ex, const char* what) {
  for (const DItem& it : p.items) {
    if (it.rows <= 0 || it.cols <= 0) continue;
    const int64_t so = (int64_t)(it.src & 0x00FFFFFFFFFFFFFFull), d = (int64_t)(it.dst & 0x00FFFFFFFFFFFFFFull),
                  eo = (int64_t)(it.e & 0x00FFFFFFFFFFFFFFull);
    check_ref(it.src, so + (int64_t)(it.rows - 1) * it.s_r + (int64_t)(it.cols - 1) * it.s_k, c, what, "src");
    check_ref(it.dst, d + (int64_t)(it.rows - 1) * it.dst_rs + it.cols - 1, c, what, "dst");
    check_ref(it.e, eo + (int64_t)(it.rows - 1) * it.e_rs, ex, what, "exponents");
    if (it.cols > tcz_max_k()) throw Err{TT_ERR_INVALID_ARG, std::string("exact split: a digit row longer than ") +
                                                               std::to_string(tcz_max_k()) + " in " + what};
  }
}

void check_plan(const GatherPlan& p, const Caps& c, const char* what) {
  for (const GItem& it : p.items) {
    if (it.rows <= 0 || it.cols <= 0) continue;
    int64_t o = (int64_t)(it.dst & 0x00FFFFFFFFFFFFFFull);
    check_ref(it.dst, o + (int64_t)(it.rows - 1) * it.dst_rs + it.cols - 1, c, what, "dst");
    for (int k = it.c0; k < it.c1; ++k) {
      const GContrib& cb = p.contribs[k];
      int64_t so = (int64_t)(cb.src & 0x00FFFFFFFFFFFFFFull);
      check_ref(cb.src, so + (int64_t)(it.rows - 1) * cb.src_rs + it.cols - 1, c, what, "src");
    }
  }
}

void check_plan(const CopyPlan& p, const Caps& c, const char* what) {
  for (const CItem& it : p.items) {
    if (it.rows <= 0 || it.cols <= 0) continue;
    int64_t so = (int64_t)(it.src & 0x00FFFFFFFFFFFFFFull), d = (int64_t)(it.dst & 0x00FFFFFFFFFFFFFFull);
    check_ref(it.src, so + (int64_t)(it.rows - 1) * it.src_rs + (int64_t)(it.cols - 1) * it.src_cs, c, what, "src");
    check_ref(it.dst, d + (int64_t)(it.rows - 1) * it.dst_rs + (int64_t)(it.cols - 1) * it.dst_cs, c, what, "dst");
  }
}

}  // namespace tt

// ===========================================================================
// engine internals
// ===========================================================================
namespace {

Caps caps(std::initializer_list<std::pair<int, int64_t>> l) {
  Caps c;
  for (auto& kv : l) c.n[kv.first] = kv.second;
  return c;
}

struct Eng {
  tt_rho* r;
  tt_ctx* c;
  cudaStream_t st;
  explicit Eng(tt_rho* rho) : r(rho), c(rho->ctx), st(rho->ctx->st) {}

  const Mpo& M() const { return r->mpo->mpo; }
  bool mixed() const { return r->nsplit > 0; }
  // kernel of the FP64 GEMM plans while set (the environment updates of the
  // mixed modes): 0 FP64 FMA, 1 the exact-accumulation split (tt_ozaki.cu),
  // 2 double-float on the FP32 pipe (gemm_df_kernel)
  int f64_kernel = 0;
  struct OzScope {
    Eng& e;
    int saved;
    OzScope(Eng& eng, int k) : e(eng), saved(eng.f64_kernel) { e.f64_kernel = k; }
    ~OzScope() { e.f64_kernel = saved; }
  };
  double* dptr(DBuf& b) { return (double*)b.p; }

  void count(int n = 1) { r->launches_acc += n; }

  // ---- structure ----------------------------------------------------------
  void drop_graph() {
    if (r->graph) {
      cudaGraphExecDestroy(r->graph);
      r->graph = nullptr;
    }
    if (r->graph_tmpl) {
      cudaGraphDestroy(r->graph_tmpl);
      r->graph_tmpl = nullptr;
    }
    ++r->graph_gen;
  }

  void invalidate_bond(int k) {
    drop_graph();
    // plans touching bond k
    if (k - 1 >= 0) r->sp64[k - 1].valid = false;
    if (k < r->N) r->sp64[k].valid = false;
    if (k - 1 >= 0) { r->sp[k - 1].valid = false; r->qrl[k - 1].valid = false; r->lqr[k - 1].valid = false; r->meas[k - 1].valid = false; }
    if (k < r->N) { r->sp[k].valid = false; r->qrl[k].valid = false; r->lqr[k].valid = false; r->meas[k].valid = false; }
    r->bp[k].valid = false;
    r->esplit_ok[k] = 0;
    for (int j = std::max(0, k - 2); j <= std::min(r->N - 1, k + 1); ++j) { r->absl_ok[j] = 0; r->absr_ok[j] = 0; }
  }

  void relayout(int j) { r->lay[j] = make_site_layout(r->bond[j], r->bond[j + 1], M().ls); }

  // Switch the contraction precision (growth and linear stage may differ):
  // invalidates the precision-dependent plans and re-splits the environments
  // that are valid with the centre on site 0 (L[0], R[1..N]).
  void set_precision(int prec) {
    const int ns = (prec == 1) ? 2 : (prec == 2 ? 3 : (prec == 3 ? 4 : 0));
    const bool ex = prec == 3;
    if (ns == r->nsplit && ex == r->exact) return;
    drop_graph();
    r->exact = ex;
    r->nsplit = ns;
    for (auto& sp : r->sp) sp.valid = false;
    for (auto& bp : r->bp) bp.valid = false;
    for (auto& e : r->esplit_ok) e = 0;
    if (ns == 0) return;
    const int N = r->N;
    if (r->L[0].p) { ensure_env(r->L, r->Lsp, r->Lsize, 0); split_env(r->L, r->Lsp, r->Lsize, 0); }
    for (int k = 1; k <= N; ++k)
      if (r->R[k].p) { ensure_env(r->R, r->Rsp, r->Rsize, k); split_env(r->R, r->Rsp, r->Rsize, k); }
  }

  void ensure_vec_capacity() {
    int64_t nmax = 1;
    for (int j = 0; j < r->N; ++j) nmax = std::max(nmax, r->lay[j].size);
    for (int k = 0; k <= r->N; ++k) nmax = std::max(nmax, make_bondmat_layout(r->bond[k]).size);
    if (nmax > r->ldq) {
      int64_t cap = nmax + nmax / 4 + 64;
      r->ldq = cap;
      ensure(c, r->Qk, (size_t)cap * r->opts.krylov_dim * sizeof(double));
      ensure(c, r->W, (size_t)cap * sizeof(double));
      ensure(c, r->tmp, (size_t)cap * sizeof(double));
      ensure(c, r->Xn, (size_t)cap * 4 * 2);
    }
  }

  void ensure_site_buf(int j) { ensure(c, r->A[j], (size_t)r->lay[j].size * sizeof(double)); }

  // ---- plans --------------------------------------------------------------
  // FP64 plans of site j whatever the precision (the measurement's energy)
  SiteDev& site_plan_fp64(int j) {
    if (!mixed()) return site_plan(j);
    SiteDev& s = r->sp64[j];
    if (s.valid) return s;
    const Mpo& m = M();
    s.h = build_site_plan(r->bond[j], r->bond[j + 1], m.ls, m.site[j].terms, m.chan[j], m.chan[j + 1], false);
    validate_site(s.h, r->bond[j], r->bond[j + 1], m.chan[j], m.chan[j + 1], false);
    upload(c, s.h.s1, s.s1);
    upload(c, s.h.s2, s.s2);
    upload(c, s.h.s3, s.s3);
    upload(c, s.h.s3l, s.s3l);
    upload(c, s.h.r1, s.r1);
    upload(c, s.h.r2, s.r2);
    upload(c, s.h.r3, s.r3);
    ensure(c, r->T1, (size_t)std::max(s.h.t1_size, s.h.u1_size) * 8);
    ensure(c, r->T2, (size_t)std::max(s.h.t2_size, s.h.u2_size) * 8);
    s.valid = true;
    return s;
  }
  // environment updates in split-BF16 (else FP64 plans, also in mixed mode)
  bool env_mixed() const { return mixed() && !r->exact && r->opts.env_precision == -1; }
  // kernel of the FP64 environment plans (f64_kernel values): the exact-
  // accumulation split by default in every split mode, double-float with
  // env_precision 2, FP64 FMA with 1
  int env_f64_kernel() const {
    if (!mixed() || env_mixed()) return 0;
    return r->opts.env_precision == 0 ? 1 : (r->opts.env_precision == 2 ? 2 : 0);
  }
  // bytes per element of a split slot (levels, plus the int16 row exponents
  // of the digit layouts, never more rows than elements)
  size_t split_bytes() const { return (size_t)2 * (r->nsplit + (r->exact ? 1 : 0)); }
  SiteDev& site_plan(int j) {
    SiteDev& s = r->sp[j];
    if (s.valid) return s;
    const Mpo& m = M();
    s.h = build_site_plan(r->bond[j], r->bond[j + 1], m.ls, m.site[j].terms, m.chan[j], m.chan[j + 1], mixed(),
                          r->exact);
    validate_site(s.h, r->bond[j], r->bond[j + 1], m.chan[j], m.chan[j + 1], mixed(), r->exact);
    upload(c, s.h.xsplit, s.xs);
    upload(c, s.h.xdig, s.xd);
    if (mixed()) ensure(c, r->Xs, (size_t)std::max<int64_t>(s.h.xt_size, 1) * split_bytes());
    upload(c, s.h.s1, s.s1);
    upload(c, s.h.s2, s.s2);
    upload(c, s.h.s3, s.s3);
    upload(c, s.h.s3l, s.s3l);
    upload(c, s.h.r1, s.r1);
    upload(c, s.h.r2, s.r2);
    upload(c, s.h.r3, s.r3);
    ensure(c, r->T1, (size_t)std::max(s.h.t1_size, s.h.u1_size) * 8);
    // FP64, split levels or digit levels plus exponents
    ensure(c, r->T2, (size_t)std::max(s.h.t2_size, s.h.u2_size) * std::max<size_t>(8, split_bytes()));
    s.valid = true;
    return s;
  }

  static void validate_site(const SitePlanHost& h, const Bond& BL, const Bond& BR, const std::vector<Q>& chl,
                            const std::vector<Q>& chr, bool mx, bool ex = false) {
    const int64_t n = h.lay.size, el = make_env_layout(BL, chl).size, er = make_env_layout(BR, chr).size;
    const int64_t elo = make_env_layout(BL, chl, mx).size, ero = make_env_layout(BR, chr, mx).size;
    const int sx = mx ? S_AUX : S_X;  // natural-layout x operand
    check_plan(h.s1, caps({{S_X, mx ? h.xt_size : n}, {S_L, elo}, {S_T1, h.t1_size}}), "S1");
    check_plan(h.s2, caps({{S_T1, h.t1_size}, {S_T2, h.t2_size}}), "S2");
    check_plan(h.s3, caps({{S_T2, h.t2_size}, {S_R, ero}, {S_Y, n}}), "S3");
    check_plan(h.s3l, caps({{sx, n}, {S_T2, h.t2_size}, {S_Y, er}}), "S3L");
    check_plan(h.r1, caps({{sx, n}, {S_R, ero}, {S_T1, h.u1_size}}), "R1");
    check_plan(h.r2, caps({{S_T1, h.u1_size}, {S_T2, h.u2_size}}), "R2");
    check_plan(h.r3, caps({{sx, n}, {S_T2, h.u2_size}, {S_Y, el}}), "R3");
    if (mx) check_plan(h.xsplit, caps({{S_X, n}, {S_Y, h.xt_size}}), "x split");
    if (ex) {
      // exponent regions: after the four levels, one int16 per digit row
      const EnvLayout ELo = make_env_layout(BL, chl, true), ERo = make_env_layout(BR, chr, true);
      int64_t lrows = 0, rrows = 0, xrows = 0, t2e = 0;
      for (int64_t q : ELo.rows) lrows += q;
      for (int64_t q : ERo.rows) rrows += q;
      for (const SiteBlock& b : h.lay.blk) xrows += (int64_t)b.m * b.dr;
      for (const GItem& it : h.s2.items) t2e = std::max<int64_t>(t2e, (int64_t)(it.e & 0x00FFFFFFFFFFFFFFull) +
                                                                           (int64_t)(it.rows - 1) * it.e_rs + 1);
      const Caps ex1 = caps({{S_L, 4 * elo + lrows}, {S_X, 4 * h.xt_size + xrows}});
      const Caps ex3 = caps({{S_T2, std::max<int64_t>(t2e, 4 * h.t2_size + 1)}, {S_R, 4 * ero + rrows}});
      check_exps(h.s1, ex1, "S1 exponents");
      check_exps(h.s3, ex3, "S3 exponents");
      check_plan(h.xdig, caps({{S_X, n}, {S_Y, h.xt_size}}), caps({{S_Y, 4 * h.xt_size + xrows}}), "x digits");
      check_plan(h.s2, caps({{S_T1, h.t1_size}, {S_T2, h.t2_size}}), "S2");
      if (t2e > 4 * h.t2_size + h.t2_size) throw Err{TT_ERR_STATE, "T2 exponents exceed the slot"};
      for (const GItem& it : h.s2.items) {
        if (it.cols > gather_digits_max_cols())
          throw Err{TT_ERR_INVALID_ARG, "exact split: a sector longer than " + std::to_string(gather_digits_max_cols())};
        if (it.c1 - it.c0 > gather_digits_max_contribs())
          throw Err{TT_ERR_INVALID_ARG, "exact split: more than " + std::to_string(gather_digits_max_contribs()) +
                                            " MPO terms feed one W-gather item"};
        // the digit gather stores column pairs (a BF16 pair per 32-bit word;
        // an odd row's last pair ends in the row's zero padding)
        if (((it.dst & 0x00FFFFFFFFFFFFFFull) | (uint64_t)it.dst_rs | (uint64_t)h.t2_size) & 1)
          throw Err{TT_ERR_STATE, "S2 digit rows not at even BF16 offsets"};
      }
    }
  }

  BondDev& bond_plan(int k) {
    BondDev& b = r->bp[k];
    if (b.valid) return b;
    b.h = build_bond_plan(r->bond[k], M().chan[k], mixed(), r->exact);
    {
      int64_t e = make_env_layout(r->bond[k], M().chan[k], mixed()).size;
      const int64_t xcap = mixed() ? b.h.xt_size : b.h.mat.size, tcap = mixed() ? b.h.tp_size : b.h.t_size;
      check_plan(b.h.b1, caps({{S_X, xcap}, {S_L, e}, {S_T1, b.h.t_size}}), "B1");
      check_plan(b.h.b2, caps({{S_T2, tcap}, {S_R, e}, {S_Y, b.h.mat.size}}), "B2");
      if (mixed()) {
        check_plan(b.h.xsplit, caps({{S_X, b.h.mat.size}, {S_Y, b.h.xt_size}}), "B x split");
        check_plan(b.h.tsplit, caps({{S_T1, b.h.t_size}, {S_Y, b.h.tp_size}}), "B T split");
      }
      if (r->exact) {
        int64_t erows = 0, xrows = 0, trows = 0;
        for (int64_t q : make_env_layout(r->bond[k], M().chan[k], true).rows) erows += q;
        for (int d : r->bond[k].dim) xrows += d;
        for (const DItem& it : b.h.tdig.items) trows += it.rows;
        check_exps(b.h.b1, caps({{S_L, 4 * e + erows}, {S_X, 4 * b.h.xt_size + xrows}}), "B1 exponents");
        check_exps(b.h.b2, caps({{S_T2, 4 * b.h.tp_size + trows}, {S_R, 4 * e + erows}}), "B2 exponents");
        check_plan(b.h.xdig, caps({{S_X, b.h.mat.size}, {S_Y, b.h.xt_size}}), caps({{S_Y, 4 * b.h.xt_size + xrows}}),
                   "B x digits");
        check_plan(b.h.tdig, caps({{S_T1, b.h.t_size}, {S_Y, b.h.tp_size}}), caps({{S_Y, 4 * b.h.tp_size + trows}}),
                   "B T digits");
      }
    }
    upload(c, b.h.b1, b.b1);
    upload(c, b.h.b2, b.b2);
    if (mixed()) {
      upload(c, b.h.xsplit, b.xs);
      upload(c, b.h.tsplit, b.ts);
      upload(c, b.h.xdig, b.xd);
      upload(c, b.h.tdig, b.td);
      ensure(c, r->Xs, (size_t)std::max<int64_t>(b.h.xt_size, 1) * split_bytes());
      ensure(c, r->T2, (size_t)std::max<int64_t>(b.h.tp_size, 1) * split_bytes());
    }
    ensure(c, r->T1, (size_t)b.h.t_size * 8);
    ensure(c, r->T2, (size_t)b.h.t_size * 8);
    b.valid = true;
    return b;
  }

  QrDev& qr_plan(int j, bool left) {
    QrDev& q = left ? r->qrl[j] : r->lqr[j];
    if (q.valid) return q;
    q.h = left ? build_qr_left(r->lay[j], r->bond[j + 1]) : build_lq_right(r->lay[j], r->bond[j], false);
    if (!left) {
      // scatter Q'^T into the (unchanged) layout
      const SiteLayout& S = r->lay[j];
      size_t bi = 0;
      for (int l = 0; l < r->bond[j].nsec(); ++l) {
        const QrJob& J = q.h.jobs[l];
        int k = q.h.new_dim[l];
        for (; bi < q.h.scatter_blocks.size() && S.blk[q.h.scatter_blocks[bi].first].l == l; ++bi) {
          const SiteBlock& b = S.blk[q.h.scatter_blocks[bi].first];
          int C = b.m * b.dr;
          q.h.scatter.items.push_back(
              CItem{mkref(S_AUX2, J.q + q.h.scatter_blocks[bi].second), mkref(S_Y, b.off), J.m, 1, C, 1, k, C});
        }
      }
    }
    {
      const int64_t n = r->lay[j].size;
      check_plan(q.h.gather, caps({{S_X, n}, {S_AUX2, q.h.ws_size}}), "QR gather");
      check_plan(q.h.scatter, caps({{S_AUX2, q.h.ws_size}, {S_Y, n}}), "QR scatter");
      check_plan(q.h.rout, caps({{S_AUX2, q.h.ws_size}, {S_AUX, q.h.s_size}}), "QR R");
      for (const QrJob& J : q.h.jobs)
        if (J.a + (int64_t)J.m * J.n > q.h.ws_size || J.q + (int64_t)J.m * J.n > q.h.ws_size ||
            J.r + (int64_t)J.n * J.n > q.h.ws_size || J.n > 2048)
          throw Err{TT_ERR_STATE, "QR job outside the workspace or wider than 2048"};
    }
    ensure(c, q.jobs, q.h.jobs.size() * sizeof(QrJob));
    if (!q.h.jobs.empty())
      CK(cudaMemcpyAsync(q.jobs.p, q.h.jobs.data(), q.h.jobs.size() * sizeof(QrJob), cudaMemcpyHostToDevice, st));
    upload(c, q.h.gather, q.gather);
    upload(c, q.h.scatter, q.scatter);
    upload(c, q.h.rout, q.rout);
    int64_t wsz = q.h.ws_size;
    if (r->use_cholqr) {
      CholQrPlan cp = build_cholqr(q.h.jobs, q.h.ws_size);
      wsz = cp.ws_end;
      const Caps cw = caps({{S_AUX2, wsz}});
      for (int p = 0; p < 3; ++p) {
        check_plan(cp.gram[p], cw, "CholQR gram");
        check_plan(cp.app[p], cw, "CholQR apply");
        upload(c, cp.gram[p], q.gram[p]);
        upload(c, cp.app[p], q.app[p]);
        for (const CholJob& J : cp.cj[p])
          if (J.g + (int64_t)J.parts * J.n * J.n > wsz || J.parts < 1 || J.r + (int64_t)J.n * J.n > wsz ||
              J.ri + (int64_t)J.n * J.n > wsz || J.pk < 0 || J.pk + (int64_t)J.n * (J.n + 1) / 2 > wsz)
            throw Err{TT_ERR_STATE, "Cholesky job outside the workspace"};
        q.ncj[p] = (int)cp.cj[p].size();
        q.maxn[p] = 0;
        for (const CholJob& cj : cp.cj[p]) q.maxn[p] = std::max(q.maxn[p], cj.n);
        ensure(c, q.cjobs[p], cp.cj[p].size() * sizeof(CholJob) + 16);
        if (!cp.cj[p].empty())
          CK(cudaMemcpyAsync(q.cjobs[p].p, cp.cj[p].data(), cp.cj[p].size() * sizeof(CholJob), cudaMemcpyHostToDevice,
                             st));
      }
      check_plan(cp.tt, cw, "CholQR T");
      check_plan(cp.rf, cw, "CholQR R");
      upload(c, cp.tt, q.tt);
      upload(c, cp.rf, q.rf);
      ensure(c, q.fail, q.h.jobs.size() * sizeof(int) + 16);
    }
    ensure(c, r->ws, (size_t)wsz * 8);
    ensure(c, r->Sb, (size_t)q.h.s_size * 8);
    q.valid = true;
    return q;
  }

  DevGemmBuf& absorb_left_plan(int j) {  // into site j from the bond on its left
    if (!r->absl_ok[j]) {
      std::vector<int> ident(r->bond[j].nsec());
      std::iota(ident.begin(), ident.end(), 0);
      BondMatLayout bm = make_bondmat_layout(r->bond[j]);
      GemmPlan g = build_absorb_left(r->lay[j], r->lay[j], r->bond[j], r->bond[j], bm.off, ident);
      check_plan(g, caps({{S_X, r->lay[j].size}, {S_AUX, bm.size}, {S_Y, r->lay[j].size}}), "absorb L");
      upload(c, g, r->absl[j]);
      r->absl_ok[j] = 1;
    }
    return r->absl[j];
  }
  DevGemmBuf& absorb_right_plan(int j) {  // into site j from the bond on its right
    if (!r->absr_ok[j]) {
      std::vector<int> ident(r->bond[j + 1].nsec());
      std::iota(ident.begin(), ident.end(), 0);
      BondMatLayout bm = make_bondmat_layout(r->bond[j + 1]);
      GemmPlan g = build_absorb_right(r->lay[j], r->lay[j], r->bond[j + 1], r->bond[j + 1], bm.off, ident);
      check_plan(g, caps({{S_X, r->lay[j].size}, {S_AUX, bm.size}, {S_Y, r->lay[j].size}}), "absorb R");
      upload(c, g, r->absr[j]);
      r->absr_ok[j] = 1;
    }
    return r->absr[j];
  }

  // ---- GEMM / gather dispatch ---------------------------------------------
  // Event pair around a launch or a whole phase; pairs may nest.  Returns the
  // pair's index (or -1 when profiling is off).
  long prof_begin(int kind, double flops) {
    if (!r->prof) return -1;
    std::vector<cudaEvent_t>& pool = r->capturing ? r->gpool : r->evpool;
    std::vector<int>& kinds = r->capturing ? r->gkind : r->evkind;
    size_t& used = r->capturing ? r->gused : r->evused;
    if (used + 2 > pool.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        pool.push_back(e);
        kinds.push_back(0);
      }
    }
    const long idx = (long)used;
    kinds[used] = kind;
    used += 2;
    if (r->capturing) r->graph_kind_flops[kind] += flops;
    else r->kind_flops[kind] += flops;
    record(pool[idx]);
    return idx;
  }
  void prof_end(long idx) {
    if (idx < 0) return;
    const std::vector<cudaEvent_t>& pool = r->capturing ? r->gpool : r->evpool;
    record(pool[idx + 1]);
  }
  // inside a stream capture a plain record only orders the graph; the external
  // flag makes it a record node whose time the replay writes
  void record(cudaEvent_t e) {
    if (r->capturing) CK(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
    else CK(cudaEventRecord(e, st));
  }

  // tcgen05 eligibility (K-major A and B, 16-byte aligned rows and offsets) and
  // the per-segment tensor maps for the current slot bases.
  bool prep_tc(DevGemmBuf& g, const Bases& b) {
    if (!g.tc_checked) {
      g.tc_checked = true;
      g.tc_ok = !g.host.segs.empty();
      for (const GSeg& sg : g.host.segs) {
        const int64_t oa = (int64_t)(sg.A & 0x00FFFFFFFFFFFFFFull), ob = (int64_t)(sg.B & 0x00FFFFFFFFFFFFFFull);
        if (sg.tA != 0 || sg.tB != 1 || sg.lda % 8 || sg.ldb % 8 || oa % 8 || ob % 8) g.tc_ok = false;
      }
      if (!g.tc_ok) return false;
      // tile lists of both tcgen05 kernels: 128 x 128 and 128 x 64; the
      // persistent kernel's list is ordered longest group first (more K
      // chunks), so the long tiles start in the first wave
      std::vector<GTile> tiles, tp;
      std::vector<int> chunks(g.host.groups.size(), 0);
      for (size_t gi = 0; gi < g.host.groups.size(); ++gi) {
        const GGroup& gg = g.host.groups[gi];
        for (int si = gg.seg0; si < gg.seg1; ++si) chunks[gi] += (g.host.segs[si].K + 63) / 64;
        for (int m0 = 0; m0 < gg.M; m0 += 128) {
          for (int n0 = 0; n0 < gg.N; n0 += 128) tiles.push_back(GTile{(int)gi, m0, n0, 0});
          for (int n0 = 0; n0 < gg.N; n0 += 64) tp.push_back(GTile{(int)gi, m0, n0, 0});
        }
      }
      std::stable_sort(tp.begin(), tp.end(), [&](const GTile& a, const GTile& b2) { return chunks[a.g] > chunks[b2.g]; });
      ensure(c, g.tiles128, tiles.size() * sizeof(GTile) + 16);
      ensure(c, g.tilesp, tp.size() * sizeof(GTile) + 16);
      if (!tiles.empty())
        CK(cudaMemcpyAsync(g.tiles128.p, tiles.data(), tiles.size() * sizeof(GTile), cudaMemcpyHostToDevice, st));
      if (!tp.empty()) CK(cudaMemcpyAsync(g.tilesp.p, tp.data(), tp.size() * sizeof(GTile), cudaMemcpyHostToDevice, st));
      g.ntiles128 = (int)tiles.size();
      g.ntilesp = (int)tp.size();
    }
    if (!g.tc_ok) return false;
    // the maps depend only on the slots the A and B operands live in
    unsigned used = 0;
    for (const GSeg& sg : g.host.segs) used |= (1u << (int)(sg.A >> 56)) | (1u << (int)(sg.B >> 56));
    bool same = true;
    for (int i = 0; i < 8; ++i)
      if (used & (1u << i)) same = same && g.key_p[i] == b.p[i] && g.key_lo[i] == b.lo[i];
    if (same && g.maps.p) return true;
    // a captured step must replay the uploads of the uncaptured one
    if (r->capturing) throw Err{TT_ERR_STATE, "tensor-map operands moved during graph capture"};
    // looked up once per process (thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
      cudaDriverEntryPointQueryResult q;
      void* fn = nullptr;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess) {
        cudaGetLastError();
        fn = nullptr;
      }
      return (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }();
    if (!encode) {
      g.tc_ok = false;
      return false;
    }
    const size_t nseg = g.host.segs.size();
    std::vector<CUtensorMap> maps(3 * nseg);
    std::vector<int> seg_group(nseg, 0);
    for (size_t gi = 0; gi < g.host.groups.size(); ++gi)
      for (int si = g.host.groups[gi].seg0; si < g.host.groups[gi].seg1; ++si) seg_group[si] = (int)gi;
    for (size_t si = 0; si < nseg; ++si) {
      const GSeg& sg = g.host.segs[si];
      const GGroup& gg = g.host.groups[seg_group[si]];
      for (int w = 0; w < 3; ++w) {  // A (box 64 x 128), B (64 x 128), B (64 x 64)
        const Ref ref = w == 0 ? sg.A : sg.B;
        const int sl = (int)(ref >> 56);
        const int64_t off = (int64_t)(ref & 0x00FFFFFFFFFFFFFFull);
        const long long lo = b.lo[sl];
        if (!b.p[sl] || lo % 8 || sg.K < 1) { g.tc_ok = false; return false; }
        cuuint64_t dims[3] = {(cuuint64_t)sg.K, (cuuint64_t)std::max(1, w == 0 ? gg.M : gg.N), (cuuint64_t)r->nsplit};
        cuuint64_t strides[2] = {(cuuint64_t)(w == 0 ? sg.lda : sg.ldb) * 2, (cuuint64_t)lo * 2};
        cuuint32_t box[3] = {64, (cuuint32_t)(w == 2 ? 64 : 128), 1};
        cuuint32_t estr[3] = {1, 1, 1};
        void* base = (char*)b.p[sl] + off * 2;
        CUresult cr = encode(&maps[3 * si + w], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
          if (std::getenv("TT_DEBUG"))
            std::fprintf(stderr, "[tc] tensor map encode failed (%d) seg %zu K %d ld %d lo %lld\n", (int)cr, si, sg.K,
                         w == 0 ? sg.lda : sg.ldb, lo);
          g.tc_ok = false;
          return false;
        }
      }
    }
    ensure(c, g.maps, maps.size() * sizeof(CUtensorMap) + 128);
    CK(cudaMemcpyAsync(g.maps.p, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < 8; ++i) { g.key_p[i] = b.p[i]; g.key_lo[i] = b.lo[i]; }
    return true;
  }

  // one launch of a split-BF16 plan on kernel k (tcgen05 kernels need prep_tc)
  void launch_split(DevGemmBuf& g, const Bases& b, int k) {
    if (k != TK_MMA64 && !r->tcerr.p) {
      ensure(c, r->tcerr, 16);
      CK(cudaMemsetAsync(r->tcerr.p, 0, 16, st));
    }
    if (k == TK_TC128)
      CK(launch_gemm_tc(g.d.groups, g.d.segs, (const GTile*)g.tiles128.p, g.ntiles128, g.maps.p, b, r->nsplit,
                        (int*)r->tcerr.p, c->wait_ns, st));
    else if (k == TK_TCP128X64)
      CK(launch_gemm_tcp(g.d.groups, g.d.segs, (const GTile*)g.tilesp.p, g.ntilesp, g.maps.p, b, r->nsplit,
                         (int*)r->tcerr.p, c->wait_ns, st));
    else
      CK(launch_gemm_bf16(g.d, b, r->nsplit, st));
  }

  // Tile-shape autotuner: the first uncaptured launch of a split-BF16 plan
  // times every eligible kernel (128 x 128 tcgen05, persistent 128 x 64
  // tcgen05, 64 x 64 mma.sync) with CUDA events, second of two runs each,
  // and keeps the fastest for the plan; plans of the same shape signature
  // (split levels, groups, tiles, K chunks) reuse the choice process-wide.
  // Every candidate overwrites the plan's whole output (no plan here
  // accumulates into C), and the chosen kernel runs last, so the output is
  // the chosen kernel's.  TT_GEMM=tc|tcp|mma forces one kernel.
  int tune(DevGemmBuf& g, const Bases& b, bool tc) {
    static const int forced = [] {
      const char* v = std::getenv("TT_GEMM");
      if (!v) return -1;
      if (!std::strcmp(v, "tc")) return (int)TK_TC128;
      if (!std::strcmp(v, "tcp")) return (int)TK_TCP128X64;
      if (!std::strcmp(v, "mma")) return (int)TK_MMA64;
      return -1;
    }();
    if (forced >= 0) return (forced == TK_MMA64 || tc) ? forced : (int)TK_MMA64;
    if (!tc) return TK_MMA64;
    if (r->capturing) return TK_TCP128X64;  // plans are tuned in the uncaptured step; this is a fallback
    long long chunks = 0, msum = 0, nsum = 0;
    for (const GSeg& sg : g.host.segs) chunks += (sg.K + 63) / 64;
    for (const GGroup& gg : g.host.groups) { msum += gg.M; nsum += gg.N; }
    char key[160];
    std::snprintf(key, sizeof key, "%d/%zu/%zu/%d/%lld/%lld/%lld", r->nsplit, g.host.groups.size(), g.host.segs.size(),
                  g.ntiles128, chunks, msum, nsum);
    static std::mutex mu;
    static std::map<std::string, int> cache;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = cache.find(key);
      if (it != cache.end()) return it->second;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = TK_MMA64;
    float best_ms = 1e30f;
    for (int k : {(int)TK_MMA64, (int)TK_TC128, (int)TK_TCP128X64}) {
      launch_split(g, b, k);
      CK(cudaEventRecord(e0, st));
      launch_split(g, b, k);
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_tc();
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    return best;
  }

  void gemm(DevGemmBuf& g, const Bases& b, bool use_mixed, int kind = 4) {
    if (use_mixed && r->exact) {
      if (!r->use_tc || !prep_tc(g, b))
        throw Err{TT_ERR_INVALID_ARG, "exact split: a GEMM plan is not eligible for the tcgen05 digit kernel"};
      for (const GSeg& sg : g.host.segs)
        if (sg.K > tcz_max_k())
          throw Err{TT_ERR_INVALID_ARG, "exact split: a sector longer than " + std::to_string(tcz_max_k())};
      if (!r->tcerr.p) {
        ensure(c, r->tcerr, 16);
        CK(cudaMemsetAsync(r->tcerr.p, 0, 16, st));
      }
      // one output form per launch (the digit kernel is specialised on it)
      const bool pair = !g.host.groups.empty() && (g.host.groups[0].flags & 2);
      for (const GGroup& gg : g.host.groups)
        if (((gg.flags & 2) != 0) != pair) throw Err{TT_ERR_STATE, "exact split: mixed output forms in one GEMM plan"};
      const long e = prof_begin(kind, g.d.flops);
      CK(launch_gemm_tcz(g.d.groups, g.d.segs, (const GTile*)g.tilesp.p, g.ntilesp, g.maps.p, b, (int*)r->tcerr.p,
                         c->wait_ns, pair, st));
      prof_end(e);
      count();
      return;
    }
    if (use_mixed) {
      const bool tc = r->use_tc && prep_tc(g, b);
      if (g.choice < 0 || (!tc && g.choice != TK_MMA64)) {
        g.choice = tune(g, b, tc);
        ++r->tuned[g.choice];
      }
    }
    const long e = prof_begin(kind, g.d.flops);
    if (use_mixed) {
      launch_split(g, b, g.choice);
    } else if (f64_kernel == 1) {
      CK(launch_gemm_oz(g.d, b, st));
    } else if (f64_kernel == 2) {
      CK(launch_gemm_df(g.d, b, st));
    } else {
      CK(launch_gemm_f64(g.d, b, st));
    }
    prof_end(e);
    count();
  }
  void gather_digits(const DevGatherBuf& g, const Bases& b) {
    const long e = prof_begin(3, 0);
    CK(launch_gather_digits(g.d, b, st));
    prof_end(e);
    count();
  }
  void gather(const DevGatherBuf& g, const Bases& b, int in, int out) {
    const long e = prof_begin(3, 0);
    CK(launch_gather(g.d, b, in, out, st));
    prof_end(e);
    count();
  }

  void split(const double* x, int64_t n, void* out) {
    CK(launch_split_bf16(x, n, r->nsplit, out, st));
    count();
  }

  // environment buffers
  void ensure_env(std::vector<DBuf>& v, std::vector<DBuf>& vsp, std::vector<int64_t>& sz, int k) {
    int64_t n = make_env_layout(r->bond[k], M().chan[k]).size;
    int64_t np = make_env_layout(r->bond[k], M().chan[k], true).size;
    sz[k] = n;
    (&sz == &r->Lsize ? r->Lpsize : r->Rpsize)[k] = np;
    ensure(c, v[k], (size_t)n * 8);
    if (mixed()) ensure(c, vsp[k], (size_t)std::max<int64_t>(np, 1) * split_bytes());
  }
  // FP64 environment -> split-bf16 copy with rows padded to 8 elements
  void split_env(std::vector<DBuf>& v, std::vector<DBuf>& vsp, std::vector<int64_t>& sz, int k) {
    if (!mixed()) return;
    if (!r->esplit_ok[k]) {
      const EnvLayout E = make_env_layout(r->bond[k], M().chan[k]), P = make_env_layout(r->bond[k], M().chan[k], true);
      if (r->exact) {
        DigitPlan dp = build_env_digits(r->bond[k], M().chan[k]);
        int64_t rows = 0;
        for (int64_t q : P.rows) rows += q;
        check_plan(dp, caps({{S_X, E.size}, {S_Y, P.size}}), caps({{S_Y, 4 * P.size + rows}}), "env digits");
        upload(c, dp, r->edig[k]);
      } else {
        CopyPlan cp = build_env_split(r->bond[k], M().chan[k]);
        check_plan(cp, caps({{S_X, E.size}, {S_Y, P.size}}), "env split");
        upload(c, cp, r->esplit[k]);
      }
      r->esplit_ok[k] = 1;
    }
    Bases b{};
    b.p[S_X] = v[k].p;
    b.p[S_Y] = vsp[k].p;
    b.lo[S_Y] = (&sz == &r->Lsize ? r->Lpsize : r->Rpsize)[k];
    if (r->exact) CK(launch_digit_copy(r->edig[k].d, b, st));
    else CK(launch_split_copy(r->esplit[k].d, b, r->nsplit, st));
    count();
  }
  // x -> transposed padded split (or digit) copy for S1's B operand (Xs)
  void split_x_transposed(SiteDev& s, const double* x) {
    Bases b{};
    b.p[S_X] = (void*)x;
    b.p[S_Y] = r->Xs.p;
    b.lo[S_Y] = s.h.xt_size;
    if (r->exact) CK(launch_digit_copy(s.xd.d, b, st));
    else CK(launch_split_copy(s.xs.d, b, r->nsplit, st));
    count();
  }

  static void need(const DBuf& b, int64_t bytes, const char* what) {
    if (!b.p || (int64_t)b.bytes < bytes)
      throw Err{TT_ERR_STATE, std::string("buffer too small for ") + what + ": " + std::to_string(b.bytes) + " < " +
                                  std::to_string(bytes)};
  }
  void need_site(int j, const SiteDev& s, bool left_env_in, bool right_env_in) {
    const int64_t el = mixed() ? (int64_t)split_bytes() : 8;
    if (left_env_in) { need(r->L[j], r->Lsize[j] * 8, "L"); if (mixed()) need(r->Lsp[j], r->Lpsize[j] * el, "Lsp"); }
    if (right_env_in) { need(r->R[j + 1], r->Rsize[j + 1] * 8, "R"); if (mixed()) need(r->Rsp[j + 1], r->Rpsize[j + 1] * el, "Rsp"); }
    if (mixed() && s.h.xt_size > 0) need(r->Xs, s.h.xt_size * el, "Xs");  // split-BF16 plans only
    if (left_env_in && r->Lsize[j] != make_env_layout(r->bond[j], M().chan[j]).size) throw Err{TT_ERR_STATE, "stale L"};
    if (right_env_in && r->Rsize[j + 1] != make_env_layout(r->bond[j + 1], M().chan[j + 1]).size) throw Err{TT_ERR_STATE, "stale R"};
    need(r->T1, std::max(s.h.t1_size, s.h.u1_size) * 8, "T1");
    need(r->T2, std::max(s.h.t2_size, s.h.u2_size) * 8, "T2");
    need(r->W, s.h.lay.size * 8, "W");
    need(r->Xn, s.h.lay.size * 2 * std::max(r->nsplit, 1), "Xn");
    if (r->ldq < s.h.lay.size) throw Err{TT_ERR_STATE, "Krylov capacity"};
  }

  // ---- applies ------------------------------------------------------------
  // y = H^(1)_j x   (x, y device FP64 in the site-j layout)
  void apply_site(int j, const double* x, double* y, bool force_fp64 = false) {
    SiteDev& s = force_fp64 ? site_plan_fp64(j) : site_plan(j);
    need_site(j, s, true, true);
    Bases b{};
    b.p[S_Y] = y;
    b.p[S_T1] = r->T1.p;
    b.p[S_T2] = r->T2.p;
    if (mixed() && !force_fp64) {
      split_x_transposed(s, x);
      b.p[S_X] = r->Xs.p; b.lo[S_X] = s.h.xt_size;
      b.p[S_L] = r->Lsp[j].p; b.lo[S_L] = r->Lpsize[j];
      b.p[S_R] = r->Rsp[j + 1].p; b.lo[S_R] = r->Rpsize[j + 1];
      b.lo[S_T2] = s.h.t2_size;
      gemm(s.s1, b, true, 0);
      if (r->exact) gather_digits(s.s2, b);
      else gather(s.s2, b, 1, r->nsplit);
      gemm(s.s3, b, true, 0);
    } else {
      b.p[S_X] = (void*)x;
      b.p[S_L] = r->L[j].p;
      b.p[S_R] = r->R[j + 1].p;
      gemm(s.s1, b, false, 0);
      gather(s.s2, b, 0, 0);
      gemm(s.s3, b, false, 0);
    }
    r->heff_flops_acc += s.s1.d.flops + s.s3.d.flops;
    r->step_flops_acc += s.s1.d.flops + s.s3.d.flops;
  }

  // y = H^(0)_k S
  void apply_bond(int k, const double* x, double* y) {
    BondDev& bd = bond_plan(k);
    {
      const int64_t el = mixed() ? (int64_t)split_bytes() : 8;
      int64_t e = make_env_layout(r->bond[k], M().chan[k]).size;
      if (r->Lsize[k] != e || r->Rsize[k] != e) throw Err{TT_ERR_STATE, "stale bond environments"};
      need(r->L[k], e * 8, "L");
      need(r->R[k], e * 8, "R");
      if (mixed()) { need(r->Lsp[k], r->Lpsize[k] * el, "Lsp"); need(r->Rsp[k], r->Rpsize[k] * el, "Rsp"); }
      need(r->T1, bd.h.t_size * 8, "T1");
      need(r->T2, (mixed() ? bd.h.tp_size : bd.h.t_size) * el, "T2");
      if (mixed()) need(r->Xs, std::max<int64_t>(bd.h.xt_size, 1) * el, "Xs");
    }
    Bases b{};
    b.p[S_Y] = y;
    b.p[S_T1] = r->T1.p;
    if (mixed()) {
      {  // x -> transposed padded split (B operand of B1)
        Bases bx{};
        bx.p[S_X] = (void*)x;
        bx.p[S_Y] = r->Xs.p; bx.lo[S_Y] = bd.h.xt_size;
        if (r->exact) CK(launch_digit_copy(bd.xd.d, bx, st));
        else CK(launch_split_copy(bd.xs.d, bx, r->nsplit, st));
        count();
      }
      b.p[S_X] = r->Xs.p; b.lo[S_X] = bd.h.xt_size;
      b.p[S_L] = r->Lsp[k].p; b.lo[S_L] = r->Lpsize[k];
      b.p[S_R] = r->Rsp[k].p; b.lo[S_R] = r->Rpsize[k];
      gemm(bd.b1, b, true, 2);  // T1 in FP64
      {  // T1 -> padded split (A operand of B2)
        Bases bt{};
        bt.p[S_T1] = r->T1.p;
        bt.p[S_Y] = r->T2.p; bt.lo[S_Y] = bd.h.tp_size;
        if (r->exact) CK(launch_digit_copy(bd.td.d, bt, st));
        else CK(launch_split_copy(bd.ts.d, bt, r->nsplit, st));
        count();
      }
      b.p[S_T2] = r->T2.p; b.lo[S_T2] = bd.h.tp_size;
      gemm(bd.b2, b, true, 2);
    } else {
      b.p[S_X] = (void*)x;
      b.p[S_L] = r->L[k].p;
      b.p[S_R] = r->R[k].p;
      b.p[S_T2] = r->T1.p;
      gemm(bd.b1, b, false, 2);
      gemm(bd.b2, b, false, 2);
    }
    r->step_flops_acc += bd.b1.d.flops + bd.b2.d.flops;
  }

  // L[j+1] from L[j] and the left-canonical A_j
  void update_left_env(int j) {
    SiteDev& s = env_mixed() ? site_plan(j) : site_plan_fp64(j);
    ensure_env(r->L, r->Lsp, r->Lsize, j + 1);
    need_site(j, s, true, false);
    need(r->A[j], s.h.lay.size * 8, "A");
    Bases b{};
    b.p[S_Y] = r->L[j + 1].p;
    b.p[S_T1] = r->T1.p;
    b.p[S_T2] = r->T2.p;
    if (env_mixed()) {
      int64_t n = s.h.lay.size;
      split_x_transposed(s, dptr(r->A[j]));
      split(dptr(r->A[j]), n, r->Xn.p);
      b.p[S_X] = r->Xs.p; b.lo[S_X] = s.h.xt_size;
      b.p[S_AUX] = r->Xn.p; b.lo[S_AUX] = n;
      b.p[S_L] = r->Lsp[j].p; b.lo[S_L] = r->Lpsize[j];
      b.lo[S_T2] = s.h.t2_size;
      gemm(s.s1, b, true, 1);
      gather(s.s2, b, 1, r->nsplit);
      gemm(s.s3l, b, true, 1);
    } else {
      OzScope oz(*this, env_f64_kernel());
      b.p[S_X] = r->A[j].p;
      b.p[S_L] = r->L[j].p;
      gemm(s.s1, b, false, 1);
      gather(s.s2, b, 0, 0);
      gemm(s.s3l, b, false, 1);
    }
    split_env(r->L, r->Lsp, r->Lsize, j + 1);
    r->step_flops_acc += s.s1.d.flops + s.s3l.d.flops;
  }

  // R[j] from R[j+1] and the right-canonical A_j
  void update_right_env(int j) {
    SiteDev& s = env_mixed() ? site_plan(j) : site_plan_fp64(j);
    ensure_env(r->R, r->Rsp, r->Rsize, j);
    need_site(j, s, false, true);
    need(r->A[j], s.h.lay.size * 8, "A");
    Bases b{};
    b.p[S_Y] = r->R[j].p;
    b.p[S_T1] = r->T1.p;
    b.p[S_T2] = r->T2.p;
    if (env_mixed()) {
      int64_t n = s.h.lay.size;
      split(dptr(r->A[j]), n, r->Xn.p);
      b.p[S_AUX] = r->Xn.p; b.lo[S_AUX] = n;
      b.p[S_R] = r->Rsp[j + 1].p; b.lo[S_R] = r->Rpsize[j + 1];
      b.lo[S_T2] = s.h.u2_size;
      gemm(s.r1, b, true, 1);
      gather(s.r2, b, 1, r->nsplit);
      gemm(s.r3, b, true, 1);
    } else {
      OzScope oz(*this, env_f64_kernel());
      b.p[S_X] = r->A[j].p;
      b.p[S_R] = r->R[j + 1].p;
      gemm(s.r1, b, false, 1);
      gather(s.r2, b, 0, 0);
      gemm(s.r3, b, false, 1);
    }
    split_env(r->R, r->Rsp, r->Rsize, j);
    r->step_flops_acc += s.r1.d.flops + s.r3.d.flops;
  }

  // ---- Lanczos exponential: x <- exp(t H) x / ||.||, logscale += ln ||.|| ---
  template <class F>
  void lanczos(double* x, int64_t n, double t, F apply) {
    const int K = r->opts.krylov_dim;
    double* Q = dptr(r->Qk);
    double* w = dptr(r->W);
    double* part = dptr(r->partial);
    KrylovState* ks = (KrylovState*)r->ks.p;
    const int64_t ldq = r->ldq;
    CK(k_norm_init(x, n, part, ks, Q, st)); count(3);
    for (int k = 0; k < K; ++k) {
      apply(Q + (int64_t)k * ldq, w);
      CK(k_dots_alpha(Q, ldq, k, w, n, part, ks, st)); count(2);
      CK(k_three_term(Q, ldq, k, w, n, ks, st)); count();
      CK(k_cgs_pass(Q, ldq, k, w, n, part, ks, 0, BREAKDOWN_TOL, K, nullptr, st)); count(3);
      CK(k_cgs_pass(Q, ldq, k, w, n, part, ks, 1, BREAKDOWN_TOL, K, k + 1 < K ? Q + (int64_t)(k + 1) * ldq : nullptr, st));
      count(k + 1 < K ? 5 : 4);
    }
    CK(k_krylov_exp(ks, t, K, st)); count();
    CK(k_combine(Q, ldq, ks, x, n, part, nullptr, st)); count();
    CK(k_finish_normalise(x, n, part, ks, (RhoScalars*)r->rs.p, st)); count(2);
  }

  void site_exp(int j, double t) {
    double* x = dptr(r->A[j]);
    const long e = prof_begin(6, 0);
    lanczos(x, r->lay[j].size, t, [&](const double* q, double* y) { apply_site(j, q, y); });
    prof_end(e);
  }
  void bond_exp(int k, double t) {
    double* S = dptr(r->Sb);
    const long e = prof_begin(7, 0);
    lanczos(S, make_bondmat_layout(r->bond[k]).size, t, [&](const double* q, double* y) { apply_bond(k, q, y); });
    prof_end(e);
  }

  // ---- gauge moves ----------------------------------------------------------
  // QR of the gathered sector matrices: shifted CholeskyQR3 on all SMs, then
  // the Householder kernel for the sectors whose Cholesky failed (rank
  // deficient or too ill-conditioned), or Householder for every sector.
  void run_qr(QrDev& q, const Bases& b) {
    const long e = prof_begin(5, 0);
    run_qr_inner(q, b);
    prof_end(e);
  }
  void run_qr_inner(QrDev& q, const Bases& b) {
    if (!r->use_cholqr) {
      CK(launch_qr((const QrJob*)q.jobs.p, (int)q.h.jobs.size(), dptr(r->ws), st));
      count();
      return;
    }
    CK(cudaMemsetAsync(q.fail.p, 0, q.h.jobs.size() * sizeof(int), st));
    // the mixed modes run the Gram and apply GEMMs in double-float on the
    // FP32 pipe (their error budget is far above ~2^-46), FP64 mode in FP64
    auto qr_gemm = [&](const DevGemmBuf& g) { CK(mixed() ? launch_gemm_df(g.d, b, st) : launch_gemm_f64(g.d, b, st)); };
    for (int p = 0; p < 3; ++p) {
      long e = prof_begin(11, q.gram[p].d.flops);
      qr_gemm(q.gram[p]);
      prof_end(e);
      e = prof_begin(12, 0);
      // the mixed modes factorise in double-float (their error budget is far
      // above ~2^-46), FP64 mode in FP64
      CK(launch_chol_inv((const CholJob*)q.cjobs[p].p, q.ncj[p], dptr(r->ws), (int*)q.fail.p, st, q.maxn[p], mixed()));
      prof_end(e);
      e = prof_begin(11, q.app[p].d.flops);
      qr_gemm(q.app[p]);
      prof_end(e);
      count(3);
    }
    const long e2 = prof_begin(11, q.tt.d.flops + q.rf.d.flops);
    CK(launch_gemm_f64(q.tt.d, b, st));
    CK(launch_gemm_f64(q.rf.d, b, st));
    prof_end(e2);
    count(2);
    if (!r->qrfb.p) {
      ensure(c, r->qrfb, 16);
      CK(cudaMemsetAsync(r->qrfb.p, 0, 16, st));
    }
    r->qr_sectors_acc += (long long)q.h.jobs.size();
    CK(launch_qr_masked((const QrJob*)q.jobs.p, (int)q.h.jobs.size(), dptr(r->ws), (const int*)q.fail.p,
                        (int*)r->qrfb.p, st));
    count();
  }
  void qr_left_move(int j) {  // A_j = A_j^L S ; S -> Sb (bond j+1)
    QrDev& q = qr_plan(j, true);
    Bases b{};
    b.p[S_X] = r->A[j].p;
    b.p[S_Y] = r->A[j].p;
    b.p[S_AUX] = r->Sb.p;
    b.p[S_AUX2] = r->ws.p;
    CK(launch_copy(q.gather.d, b, st));
    run_qr(q, b);
    CK(launch_copy(q.scatter.d, b, st));
    CK(launch_copy(q.rout.d, b, st));
    count(3);
  }
  void lq_right_move(int j) {  // A_j = S A_j^R ; S -> Sb (bond j)
    QrDev& q = qr_plan(j, false);
    Bases b{};
    b.p[S_X] = r->A[j].p;
    b.p[S_Y] = r->A[j].p;
    b.p[S_AUX] = r->Sb.p;
    b.p[S_AUX2] = r->ws.p;
    CK(launch_copy(q.gather.d, b, st));
    run_qr(q, b);
    CK(launch_copy(q.scatter.d, b, st));
    CK(launch_copy(q.rout.d, b, st));
    count(3);
  }
  void absorb_into_left_of(int j) {  // A_j <- S A_j
    DevGemmBuf& g = absorb_left_plan(j);
    Bases b{};
    b.p[S_X] = r->A[j].p;
    b.p[S_AUX] = r->Sb.p;
    b.p[S_Y] = r->tmp.p;
    gemm(g, b, false);
    CK(cudaMemcpyAsync(r->A[j].p, r->tmp.p, r->lay[j].size * 8, cudaMemcpyDeviceToDevice, st));
    r->step_flops_acc += g.d.flops;
  }
  void absorb_into_right_of(int j) {  // A_j <- A_j S
    DevGemmBuf& g = absorb_right_plan(j);
    Bases b{};
    b.p[S_X] = r->A[j].p;
    b.p[S_AUX] = r->Sb.p;
    b.p[S_Y] = r->tmp.p;
    gemm(g, b, false);
    CK(cudaMemcpyAsync(r->A[j].p, r->tmp.p, r->lay[j].size * 8, cudaMemcpyDeviceToDevice, st));
    r->step_flops_acc += g.d.flops;
  }

  // ---- 1-TDVP ---------------------------------------------------------------
  // phase timing (profiling mode): 6 site exponentials, 7 bond
  // exponentials, 8 environment updates, 9 absorbs, 10 gauge moves
  template <class F>
  void phase(int kind, F&& f) {
    const long e = prof_begin(kind, 0);
    f();
    prof_end(e);
  }
  void sweep_lr(double tau) {
    const int N = r->N;
    for (int j = 0; j < N; ++j) {
      site_exp(j, -tau);
      if (j == N - 1) break;
      phase(10, [&] { qr_left_move(j); });
      phase(8, [&] { update_left_env(j); });
      bond_exp(j + 1, +tau);
      phase(9, [&] { absorb_into_left_of(j + 1); });
    }
  }
  void sweep_rl(double tau) {
    for (int j = r->N - 1; j >= 0; --j) {
      site_exp(j, -tau);
      if (j == 0) break;
      phase(10, [&] { lq_right_move(j); });
      phase(8, [&] { update_right_env(j); });
      bond_exp(j, +tau);
      phase(9, [&] { absorb_into_right_of(j - 1); });
    }
  }

  void prepare_all() {
    ensure_vec_capacity();
    for (int j = 0; j < r->N; ++j) {
      site_plan(j);
      qr_plan(j, true);
      qr_plan(j, false);
    }
    for (int k = 1; k < r->N; ++k) bond_plan(k);
    for (int j = 0; j < r->N; ++j) {
      if (j > 0) absorb_left_plan(j);
      if (j + 1 < r->N) absorb_right_plan(j);
    }
  }

  // ---- initial state ---------------------------------------------------------
  void init_state(double beta0) {
    const Mpo& m = M();
    const int N = m.N;
    // bonds from the MPO channel charges; channel w -> (sector, index)
    std::vector<std::vector<std::pair<int, int>>> where(N + 1);
    r->bond.assign(N + 1, Bond());
    for (int k = 0; k <= N; ++k) {
      std::map<Q, int> cnt;
      for (const Q& q : m.chan[k]) cnt[q]++;
      for (auto& kv : cnt) { r->bond[k].q.push_back(kv.first); r->bond[k].dim.push_back(kv.second); }
      std::map<Q, int> next;
      for (const Q& q : m.chan[k]) {
        int s = r->bond[k].find(q);
        where[k].push_back({s, next[q]++});
      }
    }
    r->lay.resize(N);
    for (int j = 0; j < N; ++j) relayout(j);
    // host assembly of I - beta0 H / 2 from the MPO coefficients
    for (int j = 0; j < N; ++j) {
      const SiteLayout& S = r->lay[j];
      std::vector<double> h(S.size, 0.0);
      auto put = [&](int wl, int wr, int sig, int tau, double v) {
        auto a = where[j][wl], b = where[j + 1][wr];
        int p = m.ls.sec_of[sig * 4 + tau], pos = m.ls.pos_of[sig * 4 + tau];
        int bi = S.block_of(a.first, p);
        if (bi < 0) throw Err{TT_ERR_INVALID_ARG, "MPO term outside the block structure"};
        const SiteBlock& B = S.blk[bi];
        h[B.off + ((int64_t)a.second * B.m + pos) * B.dr + b.second] += v;
      };
      const bool last = (j == N - 1);
      for (const MpoTerm& t : m.site[j].terms) put(t.wl, t.wr, t.sig, t.tau, last ? -0.5 * beta0 * t.v : t.v);
      if (last)
        for (int s = 0; s < 4; ++s) put(m.start_ch[j], 0, s, s, 1.0);
      ensure_site_buf(j);
      CK(cudaMemcpyAsync(r->A[j].p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    }
    r->beta = beta0;
    right_canonicalise_shrinking();
    compress_sweep(1e-14);
    right_canonicalise_shrinking();
    ensure_vec_capacity();
    KrylovState* ks = (KrylovState*)r->ks.p;
    CK(k_normalise_inplace(dptr(r->A[0]), r->lay[0].size, dptr(r->partial), ks, (RhoScalars*)r->rs.p, st));
    build_boundary_envs();
    for (int j = N - 1; j >= 1; --j) update_right_env(j);
    CK(cudaStreamSynchronize(st));
  }

  // One Horner step of the series-expansion initial state (SETTN, Supplement
  // "Error analysis": rho_0 = sum_n (-tau_0 H)^n / n!):  rho <- I + alpha H
  // rho, with rho = exp(logscale) x (the super-MPS on the device).  The
  // product H rho is local (W_j acts on sigma of A_j; bond space (w, a) of the
  // MPO channel and the state's bond), the identity is added as a direct sum
  // (one extra state of charge 0 on every interior bond; the first site's
  // right bond and the last site's left bond are concatenated), assembled on
  // the host, uploaded and compressed exactly like the first-order state.
  void horner_step(double alpha) {
    const Mpo& m = M();
    const int N = r->N;
    const LocalSpace& ls = m.ls;
    const int d = ls.d;
    CK(cudaStreamSynchronize(st));
    std::vector<std::vector<double>> A(N);
    for (int j = 0; j < N; ++j) {
      A[j].resize(r->lay[j].size);
      CK(cudaMemcpyAsync(A[j].data(), r->A[j].p, A[j].size() * 8, cudaMemcpyDeviceToHost, st));
    }
    RhoScalars rs;
    CK(cudaMemcpyAsync(&rs, r->rs.p, sizeof(rs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double coef = alpha * std::exp(rs.logscale);
    // new bonds: interior k: identity state (charge 0) first, then (w, a)
    std::vector<Bond> nb(N + 1);
    // place[k][w][s] = (new sector, first index) of the states (w, a in sector s)
    std::vector<std::vector<std::vector<std::pair<int, int>>>> place(N + 1);
    std::vector<std::pair<int, int>> ident(N + 1, {-1, -1});
    for (int k = 0; k <= N; ++k) {
      const Bond& B = r->bond[k];
      const bool interior = k > 0 && k < N;
      std::map<Q, int> dim;
      if (interior) dim[Q{0, 0}] += 1;
      for (size_t w = 0; w < m.chan[k].size(); ++w)
        for (int q = 0; q < B.nsec(); ++q) dim[m.chan[k][w] + B.q[q]] += B.dim[q];
      for (auto& kv : dim) { nb[k].q.push_back(kv.first); nb[k].dim.push_back(kv.second); }
      std::map<Q, int> next;
      if (interior) { ident[k] = {nb[k].find(Q{0, 0}), 0}; next[Q{0, 0}] = 1; }
      place[k].assign(m.chan[k].size(), std::vector<std::pair<int, int>>(B.nsec()));
      for (size_t w = 0; w < m.chan[k].size(); ++w)
        for (int q = 0; q < B.nsec(); ++q) {
          const Q c = m.chan[k][w] + B.q[q];
          place[k][w][q] = {nb[k].find(c), next[c]};
          next[c] += B.dim[q];
        }
    }
    if (nb[0].total() != 1 || nb[N].total() != 1) throw Err{TT_ERR_STATE, "series step: boundary bonds must stay one-dimensional"};
    std::vector<SiteLayout> nl(N);
    std::vector<std::vector<double>> P(N);
    for (int j = 0; j < N; ++j) {
      nl[j] = make_site_layout(nb[j], nb[j + 1], ls);
      P[j].assign(nl[j].size, 0.0);
      const SiteLayout& S = r->lay[j];
      const SiteLayout& T = nl[j];
      auto at = [&](int L, int li, int pair, int R, int ri) -> double& {
        const int p = ls.sec_of[pair], pos = ls.pos_of[pair];
        const int bi = T.block_of(L, p);
        if (bi < 0 || T.blk[bi].r != R) throw Err{TT_ERR_STATE, "series step: block outside the charge structure"};
        const SiteBlock& B = T.blk[bi];
        return P[j][B.off + ((int64_t)li * B.m + pos) * B.dr + ri];
      };
      // H rho: W_j[wl, sig, tau, wr] A_j[a, (tau, sp), b]
      const double scale = (j == 0) ? coef : 1.0;
      for (const MpoTerm& t : m.site[j].terms)
        for (const SiteBlock& b : S.blk)
          for (int pos = 0; pos < b.m; ++pos) {
            const int tau = ls.pairs[b.p][pos].first, sp = ls.pairs[b.p][pos].second;
            if (tau != t.tau) continue;
            const auto pl = place[j][t.wl][b.l], pr = place[j + 1][t.wr][b.r];
            for (int a = 0; a < b.dl; ++a)
              for (int c2 = 0; c2 < b.dr; ++c2)
                at(pl.first, pl.second + a, t.sig * d + sp, pr.first, pr.second + c2) +=
                    scale * t.v * A[j][b.off + ((int64_t)a * b.m + pos) * b.dr + c2];
          }
      // + I: one identity state on the interior bonds (boundary bonds shared)
      const int Li = j == 0 ? 0 : ident[j].first, li = j == 0 ? 0 : ident[j].second;
      const int Ri = j == N - 1 ? 0 : ident[j + 1].first, ri = j == N - 1 ? 0 : ident[j + 1].second;
      for (int sg = 0; sg < d; ++sg) at(Li, li, sg * d + sg, Ri, ri) += 1.0;
    }
    // replace the state
    for (int k = 0; k <= N; ++k) r->bond[k] = nb[k];
    for (int k = 0; k <= N; ++k) invalidate_bond(k);
    for (int j = 0; j < N; ++j) {
      r->lay[j] = nl[j];
      ensure_site_buf(j);
      CK(cudaMemcpyAsync(r->A[j].p, P[j].data(), P[j].size() * 8, cudaMemcpyHostToDevice, st));
    }
    rs.logscale = 0.0;
    CK(cudaMemcpyAsync(r->rs.p, &rs, sizeof(rs), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    right_canonicalise_shrinking();
    compress_sweep(1e-14);
    right_canonicalise_shrinking();
    ensure_vec_capacity();
    KrylovState* ks = (KrylovState*)r->ks.p;
    CK(k_normalise_inplace(dptr(r->A[0]), r->lay[0].size, dptr(r->partial), ks, (RhoScalars*)r->rs.p, st));
    CK(cudaStreamSynchronize(st));
  }

  // rho_0 = sum_{n <= order} (-beta0 H / 2)^n / n! by Horner's rule:
  // P_{order-1} = I - (beta0 / (2 order)) H (the compact first-order state),
  // P_k = I - (beta0 / (2 (k + 1))) H P_{k+1}, rho_0 = P_0.
  void init_series(double beta0, int order) {
    init_state(beta0 / order);
    for (int k = order - 2; k >= 0; --k) horner_step(-beta0 / (2.0 * (k + 1)));
    r->beta = beta0;
    build_boundary_envs();
    for (int j = r->N - 1; j >= 1; --j) update_right_env(j);
    CK(cudaStreamSynchronize(st));
  }

  void build_boundary_envs() {
    const int N = r->N;
    ensure_env(r->L, r->Lsp, r->Lsize, 0);
    ensure_env(r->R, r->Rsp, r->Rsize, N);
    double one = 1.0;
    CK(cudaMemcpyAsync(r->L[0].p, &one, 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(r->R[N].p, &one, 8, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    split_env(r->L, r->Lsp, r->Lsize, 0);
    split_env(r->R, r->Rsp, r->Rsize, N);
  }

  // LQ sweep from the right; bonds may shrink to min(rows, cols) per sector.
  void right_canonicalise_shrinking() {
    const int N = r->N;
    for (int j = N - 1; j >= 1; --j) {
      QrPlanHost h = build_lq_right(r->lay[j], r->bond[j], true);
      Bond nb;
      std::vector<int> new_of_old(r->bond[j].nsec(), -1);
      for (int l = 0; l < r->bond[j].nsec(); ++l)
        if (h.new_dim[l] > 0) {
          new_of_old[l] = nb.nsec();
          nb.q.push_back(r->bond[j].q[l]);
          nb.dim.push_back(h.new_dim[l]);
        }
      SiteLayout oldj = r->lay[j];
      SiteLayout newj = make_site_layout(nb, r->bond[j + 1], M().ls);
      // scatter Q'^T into the new layout of A_j
      size_t bi = 0;
      for (int l = 0; l < r->bond[j].nsec(); ++l) {
        const QrJob& J = h.jobs[l];
        int k = h.new_dim[l];
        for (; bi < h.scatter_blocks.size() && oldj.blk[h.scatter_blocks[bi].first].l == l; ++bi) {
          const SiteBlock& ob = oldj.blk[h.scatter_blocks[bi].first];
          if (k == 0) continue;
          int nbi = newj.block_of(new_of_old[l], ob.p);
          const SiteBlock& b = newj.blk[nbi];
          int C = b.m * b.dr;
          h.scatter.items.push_back(
              CItem{mkref(S_AUX2, J.q + h.scatter_blocks[bi].second), mkref(S_Y, b.off), J.m, 1, C, 1, k, C});
        }
      }
      check_plan(h.gather, caps({{S_X, oldj.size}, {S_AUX2, h.ws_size}}), "init LQ gather");
      check_plan(h.scatter, caps({{S_AUX2, h.ws_size}, {S_Y, newj.size}}), "init LQ scatter");
      check_plan(h.rout, caps({{S_AUX2, h.ws_size}, {S_AUX, h.s_size}}), "init LQ R");
      DBuf jobs, newA;
      DevCopyBuf g, s, ro;
      ensure(c, jobs, h.jobs.size() * sizeof(QrJob) + 8);
      if (!h.jobs.empty()) CK(cudaMemcpyAsync(jobs.p, h.jobs.data(), h.jobs.size() * sizeof(QrJob), cudaMemcpyHostToDevice, st));
      upload(c, h.gather, g);
      upload(c, h.scatter, s);
      upload(c, h.rout, ro);
      ensure(c, r->ws, (size_t)h.ws_size * 8);
      ensure(c, r->Sb, (size_t)h.s_size * 8);
      ensure(c, newA, (size_t)newj.size * 8);
      CK(cudaMemsetAsync(newA.p, 0, (size_t)newj.size * 8, st));
      Bases b{};
      b.p[S_X] = r->A[j].p;
      b.p[S_Y] = newA.p;
      b.p[S_AUX] = r->Sb.p;
      b.p[S_AUX2] = r->ws.p;
      CK(launch_copy(g.d, b, st));
      CK(launch_qr((const QrJob*)jobs.p, (int)h.jobs.size(), dptr(r->ws), st));
      CK(launch_copy(s.d, b, st));
      CK(launch_copy(ro.d, b, st));
      // A_{j-1} <- A_{j-1} S  (S: old d x new k, row-major, offsets per old sector)
      std::vector<int64_t> soff(r->bond[j].nsec());
      int64_t o = 0;
      for (int l = 0; l < r->bond[j].nsec(); ++l) { soff[l] = o; o += (int64_t)r->bond[j].dim[l] * h.new_dim[l]; }
      SiteLayout oldp = r->lay[j - 1];
      SiteLayout newp = make_site_layout(r->bond[j - 1], nb, M().ls);
      GemmPlan ab = build_absorb_right(oldp, newp, r->bond[j], nb, soff, new_of_old);
      check_plan(ab, caps({{S_X, oldp.size}, {S_AUX, h.s_size}, {S_Y, newp.size}}), "init absorb");
      DevGemmBuf abd;
      upload(c, ab, abd);
      DBuf newP;
      ensure(c, newP, (size_t)newp.size * 8);
      CK(cudaMemsetAsync(newP.p, 0, (size_t)newp.size * 8, st));
      Bases b2{};
      b2.p[S_X] = r->A[j - 1].p;
      b2.p[S_AUX] = r->Sb.p;
      b2.p[S_Y] = newP.p;
      CK(launch_gemm_f64(abd.d, b2, st));
      CK(cudaStreamSynchronize(st));
      std::swap(r->A[j], newA);
      std::swap(r->A[j - 1], newP);
      dfree(c, newA);
      dfree(c, newP);
      dfree(c, jobs);
      release(c, g);
      release(c, s);
      release(c, ro);
      release(c, abd);
      r->bond[j] = nb;
      r->lay[j] = newj;
      r->lay[j - 1] = newp;
      invalidate_bond(j);
    }
  }

  // Left-to-right SVD sweep (compact form of the initial MPO): at every bond
  // keep the singular values s > cut * s_max of that bond; A_j <- U,
  // A_{j+1} <- s V^T A_{j+1}.  cuSOLVER gesvd per right sector (untimed).
  void compress_sweep(double cut) {
    const int N = r->N;
    const LocalSpace& ls = M().ls;
    if (!c->sol) {
      if (cusolverDnCreate(&c->sol) != CUSOLVER_STATUS_SUCCESS) throw Err{TT_ERR_CUDA, "cusolverDnCreate failed"};
    }
    cusolverDnSetStream(c->sol, st);
    for (int j = 0; j + 1 < N; ++j) {
      const SiteLayout S = r->lay[j];
      const Bond B = r->bond[j + 1];
      struct Sec { int rows, cols, ldt; bool trans; int64_t th, u, vt, sv; int kept; };
      std::vector<Sec> sec(B.nsec());
      int64_t ws = 0;
      CopyPlan gp;
      for (int q = 0; q < B.nsec(); ++q) {
        Sec& x = sec[q];
        x.rows = (int)S.grp_rows[q];
        x.cols = B.dim[q];
        x.trans = x.rows < x.cols;
        int mm = std::max(x.rows, x.cols), nn = std::min(x.rows, x.cols);
        x.ldt = mm;
        x.th = ws; ws += (int64_t)mm * nn;
        x.u = ws; ws += (int64_t)mm * nn;
        x.vt = ws; ws += (int64_t)nn * nn;
        x.sv = ws; ws += nn;
        x.kept = 0;
        if (nn == 0) continue;
        // group (row-major rows x cols) -> Theta column-major, or Theta^T column-major
        if (!x.trans) gp.items.push_back(CItem{mkref(S_X, S.grp_off[q]), mkref(S_AUX2, x.th), x.cols, 1, 1, x.ldt, x.rows, x.cols});
        else gp.items.push_back(CItem{mkref(S_X, S.grp_off[q]), mkref(S_AUX2, x.th), x.cols, 1, x.ldt, 1, x.rows, x.cols});
      }
      check_plan(gp, caps({{S_X, S.size}, {S_AUX2, ws}}), "compress gather");
      ensure(c, r->ws, (size_t)std::max<int64_t>(ws, 1) * 8);
      CK(cudaMemsetAsync(r->ws.p, 0, (size_t)std::max<int64_t>(ws, 1) * 8, st));
      DevCopyBuf gd;
      upload(c, gp, gd);
      Bases b{};
      b.p[S_X] = r->A[j].p;
      b.p[S_AUX2] = r->ws.p;
      CK(launch_copy(gd.d, b, st));
      release(c, gd);
      double* wsp = dptr(r->ws);
      DBuf work, info;
      ensure(c, info, 64);
      for (auto& x : sec) {
        int mm = std::max(x.rows, x.cols), nn = std::min(x.rows, x.cols);
        if (nn == 0) continue;
        int lwork = 0;
        if (cusolverDnDgesvd_bufferSize(c->sol, mm, nn, &lwork) != CUSOLVER_STATUS_SUCCESS) throw Err{TT_ERR_CUDA, "gesvd_bufferSize"};
        ensure(c, work, (size_t)std::max(lwork, 1) * 8 + (size_t)nn * 8);
        if (cusolverDnDgesvd(c->sol, 'S', 'S', mm, nn, wsp + x.th, x.ldt, wsp + x.sv, wsp + x.u, mm, wsp + x.vt, nn,
                             dptr(work), lwork, dptr(work) + lwork, (int*)info.p) != CUSOLVER_STATUS_SUCCESS)
          throw Err{TT_ERR_CUDA, "cusolverDnDgesvd failed"};
      }
      std::vector<double> hs(std::max<int64_t>(ws, 1));
      CK(cudaMemcpyAsync(hs.data(), wsp, (size_t)ws * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      dfree(c, work);
      dfree(c, info);
      double smax = 0;
      for (auto& x : sec)
        for (int i = 0; i < std::min(x.rows, x.cols); ++i) smax = std::max(smax, hs[x.sv + i]);
      Bond nb;
      std::vector<int> new_of_old(B.nsec(), -1);
      for (int q = 0; q < B.nsec(); ++q) {
        Sec& x = sec[q];
        for (int i = 0; i < std::min(x.rows, x.cols); ++i) x.kept += hs[x.sv + i] > cut * smax;
        if (x.kept > 0) {
          new_of_old[q] = nb.nsec();
          nb.q.push_back(B.q[q]);
          nb.dim.push_back(x.kept);
        }
      }
      SiteLayout nj = make_site_layout(r->bond[j], nb, ls);
      // S = diag(s) V^T (kept x old), row-major, per old sector; scale rows by s
      std::vector<int64_t> soff(B.nsec(), 0);
      int64_t so = 0;
      CopyPlan sc;
      for (int q = 0; q < B.nsec(); ++q) {
        const Sec& x = sec[q];
        soff[q] = so;
        if (x.kept == 0) continue;
        int nn = std::min(x.rows, x.cols);
        int64_t ubase, urs, ucs, vbase, vrs, vcs;
        if (!x.trans) { ubase = x.u; urs = 1; ucs = x.ldt; vbase = x.vt; vrs = 1; vcs = nn; }
        else { ubase = x.vt; urs = nn; ucs = 1; vbase = x.u; vrs = x.ldt; vcs = 1; }
        int mn = new_of_old[q];
        sc.items.push_back(CItem{mkref(S_AUX2, ubase), mkref(S_Y, nj.grp_off[mn]), urs, ucs, x.kept, 1, x.rows, x.kept});
        sc.items.push_back(CItem{mkref(S_AUX2, vbase), mkref(S_AUX, so), vrs, vcs, x.cols, 1, x.kept, x.cols});
        so += (int64_t)x.kept * x.cols;
      }
      check_plan(sc, caps({{S_AUX2, ws}, {S_Y, nj.size}, {S_AUX, std::max<int64_t>(so, 1)}}), "compress scatter");
      DBuf newA, Sm;
      ensure(c, newA, (size_t)nj.size * 8);
      ensure(c, Sm, (size_t)std::max<int64_t>(so, 1) * 8);
      DevCopyBuf sd;
      upload(c, sc, sd);
      Bases b2{};
      b2.p[S_AUX2] = r->ws.p;
      b2.p[S_Y] = newA.p;
      b2.p[S_AUX] = Sm.p;
      CK(launch_copy(sd.d, b2, st));
      release(c, sd);
      for (int q = 0; q < B.nsec(); ++q) {
        const Sec& x = sec[q];
        if (x.kept == 0) continue;
        // S block (kept x cols row-major) = column-major (cols x kept) with ld = cols: scale columns by s
        CK(launch_scale_rc((double*)Sm.p + soff[q], x.cols, x.cols, x.kept, wsp + x.sv, 1, st));
      }
      // A_{j+1} <- S A_{j+1}
      SiteLayout oldn = r->lay[j + 1];
      SiteLayout newn = make_site_layout(nb, r->bond[j + 2], ls);
      GemmPlan ab = build_absorb_left(oldn, newn, B, nb, soff, new_of_old);
      // S is (new x old) row-major with lda = old dim: build_absorb_left uses lda = Bold.dim
      check_plan(ab, caps({{S_X, oldn.size}, {S_AUX, std::max<int64_t>(so, 1)}, {S_Y, newn.size}}), "compress absorb");
      DevGemmBuf abd;
      upload(c, ab, abd);
      DBuf newN;
      ensure(c, newN, (size_t)newn.size * 8);
      CK(cudaMemsetAsync(newN.p, 0, (size_t)newn.size * 8, st));
      Bases b3{};
      b3.p[S_X] = r->A[j + 1].p;
      b3.p[S_AUX] = Sm.p;
      b3.p[S_Y] = newN.p;
      CK(launch_gemm_f64(abd.d, b3, st));
      CK(cudaStreamSynchronize(st));
      release(c, abd);
      std::swap(r->A[j], newA);
      std::swap(r->A[j + 1], newN);
      dfree(c, newA);
      dfree(c, newN);
      dfree(c, Sm);
      r->bond[j + 1] = nb;
      r->lay[j] = nj;
      r->lay[j + 1] = newn;
      invalidate_bond(j + 1);
    }
  }

  // Pad every bond to (about) D_target states with zero-weight directions.
  // Per sector the dimension scales by D_target / D_current (kept within what
  // both neighbouring site tensors can hold).  With the centre on site 0 and
  // sites 1..N-1 right-canonical, the new rows of A_k are the orthonormal
  // completion returned by the Householder QR of [M^T | 0] (M the rows of the
  // left sector, already orthonormal, so Q starts with M^T), and A_{k-1} gets
  // zero columns: the state is unchanged, the manifold is larger.
  void pad_bonds(int D_target) {
    const int N = r->N;
    const LocalSpace& ls = M().ls;
    // targets
    std::vector<Bond> tgt = r->bond;
    for (int k = 1; k < N; ++k) {
      int64_t cur = r->bond[k].total();
      if (cur >= D_target) continue;
      double f = (double)D_target / (double)cur;
      for (size_t q = 0; q < tgt[k].dim.size(); ++q) tgt[k].dim[q] = (int)std::floor(r->bond[k].dim[q] * f);
    }
    // feasibility: d'_q <= rows and cols of the neighbouring blocks (iterate)
    for (int it = 0; it < 4; ++it)
      for (int k = 1; k < N; ++k)
        for (int q = 0; q < tgt[k].nsec(); ++q) {
          int64_t cols = 0, rows = 0;
          for (int p = 0; p < (int)ls.pq.size(); ++p) {
            int rr = tgt[k + 1].find(tgt[k].q[q] + ls.pq[p]);
            if (rr >= 0) cols += (int64_t)ls.pairs[p].size() * tgt[k + 1].dim[rr];
            int ll = tgt[k - 1].find(tgt[k].q[q] - ls.pq[p]);
            if (ll >= 0) rows += (int64_t)ls.pairs[p].size() * tgt[k - 1].dim[ll];
          }
          int64_t cap = std::min(cols, rows);
          tgt[k].dim[q] = (int)std::max<int64_t>(r->bond[k].dim[q], std::min<int64_t>(tgt[k].dim[q], cap));
        }
    for (int k = N - 1; k >= 1; --k) {
      const Bond& Bo = r->bond[k];
      const Bond& Bn = tgt[k];
      bool same = true;
      for (int q = 0; q < Bo.nsec(); ++q) same = same && Bo.dim[q] == Bn.dim[q];
      if (same) continue;
      const SiteLayout oldk = r->lay[k];
      const SiteLayout newk = make_site_layout(Bn, r->bond[k + 1], ls);
      // QR of [M_q^T | 0] per left sector q (cols_q x d'_q, column-major)
      int64_t ws = 0;
      std::vector<QrJob> jobs;
      CopyPlan g, sc;
      for (int q = 0; q < Bo.nsec(); ++q) {
        int64_t cols = 0;
        std::vector<std::pair<int, int64_t>> segs;
        for (int p = 0; p < oldk.npq; ++p) {
          int bi = oldk.block_of(q, p);
          if (bi < 0) continue;
          segs.push_back({bi, cols});
          cols += (int64_t)oldk.blk[bi].m * oldk.blk[bi].dr;
        }
        QrJob J;
        J.m = (int)cols;
        J.n = Bn.dim[q];
        if (J.n > 2048 || cols < J.n) throw Err{TT_ERR_STATE, "padding target exceeds the sector capacity"};
        J.a = ws; ws += (int64_t)J.m * J.n;
        J.q = ws; ws += (int64_t)J.m * J.n;
        J.r = ws; ws += (int64_t)J.n * J.n;
        jobs.push_back(J);
        for (auto& sg : segs) {
          const SiteBlock& b = oldk.blk[sg.first];
          const int C = b.m * b.dr;
          g.items.push_back(CItem{mkref(S_X, b.off), mkref(S_AUX2, J.a + sg.second), C, 1, J.m, 1, b.dl, C});
          const SiteBlock& nb = newk.blk[newk.block_of(q, b.p)];
          sc.items.push_back(CItem{mkref(S_AUX2, J.q + sg.second), mkref(S_Y, nb.off), J.m, 1, C, 1, J.n, C});
        }
      }
      check_plan(g, caps({{S_X, oldk.size}, {S_AUX2, ws}}), "pad gather");
      check_plan(sc, caps({{S_AUX2, ws}, {S_Y, newk.size}}), "pad scatter");
      // A_{k-1}: zero-padded columns of every right group
      const SiteLayout oldp = r->lay[k - 1];
      const SiteLayout newp = make_site_layout(r->bond[k - 1], Bn, ls);
      CopyPlan zp;
      for (int q = 0; q < Bo.nsec(); ++q)
        if (oldp.grp_rows[q] > 0)
          zp.items.push_back(CItem{mkref(S_X, oldp.grp_off[q]), mkref(S_Y, newp.grp_off[q]), Bo.dim[q], 1, Bn.dim[q], 1,
                                   (int)oldp.grp_rows[q], Bo.dim[q]});
      check_plan(zp, caps({{S_X, oldp.size}, {S_Y, newp.size}}), "pad columns");
      DBuf jb, nA, nP;
      DevCopyBuf gd, sd, zd;
      ensure(c, jb, jobs.size() * sizeof(QrJob) + 8);
      CK(cudaMemcpyAsync(jb.p, jobs.data(), jobs.size() * sizeof(QrJob), cudaMemcpyHostToDevice, st));
      upload(c, g, gd);
      upload(c, sc, sd);
      upload(c, zp, zd);
      ensure(c, r->ws, (size_t)std::max<int64_t>(ws, 1) * 8);
      CK(cudaMemsetAsync(r->ws.p, 0, (size_t)std::max<int64_t>(ws, 1) * 8, st));
      ensure(c, nA, (size_t)newk.size * 8);
      ensure(c, nP, (size_t)newp.size * 8);
      CK(cudaMemsetAsync(nA.p, 0, (size_t)newk.size * 8, st));
      CK(cudaMemsetAsync(nP.p, 0, (size_t)newp.size * 8, st));
      Bases b{};
      b.p[S_X] = r->A[k].p;
      b.p[S_Y] = nA.p;
      b.p[S_AUX2] = r->ws.p;
      CK(launch_copy(gd.d, b, st));
      CK(launch_qr((const QrJob*)jb.p, (int)jobs.size(), dptr(r->ws), st));
      CK(launch_copy(sd.d, b, st));
      Bases b2{};
      b2.p[S_X] = r->A[k - 1].p;
      b2.p[S_Y] = nP.p;
      CK(launch_copy(zd.d, b2, st));
      CK(cudaStreamSynchronize(st));
      release(c, gd);
      release(c, sd);
      release(c, zd);
      dfree(c, jb);
      std::swap(r->A[k], nA);
      std::swap(r->A[k - 1], nP);
      dfree(c, nA);
      dfree(c, nP);
      r->bond[k] = Bn;
      r->lay[k] = newk;
      r->lay[k - 1] = newp;
      invalidate_bond(k);
    }
    ensure_vec_capacity();
    for (int j = N - 1; j >= 1; --j) update_right_env(j);
    CK(cudaStreamSynchronize(st));
  }

  // ---- measurement --------------------------------------------------------------
  MeasDev& meas_plan(int j) {
    MeasDev& md = r->meas[j];
    if (md.valid) return md;
    const SiteLayout& S = r->lay[j];
    BondMatLayout el = make_bondmat_layout(r->bond[j]);
    md.next = make_bondmat_layout(r->bond[j + 1]);
    GemmPlan t, e;
    for (const SiteBlock& b : S.blk) {
      int N = b.m * b.dr;
      t.add_group(b.dl, N, mkref(S_T1, b.off), N, 0);
      t.add_seg(mkref(S_AUX, el.off[b.l]), b.dl, 0, mkref(S_X, b.off), N, 0, b.dl);
    }
    for (int rr = 0; rr < r->bond[j + 1].nsec(); ++rr) {
      int d = r->bond[j + 1].dim[rr];
      e.add_group(d, d, mkref(S_AUX2, md.next.off[rr]), d, 0);
      if (S.grp_rows[rr] > 0) e.add_seg(mkref(S_X, S.grp_off[rr]), d, 1, mkref(S_T1, S.grp_off[rr]), d, 0, (int)S.grp_rows[rr]);
    }
    check_plan(t, caps({{S_AUX, el.size}, {S_X, S.size}, {S_T1, S.size}}), "measure T");
    check_plan(e, caps({{S_X, S.size}, {S_T1, S.size}, {S_AUX2, md.next.size}}), "measure EL");
    upload(c, t, md.t);
    upload(c, e, md.el);
    std::vector<ObsItem> items;
    for (const SiteBlock& b : S.blk) {
      ObsItem it{};
      it.off = b.off;
      it.dl = b.dl;
      it.m = b.m;
      it.dr = b.dr;
      for (int s = 0; s < b.m; ++s) {
        int sig = M().ls.pairs[b.p][s].first;
        int nu = sig & 1, nd = (sig >> 1) & 1;
        it.wn[s] = nu + nd;
        it.wd[s] = nu * nd;
      }
      items.push_back(it);
    }
    ensure(c, md.items, items.size() * sizeof(ObsItem) + 8);
    if (!items.empty()) CK(cudaMemcpyAsync(md.items.p, items.data(), items.size() * sizeof(ObsItem), cudaMemcpyHostToDevice, st));
    md.nitems = (int)items.size();
    md.valid = true;
    return md;
  }

  void measure(tt_obs* out) {
    const int N = r->N;
    ensure_vec_capacity();
    // obs buffer: [0] n-sum, [1] d-sum, [2] <A|H A>, [3] <A|A>
    ensure(c, r->obs, 8 * 8);
    CK(cudaMemsetAsync(r->obs.p, 0, 8 * 8, st));
    double* ob = dptr(r->obs);
    // energy at the canonical centre (site 0)
    apply_site(0, dptr(r->A[0]), dptr(r->W), true);  // FP64 contraction for the energy
    CK(k_dot_plain(dptr(r->A[0]), dptr(r->W), r->lay[0].size, dptr(r->partial), ob + 2, st));
    CK(k_dot_plain(dptr(r->A[0]), dptr(r->A[0]), r->lay[0].size, dptr(r->partial), ob + 3, st));
    // local densities with the left transfer matrices (sites > j right-canonical)
    size_t maxel = 8;
    for (int k = 0; k <= N; ++k) maxel = std::max<size_t>(maxel, make_bondmat_layout(r->bond[k]).size * 8);
    ensure(c, r->el0, maxel);
    ensure(c, r->el1, maxel);
    int64_t maxsite = 1;
    for (int j = 0; j < N; ++j) maxsite = std::max(maxsite, r->lay[j].size);
    ensure(c, r->T1, (size_t)maxsite * 8);
    double one = 1.0;
    CK(cudaMemcpyAsync(r->el0.p, &one, 8, cudaMemcpyHostToDevice, st));
    size_t maxitems = 1;
    for (int j = 0; j < N; ++j) maxitems = std::max(maxitems, r->lay[j].blk.size());
    DBuf part2;
    ensure(c, part2, maxitems * 2 * 8);
    for (int j = 0; j < N; ++j) {
      MeasDev& md = meas_plan(j);
      Bases b{};
      b.p[S_X] = r->A[j].p;
      b.p[S_T1] = r->T1.p;
      b.p[S_AUX] = r->el0.p;
      b.p[S_AUX2] = r->el1.p;
      CK(launch_gemm_f64(md.t.d, b, st));
      CK(launch_local_obs((const ObsItem*)md.items.p, md.nitems, dptr(r->A[j]), dptr(r->T1), dptr(part2), ob, st));
      CK(launch_gemm_f64(md.el.d, b, st));
      std::swap(r->el0, r->el1);
    }
    double hv[4];
    RhoScalars rs;
    CK(cudaMemcpyAsync(hv, ob, 4 * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&rs, r->rs.p, sizeof(rs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    dfree(c, part2);
    check_tc();  // an aborted GEMM leaves garbage behind: report the cause first
    if (rs.bad) throw Err{TT_ERR_NUMERIC, "non-finite or zero norm in a Krylov update"};
    double nrm2 = hv[3];
    out->beta = r->beta;
    out->energy_per_site = hv[2] / nrm2 / N;
    out->density = hv[0] / nrm2 / N;
    out->double_occ = hv[1] / nrm2 / N;
    out->lnZ = 2.0 * rs.logscale + std::log(nrm2);
    out->free_energy_per_site = -out->lnZ / (r->beta * N);
    int mb = 1;
    for (auto& b : r->bond) mb = std::max<int>(mb, (int)b.total());
    out->max_bond = mb;
    out->krylov_resid_max = rs.resid_max;
    if (!std::isfinite(out->lnZ) || !std::isfinite(out->energy_per_site))
      throw Err{TT_ERR_NUMERIC, "non-finite observable"};
  }

  // ---- 2-TDVP growth ----------------------------------------------------------
  void merge_two(int j, const SiteLayout& C2, DBuf& Cbuf) {
    const SiteLayout& A1 = r->lay[j];
    const SiteLayout& A2 = r->lay[j + 1];
    const LocalSpace& ls = M().ls;
    const LocalSpace& ls2 = r->mpo->ls2;
    GemmPlan g;
    CopyPlan cp;
    int64_t cur = 0;
    for (const SiteBlock& b1 : A1.blk)
      for (int p2 = 0; p2 < A2.npq; ++p2) {
        int b2i = A2.block_of(b1.r, p2);
        if (b2i < 0) continue;
        const SiteBlock& b2 = A2.blk[b2i];
        int M_ = b1.dl * b1.m, N_ = b2.m * b2.dr;
        g.add_group(M_, N_, mkref(S_T1, cur), N_, 0);
        g.add_seg(mkref(S_X, b1.off), b1.dr, 0, mkref(S_AUX, b2.off), N_, 0, b1.dr);
        for (int s1 = 0; s1 < b1.m; ++s1)
          for (int s2 = 0; s2 < b2.m; ++s2) {
            auto pr1 = ls.pairs[b1.p][s1];
            auto pr2 = ls.pairs[b2.p][s2];
            int sig = pr1.first * 4 + pr2.first, sgp = pr1.second * 4 + pr2.second;
            int pidx = sig * 16 + sgp;
            int P = ls2.sec_of[pidx], pos = ls2.pos_of[pidx];
            int cbi = C2.block_of(b1.l, P);
            const SiteBlock& cb = C2.blk[cbi];
            cp.items.push_back(CItem{mkref(S_T1, cur + (int64_t)s1 * N_ + (int64_t)s2 * b2.dr), mkref(S_Y, cb.off + (int64_t)pos * cb.dr),
                                     (int64_t)b1.m * N_, 1, (int64_t)cb.m * cb.dr, 1, b1.dl, b2.dr});
          }
        cur += (int64_t)M_ * N_;
      }
    check_plan(g, caps({{S_X, A1.size}, {S_AUX, A2.size}, {S_T1, cur}}), "merge GEMM");
    check_plan(cp, caps({{S_T1, cur}, {S_Y, C2.size}}), "merge copy");
    DevGemmBuf gd;
    DevCopyBuf cd;
    upload(c, g, gd);
    upload(c, cp, cd);
    ensure(c, r->T1, (size_t)std::max<int64_t>(cur, 1) * 8);
    ensure(c, Cbuf, (size_t)C2.size * 8);
    CK(cudaMemsetAsync(Cbuf.p, 0, (size_t)C2.size * 8, st));
    Bases b{};
    b.p[S_X] = r->A[j].p;
    b.p[S_AUX] = r->A[j + 1].p;
    b.p[S_T1] = r->T1.p;
    b.p[S_Y] = Cbuf.p;
    CK(launch_gemm_f64(gd.d, b, st));
    CK(launch_copy(cd.d, b, st));
    CK(cudaStreamSynchronize(st));
    release(c, gd);
    release(c, cd);
  }

  struct SvdSector {
    Q q;
    int rows, cols;
    int64_t theta, u, vt, s;  // ws offsets
    int ldt;
    bool trans;               // Theta stored transposed (rows < cols)
    std::vector<std::pair<int, int>> rowseg;  // (l, p1) -> rowoff order (implicit)
    int kept = 0;
  };

  // Split the two-site tensor C (bond j -> bond j+2) into A_j A_{j+1} with a
  // new bond j+1.  left_canonical: A_j = U, A_{j+1} = s V^T; else A_j = U s,
  // A_{j+1} = V^T.
  void split_two(int j, const SiteLayout& C2, DBuf& Cbuf, bool left_canonical) {
    const Bond& BL = r->bond[j];
    const Bond& BR = r->bond[j + 2];
    const LocalSpace& ls = M().ls;
    const LocalSpace& ls2 = r->mpo->ls2;
    // middle sectors
    std::map<Q, int> mid;
    for (int l = 0; l < BL.nsec(); ++l)
      for (int p = 0; p < (int)ls.pq.size(); ++p) {
        Q m = BL.q[l] + ls.pq[p];
        bool ok = false;
        for (int rr = 0; rr < BR.nsec() && !ok; ++rr) ok = ls.find(BR.q[rr] - m) >= 0;
        if (ok) mid[m] = 0;
      }
    std::vector<SvdSector> sec;
    for (auto& kv : mid) { kv.second = (int)sec.size(); sec.push_back(SvdSector{kv.first, 0, 0, 0, 0, 0, 0, 0, false, {}, 0}); }
    // row offsets per (l, p1), col offsets per r
    std::map<std::pair<int, int>, int64_t> rowoff;
    std::vector<std::map<int, int64_t>> coloff(sec.size());
    for (int l = 0; l < BL.nsec(); ++l)
      for (int p = 0; p < (int)ls.pq.size(); ++p) {
        auto it = mid.find(BL.q[l] + ls.pq[p]);
        if (it == mid.end()) continue;
        SvdSector& S = sec[it->second];
        rowoff[{l, p}] = S.rows;
        S.rows += BL.dim[l] * (int)ls.pairs[p].size();
      }
    for (size_t si = 0; si < sec.size(); ++si)
      for (int rr = 0; rr < BR.nsec(); ++rr) {
        int p2 = ls.find(BR.q[rr] - sec[si].q);
        if (p2 < 0) continue;
        coloff[si][rr] = sec[si].cols;
        sec[si].cols += (int)ls.pairs[p2].size() * BR.dim[rr];
      }
    int64_t ws = 0;
    for (auto& S : sec) {
      S.trans = S.rows < S.cols;
      int mm = std::max(S.rows, S.cols), nn = std::min(S.rows, S.cols);
      S.ldt = mm;
      S.theta = ws; ws += (int64_t)mm * nn;
      S.u = ws; ws += (int64_t)mm * nn;
      S.vt = ws; ws += (int64_t)nn * nn;
      S.s = ws; ws += nn;
    }
    ensure(c, r->ws, (size_t)std::max<int64_t>(ws, 1) * 8);
    CK(cudaMemsetAsync(r->ws.p, 0, (size_t)std::max<int64_t>(ws, 1) * 8, st));
    // gather C -> Theta
    CopyPlan gp;
    for (const SiteBlock& cb : C2.blk)
      for (int pos = 0; pos < cb.m; ++pos) {
        auto pr = ls2.pairs[cb.p][pos];
        int s1a = pr.first / 4, s2a = pr.first % 4, s1b = pr.second / 4, s2b = pr.second % 4;
        int i1 = s1a * 4 + s1b, i2 = s2a * 4 + s2b;
        int p1 = ls.sec_of[i1], q1 = ls.pos_of[i1];
        int p2 = ls.sec_of[i2], q2 = ls.pos_of[i2];
        Q m = BL.q[cb.l] + ls.pq[p1];
        int si = mid.at(m);
        SvdSector& S = sec[si];
        int64_t row = rowoff.at({cb.l, p1}) + q1;
        int64_t col = coloff[si].at(cb.r) + (int64_t)q2 * BR.dim[cb.r];
        int m1 = (int)ls.pairs[p1].size();
        CItem it;
        it.src = mkref(S_X, cb.off + (int64_t)pos * cb.dr);
        it.src_rs = (int64_t)cb.m * cb.dr;
        it.src_cs = 1;
        if (!S.trans) {
          it.dst = mkref(S_AUX2, S.theta + row + col * S.ldt);
          it.dst_rs = m1;
          it.dst_cs = S.ldt;
        } else {
          it.dst = mkref(S_AUX2, S.theta + col + row * S.ldt);
          it.dst_rs = (int64_t)m1 * S.ldt;
          it.dst_cs = 1;
        }
        it.rows = cb.dl;
        it.cols = cb.dr;
        gp.items.push_back(it);
      }
    check_plan(gp, caps({{S_X, C2.size}, {S_AUX2, ws}}), "split gather");
    DevCopyBuf gd;
    upload(c, gp, gd);
    Bases b{};
    b.p[S_X] = Cbuf.p;
    b.p[S_AUX2] = r->ws.p;
    CK(launch_copy(gd.d, b, st));
    release(c, gd);
    // SVD per sector (cuSOLVER gesvd, m >= n)
    if (!c->sol) {
      if (cusolverDnCreate(&c->sol) != CUSOLVER_STATUS_SUCCESS) throw Err{TT_ERR_CUDA, "cusolverDnCreate failed"};
    }
    cusolverDnSetStream(c->sol, st);
    DBuf work, info;
    ensure(c, info, 64);
    double* wsp = dptr(r->ws);
    for (auto& S : sec) {
      int mm = std::max(S.rows, S.cols), nn = std::min(S.rows, S.cols);
      if (nn == 0) continue;
      int lwork = 0;
      if (cusolverDnDgesvd_bufferSize(c->sol, mm, nn, &lwork) != CUSOLVER_STATUS_SUCCESS)
        throw Err{TT_ERR_CUDA, "gesvd_bufferSize failed"};
      ensure(c, work, (size_t)std::max(lwork, 1) * 8 + (size_t)nn * 8);
      cusolverStatus_t cs = cusolverDnDgesvd(c->sol, 'S', 'S', mm, nn, wsp + S.theta, S.ldt, wsp + S.s, wsp + S.u, mm,
                                             wsp + S.vt, nn, dptr(work), lwork, dptr(work) + lwork, (int*)info.p);
      if (cs != CUSOLVER_STATUS_SUCCESS) throw Err{TT_ERR_CUDA, "cusolverDnDgesvd failed"};
    }
    // singular values to the host; global truncation (same rule as the oracle)
    std::vector<double> hs(std::max<int64_t>(ws, 1));
    CK(cudaMemcpyAsync(hs.data(), wsp, (size_t)ws * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    dfree(c, work);
    dfree(c, info);
    struct SV { double s; int sec, idx; };
    std::vector<SV> all;
    for (size_t si = 0; si < sec.size(); ++si) {
      int nn = std::min(sec[si].rows, sec[si].cols);
      for (int i = 0; i < nn; ++i) all.push_back(SV{hs[sec[si].s + i], (int)si, i});
    }
    std::stable_sort(all.begin(), all.end(), [](const SV& a, const SV& b) { return a.s > b.s; });
    int k = 0;
    if (!all.empty() && all[0].s > 0) {
      const double s0 = all[0].s;
      int cnt = 0;
      for (auto& x : all) cnt += (x.s > r->opts.svd_cut * s0);
      k = std::min(r->opts.D_max, cnt);
      if (k > 0 && k < (int)all.size()) {
        int k0 = k;
        double ta = DEGEN_ABS * s0;
        while (k > 0 && all[k - 1].s - all[k].s <= r->opts.degen_tol * all[k - 1].s + ta) --k;
        if (k == 0) {
          k = k0;
          while (k < (int)all.size() && all[k - 1].s - all[k].s <= r->opts.degen_tol * all[k - 1].s + ta) ++k;
        }
      }
    }
    for (int i = 0; i < k; ++i) sec[all[i].sec].kept++;
    if (std::getenv("TT_DEBUG")) {
      std::fprintf(stderr, "[split j=%d] nsv=%zu kept=%d s0=%.6e", j, all.size(), k, all.empty() ? 0.0 : all[0].s);
      for (int i = std::max(0, k - 3); i < std::min((int)all.size(), k + 3); ++i)
        std::fprintf(stderr, " s[%d]=%.9e(sec%d)", i, all[i].s / all[0].s, all[i].sec);
      std::fprintf(stderr, "\n");
    }
    // new middle bond
    Bond nb;
    std::vector<int> newidx(sec.size(), -1);
    for (size_t si = 0; si < sec.size(); ++si)
      if (sec[si].kept > 0) {
        newidx[si] = nb.nsec();
        nb.q.push_back(sec[si].q);
        nb.dim.push_back(sec[si].kept);
      }
    if (nb.nsec() == 0) throw Err{TT_ERR_NUMERIC, "two-site split kept no state"};
    SiteLayout n1 = make_site_layout(BL, nb, ls);
    SiteLayout n2 = make_site_layout(nb, BR, ls);
    DBuf A1, A2;
    ensure(c, A1, (size_t)n1.size * 8);
    ensure(c, A2, (size_t)n2.size * 8);
    CopyPlan sc;
    for (size_t si = 0; si < sec.size(); ++si) {
      const SvdSector& S = sec[si];
      if (S.kept == 0) continue;
      int mn = newidx[si];
      int mm = std::max(S.rows, S.cols), nn = std::min(S.rows, S.cols);
      // U (rows x nn) and V^T (nn x cols) in strided form
      int64_t ubase, urs, ucs, vbase, vrs, vcs;
      if (!S.trans) { ubase = S.u; urs = 1; ucs = mm; vbase = S.vt; vrs = 1; vcs = nn; }
      else { ubase = S.vt; urs = nn; ucs = 1; vbase = S.u; vrs = mm; vcs = 1; }
      // A_j group for middle sector mn: rows x kept (row-major)
      sc.items.push_back(CItem{mkref(S_AUX2, ubase), mkref(S_X, n1.grp_off[mn]), urs, ucs, S.kept, 1, S.rows, S.kept});
      for (auto& kv : coloff[si]) {
        int rr = kv.first;
        int p2 = ls.find(BR.q[rr] - S.q);
        int bi = n2.block_of(mn, p2);
        const SiteBlock& B = n2.blk[bi];
        int C = B.m * B.dr;
        sc.items.push_back(CItem{mkref(S_AUX2, vbase + kv.second * vcs), mkref(S_Y, B.off), vrs, vcs, C, 1, S.kept, C});
      }
    }
    check_plan(sc, caps({{S_AUX2, ws}, {S_X, n1.size}, {S_Y, n2.size}}), "split scatter");
    DevCopyBuf sd;
    upload(c, sc, sd);
    Bases b2{};
    b2.p[S_X] = A1.p;
    b2.p[S_Y] = A2.p;
    b2.p[S_AUX2] = r->ws.p;
    CK(launch_copy(sd.d, b2, st));
    release(c, sd);
    // absorb singular values
    for (size_t si = 0; si < sec.size(); ++si) {
      const SvdSector& S = sec[si];
      if (S.kept == 0) continue;
      int mn = newidx[si];
      const double* sv = wsp + S.s;
      if (left_canonical) {
        for (const SiteBlock& B : n2.blk)
          if (B.l == mn) {
            int C = B.m * B.dr;
            CK(launch_scale_rc((double*)A2.p + B.off, C, C, S.kept, sv, 1, st));
          }
      } else {
        CK(launch_scale_rc((double*)A1.p + n1.grp_off[mn], S.kept, S.kept, (int)n1.grp_rows[mn], sv, 0, st));
      }
    }
    CK(cudaStreamSynchronize(st));
    std::swap(r->A[j], A1);
    std::swap(r->A[j + 1], A2);
    dfree(c, A1);
    dfree(c, A2);
    r->bond[j + 1] = nb;
    r->lay[j] = n1;
    r->lay[j + 1] = n2;
    invalidate_bond(j + 1);
    ensure_vec_capacity();
  }

  void two_site_exp(int j, const SiteLayout& C2, DBuf& Cbuf, double t) {
    const Mpo& m = M();
    MpoSite w12 = combine_two_sites(m, j, r->mpo->ls2);
    SitePlanHost h = build_site_plan(r->bond[j], r->bond[j + 2], r->mpo->ls2, w12.terms, m.chan[j], m.chan[j + 2], mixed());
    validate_site(h, r->bond[j], r->bond[j + 2], m.chan[j], m.chan[j + 2], mixed());
    DevGemmBuf s1, s3;
    DevGatherBuf s2;
    DevCopyBuf xs;
    upload(c, h.s1, s1);
    upload(c, h.s2, s2);
    upload(c, h.s3, s3);
    upload(c, h.xsplit, xs);
    if (mixed()) ensure(c, r->Xs, (size_t)std::max<int64_t>(h.xt_size, 1) * 2 * r->nsplit);
    ensure(c, r->T1, (size_t)std::max<int64_t>(h.t1_size, 1) * 8);
    ensure(c, r->T2, (size_t)std::max<int64_t>(h.t2_size, 1) * 8);
    int64_t n = C2.size;
    if (n > r->ldq) {
      r->ldq = n + n / 4 + 64;
      ensure(c, r->Qk, (size_t)r->ldq * r->opts.krylov_dim * 8);
      ensure(c, r->W, (size_t)r->ldq * 8);
      ensure(c, r->tmp, (size_t)r->ldq * 8);
      ensure(c, r->Xn, (size_t)r->ldq * 4 * 2);
    }
    auto apply = [&](const double* x, double* y) {
      Bases b{};
      b.p[S_Y] = y;
      b.p[S_T1] = r->T1.p;
      b.p[S_T2] = r->T2.p;
      if (mixed()) {
        Bases bx{};
        bx.p[S_X] = (void*)x;
        bx.p[S_Y] = r->Xs.p;
        bx.lo[S_Y] = h.xt_size;
        CK(launch_split_copy(xs.d, bx, r->nsplit, st));
        b.p[S_X] = r->Xs.p; b.lo[S_X] = h.xt_size;
        b.p[S_L] = r->Lsp[j].p; b.lo[S_L] = r->Lpsize[j];
        b.p[S_R] = r->Rsp[j + 2].p; b.lo[S_R] = r->Rpsize[j + 2];
        b.lo[S_T2] = h.t2_size;
        CK(launch_gemm_bf16(s1.d, b, r->nsplit, st));
        CK(launch_gather(s2.d, b, 1, r->nsplit, st));
        CK(launch_gemm_bf16(s3.d, b, r->nsplit, st));
      } else {
        b.p[S_X] = (void*)x;
        b.p[S_L] = r->L[j].p;
        b.p[S_R] = r->R[j + 2].p;
        CK(launch_gemm_f64(s1.d, b, st));
        CK(launch_gather(s2.d, b, 0, 0, st));
        CK(launch_gemm_f64(s3.d, b, st));
      }
    };
    lanczos(dptr(Cbuf), n, t, apply);
    CK(cudaStreamSynchronize(st));
    release(c, s1);
    release(c, s2);
    release(c, s3);
    release(c, xs);
  }

  void grow_sweep_lr(double tau) {
    const int N = r->N;
    for (int j = 0; j + 1 < N; ++j) {
      SiteLayout C2 = make_site_layout(r->bond[j], r->bond[j + 2], r->mpo->ls2);
      DBuf Cbuf;
      merge_two(j, C2, Cbuf);
      two_site_exp(j, C2, Cbuf, -tau);
      split_two(j, C2, Cbuf, true);
      dfree(c, Cbuf);
      update_left_env(j);
      if (j < N - 2) site_exp(j + 1, +tau);
    }
  }
  void grow_sweep_rl(double tau) {
    for (int j = r->N - 2; j >= 0; --j) {
      SiteLayout C2 = make_site_layout(r->bond[j], r->bond[j + 2], r->mpo->ls2);
      DBuf Cbuf;
      merge_two(j, C2, Cbuf);
      two_site_exp(j, C2, Cbuf, -tau);
      split_two(j, C2, Cbuf, false);
      dfree(c, Cbuf);
      update_right_env(j + 1);
      if (j > 0) site_exp(j, +tau);
    }
  }

  bool saturated() const {
    const int N = r->N;
    for (int k = 1; k < N; ++k) {
      int64_t cap = r->opts.D_max;
      int e = std::min(k, N - k);
      int64_t p = 1;
      for (int i = 0; i < e && p < cap; ++i) p *= 16;
      cap = std::min(cap, p);
      if (r->bond[k].total() != cap) return false;
    }
    return true;
  }

  void check_bad() {
    RhoScalars rs;
    CK(cudaMemcpyAsync(&rs, r->rs.p, sizeof(rs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    check_tc();  // an aborted GEMM leaves garbage behind: report the cause first
    if (rs.bad) throw Err{TT_ERR_NUMERIC, "non-finite or zero norm in a Krylov update"};
  }
  void check_tc() {
    if (!r->tcerr.p) return;
    int e = 0;
    CK(cudaMemcpyAsync(&e, r->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (e) throw Err{TT_ERR_TIMEOUT, "a bounded mbarrier wait of the tcgen05 GEMM expired"};
  }
};

tt_status fail(tt_ctx* c, const Err& e) {
  if (c) c->err = e.msg;
  return e.st;
}

template <class F>
tt_status guarded(tt_ctx* c, tt_rho* r, F f) {
  if (r && r->poisoned) {
    if (c) c->err = "object poisoned by an earlier error";
    return TT_ERR_STATE;
  }
  try {
    f();
    return TT_OK;
  } catch (const Err& e) {
    if (r && (e.st == TT_ERR_CUDA || e.st == TT_ERR_NUMERIC || e.st == TT_ERR_TIMEOUT)) r->poisoned = true;
    return fail(c, e);
  } catch (const std::bad_alloc&) {
    if (r) r->poisoned = true;
    return fail(c, Err{TT_ERR_OOM, "host allocation failed"});
  } catch (const std::exception& e) {
    if (r) r->poisoned = true;
    return fail(c, Err{TT_ERR_STATE, e.what()});
  }
}

void alloc_rho_arrays(tt_rho* r) {
  const int N = r->N;
  r->A.assign(N, DBuf());
  r->L.assign(N + 1, DBuf());
  r->R.assign(N + 1, DBuf());
  r->Lsp.assign(N + 1, DBuf());
  r->Rsp.assign(N + 1, DBuf());
  r->Lsize.assign(N + 1, 0);
  r->Rsize.assign(N + 1, 0);
  r->Lpsize.assign(N + 1, 0);
  r->Rpsize.assign(N + 1, 0);
  r->esplit.assign(N + 1, DevCopyBuf());
  r->edig.assign(N + 1, DevDigitBuf());
  r->esplit_ok.assign(N + 1, 0);
  {
    const char* gk = std::getenv("TT_GEMM_KERNEL");
    r->use_tc = !(gk && std::strcmp(gk, "mma") == 0);
    const char* gg = std::getenv("TT_CUDA_GRAPH");
    r->use_graph = !(gg && std::strcmp(gg, "0") == 0);
    const char* gq = std::getenv("TT_QR");
    r->use_cholqr = !(gq && std::strcmp(gq, "householder") == 0);
  }
  r->sp.assign(N, SiteDev());
  r->sp64.assign(N, SiteDev());
  r->bp.assign(N + 1, BondDev());
  r->qrl.assign(N, QrDev());
  r->lqr.assign(N, QrDev());
  r->absl.assign(N, DevGemmBuf());
  r->absr.assign(N, DevGemmBuf());
  r->absl_ok.assign(N, 0);
  r->absr_ok.assign(N, 0);
  r->meas.assign(N, MeasDev());
  tt_ctx* c = r->ctx;
  ensure(c, r->partial, (size_t)lanczos_nblk() * 17 * 8);
  ensure(c, r->ks, sizeof(KrylovState));
  ensure(c, r->rs, sizeof(RhoScalars));
  CK(cudaMemsetAsync(r->rs.p, 0, sizeof(RhoScalars), c->st));
}

void free_rho(tt_rho* r) {
  tt_ctx* c = r->ctx;
  for (auto& b : r->A) dfree(c, b);
  for (auto* v : {&r->L, &r->R, &r->Lsp, &r->Rsp})
    for (auto& b : *v) dfree(c, b);
  for (auto* v : {&r->sp, &r->sp64})
    for (auto& s : *v) {
      release(c, s.s1); release(c, s.s2); release(c, s.s3); release(c, s.s3l); release(c, s.r1); release(c, s.r2);
      release(c, s.r3); release(c, s.xs); release(c, s.xd);
    }
  for (auto& e : r->esplit) release(c, e);
  for (auto& e : r->edig) release(c, e);
  for (auto& s : r->bp) {
    release(c, s.b1); release(c, s.b2); release(c, s.xs); release(c, s.ts); release(c, s.xd); release(c, s.td);
  }
  for (auto* v : {&r->qrl, &r->lqr})
    for (auto& q : *v) {
      dfree(c, q.jobs); release(c, q.gather); release(c, q.scatter); release(c, q.rout);
      for (int p = 0; p < 3; ++p) { release(c, q.gram[p]); release(c, q.app[p]); dfree(c, q.cjobs[p]); }
      release(c, q.tt); release(c, q.rf); dfree(c, q.fail);
    }
  for (auto& g : r->absl) release(c, g);
  for (auto& g : r->absr) release(c, g);
  for (auto& m : r->meas) { release(c, m.t); release(c, m.el); dfree(c, m.items); }
  for (DBuf* b : {&r->Qk, &r->W, &r->Xs, &r->Xn, &r->T1, &r->T2, &r->Sb, &r->ws, &r->partial, &r->ks, &r->rs, &r->tmp, &r->obs, &r->el0, &r->el1, &r->tcerr, &r->qrfb})
    dfree(c, *b);
}

// the growth stage's two-site contractions have no digit path: the exact
// split grows in FP64
int growth_arith(int prec) { return prec == 3 ? 0 : prec; }

bool valid_opts(const tt_run_opts* o) {
  return o && o->D_max >= 1 && o->krylov_dim >= 1 && o->krylov_dim <= 16 && o->precision >= 0 && o->precision <= 3 &&
         o->growth_precision >= -1 && o->growth_precision <= 3 && o->svd_cut >= 0 && o->degen_tol >= 0 &&
         o->env_precision >= -1 && o->env_precision <= 2;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

// the statistics window: opened by the first step call after tt_stats_get
void stats_open(tt_rho* rho, cudaStream_t st) {
  if (rho->stats_pending) return;
  rho->heff_flops_acc = rho->step_flops_acc = 0;
  rho->launches_acc = 0;
  rho->qr_sectors_acc = 0;
  rho->evused = 0;
  for (int k = 0; k < 13; ++k) { rho->kind_ms[k] = 0; rho->kind_n[k] = 0; rho->kind_flops[k] = 0; }
  CK(cudaEventRecord(rho->ev0, st));
}

void count_replay(tt_rho* rho) {
  rho->heff_flops_acc += rho->graph_heff_flops;
  rho->step_flops_acc += rho->graph_step_flops;
  rho->launches_acc += rho->graph_launches;
  rho->qr_sectors_acc += rho->graph_qr_sectors;
  ++rho->graph_replays;
}

void stats_close(tt_rho* rho, cudaStream_t st) {
  CK(cudaEventRecord(rho->ev1, st));
  rho->stats.heff_flops = rho->heff_flops_acc;
  rho->stats.step_flops = rho->step_flops_acc;
  rho->stats.launches = rho->launches_acc;
  rho->stats.qr_sectors = rho->qr_sectors_acc;
  rho->stats.n_sites = rho->N;
  rho->stats_pending = true;
}

}  // namespace

namespace tt {

bool rho_graph_current(const tt_rho* rho, double dtau) {
  return rho && rho->graph && rho->graph_tmpl && !rho->poisoned && !rho->prof && !rho->graph_prof &&
         rho->graph_dtau == dtau && rho->graph_buf_gen == rho->ctx->buf_gen && rho->graph_wait_ns == rho->ctx->wait_ns;
}

void rho_account_replays(tt_rho* rho, double dtau, int n, cudaStream_t st, bool before) {
  if (before) {
    stats_open(rho, st);
    return;
  }
  for (int i = 0; i < n; ++i) {
    count_replay(rho);
    rho->beta += dtau;
  }
  stats_close(rho, st);
}

}  // namespace tt

extern "C" {

tt_status tt_ctx_create(const tt_alloc_cb* alloc, void* cuda_stream, tt_ctx** out) {
  if (!out) return TT_ERR_INVALID_ARG;
  *out = nullptr;
  tt_ctx* c = new (std::nothrow) tt_ctx();
  if (!c) return TT_ERR_OOM;
  c->st = (cudaStream_t)cuda_stream;
  if (alloc) {
    if (!alloc->alloc || !alloc->free) { delete c; return TT_ERR_INVALID_ARG; }
    c->cb = *alloc;
    c->has_cb = true;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TT_ERR_CUDA;
  }
  *out = c;
  return TT_OK;
}

void tt_ctx_destroy(tt_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  if (ctx->sol) cusolverDnDestroy(ctx->sol);
  delete ctx;
}

const char* tt_last_error(const tt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tt_status tt_ctx_set_wait_limit(tt_ctx* ctx, double seconds) {
  if (!ctx || !std::isfinite(seconds) || seconds < 0 || seconds > 60) return TT_ERR_INVALID_ARG;
  ctx->wait_ns = (long long)(seconds * 1e9);
  return TT_OK;
}

tt_status tt_hubbard_mpo_create(tt_ctx* ctx, const tt_model* m, tt_mpo** out) {
  if (!ctx || !m || !out) return TT_ERR_INVALID_ARG;
  *out = nullptr;
  if (m->Lx < 1 || m->Wy < 1 || (long long)m->Lx * m->Wy > 512 || m->Lx * m->Wy < 2) {
    ctx->err = "geometry must satisfy Lx, Wy >= 1, 2 <= Lx*Wy <= 512";
    return TT_ERR_INVALID_ARG;
  }
  if (!std::isfinite(m->tp)) {
    ctx->err = "next-nearest hopping tp must be finite";
    return TT_ERR_INVALID_ARG;
  }
  if (m->interaction_form != 0 && m->interaction_form != 1) {
    ctx->err = "interaction_form must be 0 or 1";
    return TT_ERR_INVALID_ARG;
  }
  if (!std::isfinite(m->t) || !std::isfinite(m->U) || !std::isfinite(m->mu)) {
    ctx->err = "non-finite model parameter";
    return TT_ERR_INVALID_ARG;
  }
  tt_mpo* p = new (std::nothrow) tt_mpo();
  if (!p) return TT_ERR_OOM;
  p->ctx = ctx;
  p->spec = ModelSpec{m->Lx, m->Wy, m->bc_y_periodic, m->t, m->U, m->mu, m->interaction_form, m->tp};
  p->mpo = build_hubbard_mpo(p->spec);
  p->ls2 = product_space(p->mpo.ls, p->mpo.ls);
  *out = p;
  return TT_OK;
}

void tt_mpo_destroy(tt_mpo* mpo) { delete mpo; }

int tt_mpo_num_sites(const tt_mpo* mpo) { return mpo ? mpo->mpo.N : 0; }

int tt_mpo_bond_dim(const tt_mpo* mpo, int k) {
  if (!mpo || k < 0 || k > mpo->mpo.N) return 0;
  return (int)mpo->mpo.chan[k].size();
}

tt_status tt_mpo_channel_charge(const tt_mpo* mpo, int k, int w, int* qn, int* qs) {
  if (!mpo || k < 0 || k > mpo->mpo.N || w < 0 || w >= (int)mpo->mpo.chan[k].size() || !qn || !qs)
    return TT_ERR_INVALID_ARG;
  *qn = mpo->mpo.chan[k][w].n;
  *qs = mpo->mpo.chan[k][w].s;
  return TT_OK;
}

tt_status tt_rho_create(tt_ctx* ctx, const tt_mpo* mpo, double beta0, int taylor_order, const tt_run_opts* opts,
                        tt_rho** out) {
  if (!ctx || !mpo || !out || !valid_opts(opts) || taylor_order < 1 || taylor_order > 8 || !(beta0 > 0) ||
      !std::isfinite(beta0)) {
    if (ctx) ctx->err = "invalid argument to tt_rho_create";
    return TT_ERR_INVALID_ARG;
  }
  *out = nullptr;
  tt_rho* r = new (std::nothrow) tt_rho();
  if (!r) return TT_ERR_OOM;
  r->ctx = ctx;
  r->mpo = mpo;
  r->opts = *opts;
  r->N = mpo->mpo.N;
  r->nsplit = opts->growth_precision == 1 ? 2 : (opts->growth_precision == 2 ? 3 : 0);
  tt_status s = guarded(ctx, r, [&] {
    alloc_rho_arrays(r);
    Eng e(r);
    if (taylor_order == 1) e.init_state(beta0);
    else e.init_series(beta0, taylor_order);
  });
  if (s != TT_OK) {
    free_rho(r);
    delete r;
    return s;
  }
  *out = r;
  return TT_OK;
}

void tt_rho_destroy(tt_rho* rho) {
  if (!rho) return;
  cudaStreamSynchronize(rho->ctx->st);
  for (cudaEvent_t e : rho->evpool) cudaEventDestroy(e);
  for (cudaEvent_t e : rho->gpool) cudaEventDestroy(e);
  if (rho->graph) cudaGraphExecDestroy(rho->graph);
  if (rho->graph_tmpl) cudaGraphDestroy(rho->graph_tmpl);
  if (rho->ev0) cudaEventDestroy(rho->ev0);
  if (rho->ev1) cudaEventDestroy(rho->ev1);
  free_rho(rho);
  cudaStreamSynchronize(rho->ctx->st);
  delete rho;
}

tt_status tt_rho_grow(tt_rho* rho, const tt_mpo* mpo, double dtau, double beta_max, double* beta_reached) {
  if (!rho || mpo != rho->mpo || !(dtau > 0)) return TT_ERR_INVALID_ARG;
  return guarded(rho->ctx, rho, [&] {
    Eng e(rho);
    e.set_precision(growth_arith(rho->opts.growth_precision));
    while (rho->beta < beta_max - 1e-12 && !e.saturated()) {
      e.grow_sweep_lr(dtau / 4);
      e.grow_sweep_rl(dtau / 4);
      rho->beta += dtau;
      e.check_bad();
    }
    if (beta_reached) *beta_reached = rho->beta;
  });
}

tt_status tt_rho_grow_exp(tt_rho* rho, const tt_mpo* mpo, double ratio, double beta_max, double* beta_reached) {
  if (!rho || mpo != rho->mpo || !(ratio > 1.0) || !(ratio <= 4.0) || !std::isfinite(beta_max))
    return TT_ERR_INVALID_ARG;
  return guarded(rho->ctx, rho, [&] {
    Eng e(rho);
    e.set_precision(growth_arith(rho->opts.growth_precision));
    while (rho->beta < beta_max - 1e-12 && !e.saturated()) {
      const double dtau = std::min(rho->beta * (ratio - 1.0), beta_max - rho->beta);
      e.grow_sweep_lr(dtau / 4);
      e.grow_sweep_rl(dtau / 4);
      rho->beta += dtau;
      e.check_bad();
    }
    if (beta_reached) *beta_reached = rho->beta;
  });
}

tt_status tt_tdvp_step(tt_rho* rho, const tt_mpo* mpo, double dtau, int n_steps) {
  if (!rho || mpo != rho->mpo || !(dtau > 0) || n_steps < 0) return TT_ERR_INVALID_ARG;
  return guarded(rho->ctx, rho, [&] {
    Eng e(rho);
    e.set_precision(rho->opts.precision);
    e.prepare_all();
    if (!rho->ev0) CK(cudaEventCreate(&rho->ev0));
    if (!rho->ev1) CK(cudaEventCreate(&rho->ev1));
    cudaStream_t st = rho->ctx->st;
    // statistics accumulate over the calls since the last tt_stats_get
    stats_open(rho, st);
    if (rho->graph && (rho->graph_dtau != dtau || rho->graph_prof != rho->prof ||
                       rho->graph_buf_gen != rho->ctx->buf_gen || rho->graph_wait_ns != rho->ctx->wait_ns))
      e.drop_graph();
    int s = 0;
    if (!rho->graph && rho->use_graph && n_steps > 0 && st != nullptr && !rho->stats_pending) {
      // one uncaptured step builds every plan, tensor map and buffer, then one
      // step is captured (no allocation or host synchronisation happens in it)
      e.sweep_lr(dtau / 4);
      e.sweep_rl(dtau / 4);
      rho->beta += dtau;
      ++s;
      const double hf = rho->heff_flops_acc, sf = rho->step_flops_acc;
      const long long ln = rho->launches_acc, qn = rho->qr_sectors_acc;
      // profiling events of the captured step live in their own pool, created
      // before the capture
      rho->gused = 0;
      for (int k = 0; k < 13; ++k) rho->graph_kind_flops[k] = 0;
      if (rho->prof)
        while (rho->gpool.size() < rho->evused + 512) {
          cudaEvent_t x;
          CK(cudaEventCreate(&x));
          rho->gpool.push_back(x);
          rho->gkind.push_back(0);
        }
      cudaGraph_t g = nullptr;
      const unsigned long long gen0 = rho->ctx->buf_gen;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      rho->capturing = true;
      bool ok = true;
      try {
        e.sweep_lr(dtau / 4);
        e.sweep_rl(dtau / 4);
      } catch (...) {
        ok = false;
      }
      rho->capturing = false;
      cudaError_t ce = cudaStreamEndCapture(st, &g);
      if (rho->ctx->buf_gen != gen0) ok = false;  // a buffer was replaced inside the capture
      if (!ok || ce != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        throw Err{TT_ERR_CUDA, "capture of the beta-step failed"};
      }
      cudaError_t ie = cudaGraphInstantiate(&rho->graph, g, 0);
      if (ie != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        rho->graph = nullptr;
        throw Err{TT_ERR_CUDA, "graph instantiation failed"};
      }
      rho->graph_tmpl = g;
      ++rho->graph_gen;
      rho->graph_dtau = dtau;
      rho->graph_prof = rho->prof;
      rho->graph_wait_ns = rho->ctx->wait_ns;
      rho->graph_buf_gen = rho->ctx->buf_gen;
      rho->graph_heff_flops = rho->heff_flops_acc - hf;
      rho->graph_step_flops = rho->step_flops_acc - sf;
      rho->graph_launches = rho->launches_acc - ln;
      rho->graph_qr_sectors = rho->qr_sectors_acc - qn;
      rho->qr_sectors_acc = qn;
      // the captured step has not run yet: undo its host-side bookkeeping
      rho->heff_flops_acc = hf;
      rho->step_flops_acc = sf;
      rho->launches_acc = ln;
      rho->graph_replays = 0;
    }
    for (; s < n_steps; ++s) {
      if (rho->graph) {
        CK(cudaGraphLaunch(rho->graph, st));
        count_replay(rho);
      } else {
        e.sweep_lr(dtau / 4);
        e.sweep_rl(dtau / 4);
      }
      rho->beta += dtau;
    }
    stats_close(rho, st);
  });
}



tt_status tt_measure(tt_rho* rho, const tt_mpo* mpo, tt_obs* out) {
  if (!rho || mpo != rho->mpo || !out) return TT_ERR_INVALID_ARG;
  return guarded(rho->ctx, rho, [&] {
    Eng e(rho);
    e.measure(out);
  });
}

tt_status tt_stats_get(const tt_rho* rho_c, tt_stats* out) {
  if (!rho_c || !out) return TT_ERR_INVALID_ARG;
  tt_rho* rho = const_cast<tt_rho*>(rho_c);
  if (rho->stats_pending) {
    float ms = 0;
    cudaError_t ce = cudaEventSynchronize(rho->ev1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, rho->ev0, rho->ev1);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      rho->ctx->err = std::string("step timing events: ") + cudaGetErrorString(ce);
      return TT_ERR_CUDA;
    }
    rho->stats.step_ms = ms;
    for (size_t i = 0; i + 1 < rho->evused; i += 2) {
      float t = 0;
      cudaError_t ee = cudaEventElapsedTime(&t, rho->evpool[i], rho->evpool[i + 1]);
      if (ee != cudaSuccess) {
        cudaGetLastError();
        rho->ctx->err = std::string("profiling events: ") + cudaGetErrorString(ee);
        return TT_ERR_CUDA;
      }
      rho->kind_ms[rho->evkind[i]] += t;
      rho->kind_n[rho->evkind[i]] += 1;
    }
    // events inside the graph hold the times of its last replay; every replay
    // runs the same launches, so they stand for all replays since the reset
    if (rho->graph_replays > 0 && rho->graph_prof) {
      for (size_t i = 0; i + 1 < rho->gused; i += 2) {
        float t = 0;
        cudaError_t ee = cudaEventElapsedTime(&t, rho->gpool[i], rho->gpool[i + 1]);
        if (ee != cudaSuccess) {
          cudaGetLastError();
          rho->ctx->err = std::string("profiling events inside the graph: ") + cudaGetErrorString(ee);
          return TT_ERR_CUDA;
        }
        rho->kind_ms[rho->gkind[i]] += t * rho->graph_replays;
        rho->kind_n[rho->gkind[i]] += rho->graph_replays;
      }
      for (int k = 0; k < 13; ++k) rho->kind_flops[k] += rho->graph_kind_flops[k] * rho->graph_replays;
    }
    rho->graph_replays = 0;
    rho->stats.heff_ms = rho->kind_ms[0];
    rho->stats.heff_launches = rho->kind_n[0];
    rho->stats.env_ms = rho->kind_ms[1];
    rho->stats.env_flops = rho->kind_flops[1];
    rho->stats.bond_ms = rho->kind_ms[2];
    rho->stats.bond_flops = rho->kind_flops[2];
    rho->stats.gather_ms = rho->kind_ms[3];
    rho->stats.gather_launches = rho->kind_n[3];
    rho->stats.qr_ms = rho->kind_ms[5];
    rho->stats.site_exp_ms = rho->kind_ms[6];
    rho->stats.bond_exp_ms = rho->kind_ms[7];
    rho->stats.env_update_ms = rho->kind_ms[8];
    rho->stats.absorb_ms = rho->kind_ms[9];
    rho->stats.gauge_ms = rho->kind_ms[10];
    rho->stats.qr_gemm_ms = rho->kind_ms[11];
    rho->stats.qr_gemm_flops = rho->kind_flops[11];
    rho->stats.qr_chol_ms = rho->kind_ms[12];
    rho->stats.qr_fallbacks = 0;
    if (rho->qrfb.p) {
      int nfb = 0;
      cudaStream_t cs = rho->ctx->st;
      cudaError_t fe = cudaMemcpyAsync(&nfb, rho->qrfb.p, sizeof(int), cudaMemcpyDeviceToHost, cs);
      if (fe == cudaSuccess) fe = cudaMemsetAsync(rho->qrfb.p, 0, sizeof(int), cs);
      if (fe == cudaSuccess) fe = cudaStreamSynchronize(cs);
      if (fe != cudaSuccess) {
        cudaGetLastError();
        rho->ctx->err = std::string("QR fallback counter: ") + cudaGetErrorString(fe);
        return TT_ERR_CUDA;
      }
      rho->stats.qr_fallbacks = nfb;
    }
    rho->stats_pending = false;
  }
  *out = rho->stats;
  int mb = 1, ns = 1;
  for (auto& b : rho->bond) { mb = std::max<int>(mb, (int)b.total()); ns = std::max(ns, b.nsec()); }
  out->max_bond = mb;
  out->n_sectors_max = ns;
  out->tuned_tc128 = rho->tuned[TK_TC128];
  out->tuned_tcp128x64 = rho->tuned[TK_TCP128X64];
  out->tuned_mma64 = rho->tuned[TK_MMA64];
  return TT_OK;
}

tt_status tt_rho_bond_dims(const tt_rho* rho, int* dims, int n) {
  if (!rho || !dims || n < rho->N + 1) return TT_ERR_INVALID_ARG;
  for (int k = 0; k <= rho->N; ++k) dims[k] = (int)rho->bond[k].total();
  return TT_OK;
}

tt_status tt_rho_bond_sectors(const tt_rho* rho, int k, int* qn, int* qs, int* dims, int cap, int* nsec) {
  if (!rho || !nsec || k < 0 || k > rho->N) return TT_ERR_INVALID_ARG;
  const tt::Bond& B = rho->bond[k];
  *nsec = B.nsec();
  if (cap < B.nsec() || !qn || !qs || !dims) return TT_ERR_INVALID_ARG;
  for (int i = 0; i < B.nsec(); ++i) {
    qn[i] = B.q[i].n;
    qs[i] = B.q[i].s;
    dims[i] = B.dim[i];
  }
  return TT_OK;
}


static bool read_bonds_lr(const tt_mpo* mpo, int site, const int* nsec_lr, const int* qn, const int* qs,
                          const int* qd, Bond& BL, Bond& BR) {
  if (!mpo || !nsec_lr || !qn || !qs || !qd || site < 0 || site >= mpo->mpo.N) return false;
  int o = 0;
  for (int side = 0; side < 2; ++side) {
    Bond& B = side == 0 ? BL : BR;
    int n = nsec_lr[side];
    if (n < 1 || n > 100000) return false;
    for (int i = 0; i < n; ++i, ++o) {
      if (qd[o] < 1) return false;
      Q q{qn[o], qs[o]};
      if (!B.q.empty() && !(B.q.back() < q)) return false;
      B.q.push_back(q);
      B.dim.push_back(qd[o]);
    }
  }
  return true;
}

tt_status tt_layout_sizes(const tt_mpo* mpo, int site, const int* nsec_lr, const int* qn, const int* qs, const int* qd,
                          int64_t* x_size, int64_t* l_size, int64_t* r_size) {
  Bond BL, BR;
  if (!read_bonds_lr(mpo, site, nsec_lr, qn, qs, qd, BL, BR)) return TT_ERR_INVALID_ARG;
  const Mpo& m = mpo->mpo;
  if (x_size) *x_size = make_site_layout(BL, BR, m.ls).size;
  if (l_size) *l_size = make_env_layout(BL, m.chan[site]).size;
  if (r_size) *r_size = make_env_layout(BR, m.chan[site + 1]).size;
  return TT_OK;
}

static tt_status heff_apply_impl(tt_ctx* ctx, const tt_mpo* mpo, int site, int precision, const Bond& BL,
                                 const Bond& BR, const double* Lh, const double* Rh, const double* xh, double* yh) {
  tt_rho* r = new (std::nothrow) tt_rho();
  if (!r) return TT_ERR_OOM;
  r->ctx = ctx;
  r->mpo = mpo;
  r->opts = tt_run_opts{1, 1, precision, precision, 1e-12, 1e-10, 0};
  r->N = mpo->mpo.N;
  r->nsplit = (precision == 1) ? 2 : (precision == 2 ? 3 : (precision == 3 ? 4 : 0));
  r->exact = precision == 3;
  tt_status s = guarded(ctx, nullptr, [&] {
    alloc_rho_arrays(r);
    r->bond.assign(r->N + 1, Bond());
    r->bond[site] = BL;
    r->bond[site + 1] = BR;
    r->lay.assign(r->N, SiteLayout());
    Eng e(r);
    e.relayout(site);
    e.ensure_vec_capacity();
    e.ensure_site_buf(site);
    e.ensure_env(r->L, r->Lsp, r->Lsize, site);
    e.ensure_env(r->R, r->Rsp, r->Rsize, site + 1);
    const int64_t nx = r->lay[site].size;
    CK(cudaMemcpyAsync(r->A[site].p, xh, nx * 8, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(r->L[site].p, Lh, r->Lsize[site] * 8, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(r->R[site + 1].p, Rh, r->Rsize[site + 1] * 8, cudaMemcpyHostToDevice, ctx->st));
    e.split_env(r->L, r->Lsp, r->Lsize, site);
    e.split_env(r->R, r->Rsp, r->Rsize, site + 1);
    e.apply_site(site, (const double*)r->A[site].p, (double*)r->W.p);
    CK(cudaMemcpyAsync(yh, r->W.p, nx * 8, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    e.check_tc();
  });
  cudaStreamSynchronize(ctx->st);
  free_rho(r);
  cudaStreamSynchronize(ctx->st);
  delete r;
  return s;
}

tt_status tt_heff_apply_host(tt_ctx* ctx, const tt_mpo* mpo, int site, int precision, const int* nsec_lr,
                             const int* qn, const int* qs, const int* qd, const double* Lh, const double* Rh,
                             const double* xh, double* yh) {
  if (!ctx || !mpo || !Lh || !Rh || !xh || !yh || precision < 0 || precision > 3) return TT_ERR_INVALID_ARG;
  Bond BL, BR;
  if (!read_bonds_lr(mpo, site, nsec_lr, qn, qs, qd, BL, BR)) {
    ctx->err = "invalid sector tables";
    return TT_ERR_INVALID_ARG;
  }
  return heff_apply_impl(ctx, mpo, site, precision, BL, BR, Lh, Rh, xh, yh);
}

tt_status tt_heff_apply_terms_host(tt_ctx* ctx, int nw_l, const int* chl_qn, const int* chl_qs, int nw_r,
                                   const int* chr_qn, const int* chr_qs, int nterms, const int* t_wl, const int* t_wr,
                                   const int* t_sig, const int* t_tau, const double* t_val, int precision,
                                   const int* nsec_lr, const int* qn, const int* qs, const int* qd, const double* Lh,
                                   const double* Rh, const double* xh, double* yh) {
  if (!ctx || !chl_qn || !chl_qs || !chr_qn || !chr_qs || nw_l < 1 || nw_r < 1 || nw_l > 4096 || nw_r > 4096 ||
      nterms < 0 || (nterms > 0 && (!t_wl || !t_wr || !t_sig || !t_tau || !t_val)) || !Lh || !Rh || !xh || !yh ||
      precision < 0 || precision > 3)
    return TT_ERR_INVALID_ARG;
  tt_mpo m;
  m.ctx = ctx;
  m.mpo.N = 1;
  m.mpo.Lx = 1;
  m.mpo.Wy = 1;
  m.mpo.ls = hubbard_site_space();
  m.mpo.chan.assign(2, std::vector<Q>());
  for (int w = 0; w < nw_l; ++w) m.mpo.chan[0].push_back(Q{chl_qn[w], chl_qs[w]});
  for (int w = 0; w < nw_r; ++w) m.mpo.chan[1].push_back(Q{chr_qn[w], chr_qs[w]});
  m.mpo.start_ch.assign(2, -1);
  m.mpo.done_ch.assign(2, -1);
  MpoSite site;
  const LocalSpace& ls = m.mpo.ls;
  for (int i = 0; i < nterms; ++i) {
    const int wl = t_wl[i], wr = t_wr[i], sg = t_sig[i], ta = t_tau[i];
    if (wl < 0 || wl >= nw_l || wr < 0 || wr >= nw_r || sg < 0 || sg >= ls.d || ta < 0 || ta >= ls.d ||
        !std::isfinite(t_val[i]) || m.mpo.chan[1][wr] != m.mpo.chan[0][wl] + ls.q[sg] - ls.q[ta]) {
      ctx->err = "invalid MPO term " + std::to_string(i) + " (index out of range, non-finite value, or channel " +
                 "charges violating c_wr = c_wl + q(sig) - q(tau))";
      return TT_ERR_INVALID_ARG;
    }
    site.terms.push_back(MpoTerm{wl, wr, sg, ta, t_val[i]});
  }
  std::sort(site.terms.begin(), site.terms.end(), [](const MpoTerm& a, const MpoTerm& b) {
    return std::make_tuple(a.wr, a.sig, a.wl, a.tau) < std::make_tuple(b.wr, b.sig, b.wl, b.tau);
  });
  m.mpo.site.push_back(site);
  Bond BL, BR;
  if (!read_bonds_lr(&m, 0, nsec_lr, qn, qs, qd, BL, BR)) {
    ctx->err = "invalid sector tables";
    return TT_ERR_INVALID_ARG;
  }
  return heff_apply_impl(ctx, &m, 0, precision, BL, BR, Lh, Rh, xh, yh);
}

tt_status tt_layout_sizes_terms(int nw_l, const int* chl_qn, const int* chl_qs, int nw_r, const int* chr_qn,
                                const int* chr_qs, const int* nsec_lr, const int* qn, const int* qs, const int* qd,
                                int64_t* x_size, int64_t* l_size, int64_t* r_size) {
  if (!chl_qn || !chl_qs || !chr_qn || !chr_qs || nw_l < 1 || nw_r < 1) return TT_ERR_INVALID_ARG;
  tt_mpo m;
  m.mpo.N = 1;
  m.mpo.ls = hubbard_site_space();
  m.mpo.chan.assign(2, std::vector<Q>());
  for (int w = 0; w < nw_l; ++w) m.mpo.chan[0].push_back(Q{chl_qn[w], chl_qs[w]});
  for (int w = 0; w < nw_r; ++w) m.mpo.chan[1].push_back(Q{chr_qn[w], chr_qs[w]});
  return tt_layout_sizes(&m, 0, nsec_lr, qn, qs, qd, x_size, l_size, r_size);
}

static const char kMagic[8] = {'T', 'T', 'R', 'H', 'O', '0', '0', '1'};

tt_status tt_rho_save(tt_rho* rho, const char* path) {
  if (!rho || !path) return TT_ERR_INVALID_ARG;
  return guarded(rho->ctx, rho, [&] {
    RhoScalars rs;
    CK(cudaMemcpyAsync(&rs, rho->rs.p, sizeof(rs), cudaMemcpyDeviceToHost, rho->ctx->st));
    CK(cudaStreamSynchronize(rho->ctx->st));
    std::ofstream f(path, std::ios::binary);
    if (!f) throw Err{TT_ERR_INVALID_ARG, std::string("cannot open ") + path};
    int32_t N = rho->N;
    f.write(kMagic, 8);
    f.write((const char*)&N, 4);
    f.write((const char*)&rho->beta, 8);
    f.write((const char*)&rs.logscale, 8);
    f.write((const char*)&rs.resid_max, 8);
    for (const Bond& B : rho->bond) {
      int32_t n = B.nsec();
      f.write((const char*)&n, 4);
      for (int i = 0; i < n; ++i) {
        int32_t v[3] = {B.q[i].n, B.q[i].s, B.dim[i]};
        f.write((const char*)v, 12);
      }
    }
    for (int j = 0; j < rho->N; ++j) {
      std::vector<double> h(rho->lay[j].size);
      CK(cudaMemcpyAsync(h.data(), rho->A[j].p, h.size() * 8, cudaMemcpyDeviceToHost, rho->ctx->st));
      CK(cudaStreamSynchronize(rho->ctx->st));
      int64_t n = (int64_t)h.size();
      f.write((const char*)&n, 8);
      f.write((const char*)h.data(), n * 8);
    }
    if (!f) throw Err{TT_ERR_INVALID_ARG, "write failed"};
  });
}

tt_status tt_rho_load(tt_ctx* ctx, const tt_mpo* mpo, const char* path, const tt_run_opts* opts, tt_rho** out) {
  if (!ctx || !mpo || !path || !out || !valid_opts(opts)) return TT_ERR_INVALID_ARG;
  *out = nullptr;
  std::ifstream f(path, std::ios::binary);
  if (!f) {
    ctx->err = std::string("cannot open ") + path;
    return TT_ERR_INVALID_ARG;
  }
  char mg[8];
  int32_t N;
  double beta, logscale, resid;
  f.read(mg, 8);
  f.read((char*)&N, 4);
  f.read((char*)&beta, 8);
  f.read((char*)&logscale, 8);
  f.read((char*)&resid, 8);
  if (!f || std::memcmp(mg, kMagic, 8) != 0 || N != mpo->mpo.N) {
    ctx->err = "not a checkpoint of this model";
    return TT_ERR_INVALID_ARG;
  }
  tt_rho* r = new (std::nothrow) tt_rho();
  if (!r) return TT_ERR_OOM;
  r->ctx = ctx;
  r->mpo = mpo;
  r->opts = *opts;
  r->N = N;
  r->nsplit = 0;  // environments are rebuilt in FP64; the step switches precision
  r->beta = beta;
  tt_status s = guarded(ctx, r, [&] {
    alloc_rho_arrays(r);
    r->bond.assign(N + 1, Bond());
    for (int k = 0; k <= N; ++k) {
      int32_t n;
      f.read((char*)&n, 4);
      if (!f || n < 1 || n > 1000000) throw Err{TT_ERR_INVALID_ARG, "corrupt checkpoint"};
      for (int i = 0; i < n; ++i) {
        int32_t v[3];
        f.read((char*)v, 12);
        r->bond[k].q.push_back(Q{v[0], v[1]});
        r->bond[k].dim.push_back(v[2]);
      }
    }
    r->lay.assign(N, SiteLayout());
    Eng e(r);
    for (int j = 0; j < N; ++j) {
      e.relayout(j);
      int64_t n;
      f.read((char*)&n, 8);
      if (!f || n != r->lay[j].size) throw Err{TT_ERR_INVALID_ARG, "corrupt checkpoint"};
      std::vector<double> h(n);
      f.read((char*)h.data(), n * 8);
      if (!f) throw Err{TT_ERR_INVALID_ARG, "truncated checkpoint"};
      e.ensure_site_buf(j);
      CK(cudaMemcpyAsync(r->A[j].p, h.data(), n * 8, cudaMemcpyHostToDevice, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
    RhoScalars rs{logscale, resid, 0, 0};
    CK(cudaMemcpyAsync(r->rs.p, &rs, sizeof(rs), cudaMemcpyHostToDevice, ctx->st));
    e.ensure_vec_capacity();
    e.build_boundary_envs();
    for (int j = N - 1; j >= 1; --j) e.update_right_env(j);
    CK(cudaStreamSynchronize(ctx->st));
  });
  if (s != TT_OK) {
    free_rho(r);
    delete r;
    return s;
  }
  *out = r;
  return TT_OK;
}

tt_status tt_rho_pad(tt_rho* rho, const tt_mpo* mpo, int D_target) {
  if (!rho || mpo != rho->mpo || D_target < 1) return TT_ERR_INVALID_ARG;
  return guarded(rho->ctx, rho, [&] {
    Eng e(rho);
    e.pad_bonds(D_target);
  });
}

tt_status tt_rho_set_profiling(tt_rho* rho, int on) {
  if (!rho) return TT_ERR_INVALID_ARG;
  rho->prof = on != 0;
  return TT_OK;
}

tt_status tt_qr_device(tt_ctx* ctx, const double* A, int m, int n, double* Q, double* R) {
  if (!ctx || !A || !Q || !R || m < 1 || n < 1 || n > 2048 || m < n) {
    if (ctx) ctx->err = "tt_qr_device: need device pointers and 1 <= n <= min(m, 2048)";
    return TT_ERR_INVALID_ARG;
  }
  DBuf ws, job;
  tt_status st = guarded(ctx, nullptr, [&] {
    const int64_t mn = (int64_t)m * n;
    ensure(ctx, ws, (size_t)(2 * mn + (int64_t)n * n) * sizeof(double));
    ensure(ctx, job, sizeof(QrJob));
    QrJob J{0, mn, 2 * mn, m, n};
    CK(cudaMemcpyAsync(job.p, &J, sizeof(J), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ws.p, A, mn * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(launch_qr((const QrJob*)job.p, 1, (double*)ws.p, ctx->st));
    CK(cudaMemcpyAsync(Q, (double*)ws.p + mn, mn * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(R, (double*)ws.p + 2 * mn, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  });
  dfree(ctx, ws);
  dfree(ctx, job);
  return st;
}

}  // extern "C"
