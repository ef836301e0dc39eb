// Batch of independent tanTRG instances (many small models evolved together).
//
// Every instance is an ordinary tt_rho with its own context and CUDA stream,
// and its beta-step is captured as its own CUDA graph.  The batch composes
// the instances' step graphs as child nodes of one parent graph (no edges
// between them: the instances share nothing), so a batch beta-step is one
// graph launch on the caller's stream and the device runs every instance's
// kernels concurrently, filling the GPU that one small instance cannot.  The
// first step of a batch (and any step after an instance's graph was replaced,
// or with profiling on) runs per instance on the instance streams, forked
// from and joined back to the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tantrg.h"
#include "tt_engine.h"

struct tt_batch {
  tt_ctx* ctx = nullptr;  // caller's context: stream to order against, error text
  struct Inst {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    tt_ctx* c = nullptr;
    tt_mpo* mpo = nullptr;
    tt_rho* rho = nullptr;
    int D_max = 0;
  };
  std::vector<Inst> inst;
  cudaEvent_t fork = nullptr;
  // parent graph of one batch beta-step, and the instances' graph generations
  // it was composed from
  cudaGraphExec_t parent = nullptr;
  double parent_dtau = 0.0;
  std::vector<unsigned long long> parent_gen;
};

namespace {

void destroy_inst(tt_batch::Inst& in) {
  if (in.rho) tt_rho_destroy(in.rho);
  if (in.mpo) tt_mpo_destroy(in.mpo);
  if (in.c) tt_ctx_destroy(in.c);
  if (in.done) cudaEventDestroy(in.done);
  if (in.st) cudaStreamDestroy(in.st);
  in = tt_batch::Inst();
}

tt_status fail_inst(tt_batch* b, size_t i, tt_status s) {
  const char* msg = b->inst[i].c ? tt_last_error(b->inst[i].c) : "";
  b->ctx->err = "instance " + std::to_string(i) + ": " + (msg ? msg : "");
  return s;
}

// Runs f(i) for every instance on up to 16 host threads (each instance has its
// own context and stream, so their host-side synchronisations overlap);
// returns the first failure in instance order.
template <class F>
tt_status for_each_instance(tt_batch* b, F&& f) {
  const size_t n = b->inst.size();
  std::vector<tt_status> st(n, TT_OK);
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t i; (i = next.fetch_add(1)) < n;) st[i] = f(i);
  };
  const size_t nt = std::min<size_t>(n, 16);
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  for (size_t i = 0; i < n; ++i)
    if (st[i] != TT_OK) return fail_inst(b, i, st[i]);
  return TT_OK;
}

void drop_parent(tt_batch* b) {
  if (b->parent) cudaGraphExecDestroy(b->parent);
  b->parent = nullptr;
}

bool parent_current(const tt_batch* b, double dtau) {
  if (!b->parent || b->parent_dtau != dtau) return false;
  for (size_t i = 0; i < b->inst.size(); ++i)
    if (!tt::rho_graph_current(b->inst[i].rho, dtau) || b->inst[i].rho->graph_gen != b->parent_gen[i]) return false;
  return true;
}

// The parent graph from every instance's current step graph; none (and the
// per-instance path) when some instance has no replayable graph.
void build_parent(tt_batch* b, double dtau) {
  drop_parent(b);
  for (const auto& in : b->inst)
    if (!tt::rho_graph_current(in.rho, dtau)) return;
  cudaGraph_t pg = nullptr;
  if (cudaGraphCreate(&pg, 0) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  bool ok = true;
  for (const auto& in : b->inst) {
    cudaGraphNode_t node;
    if (cudaGraphAddChildGraphNode(&node, pg, nullptr, 0, in.rho->graph_tmpl) != cudaSuccess) {
      ok = false;
      break;
    }
  }
  if (ok && cudaGraphInstantiate(&b->parent, pg, 0) != cudaSuccess) {
    b->parent = nullptr;
    ok = false;
  }
  if (!ok) cudaGetLastError();
  cudaGraphDestroy(pg);
  if (!b->parent) return;
  b->parent_dtau = dtau;
  b->parent_gen.resize(b->inst.size());
  for (size_t i = 0; i < b->inst.size(); ++i) b->parent_gen[i] = b->inst[i].rho->graph_gen;
}

// n beta-steps, one per instance on its own stream (forked from and joined
// back to the caller's stream); captures the instances' graphs when needed
tt_status step_per_instance(tt_batch* b, double dtau, int n) {
  if (cudaEventRecord(b->fork, b->ctx->st) != cudaSuccess) {
    cudaGetLastError();
    b->ctx->err = "batch fork event failed";
    return TT_ERR_CUDA;
  }
  for (size_t i = 0; i < b->inst.size(); ++i) {
    tt_batch::Inst& in = b->inst[i];
    if (cudaStreamWaitEvent(in.st, b->fork, 0) != cudaSuccess) {
      cudaGetLastError();
      return fail_inst(b, i, TT_ERR_CUDA);
    }
    tt_status s = tt_tdvp_step(in.rho, in.mpo, dtau, n);
    if (s != TT_OK) return fail_inst(b, i, s);
    if (cudaEventRecord(in.done, in.st) != cudaSuccess || cudaStreamWaitEvent(b->ctx->st, in.done, 0) != cudaSuccess) {
      cudaGetLastError();
      return fail_inst(b, i, TT_ERR_CUDA);
    }
  }
  return TT_OK;
}

// n replays of the parent graph on the caller's stream, ordered after all
// earlier work of the instance streams and before all later work on them
tt_status step_parent(tt_batch* b, double dtau, int n) {
  cudaStream_t st = b->ctx->st;
  try {
    for (size_t i = 0; i < b->inst.size(); ++i) {
      tt_batch::Inst& in = b->inst[i];
      if (cudaEventRecord(in.done, in.st) != cudaSuccess || cudaStreamWaitEvent(st, in.done, 0) != cudaSuccess)
        throw tt::Err{TT_ERR_CUDA, "batch join event failed"};
    }
    for (auto& in : b->inst) tt::rho_account_replays(in.rho, dtau, n, st, true);
    for (int s = 0; s < n; ++s)
      if (cudaGraphLaunch(b->parent, st) != cudaSuccess) throw tt::Err{TT_ERR_CUDA, "batch graph launch failed"};
    for (auto& in : b->inst) tt::rho_account_replays(in.rho, dtau, n, st, false);
    if (cudaEventRecord(b->fork, st) != cudaSuccess) throw tt::Err{TT_ERR_CUDA, "batch fork event failed"};
    for (auto& in : b->inst)
      if (cudaStreamWaitEvent(in.st, b->fork, 0) != cudaSuccess) throw tt::Err{TT_ERR_CUDA, "batch fork event failed"};
  } catch (const tt::Err& e) {
    cudaGetLastError();
    b->ctx->err = e.msg;
    return e.st;
  }
  return TT_OK;
}

}  // namespace

extern "C" {

tt_status tt_batch_create(tt_ctx* ctx, int n, const tt_model* models, const int* D_max, double beta0,
                          const tt_run_opts* opts, tt_batch** out) {
  if (!ctx || n < 1 || !models || !D_max || !opts || !out) {
    if (ctx) ctx->err = "invalid argument to tt_batch_create";
    return TT_ERR_INVALID_ARG;
  }
  *out = nullptr;
  tt_batch* b = new (std::nothrow) tt_batch();
  if (!b) return TT_ERR_OOM;
  b->ctx = ctx;
  b->inst.resize(n);
  tt_status s = TT_OK;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    s = TT_ERR_CUDA;
  }
  for (int i = 0; i < n && s == TT_OK; ++i) {
    tt_batch::Inst& in = b->inst[i];
    if (cudaStreamCreateWithFlags(&in.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&in.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "stream or event creation failed for instance " + std::to_string(i);
      s = TT_ERR_CUDA;
      break;
    }
    s = tt_ctx_create(ctx->has_cb ? &ctx->cb : nullptr, in.st, &in.c);
    if (s != TT_OK) break;
    tt_run_opts o = *opts;
    o.D_max = D_max[i];
    in.D_max = D_max[i];
    if ((s = tt_hubbard_mpo_create(in.c, &models[i], &in.mpo)) != TT_OK ||
        (s = tt_rho_create(in.c, in.mpo, beta0, 1, &o, &in.rho)) != TT_OK) {
      s = fail_inst(b, i, s);
      break;
    }
  }
  if (s != TT_OK) {
    tt_batch_destroy(b);
    return s;
  }
  *out = b;
  return TT_OK;
}

void tt_batch_destroy(tt_batch* b) {
  if (!b) return;
  drop_parent(b);
  for (auto& in : b->inst) destroy_inst(in);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

int tt_batch_size(const tt_batch* b) { return b ? (int)b->inst.size() : 0; }

tt_status tt_batch_grow(tt_batch* b, double dtau, double beta_max) {
  if (!b || !(dtau > 0)) return TT_ERR_INVALID_ARG;
  return for_each_instance(b, [&](size_t i) {
    double reached = 0;
    return tt_rho_grow(b->inst[i].rho, b->inst[i].mpo, dtau, beta_max, &reached);
  });
}

tt_status tt_batch_pad(tt_batch* b) {
  if (!b) return TT_ERR_INVALID_ARG;
  return for_each_instance(b, [&](size_t i) {
    tt_status s = tt_rho_pad(b->inst[i].rho, b->inst[i].mpo, b->inst[i].D_max);
    if (s == TT_OK) s = cudaStreamSynchronize(b->inst[i].st) == cudaSuccess ? TT_OK : TT_ERR_CUDA;
    return s;
  });
}

tt_status tt_batch_step(tt_batch* b, double dtau, int n_steps) {
  if (!b || !(dtau > 0) || n_steps < 0) return TT_ERR_INVALID_ARG;
  int s = 0;
  if (n_steps > 0 && !parent_current(b, dtau)) {
    // one step per instance (captures or re-captures the instance graphs),
    // then the parent graph from them when every instance has one
    tt_status r = step_per_instance(b, dtau, 1);
    if (r != TT_OK) return r;
    s = 1;
    build_parent(b, dtau);
  }
  if (s == n_steps) return TT_OK;
  if (!b->parent) return step_per_instance(b, dtau, n_steps - s);
  return step_parent(b, dtau, n_steps - s);
}

tt_status tt_batch_measure(tt_batch* b, tt_obs* out_n) {
  if (!b || !out_n) return TT_ERR_INVALID_ARG;
  return for_each_instance(b, [&](size_t i) { return tt_measure(b->inst[i].rho, b->inst[i].mpo, &out_n[i]); });
}

tt_status tt_batch_stats(tt_batch* b, int i, tt_stats* out) {
  if (!b || i < 0 || i >= (int)b->inst.size() || !out) return TT_ERR_INVALID_ARG;
  return tt_stats_get(b->inst[i].rho, out);
}

tt_status tt_batch_set_profiling(tt_batch* b, int on) {
  if (!b) return TT_ERR_INVALID_ARG;
  for (auto& in : b->inst) {
    tt_status s = tt_rho_set_profiling(in.rho, on);
    if (s != TT_OK) return s;
  }
  return TT_OK;
}

}  // extern "C"
