// Batch of independent tanTRG instances (many small models evolved together).
//
// Every instance is an ordinary tt_rho with its own context and CUDA stream,
// so its beta-step is its own captured CUDA graph; a batch step forks all
// instance streams from the caller's stream, replays every instance's graph,
// and joins them back.  The instances share nothing, so their graphs run
// concurrently and together fill the GPU that one small instance cannot.
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
    tt_status s = tt_tdvp_step(in.rho, in.mpo, dtau, n_steps);
    if (s != TT_OK) return fail_inst(b, i, s);
    if (cudaEventRecord(in.done, in.st) != cudaSuccess || cudaStreamWaitEvent(b->ctx->st, in.done, 0) != cudaSuccess) {
      cudaGetLastError();
      return fail_inst(b, i, TT_ERR_CUDA);
    }
  }
  return TT_OK;
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
