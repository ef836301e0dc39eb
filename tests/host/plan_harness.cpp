// CPU executor of the library's host-built plans, for the CPU test suite.
//
// Builds the Hubbard MPO automaton and the block plans with the library's own
// host code (tt_model.cpp, tt_plans.cpp) and executes the GEMM, gather and
// copy records in plain FP64 loops with every access bounds-checked, so the
// index arithmetic of the plans (FP64 layouts and the padded / transposed
// split-BF16 layouts, the latter emulated with one FP64 level) can be checked
// against dense contractions without a GPU.  Test infrastructure only.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <stdexcept>
#include <tuple>
#include <string>
#include <vector>

#include "tt_core.h"
#include "tt_plans.h"

using namespace tt;

namespace {

struct Slots {
  double* p[8] = {nullptr};
  int64_t n[8] = {0};
  double& at(Ref r, int64_t i) {
    const int s = (int)(r >> 56);
    const int64_t o = (int64_t)(r & 0x00FFFFFFFFFFFFFFull) + i;
    if (s < 0 || s > 7 || !p[s] || o < 0 || o >= n[s])
      throw std::runtime_error("plan access out of bounds: slot " + std::to_string(s) + " index " +
                               std::to_string(o) + " size " + std::to_string(s >= 0 && s < 8 ? n[s] : -1));
    return p[s][o];
  }
};

void run_gemm(const GemmPlan& P, Slots& S) {
  for (const GGroup& g : P.groups)
    for (int m = 0; m < g.M; ++m)
      for (int n = 0; n < g.N; ++n) {
        double acc = 0.0;
        for (int si = g.seg0; si < g.seg1; ++si) {
          const GSeg& sg = P.segs[si];
          for (int k = 0; k < sg.K; ++k) {
            const double a = S.at(sg.A, sg.tA ? (int64_t)k * sg.lda + m : (int64_t)m * sg.lda + k);
            const double b = S.at(sg.B, sg.tB ? (int64_t)n * sg.ldb + k : (int64_t)k * sg.ldb + n);
            acc += a * b;
          }
        }
        double& c = S.at(g.C, (int64_t)m * g.ldc + n);
        c = (g.flags & 1) ? c + acc : acc;
      }
}

void run_gather(const GatherPlan& P, Slots& S) {
  for (const GItem& it : P.items)
    for (int r = 0; r < it.rows; ++r)
      for (int c = 0; c < it.cols; ++c) {
        double acc = 0.0;
        for (int k = it.c0; k < it.c1; ++k) {
          const GContrib& cb = P.contribs[k];
          acc += cb.coef * S.at(cb.src, (int64_t)r * cb.src_rs + c);
        }
        S.at(it.dst, (int64_t)r * it.dst_rs + c) = acc;
      }
}

void run_copy(const CopyPlan& P, Slots& S) {
  for (const CItem& it : P.items)
    for (int r = 0; r < it.rows; ++r)
      for (int c = 0; c < it.cols; ++c)
        S.at(it.dst, (int64_t)r * it.dst_rs + (int64_t)c * it.dst_cs) =
            S.at(it.src, (int64_t)r * it.src_rs + (int64_t)c * it.src_cs);
}

// geom = {Lx, Wy, periodic, form}, par = {t, U, mu, tp}
Mpo model(const int* geom, const double* par) {
  ModelSpec m{geom[0], geom[1], geom[2], par[0], par[1], par[2], geom[3], par[3]};
  return build_hubbard_mpo(m);
}

Bond bond_from(const int* qn, const int* qs, const int* qd, int ns) {
  Bond b;
  for (int i = 0; i < ns; ++i) {
    b.q.push_back(Q{qn[i], qs[i]});
    b.dim.push_back(qd[i]);
  }
  return b;
}

std::string g_err;

template <class F>
int guarded(F&& f) {
  try {
    f();
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return 1;
  }
}

// split-bf16 environment copy (rows padded to 8), emulated in FP64
std::vector<double> pad_env(const Bond& B, const std::vector<Q>& ch, const double* env, int64_t n) {
  EnvLayout P = make_env_layout(B, ch, true);
  std::vector<double> out(std::max<int64_t>(P.size, 1), 0.0);
  Slots S;
  S.p[S_X] = const_cast<double*>(env); S.n[S_X] = n;
  S.p[S_Y] = out.data(); S.n[S_Y] = P.size;
  run_copy(build_env_split(B, ch), S);
  return out;
}

// Exact-split exponent bookkeeping: producers (digit copies, digit gather)
// record, per exponent slot element, which data row it describes (slot, first
// element, length); consumers (GEMM segments) must read, for every operand
// row, the exponent recorded for exactly that row, covering their K.
struct ExpBook {
  std::map<std::pair<int, int64_t>, std::tuple<int, int64_t, int>> rows;
  static int slot(Ref r) { return (int)(r >> 56); }
  static int64_t off(Ref r) { return (int64_t)(r & 0x00FFFFFFFFFFFFFFull); }
  void produce(Ref e, int64_t e_rs, Ref dst, int64_t dst_rs, int nrows, int cols, int as_slot) {
    for (int r = 0; r < nrows; ++r) {
      auto key = std::make_pair(as_slot, off(e) + r * e_rs);
      auto val = std::make_tuple(as_slot, off(dst) + r * dst_rs, cols);
      auto it = rows.find(key);
      if (it != rows.end() && it->second != val)
        throw std::runtime_error("two producers write exponent " + std::to_string(key.second) + " of slot " +
                                 std::to_string(as_slot));
      rows[key] = val;
    }
  }
  void consume(Ref e, int es, Ref data, int ld, int nrows, int K, const char* what) {
    if (es <= 0) throw std::runtime_error(std::string("missing exponents: ") + what);
    for (int m = 0; m < nrows; ++m) {
      auto it = rows.find(std::make_pair(slot(e), off(e) + (int64_t)m * es));
      if (it == rows.end())
        throw std::runtime_error(std::string(what) + ": no exponent produced for row " + std::to_string(m));
      const auto want = std::make_tuple(slot(data), off(data) + (int64_t)m * ld, 0);
      if (std::get<0>(it->second) != std::get<0>(want) || std::get<1>(it->second) != std::get<1>(want))
        throw std::runtime_error(std::string(what) + ": row " + std::to_string(m) + " reads the exponent of another row");
      if (std::get<2>(it->second) < K)
        throw std::runtime_error(std::string(what) + ": segment K exceeds the row the exponent covers");
    }
  }
  void produce_digits(const DigitPlan& p, int as_slot) {
    for (const DItem& it : p.items) produce(it.e, it.e_rs, it.dst, it.dst_rs, it.rows, it.cols, as_slot);
  }
  void consume_gemm(const GemmPlan& p, const char* what) {
    for (const GGroup& g : p.groups)
      for (int si = g.seg0; si < g.seg1; ++si) {
        const GSeg& sg = p.segs[si];
        if (sg.tA != 0 || sg.tB != 1) throw std::runtime_error(std::string(what) + ": digit operands must be K-major");
        consume(sg.eA, sg.eas, sg.A, sg.lda, g.M, sg.K, what);
        consume(sg.eB, sg.ebs, sg.B, sg.ldb, g.N, sg.K, what);
      }
  }
};

}  // namespace

extern "C" {

// Exact-split plans of site j (H_eff apply) and bond j+1 (bond apply): every
// GEMM operand row reads the exponent its producer wrote for that row.
int h_exact_exponents(const int* geom, const double* par, int j, const int* nsec_lr, const int* qn, const int* qs,
                      const int* qd) {
  return guarded([&] {
    Mpo M = model(geom, par);
    Bond BL = bond_from(qn, qs, qd, nsec_lr[0]);
    Bond BR = bond_from(qn + nsec_lr[0], qs + nsec_lr[0], qd + nsec_lr[0], nsec_lr[1]);
    SitePlanHost P = build_site_plan(BL, BR, M.ls, M.site[j].terms, M.chan[j], M.chan[j + 1], true, true);
    ExpBook site;
    site.produce_digits(P.xdig, S_X);                                 // x (transposed) -> S1's B operand
    site.produce_digits(build_env_digits(BL, M.chan[j]), S_L);        // L -> S1's A operand
    site.produce_digits(build_env_digits(BR, M.chan[j + 1]), S_R);    // R -> S3's B operand
    for (const GItem& it : P.s2.items) site.produce(it.e, it.e_rs, it.dst, it.dst_rs, it.rows, it.cols, S_T2);
    site.consume_gemm(P.s1, "S1");
    site.consume_gemm(P.s3, "S3");
    BondPlanHost B = build_bond_plan(BR, M.chan[j + 1], true, true);
    ExpBook bond;
    bond.produce_digits(B.xdig, S_X);
    bond.produce_digits(B.tdig, S_T2);
    bond.produce_digits(build_env_digits(BR, M.chan[j + 1]), S_L);
    bond.produce_digits(build_env_digits(BR, M.chan[j + 1]), S_R);
    bond.consume_gemm(B.b1, "B1");
    bond.consume_gemm(B.b2, "B2");
  });
}

// The exact split's digit W-gather items of site j, against what the kernel
// assumes: rows of at most max_cols columns, at most max_contribs MPO terms per
// item, even BF16 offsets and strides (it stores column pairs as one 32-bit
// word), every T2 element written by exactly one item, and the extra column
// an odd-width row's last pair writes lying in that row's own zero padding
// (not in another item's columns).  stats: [max cols, max terms per item,
// items with an odd width].
int h_gather_digit_items(const int* geom, const double* par, int j, const int* nsec_lr, const int* qn, const int* qs,
                         const int* qd, int max_cols, int max_contribs, int* stats) {
  return guarded([&] {
    Mpo M = model(geom, par);
    Bond BL = bond_from(qn, qs, qd, nsec_lr[0]);
    Bond BR = bond_from(qn + nsec_lr[0], qs + nsec_lr[0], qd + nsec_lr[0], nsec_lr[1]);
    SitePlanHost P = build_site_plan(BL, BR, M.ls, M.site[j].terms, M.chan[j], M.chan[j + 1], true, true);
    if (P.t2_size & 1) throw std::runtime_error("odd T2 level stride");
    std::vector<char> owner((size_t)P.t2_size, 0);
    int mc = 0, mk = 0, odd = 0;
    for (const GItem& it : P.s2.items) {
      const int64_t off = (int64_t)(it.dst & 0x00FFFFFFFFFFFFFFull);
      if ((off | it.dst_rs) & 1) throw std::runtime_error("odd digit row offset or stride");
      mc = std::max(mc, it.cols);
      mk = std::max(mk, it.c1 - it.c0);
      odd += it.cols & 1;
      for (int r = 0; r < it.rows; ++r)
        for (int c = 0; c < it.cols; ++c) {
          const int64_t e = off + (int64_t)r * it.dst_rs + c;
          if (e < 0 || e >= P.t2_size) throw std::runtime_error("T2 element outside the level");
          if (owner[(size_t)e]) throw std::runtime_error("T2 element written by two items");
          owner[(size_t)e] = 1;
        }
    }
    for (const GItem& it : P.s2.items) {
      if (!(it.cols & 1)) continue;
      const int64_t off = (int64_t)(it.dst & 0x00FFFFFFFFFFFFFFull);
      for (int r = 0; r < it.rows; ++r) {
        const int64_t e = off + (int64_t)r * it.dst_rs + it.cols;
        if (e >= P.t2_size || owner[(size_t)e]) throw std::runtime_error("pair store of an odd row leaves its padding");
      }
    }
    if (mc > max_cols) throw std::runtime_error("row longer than the kernel's limit");
    if (mk > max_contribs) throw std::runtime_error("more MPO terms per item than the kernel's limit");
    stats[0] = mc;
    stats[1] = mk;
    stats[2] = odd;
  });
}

const char* h_error() { return g_err.c_str(); }

int h_mpo_shape(const int* geom, const double* par, int* N, int* chan_dims, int cap) {
  return guarded([&] {
    Mpo M = model(geom, par);
    *N = M.N;
    if (cap < M.N + 1) throw std::runtime_error("cap");
    for (int k = 0; k <= M.N; ++k) chan_dims[k] = (int)M.chan[k].size();
  });
}

// dense W_j[w, sigma, tau, w'] (row-major, dims chl x 4 x 4 x chr)
int h_mpo_site_dense(const int* geom, const double* par, int j, double* W) {
  return guarded([&] {
    Mpo M = model(geom, par);
    const int chl = (int)M.chan[j].size(), chr = (int)M.chan[j + 1].size();
    std::memset(W, 0, sizeof(double) * chl * 16 * chr);
    for (const MpoTerm& t : M.site[j].terms) W[(((int64_t)t.wl * 4 + t.sig) * 4 + t.tau) * chr + t.wr] += t.v;
  });
}

// dense two-site W12[w, (s1 s2), (t1 t2), w''] (chan j x 16 x 16 x chan j+2)
int h_mpo_two_site_dense(const int* geom, const double* par, int j, double* W) {
  return guarded([&] {
    Mpo M = model(geom, par);
    const int chl = (int)M.chan[j].size(), chr = (int)M.chan[j + 2].size();
    std::memset(W, 0, sizeof(double) * chl * 256 * chr);
    for (const MpoTerm& t : combine_two_sites(M, j, product_space(M.ls, M.ls)).terms)
      W[(((int64_t)t.wl * 16 + t.sig) * 16 + t.tau) * chr + t.wr] += t.v;
  });
}

// channel charges of bond k (n, 2Sz)
int h_mpo_chan(const int* geom, const double* par, int k, int* qn, int* qs, int cap) {
  return guarded([&] {
    Mpo M = model(geom, par);
    if (cap < (int)M.chan[k].size()) throw std::runtime_error("cap");
    for (size_t w = 0; w < M.chan[k].size(); ++w) {
      qn[w] = M.chan[k][w].n;
      qs[w] = M.chan[k][w].s;
    }
  });
}

// start / done channel indices at the two boundary bonds
int h_mpo_boundary(const int* geom, const double* par, int* start0, int* doneN) {
  return guarded([&] {
    Mpo M = model(geom, par);
    *start0 = M.start_ch[0];
    *doneN = M.done_ch[M.N];
  });
}

// Site plans (H_eff apply, left and right environment updates) executed on
// the CPU.  op: 0 = H_eff apply (in: L (bond j), R (bond j+1), x; out: y),
// 1 = left environment update (in: L (bond j), x; out: L (bond j+1)),
// 2 = right environment update (in: R (bond j+1), x; out: R (bond j)).
// Sectors of bonds j and j+1 concatenated (nsec_lr = {nl, nr}).
// two != 0: the two-site tensor of sites j, j+1 (growth stage): product
// local space (d = 16, sigma = 4 sigma_j + sigma_{j+1}), W_j W_{j+1} summed
// over the middle channel, environments of bonds j and j+2.
int h_site_op(const int* geom, const double* par, int j, int op, int mixed, int two, const int* nsec_lr,
              const int* qn, const int* qs, const int* qd, const double* L, int64_t nL, const double* R, int64_t nR,
              const double* x, int64_t nx, double* out, int64_t nout) {
  return guarded([&] {
    Mpo M = model(geom, par);
    Bond BL = bond_from(qn, qs, qd, nsec_lr[0]);
    Bond BR = bond_from(qn + nsec_lr[0], qs + nsec_lr[0], qd + nsec_lr[0], nsec_lr[1]);
    const LocalSpace ls2 = product_space(M.ls, M.ls);
    const MpoSite w2 = two ? combine_two_sites(M, j, ls2) : MpoSite();
    const int jr = two ? j + 2 : j + 1;
    SitePlanHost P = build_site_plan(BL, BR, two ? ls2 : M.ls, two ? w2.terms : M.site[j].terms, M.chan[j],
                                     M.chan[jr], mixed != 0);
    if (nx != P.lay.size) throw std::runtime_error("x size " + std::to_string(P.lay.size));
    std::vector<double> T1(std::max<int64_t>(std::max(P.t1_size, P.u1_size), 1)),
        T2(std::max<int64_t>(std::max(P.t2_size, P.u2_size), 1), 0.0);
    std::vector<double> Lp, Rp, Xs(std::max<int64_t>(P.xt_size, 1), 0.0);
    Slots S;
    S.p[S_T1] = T1.data(); S.n[S_T1] = (int64_t)T1.size();
    S.p[S_T2] = T2.data(); S.n[S_T2] = (int64_t)T2.size();
    S.p[S_Y] = out; S.n[S_Y] = nout;
    if (mixed) {
      Slots C;
      C.p[S_X] = const_cast<double*>(x); C.n[S_X] = nx;
      C.p[S_Y] = Xs.data(); C.n[S_Y] = P.xt_size;
      run_copy(P.xsplit, C);
      S.p[S_AUX] = const_cast<double*>(x); S.n[S_AUX] = nx;  // natural split copy of x
      S.p[S_X] = Xs.data(); S.n[S_X] = P.xt_size;
    } else {
      S.p[S_X] = const_cast<double*>(x); S.n[S_X] = nx;
    }
    if (op == 0 || op == 1) {
      if (mixed) {
        Lp = pad_env(BL, M.chan[j], L, nL);
        S.p[S_L] = Lp.data(); S.n[S_L] = (int64_t)Lp.size();
      } else {
        S.p[S_L] = const_cast<double*>(L); S.n[S_L] = nL;
      }
    }
    if (op == 0 || op == 2) {
      if (mixed) {
        Rp = pad_env(BR, M.chan[jr], R, nR);
        S.p[S_R] = Rp.data(); S.n[S_R] = (int64_t)Rp.size();
      } else {
        S.p[S_R] = const_cast<double*>(R); S.n[S_R] = nR;
      }
    }
    if (op == 0) {
      if (nout != P.lay.size) throw std::runtime_error("y size");
      run_gemm(P.s1, S);
      run_gather(P.s2, S);
      run_gemm(P.s3, S);
    } else if (op == 1) {
      if (nout != P.lenv_size) throw std::runtime_error("L out size " + std::to_string(P.lenv_size));
      run_gemm(P.s1, S);
      run_gather(P.s2, S);
      run_gemm(P.s3l, S);
    } else {
      if (nout != P.renv_size) throw std::runtime_error("R out size " + std::to_string(P.renv_size));
      run_gemm(P.r1, S);
      run_gather(P.r2, S);
      run_gemm(P.r3, S);
    }
  });
}

// Bond H_eff apply y = H^(0) x on bond k (L and R both of bond k).
int h_bond_op(const int* geom, const double* par, int k, int mixed, int nsec, const int* qn, const int* qs,
              const int* qd, const double* L, int64_t nL, const double* R, int64_t nR, const double* x, int64_t nx,
              double* y) {
  return guarded([&] {
    Mpo M = model(geom, par);
    Bond B = bond_from(qn, qs, qd, nsec);
    BondPlanHost P = build_bond_plan(B, M.chan[k], mixed != 0);
    if (nx != P.mat.size) throw std::runtime_error("x size " + std::to_string(P.mat.size));
    std::vector<double> T1(std::max<int64_t>(P.t_size, 1)), Tp(std::max<int64_t>(P.tp_size, 1), 0.0),
        Xs(std::max<int64_t>(P.xt_size, 1), 0.0), Lp, Rp;
    Slots S;
    S.p[S_Y] = y; S.n[S_Y] = nx;
    S.p[S_T1] = T1.data(); S.n[S_T1] = (int64_t)T1.size();
    if (mixed) {
      Slots C;
      C.p[S_X] = const_cast<double*>(x); C.n[S_X] = nx;
      C.p[S_Y] = Xs.data(); C.n[S_Y] = P.xt_size;
      run_copy(P.xsplit, C);
      Lp = pad_env(B, M.chan[k], L, nL);
      Rp = pad_env(B, M.chan[k], R, nR);
      S.p[S_X] = Xs.data(); S.n[S_X] = P.xt_size;
      S.p[S_L] = Lp.data(); S.n[S_L] = (int64_t)Lp.size();
      S.p[S_R] = Rp.data(); S.n[S_R] = (int64_t)Rp.size();
      run_gemm(P.b1, S);
      Slots C2;
      C2.p[S_T1] = T1.data(); C2.n[S_T1] = (int64_t)T1.size();
      C2.p[S_Y] = Tp.data(); C2.n[S_Y] = P.tp_size;
      run_copy(P.tsplit, C2);
      S.p[S_T2] = Tp.data(); S.n[S_T2] = P.tp_size;
      run_gemm(P.b2, S);
    } else {
      S.p[S_X] = const_cast<double*>(x); S.n[S_X] = nx;
      S.p[S_L] = const_cast<double*>(L); S.n[S_L] = nL;
      S.p[S_R] = const_cast<double*>(R); S.n[S_R] = nR;
      S.p[S_T2] = T1.data(); S.n[S_T2] = (int64_t)T1.size();
      run_gemm(P.b1, S);
      run_gemm(P.b2, S);
    }
  });
}

// Absorb of the bond matrix into a site (identity sector map, as in the
// 1-TDVP sweep): side 0: A <- S A (S on bond j, the left bond), side 1:
// A <- A S (S on bond j+1).  S in the block-diagonal bond layout.
int h_absorb(int side, int nl, int nr, const int* qn, const int* qs, const int* qd, const double* x, int64_t nx,
             const double* S, int64_t ns, double* y) {
  return guarded([&] {
    LocalSpace ls = hubbard_site_space();
    Bond BL = bond_from(qn, qs, qd, nl), BR = bond_from(qn + nl, qs + nl, qd + nl, nr);
    SiteLayout L = make_site_layout(BL, BR, ls);
    if (nx != L.size) throw std::runtime_error("x size");
    const Bond& B = side == 0 ? BL : BR;
    BondMatLayout bm = make_bondmat_layout(B);
    if (ns != bm.size) throw std::runtime_error("S size");
    std::vector<int> ident(B.nsec());
    for (int i = 0; i < B.nsec(); ++i) ident[i] = i;
    GemmPlan G = side == 0 ? build_absorb_left(L, L, B, B, bm.off, ident) : build_absorb_right(L, L, B, B, bm.off, ident);
    Slots Sl;
    Sl.p[S_X] = const_cast<double*>(x); Sl.n[S_X] = nx;
    Sl.p[S_AUX] = const_cast<double*>(S); Sl.n[S_AUX] = ns;
    Sl.p[S_Y] = y; Sl.n[S_Y] = nx;
    run_gemm(G, Sl);
  });
}

// Left gauge move of site j by the QR plan and the shifted CholeskyQR3 plan:
// gather the right-sector group matrices, run the Gram / apply / R-product
// GEMM plans, a CPU restatement of the device Cholesky step (shift, partial
// sums, identity check and first-order factor of the last pass), then the
// scatter of Q into the site layout (q, x's size) and of R (r, s_size
// elements).  fail[r] = 1 for sectors the device would hand to Householder.
int h_qr_left(int nl, int nr, const int* qn, const int* qs, const int* qd, const double* x, int64_t nx, double* q,
              double* r, int64_t nrout, int* fail) {
  return guarded([&] {
    LocalSpace ls = hubbard_site_space();
    Bond BL = bond_from(qn, qs, qd, nl), BR = bond_from(qn + nl, qs + nl, qd + nl, nr);
    SiteLayout S = make_site_layout(BL, BR, ls);
    if (nx != S.size) throw std::runtime_error("x size " + std::to_string(S.size));
    QrPlanHost P = build_qr_left(S, BR);
    if (nrout != P.s_size) throw std::runtime_error("R size " + std::to_string(P.s_size));
    CholQrPlan CP = build_cholqr(P.jobs, P.ws_size);
    std::vector<double> ws(std::max<int64_t>(CP.ws_end, 1), 0.0);
    Slots Sx;
    Sx.p[S_X] = const_cast<double*>(x); Sx.n[S_X] = nx;
    Sx.p[S_Y] = q; Sx.n[S_Y] = nx;
    Sx.p[S_AUX] = r; Sx.n[S_AUX] = nrout;
    Sx.p[S_AUX2] = ws.data(); Sx.n[S_AUX2] = (int64_t)ws.size();
    run_copy(P.gather, Sx);
    std::vector<int> fl(P.jobs.size(), 0);
    auto chol = [&](const CholJob& J) {
      const int n = J.n;
      if (J.shift == 3) { fl[J.sec] = 1; return; }
      if (fl[J.sec]) return;
      double* G = &Sx.at(mkref(S_AUX2, J.g), 0);
      double* R = &Sx.at(mkref(S_AUX2, J.r), 0);
      double* Ri = &Sx.at(mkref(S_AUX2, J.ri), 0);
      const int64_t nn = (int64_t)n * n;
      Sx.at(mkref(S_AUX2, J.g), (int64_t)J.parts * nn - 1);  // bounds of the partials
      // the device keeps the summed upper triangle packed row by row in the
      // job's scratch (shared memory for small n); the scratch must not
      // overlap anything still needed, so it is used here for every n
      Sx.at(mkref(S_AUX2, J.pk), (int64_t)n * (n + 1) / 2 - 1);
      double* Pk = &Sx.at(mkref(S_AUX2, J.pk), 0);
      auto P = [&](int i, int j) -> double& { return Pk[(int64_t)i * n - (int64_t)i * (i - 1) / 2 + (j - i)]; };
      for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
          double acc = G[i * n + j];
          for (int p = 1; p < J.parts; ++p) acc += G[p * nn + i * n + j];
          P(i, j) = acc;
        }
      if (J.shift == 2) {
        double mx = 0.0;
        for (int i = 0; i < n; ++i)
          for (int j = i; j < n; ++j) mx = std::max(mx, std::fabs(P(i, j) - (i == j ? 1.0 : 0.0)));
        if (!(mx <= 1e-3)) { fl[J.sec] = 1; return; }
        if (n * mx <= 1e-8) {
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
              const double e = j < i ? 0.0 : P(i, j);
              R[i * n + j] = j < i ? 0.0 : (j == i ? 1.0 + 0.5 * (e - 1.0) : e);
              Ri[i * n + j] = j < i ? 0.0 : (j == i ? 1.0 - 0.5 * (e - 1.0) : -e);
            }
          return;
        }
      }
      if (J.shift == 1) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) tr += P(i, i);
        const double sft = 11.0 * ((double)J.m * n + (double)n * (n + 1)) * 1.1102230246251565e-16 * tr;
        for (int i = 0; i < n; ++i) P(i, i) += sft;
      }
      for (int64_t e = 0; e < nn; ++e) R[e] = 0.0;
      for (int k = 0; k < n; ++k) {
        const double d = P(k, k);
        if (!(d > 0.0)) { fl[J.sec] = 1; return; }
        const double pv = std::sqrt(d);
        for (int j = k; j < n; ++j) R[k * n + j] = P(k, j) / pv;
        for (int i = k + 1; i < n; ++i)
          for (int j = i; j < n; ++j) P(i, j) -= R[k * n + i] * R[k * n + j];
      }
      for (int j = 0; j < n; ++j) {
        for (int i = j + 1; i < n; ++i) Ri[i * n + j] = 0.0;
        Ri[j * n + j] = 1.0 / R[j * n + j];
        for (int i = j - 1; i >= 0; --i) {
          double acc = 0.0;
          for (int qq = i + 1; qq <= j; ++qq) acc += R[i * n + qq] * Ri[qq * n + j];
          Ri[i * n + j] = -acc / R[i * n + i];
        }
      }
    };
    for (int p = 0; p < 3; ++p) {
      run_gemm(CP.gram[p], Sx);
      for (const CholJob& J : CP.cj[p]) chol(J);
      run_gemm(CP.app[p], Sx);
    }
    run_gemm(CP.tt, Sx);
    run_gemm(CP.rf, Sx);
    run_copy(P.scatter, Sx);
    run_copy(P.rout, Sx);
    for (size_t i = 0; i < fl.size(); ++i) fail[i] = fl[i];
  });
}

}  // extern "C"
