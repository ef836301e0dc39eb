// Host-side plan compilers: every contraction of the sweep written as lists
// of GEMM groups, W-gather items and strided copies over the U(1)xU(1) blocks.
//
// H_eff site apply (Supplement, Fig. "Lanczos": L_i A_i, then H_i, then R_i):
//   S1  T1[b][(w, a_l), (s_in, b_r)] = L[(w, a_l), b_l] A[b_l, (s_in, b_r)]  per block b
//   S2  T2[r][(a_l, s_out), (w', b_r)] = sum W[w, sig, tau, w'] T1[...]     (gather)
//   S3  y[r][(a_l, s_out), a_r] = sum_w' T2[r][:, (w', .)] R[a_r, w', b_r]
// Left environment update (Fig. "optimalB"(c) contracted with A^L on the bra):
//   S1, S2, then L'[(w', a_r), b_r] = sum A[(a_l, s), a_r] T2[(a_l, s), (w', b_r)]
// Right environment update (mirror, A R first):
//   R1  U1[b][(b_l, s_in), (w', a_r)] = A[(b_l, s_in), b_r] R[(w', a_r), b_r]^T
//   R2  U2[a][(w, b_l), (s_out, a_r)] = sum W U1                            (gather)
//   R3  R'[(w, a_l), b_l] = sum A[a_l, (s, a_r)] U2[(w, b_l), (s, a_r)]^T
// Bond apply (Fig. "optimalB"(d)):
//   B1  T[(w, a), c] = L[(w, a), b] S[b, c];  B2  y[a, a'] = sum_w T[(w,a), c] R[a', w, c]
#include "tt_plans.h"

#include <algorithm>
#include <map>
#include <stdexcept>

namespace tt {

namespace {
// (wr, sig) -> terms ; (wl, sig) -> terms
struct TermIndex {
  std::map<std::pair<int, int>, std::vector<const MpoTerm*>> by_r, by_l;
  explicit TermIndex(const std::vector<MpoTerm>& t) {
    for (const auto& x : t) {
      by_r[{x.wr, x.sig}].push_back(&x);
      by_l[{x.wl, x.sig}].push_back(&x);
    }
  }
};
}  // namespace

std::vector<int64_t> env_row_starts(const EnvLayout& E) {
  std::vector<int64_t> r(E.rows.size(), 0);
  int64_t c = 0;
  for (size_t b = 0; b < E.rows.size(); ++b) {
    r[b] = c;
    c += E.rows[b];
  }
  return r;
}

SitePlanHost build_site_plan(const Bond& BL, const Bond& BR, const LocalSpace& ls, const std::vector<MpoTerm>& terms,
                             const std::vector<Q>& chl, const std::vector<Q>& chr, bool mixed, bool exact) {
  exact = exact && mixed;
  SitePlanHost P;
  P.lay = make_site_layout(BL, BR, ls);
  const SiteLayout& S = P.lay;
  EnvLayout EL = make_env_layout(BL, chl);
  EnvLayout ER = make_env_layout(BR, chr);
  // operand layouts of the contraction inputs: split-bf16 environments have
  // rows padded to 8 elements; FP64 ones are the natural layout
  EnvLayout ELo = make_env_layout(BL, chl, mixed);
  EnvLayout ERo = make_env_layout(BR, chr, mixed);
  auto wpad = [&](int x) { return mixed ? pad8i(x) : x; };
  const int nwl = (int)chl.size(), nwr = (int)chr.size();
  const int t1flag = mixed ? 2 : 0;
  TermIndex ti(terms);
  const int d = ls.d;

  // ---- S1 (mixed: B = transposed x block [(s, a_r)][a_l], rows padded: K-major)
  std::vector<int64_t> t1off(S.blk.size(), -1), t1ld(S.blk.size(), 0), xtoff(S.blk.size(), 0), xtrow(S.blk.size(), 0);
  int64_t cur = 0, xt = 0, xtr = 0;
  if (mixed)
    for (size_t bi = 0; bi < S.blk.size(); ++bi) {
      const SiteBlock& b = S.blk[bi];
      const int N = b.m * b.dr, ldt = pad8i(b.dl);
      xtoff[bi] = xt;
      xtrow[bi] = xtr;
      // x block row-major (d_l x N) -> transposed (N x ldt)
      P.xsplit.items.push_back(CItem{mkref(S_X, b.off), mkref(S_Y, xt), N, 1, 1, ldt, b.dl, N});
      xt += (int64_t)N * ldt;
      xtr += N;
    }
  P.xt_size = pad8l(xt);
  // digit exponents live after the four levels of a slot (offsets in 2-byte units)
  const int64_t xte = 4 * P.xt_size;
  if (exact)
    for (size_t bi = 0; bi < S.blk.size(); ++bi) {
      const SiteBlock& b = S.blk[bi];
      const int N = b.m * b.dr;
      // transposed: digit row j = column j of the block, K = d_l
      P.xdig.items.push_back(DItem{mkref(S_X, b.off), mkref(S_Y, xtoff[bi]), mkref(S_Y, xte + xtrow[bi]), 1, N,
                                   pad8i(b.dl), 1, N, b.dl});
    }
  const std::vector<int64_t> elrow = env_row_starts(ELo), errow = env_row_starts(ERo);
  const int64_t ele = 4 * ELo.size, ere = 4 * ERo.size;
  for (size_t bi = 0; bi < S.blk.size(); ++bi) {
    const SiteBlock& b = S.blk[bi];
    int64_t M = EL.rows[b.l];
    int64_t N = (int64_t)b.m * b.dr;
    if (M == 0 || N == 0) continue;
    t1off[bi] = cur;
    t1ld[bi] = N;
    P.s1.add_group((int)M, (int)N, mkref(S_T1, cur), (int)N, t1flag);
    if (mixed) P.s1.add_seg(mkref(S_L, ELo.off[b.l]), ELo.ld[b.l], 0, mkref(S_X, xtoff[bi]), pad8i(b.dl), 1, b.dl);
    else P.s1.add_seg(mkref(S_L, EL.off[b.l]), b.dl, 0, mkref(S_X, b.off), (int)N, 0, b.dl);
    if (exact) P.s1.set_exps(mkref(S_L, ele + elrow[b.l]), 1, mkref(S_X, xte + xtrow[bi]), 1);
    cur += M * N;
  }
  P.t1_size = cur;

  // ---- T2 layout (per right sector r of BR)
  const int nr = BR.nsec();
  std::vector<int64_t> t2off(nr, 0), t2cols(nr, 0), t2col((size_t)nr * nwr, -1);
  std::vector<int> t2ket((size_t)nr * nwr, -1), t2seg((size_t)nr * nwr, -1), nseg(nr, 0);
  std::vector<int64_t> t2e(nr, 0);
  cur = 0;
  int64_t curE = 0;
  for (int r = 0; r < nr; ++r) {
    int64_t cols = 0;
    for (int w = 0; w < nwr; ++w) {
      int b = BR.find(BR.q[r] - chr[w]);
      if (b < 0) continue;
      t2col[(size_t)r * nwr + w] = cols;
      t2ket[(size_t)r * nwr + w] = b;
      t2seg[(size_t)r * nwr + w] = nseg[r]++;
      cols += wpad(BR.dim[b]);
    }
    t2cols[r] = cols;
    t2off[r] = cur;
    cur += S.grp_rows[r] * cols;
    t2e[r] = curE;  // exponents: per group row, one per column segment
    curE += S.grp_rows[r] * nseg[r];
  }
  P.t2_size = cur;
  const int64_t t2x = 4 * P.t2_size;

  // ---- S2 gather
  for (size_t obi = 0; obi < S.blk.size(); ++obi) {
    const SiteBlock& ob = S.blk[obi];
    const int r = ob.r;
    for (int so = 0; so < ob.m; ++so) {
      const int sig = ls.pairs[ob.p][so].first, sgp = ls.pairs[ob.p][so].second;
      for (int w2 = 0; w2 < nwr; ++w2) {
        int64_t col = t2col[(size_t)r * nwr + w2];
        if (col < 0) continue;
        const int br = t2ket[(size_t)r * nwr + w2];
        GItem it;
        it.dst = mkref(S_T2, t2off[r] + (ob.grp_row + so) * t2cols[r] + col);
        it.dst_rs = (int64_t)ob.m * t2cols[r];
        it.rows = ob.dl;
        it.cols = BR.dim[br];
        it.c0 = (int)P.s2.contribs.size();
        auto f = ti.by_r.find({w2, sig});
        if (f != ti.by_r.end())
          for (const MpoTerm* t : f->second) {
            const int w = t->wl, tau = t->tau;
            int lb = BL.find(BL.q[ob.l] - chl[w]);
            if (lb < 0) continue;
            const int pidx = tau * d + sgp;
            const int pin = ls.sec_of[pidx], si = ls.pos_of[pidx];
            int bin = S.block_of(lb, pin);
            if (bin < 0 || t1off[bin] < 0) continue;
            if (S.blk[bin].r != br) throw std::logic_error("S2: charge mismatch");
            int64_t row = EL.row_of(lb, w);
            if (row < 0) continue;
            GContrib c;
            c.src = mkref(S_T1, t1off[bin] + row * t1ld[bin] + (int64_t)si * S.blk[bin].dr);
            c.src_rs = t1ld[bin];
            c.coef = t->v;
            P.s2.contribs.push_back(c);
          }
        it.c1 = (int)P.s2.contribs.size();
        if (exact) {
          it.e = mkref(S_T2, t2x + t2e[r] + (ob.grp_row + so) * nseg[r] + t2seg[(size_t)r * nwr + w2]);
          it.e_rs = (int64_t)ob.m * nseg[r];
        }
        P.s2.items.push_back(it);
        P.s2.elems += (double)it.rows * it.cols * (1 + it.c1 - it.c0);
      }
    }
  }

  // ---- S3 (H_eff output) and S3L (left environment update)
  for (int r = 0; r < nr; ++r) {
    if (S.grp_rows[r] > 0) {
      P.s3.add_group((int)S.grp_rows[r], BR.dim[r], mkref(S_Y, S.grp_off[r]), BR.dim[r], 0);
      for (int w2 = 0; w2 < nwr; ++w2) {
        int64_t col = t2col[(size_t)r * nwr + w2];
        if (col < 0) continue;
        const int b = t2ket[(size_t)r * nwr + w2];
        int64_t rrow = ER.row_of(b, w2);
        P.s3.add_seg(mkref(S_T2, t2off[r] + col), (int)t2cols[r], 0, mkref(S_R, ERo.off[b] + rrow * ERo.ld[b]),
                     ERo.ld[b], 1, BR.dim[b]);
        if (exact)
          P.s3.set_exps(mkref(S_T2, t2x + t2e[r] + t2seg[(size_t)r * nwr + w2]), nseg[r],
                        mkref(S_R, ere + errow[b] + rrow), 1);
      }
    }
    for (int w2 = 0; w2 < nwr; ++w2) {
      int64_t col = t2col[(size_t)r * nwr + w2];
      if (col < 0) continue;
      const int b = t2ket[(size_t)r * nwr + w2];
      int64_t lrow = ER.row_of(b, w2);
      P.s3l.add_group(BR.dim[r], BR.dim[b], mkref(S_Y, ER.off[b] + lrow * BR.dim[b]), BR.dim[b], 0);
      if (S.grp_rows[r] > 0)
        P.s3l.add_seg(mkref(mixed ? S_AUX : S_X, S.grp_off[r]), BR.dim[r], 1, mkref(S_T2, t2off[r] + col),
                      (int)t2cols[r], 0, (int)S.grp_rows[r]);
    }
  }
  P.lenv_size = ER.size;

  // ---- R1
  std::vector<int64_t> u1off(S.blk.size(), -1), u1ld(S.blk.size(), 0);
  cur = 0;
  for (size_t bi = 0; bi < S.blk.size(); ++bi) {
    const SiteBlock& b = S.blk[bi];
    int64_t M = (int64_t)b.dl * b.m;
    int64_t N = ER.rows[b.r];
    if (M == 0 || N == 0) continue;
    u1off[bi] = cur;
    u1ld[bi] = N;
    P.r1.add_group((int)M, (int)N, mkref(S_T1, cur), (int)N, t1flag);
    P.r1.add_seg(mkref(mixed ? S_AUX : S_X, b.off), b.dr, 0, mkref(S_R, ERo.off[b.r]), ERo.ld[b.r], 1, b.dr);
    cur += M * N;
  }
  P.u1_size = cur;

  // ---- U2 layout per bra-left sector a of BL: rows (w, b_l), cols (p, s, a_r)
  const int nl = BL.nsec();
  std::vector<int64_t> u2off(nl, 0), u2rows(nl, 0), u2cols(nl, 0);
  std::vector<int64_t> u2row((size_t)nl * nwl, -1);
  std::vector<int> u2ket((size_t)nl * nwl, -1);
  std::vector<int64_t> colseg((size_t)nl * S.npq, -1);
  cur = 0;
  for (int a = 0; a < nl; ++a) {
    int64_t rows = 0, cols = 0;
    for (int w = 0; w < nwl; ++w) {
      int lb = BL.find(BL.q[a] - chl[w]);
      if (lb < 0) continue;
      u2row[(size_t)a * nwl + w] = rows;
      u2ket[(size_t)a * nwl + w] = lb;
      rows += BL.dim[lb];
    }
    for (int p = 0; p < S.npq; ++p) {
      int bi = S.block_of(a, p);
      if (bi < 0) continue;
      colseg[(size_t)a * S.npq + p] = cols;
      cols += (int64_t)S.blk[bi].m * S.blk[bi].dr;
    }
    u2off[a] = cur;
    u2rows[a] = rows;
    u2cols[a] = cols;
    cur += rows * cols;
  }
  P.u2_size = cur;

  // ---- R2 gather
  for (int a = 0; a < nl; ++a)
    for (int w = 0; w < nwl; ++w) {
      int64_t row0 = u2row[(size_t)a * nwl + w];
      if (row0 < 0) continue;
      const int lb = u2ket[(size_t)a * nwl + w];
      for (int p = 0; p < S.npq; ++p) {
        int obi = S.block_of(a, p);
        if (obi < 0) continue;
        const SiteBlock& ob = S.blk[obi];
        for (int so = 0; so < ob.m; ++so) {
          const int sig = ls.pairs[p][so].first, sgp = ls.pairs[p][so].second;
          GItem it;
          it.dst = mkref(S_T2, u2off[a] + row0 * u2cols[a] + colseg[(size_t)a * S.npq + p] + (int64_t)so * ob.dr);
          it.dst_rs = u2cols[a];
          it.rows = BL.dim[lb];
          it.cols = ob.dr;
          it.c0 = (int)P.r2.contribs.size();
          auto f = ti.by_l.find({w, sig});
          if (f != ti.by_l.end())
            for (const MpoTerm* t : f->second) {
              const int w2 = t->wr, tau = t->tau;
              const int pidx = tau * d + sgp;
              const int pin = ls.sec_of[pidx], si = ls.pos_of[pidx];
              int bin = S.block_of(lb, pin);
              if (bin < 0 || u1off[bin] < 0) continue;
              const SiteBlock& ib = S.blk[bin];
              int64_t rrow = ER.row_of(ib.r, w2);
              if (rrow < 0) continue;
              if (ER.bra[(size_t)ib.r * ER.nw + w2] != ob.r) throw std::logic_error("R2: charge mismatch");
              GContrib c;
              c.src = mkref(S_T1, u1off[bin] + (int64_t)si * u1ld[bin] + rrow);
              c.src_rs = (int64_t)ib.m * u1ld[bin];
              c.coef = t->v;
              P.r2.contribs.push_back(c);
            }
          it.c1 = (int)P.r2.contribs.size();
          P.r2.items.push_back(it);
          P.r2.elems += (double)it.rows * it.cols * (1 + it.c1 - it.c0);
        }
      }
    }

  // ---- R3 (right environment of bond j, layout EL)
  for (int a = 0; a < nl; ++a)
    for (int w = 0; w < nwl; ++w) {
      int64_t row0 = u2row[(size_t)a * nwl + w];
      if (row0 < 0) continue;
      const int lb = u2ket[(size_t)a * nwl + w];
      int64_t erow = EL.row_of(lb, w);
      P.r3.add_group(BL.dim[a], BL.dim[lb], mkref(S_Y, EL.off[lb] + erow * BL.dim[lb]), BL.dim[lb], 0);
      for (int p = 0; p < S.npq; ++p) {
        int obi = S.block_of(a, p);
        if (obi < 0) continue;
        const SiteBlock& ob = S.blk[obi];
        int K = ob.m * ob.dr;
        P.r3.add_seg(mkref(mixed ? S_AUX : S_X, ob.off), K, 0,
                     mkref(S_T2, u2off[a] + row0 * u2cols[a] + colseg[(size_t)a * S.npq + p]), (int)u2cols[a], 1, K);
      }
    }
  P.renv_size = EL.size;
  return P;
}

CopyPlan build_env_split(const Bond& B, const std::vector<Q>& chan) {
  EnvLayout E = make_env_layout(B, chan), P = make_env_layout(B, chan, true);
  CopyPlan cp;
  for (int b = 0; b < B.nsec(); ++b)
    if (E.rows[b] > 0)
      cp.items.push_back(CItem{mkref(S_X, E.off[b]), mkref(S_Y, P.off[b]), E.ld[b], 1, P.ld[b], 1, (int)E.rows[b], B.dim[b]});
  return cp;
}

DigitPlan build_env_digits(const Bond& B, const std::vector<Q>& chan) {
  EnvLayout E = make_env_layout(B, chan), P = make_env_layout(B, chan, true);
  const std::vector<int64_t> rs = env_row_starts(P);
  DigitPlan dp;
  for (int b = 0; b < B.nsec(); ++b)
    if (E.rows[b] > 0)
      dp.items.push_back(DItem{mkref(S_X, E.off[b]), mkref(S_Y, P.off[b]), mkref(S_Y, 4 * P.size + rs[b]), E.ld[b], 1,
                               P.ld[b], 1, (int)E.rows[b], B.dim[b]});
  return dp;
}

BondPlanHost build_bond_plan(const Bond& B, const std::vector<Q>& ch, bool mixed, bool exact) {
  exact = exact && mixed;
  // y_q = sum_w L_w(q <- b) x_b R_w(q <- b)^T with b = q - ch[w]: first
  // T_b = L_b x_b for all channels at once (rows (w, a) of the environment),
  // then per output sector the sum over w of (rows of channel w of T_b) R^T.
  BondPlanHost P;
  EnvLayout E = make_env_layout(B, ch);
  EnvLayout Eo = make_env_layout(B, ch, mixed);  // operand layout of L and R
  P.mat = make_bondmat_layout(B);
  const int nw = (int)ch.size();
  std::vector<int64_t> toff(B.nsec(), -1), tpoff(B.nsec(), -1), xtoff(B.nsec(), 0), tprow(B.nsec(), 0);
  std::vector<int64_t> xtrow(B.nsec(), 0);
  int64_t cur = 0, curp = 0, xt = 0, xtr = 0, tpr = 0;
  for (int b = 0; b < B.nsec(); ++b) {
    const int d = B.dim[b], ldp = pad8i(d);
    if (mixed) {
      xtoff[b] = xt;
      xtrow[b] = xtr;
      P.xsplit.items.push_back(CItem{mkref(S_X, P.mat.off[b]), mkref(S_Y, xt), d, 1, 1, ldp, d, d});
      xt += (int64_t)d * ldp;
      xtr += d;
    }
    if (E.rows[b] == 0) continue;
    toff[b] = cur;
    P.b1.add_group((int)E.rows[b], d, mkref(S_T1, cur), d, 0);
    if (mixed) {
      P.b1.add_seg(mkref(S_L, Eo.off[b]), Eo.ld[b], 0, mkref(S_X, xtoff[b]), ldp, 1, d);
      tpoff[b] = curp;
      tprow[b] = tpr;
      P.tsplit.items.push_back(CItem{mkref(S_T1, cur), mkref(S_Y, curp), d, 1, ldp, 1, (int)E.rows[b], d});
      curp += E.rows[b] * ldp;
      tpr += E.rows[b];
    } else {
      P.b1.add_seg(mkref(S_L, Eo.off[b]), Eo.ld[b], 0, mkref(S_X, P.mat.off[b]), d, 0, d);
    }
    cur += E.rows[b] * d;
  }
  P.t_size = cur;
  P.xt_size = pad8l(xt);
  P.tp_size = pad8l(curp);
  const std::vector<int64_t> erow = env_row_starts(Eo);
  const int64_t xte = 4 * P.xt_size, tpe = 4 * P.tp_size, ee = 4 * Eo.size;
  if (exact) {
    for (int b = 0; b < B.nsec(); ++b) {
      const int d = B.dim[b], ldp = pad8i(d);
      // transposed S block: digit row c = column c of S, K = d
      P.xdig.items.push_back(DItem{mkref(S_X, P.mat.off[b]), mkref(S_Y, xtoff[b]), mkref(S_Y, xte + xtrow[b]), 1, d,
                                   ldp, 1, d, d});
      if (toff[b] >= 0)
        P.tdig.items.push_back(DItem{mkref(S_T1, toff[b]), mkref(S_Y, tpoff[b]), mkref(S_Y, tpe + tprow[b]), d, 1, ldp,
                                     1, (int)E.rows[b], d});
    }
    // B1 segments in group order: one per sector with rows
    int gi = 0;
    for (int b = 0; b < B.nsec(); ++b) {
      if (E.rows[b] == 0) continue;
      GSeg& sg = P.b1.segs[P.b1.groups[gi++].seg0];
      sg.eA = mkref(S_L, ee + erow[b]);
      sg.eas = 1;
      sg.eB = mkref(S_X, xte + xtrow[b]);
      sg.ebs = 1;
    }
  }
  for (int q = 0; q < B.nsec(); ++q) {
    P.b2.add_group(B.dim[q], B.dim[q], mkref(S_Y, P.mat.off[q]), B.dim[q], 0);
    for (int w = 0; w < nw; ++w) {
      int b = B.find(B.q[q] - ch[w]);
      if (b < 0 || toff[b] < 0) continue;
      int64_t row = E.row_of(b, w);
      if (mixed) {
        P.b2.add_seg(mkref(S_T2, tpoff[b] + row * pad8i(B.dim[b])), pad8i(B.dim[b]), 0,
                     mkref(S_R, Eo.off[b] + row * Eo.ld[b]), Eo.ld[b], 1, B.dim[b]);
        if (exact) P.b2.set_exps(mkref(S_T2, tpe + tprow[b] + row), 1, mkref(S_R, ee + erow[b] + row), 1);
      } else
        P.b2.add_seg(mkref(S_T2, toff[b] + row * B.dim[b]), B.dim[b], 0, mkref(S_R, Eo.off[b] + row * Eo.ld[b]),
                     Eo.ld[b], 1, B.dim[b]);
    }
  }
  return P;
}

GemmPlan build_absorb_left(const SiteLayout& oldl, const SiteLayout& newl, const Bond& Bold, const Bond& Bnew,
                           const std::vector<int64_t>& soff, const std::vector<int>& new_of_old) {
  // A_new[(l', p, r)] = S_l (d_new x d_old, row-major) A_old[(l, p, r)] ; l' = new_of_old[l]
  GemmPlan G;
  for (const SiteBlock& ob : oldl.blk) {
    int ln = new_of_old[ob.l];
    if (ln < 0) continue;
    int nbi = newl.block_of(ln, ob.p);
    if (nbi < 0) continue;
    const SiteBlock& nb = newl.blk[nbi];
    int N = ob.m * ob.dr;
    G.add_group(Bnew.dim[ln], N, mkref(S_Y, nb.off), N, 0);
    G.add_seg(mkref(S_AUX, soff[ob.l]), Bold.dim[ob.l], 0, mkref(S_X, ob.off), N, 0, Bold.dim[ob.l]);
  }
  return G;
}

GemmPlan build_absorb_right(const SiteLayout& oldl, const SiteLayout& newl, const Bond& Bold, const Bond& Bnew,
                            const std::vector<int64_t>& soff, const std::vector<int>& new_of_old) {
  // A_new[group r'] = A_old[group r] (rows x d_old) S_r (d_old x d_new, row-major)
  GemmPlan G;
  for (int r = 0; r < Bold.nsec(); ++r) {
    int rn = new_of_old[r];
    if (rn < 0) continue;
    if (oldl.grp_rows[r] == 0) continue;
    G.add_group((int)oldl.grp_rows[r], Bnew.dim[rn], mkref(S_Y, newl.grp_off[rn]), Bnew.dim[rn], 0);
    G.add_seg(mkref(S_X, oldl.grp_off[r]), Bold.dim[r], 0, mkref(S_AUX, soff[r]), Bnew.dim[rn], 0, Bold.dim[r]);
  }
  return G;
}

QrPlanHost build_qr_left(const SiteLayout& S, const Bond& BR) {
  // per right sector r: the (grp_rows x d_r) group matrix, QR -> A^L, R -> S
  QrPlanHost P;
  int64_t ws = 0, sm = 0;
  for (int r = 0; r < BR.nsec(); ++r) {
    int m = (int)S.grp_rows[r], n = BR.dim[r];
    QrJob J;
    J.m = m;
    J.n = n;
    J.a = ws;
    ws += (int64_t)m * n;
    J.q = ws;
    ws += (int64_t)m * n;
    J.r = ws;
    ws += (int64_t)n * n;
    P.jobs.push_back(J);
    P.gather.items.push_back(CItem{mkref(S_X, S.grp_off[r]), mkref(S_AUX2, J.a), n, 1, 1, m, m, n});
    P.scatter.items.push_back(CItem{mkref(S_AUX2, J.q), mkref(S_Y, S.grp_off[r]), 1, m, n, 1, m, n});
    P.rout.items.push_back(CItem{mkref(S_AUX2, J.r), mkref(S_AUX, sm), 1, n, n, 1, n, n});
    P.new_dim.push_back(n);
    sm += (int64_t)n * n;
  }
  P.ws_size = ws;
  P.s_size = sm;
  return P;
}

QrPlanHost build_lq_right(const SiteLayout& S, const Bond& BL, bool shrink) {
  // per left sector l: M = [blocks (l, p)] (d_l x cols); QR of M^T (cols x d_l).
  QrPlanHost P;
  int64_t ws = 0, sm = 0;
  for (int l = 0; l < BL.nsec(); ++l) {
    int n = BL.dim[l];
    int64_t cols = 0;
    std::vector<std::pair<int, int64_t>> segs;
    for (int p = 0; p < S.npq; ++p) {
      int bi = S.block_of(l, p);
      if (bi < 0) continue;
      segs.push_back({bi, cols});
      cols += (int64_t)S.blk[bi].m * S.blk[bi].dr;
    }
    int m = (int)cols;
    int k = shrink ? std::min(m, n) : n;
    QrJob J;
    J.m = m;
    J.n = n;
    J.a = ws;
    ws += (int64_t)m * n;
    J.q = ws;
    ws += (int64_t)m * n;
    J.r = ws;
    ws += (int64_t)n * n;
    P.jobs.push_back(J);
    for (auto& sg : segs) {
      const SiteBlock& b = S.blk[sg.first];
      int C = b.m * b.dr;
      // block row-major (d_l x C) -> M^T column-major rows [cs, cs + C), cols a_l
      P.gather.items.push_back(CItem{mkref(S_X, b.off), mkref(S_AUX2, J.a + sg.second), C, 1, m, 1, n, C});
      // A^R block (first k rows a_l) = Q'^T
      P.scatter_blocks.push_back({sg.first, sg.second});
    }
    P.lq_cols.push_back(m);
    P.new_dim.push_back(k);
    // S = R'^T (n x k, row-major): S[a][b] = R'[b][a] = ws[r + b + a n]
    P.rout.items.push_back(CItem{mkref(S_AUX2, J.r), mkref(S_AUX, sm), n, 1, k, 1, n, k});
    sm += (int64_t)n * k;
  }
  P.ws_size = ws;
  P.s_size = sm;
  return P;
}

CholQrPlan build_cholqr(const std::vector<QrJob>& jobs, int64_t ws0) {
  // Per sector (m x n, column-major X):
  //   G = X^T X: only the upper block triangle (row blocks of 64, columns from
  //   the block's first row on), K split into `parts` chunks that write
  //   separate partial Gram matrices (summed by the Cholesky kernel);
  //   Xo^T = RI^T X^T: RI is upper triangular, so output row block q0 needs
  //   K = min(n, q0 + 64) only.
  constexpr int RB = 64, KCHUNK = 512, MAXPARTS = 16;
  CholQrPlan P;
  int64_t w = ws0;
  for (size_t sec = 0; sec < jobs.size(); ++sec) {
    const QrJob& J = jobs[sec];
    const int m = J.m, n = J.n;
    if (m < n || n == 0) {  // rank-deficient by shape: Householder only
      if (n > 0) P.cj[0].push_back(CholJob{0, 0, 0, m, n, 3, (int)sec, 1});
      continue;
    }
    const int parts = std::max(1, std::min(MAXPARTS, (m + KCHUNK - 1) / KCHUNK));
    int kc = (m + parts - 1) / parts;
    kc = (kc + 15) / 16 * 16;
    const int64_t mn = (int64_t)m * n, nn = (int64_t)n * n;
    const int64_t q0 = w, q1 = q0 + mn, g = q1 + mn, r0 = g + parts * nn, r1 = r0 + nn, r2 = r1 + nn,
                  ri0 = r2 + nn, ri1 = ri0 + nn, ri2 = ri1 + nn, tt = ri2 + nn;
    w = tt + nn;
    const int64_t X[3] = {J.a, q0, q1}, Xo[3] = {q0, q1, J.q}, R[3] = {r0, r1, r2}, RI[3] = {ri0, ri1, ri2};
    for (int p = 0; p < 3; ++p) {
      for (int s = 0; s < parts; ++s) {
        const int k0 = s * kc, K = std::min(kc, m - k0);
        if (K <= 0) {  // empty chunk: its partial must still be written
          for (int i0 = 0; i0 < n; i0 += RB)
            P.gram[p].add_group(std::min(RB, n - i0), n - i0, mkref(S_AUX2, g + s * nn + (int64_t)i0 * n + i0), n, 0);
          continue;
        }
        for (int i0 = 0; i0 < n; i0 += RB) {
          P.gram[p].add_group(std::min(RB, n - i0), n - i0, mkref(S_AUX2, g + s * nn + (int64_t)i0 * n + i0), n, 0);
          const Ref xa = mkref(S_AUX2, X[p] + (int64_t)i0 * m + k0);
          P.gram[p].add_seg(xa, m, 0, xa, m, 1, K);
        }
      }
      const int shift = p == 0 ? 1 : (p == 2 ? 2 : 0);
      // the T region is free until the passes are done: packed scratch
      P.cj[p].push_back(CholJob{g, R[p], RI[p], m, n, shift, (int)sec, parts, tt});
      for (int r0b = 0; r0b < n; r0b += RB) {
        P.app[p].add_group(std::min(RB, n - r0b), m, mkref(S_AUX2, Xo[p] + (int64_t)r0b * m), m, 0);
        P.app[p].add_seg(mkref(S_AUX2, RI[p] + r0b), n, 1, mkref(S_AUX2, X[p]), m, 0, std::min(n, r0b + RB));
      }
    }
    // T^T = R0^T R1^T ; R^T = T^T R2^T (row-major R^T = column-major R)
    P.tt.add_group(n, n, mkref(S_AUX2, tt), n, 0);
    P.tt.add_seg(mkref(S_AUX2, r0), n, 1, mkref(S_AUX2, r1), n, 1, n);
    P.rf.add_group(n, n, mkref(S_AUX2, J.r), n, 0);
    P.rf.add_seg(mkref(S_AUX2, tt), n, 0, mkref(S_AUX2, r2), n, 1, n);
  }
  P.ws_end = w;
  return P;
}

}  // namespace tt
