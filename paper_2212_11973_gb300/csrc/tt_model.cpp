// Lattice, local spaces, block layouts and the Hubbard MPO automaton (host).
//
// Hubbard Hamiltonian: Eq. 3 (form 0) or the particle-hole symmetric on-site
// term U (n_up - 1/2)(n_dn - 1/2) of the DQMC appendix (form 1).  The lattice is
// mapped to a chain by the snake path of Fig. 1(a); hopping terms become
// long-range 1D terms with Jordan-Wigner parity strings.
//
// MPO automaton (compressed per bond): the channels of bond k are "start"
// (nothing placed), "done" (a whole term placed) and one channel per (operator
// type o, left endpoint i) of every lattice bond (i, j) that crosses bond k
// (i < k <= j).  Channel charges are the charges the left part has changed:
// c+_up F: (+1,+1), c+_dn F: (+1,-1), F c_up: (-1,-1), F c_dn: (-1,+1).
#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <stdexcept>

#include "tt_core.h"

namespace tt {

// ---------------------------------------------------------------------------
LocalSpace make_local_space(const std::vector<Q>& charges) {
  LocalSpace ls;
  ls.d = (int)charges.size();
  ls.q = charges;
  std::set<Q> ps;
  for (int a = 0; a < ls.d; ++a)
    for (int b = 0; b < ls.d; ++b) ps.insert(charges[a] - charges[b]);
  ls.pq.assign(ps.begin(), ps.end());
  ls.pairs.assign(ls.pq.size(), {});
  ls.sec_of.assign((size_t)ls.d * ls.d, -1);
  ls.pos_of.assign((size_t)ls.d * ls.d, -1);
  for (int a = 0; a < ls.d; ++a)
    for (int b = 0; b < ls.d; ++b) {
      int p = ls.find(charges[a] - charges[b]);
      ls.sec_of[(size_t)a * ls.d + b] = p;
      ls.pos_of[(size_t)a * ls.d + b] = (int)ls.pairs[p].size();
      ls.pairs[p].push_back({a, b});
    }
  return ls;
}

LocalSpace hubbard_site_space() {
  // sigma = n_up + 2 n_dn: |0>, |up>, |dn>, |up dn>
  return make_local_space({Q{0, 0}, Q{1, 1}, Q{1, -1}, Q{2, 0}});
}

LocalSpace product_space(const LocalSpace& a, const LocalSpace& b) {
  std::vector<Q> c;
  for (int x = 0; x < a.d; ++x)
    for (int y = 0; y < b.d; ++y) c.push_back(a.q[x] + b.q[y]);
  return make_local_space(c);
}

int Bond::find(Q c) const {
  auto it = std::lower_bound(q.begin(), q.end(), c);
  if (it == q.end() || *it != c) return -1;
  return (int)(it - q.begin());
}

SiteLayout make_site_layout(const Bond& L, const Bond& R, const LocalSpace& ls) {
  SiteLayout S;
  S.ls = &ls;
  S.npq = (int)ls.pq.size();
  S.lp_index.assign((size_t)L.nsec() * S.npq, -1);
  S.grp_off.assign(R.nsec(), 0);
  S.grp_rows.assign(R.nsec(), 0);
  int64_t off = 0;
  for (int r = 0; r < R.nsec(); ++r) {
    S.grp_off[r] = off;
    int64_t row = 0;
    for (int l = 0; l < L.nsec(); ++l)
      for (int p = 0; p < S.npq; ++p) {
        if (!(L.q[l] + ls.pq[p] == R.q[r])) continue;
        SiteBlock b;
        b.l = l;
        b.p = p;
        b.r = r;
        b.dl = L.dim[l];
        b.m = (int)ls.pairs[p].size();
        b.dr = R.dim[r];
        b.off = off;
        b.grp_row = row;
        S.lp_index[(size_t)l * S.npq + p] = (int)S.blk.size();
        S.blk.push_back(b);
        off += (int64_t)b.dl * b.m * b.dr;
        row += (int64_t)b.dl * b.m;
      }
    S.grp_rows[r] = row;
  }
  S.size = off;
  return S;
}

EnvLayout make_env_layout(const Bond& B, const std::vector<Q>& chan, bool pad8) {
  EnvLayout E;
  E.nw = (int)chan.size();
  E.off.assign(B.nsec(), 0);
  E.rows.assign(B.nsec(), 0);
  E.ld.assign(B.nsec(), 0);
  E.rowoff.assign((size_t)B.nsec() * E.nw, -1);
  E.bra.assign((size_t)B.nsec() * E.nw, -1);
  int64_t off = 0;
  for (int b = 0; b < B.nsec(); ++b) {
    E.off[b] = off;
    int64_t row = 0;
    for (int w = 0; w < E.nw; ++w) {
      int a = B.find(B.q[b] + chan[w]);
      if (a < 0) continue;
      E.rowoff[(size_t)b * E.nw + w] = row;
      E.bra[(size_t)b * E.nw + w] = a;
      row += B.dim[a];
    }
    E.rows[b] = row;
    E.ld[b] = pad8 ? pad8i(B.dim[b]) : B.dim[b];
    off += row * E.ld[b];
  }
  E.size = off;
  return E;
}

BondMatLayout make_bondmat_layout(const Bond& B) {
  BondMatLayout M;
  M.off.resize(B.nsec());
  int64_t off = 0;
  for (int b = 0; b < B.nsec(); ++b) {
    M.off[b] = off;
    off += (int64_t)B.dim[b] * B.dim[b];
  }
  M.size = off;
  return M;
}

// ---------------------------------------------------------------------------
static int snake(int x, int y, int W) { return x * W + ((x % 2 == 0) ? y : W - 1 - y); }

std::vector<std::pair<int, int>> lattice_bonds(const ModelSpec& m) {
  std::set<std::pair<int, int>> out;
  for (int x = 0; x < m.Lx; ++x)
    for (int y = 0; y < m.Wy; ++y) {
      int i = snake(x, y, m.Wy);
      std::vector<int> nb;
      if (x + 1 < m.Lx) nb.push_back(snake(x + 1, y, m.Wy));
      if (y + 1 < m.Wy)
        nb.push_back(snake(x, y + 1, m.Wy));
      else if (m.periodic && m.Wy > 2)
        nb.push_back(snake(x, 0, m.Wy));
      for (int j : nb) out.insert({std::min(i, j), std::max(i, j)});
    }
  return std::vector<std::pair<int, int>>(out.begin(), out.end());
}

std::map<std::pair<int, int>, double> hopping_bonds(const ModelSpec& m) {
  std::map<std::pair<int, int>, double> amp;
  for (auto& b : lattice_bonds(m)) amp[b] += m.t;
  if (m.tp != 0.0)
    for (int x = 0; x + 1 < m.Lx; ++x)
      for (int y = 0; y < m.Wy; ++y)
        for (int dy : {1, -1}) {
          int yy = y + dy;
          if (yy < 0 || yy >= m.Wy) {
            if (!(m.periodic && m.Wy > 2)) continue;
            yy = (yy + m.Wy) % m.Wy;
          }
          const int i = snake(x, y, m.Wy), j = snake(x + 1, yy, m.Wy);
          amp[{std::min(i, j), std::max(i, j)}] += m.tp;
        }
  return amp;
}

namespace {
// 4x4 local operators as dense row-major arrays, basis sigma = n_up + 2 n_dn.
struct Op4 {
  double a[16] = {0};
  double& operator()(int i, int j) { return a[i * 4 + j]; }
  double operator()(int i, int j) const { return a[i * 4 + j]; }
};
Op4 mul(const Op4& x, const Op4& y) {
  Op4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += x(i, k) * y(k, j);
      r(i, j) = s;
    }
  return r;
}
Op4 transpose(const Op4& x) {
  Op4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r(i, j) = x(j, i);
  return r;
}
Op4 diag(double a, double b, double c, double d) {
  Op4 r;
  r(0, 0) = a; r(1, 1) = b; r(2, 2) = c; r(3, 3) = d;
  return r;
}
}  // namespace

Mpo build_hubbard_mpo(const ModelSpec& m) {
  Mpo M;
  M.N = m.Lx * m.Wy;
  M.Lx = m.Lx;
  M.Wy = m.Wy;
  M.ls = hubbard_site_space();
  const int N = M.N;
  const auto amp = hopping_bonds(m);
  std::vector<std::pair<int, int>> bonds;
  for (auto& kv : amp) bonds.push_back(kv.first);

  // local operators: c_up = a_up, c_dn = F_up a_dn (up before down in a site)
  Op4 a_up, a_dn;
  a_up(0, 1) = 1; a_up(2, 3) = 1;
  a_dn(0, 2) = 1; a_dn(1, 3) = 1;
  Op4 F = diag(1, -1, -1, 1), Fup = diag(1, -1, 1, -1), I = diag(1, 1, 1, 1);
  Op4 c_up = a_up, c_dn = mul(Fup, a_dn);
  Op4 cd_up = transpose(c_up), cd_dn = transpose(c_dn);
  Op4 left[4] = {mul(cd_up, F), mul(cd_dn, F), mul(F, c_up), mul(F, c_dn)};
  Op4 right[4] = {c_up, c_dn, cd_up, cd_dn};
  Q och[4] = {Q{1, 1}, Q{1, -1}, Q{-1, -1}, Q{-1, 1}};
  Op4 nu = diag(0, 1, 0, 1), nd = diag(0, 0, 1, 1);
  Op4 onsite;
  for (int i = 0; i < 4; ++i) {
    double vu = nu(i, i), vd = nd(i, i);
    double v = (m.form == 0) ? m.U * vu * vd : m.U * (vu - 0.5) * (vd - 0.5);
    onsite(i, i) = v - m.mu * (vu + vd);
  }

  // channel lists per bond k (0..N): bond k lies between site k-1 and site k
  // key: (kind, o, i) ; kind 0 = start, 1 = done, 2 = hop channel
  struct Key {
    int kind, o, i;
    bool operator<(const Key& b) const {
      if (kind != b.kind) return kind < b.kind;
      if (o != b.o) return o < b.o;
      return i < b.i;
    }
  };
  std::vector<std::map<Key, int>> cidx(N + 1);
  M.chan.assign(N + 1, {});
  M.start_ch.assign(N + 1, -1);
  M.done_ch.assign(N + 1, -1);
  for (int k = 0; k <= N; ++k) {
    std::vector<Key> keys;
    if (k < N) keys.push_back({0, 0, 0});
    if (k > 0) keys.push_back({1, 0, 0});
    std::set<int> lefts;
    for (auto& b : bonds)
      if (b.first < k && k <= b.second) lefts.insert(b.first);
    for (int o = 0; o < 4; ++o)
      for (int i : lefts) keys.push_back({2, o, i});
    std::sort(keys.begin(), keys.end());
    for (size_t w = 0; w < keys.size(); ++w) {
      cidx[k][keys[w]] = (int)w;
      Q c = keys[w].kind == 2 ? och[keys[w].o] : Q{0, 0};
      M.chan[k].push_back(c);
      if (keys[w].kind == 0) M.start_ch[k] = (int)w;
      if (keys[w].kind == 1) M.done_ch[k] = (int)w;
    }
  }
  auto chan = [&](int k, Key key) -> int {
    auto it = cidx[k].find(key);
    return it == cidx[k].end() ? -1 : it->second;
  };

  M.site.assign(N, {});
  for (int j = 0; j < N; ++j) {
    std::vector<MpoTerm> terms;
    auto add = [&](int wl, int wr, const Op4& op, double s) {
      if (wl < 0 || wr < 0) return;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          if (op(a, b) != 0.0) terms.push_back(MpoTerm{wl, wr, a, b, s * op(a, b)});
    };
    int sl = chan(j, {0, 0, 0}), dl = chan(j, {1, 0, 0});
    int sr = chan(j + 1, {0, 0, 0}), dr = chan(j + 1, {1, 0, 0});
    add(sl, sr, I, 1.0);
    add(dl, dr, I, 1.0);
    add(sl, dr, onsite, 1.0);
    for (int o = 0; o < 4; ++o) {
      add(sl, chan(j + 1, {2, o, j}), left[o], 1.0);  // a hop starts at site j
      for (auto& b : bonds) {
        int i = b.first;
        if (i >= j) continue;
        int wl = chan(j, {2, o, i});
        if (wl < 0) continue;
        if (b.second == j) add(wl, dr, right[o], -amp.at(b));  // the hop (i, j) closes here
      }
      // pass-through: a pending channel (o, i) continues with the parity F
      for (auto& kv : cidx[j]) {
        if (kv.first.kind != 2 || kv.first.o != o) continue;
        int wr = chan(j + 1, kv.first);
        if (wr >= 0) add(kv.second, wr, F, 1.0);
      }
    }
    std::sort(terms.begin(), terms.end(), [](const MpoTerm& a, const MpoTerm& b) {
      if (a.wr != b.wr) return a.wr < b.wr;
      if (a.sig != b.sig) return a.sig < b.sig;
      if (a.wl != b.wl) return a.wl < b.wl;
      return a.tau < b.tau;
    });
    M.site[j].terms = terms;
  }
  return M;
}

MpoSite combine_two_sites(const Mpo& mpo, int j, const LocalSpace& ls2) {
  // W12[w, (s1 s2), (t1 t2), w''] = sum_w' W_j[w, s1, t1, w'] W_{j+1}[w', s2, t2, w'']
  std::map<std::tuple<int, int, int, int>, double> acc;
  const auto& A = mpo.site[j].terms;
  const auto& B = mpo.site[j + 1].terms;
  int d2 = mpo.ls.d;
  for (const auto& a : A)
    for (const auto& b : B) {
      if (a.wr != b.wl) continue;
      int s = a.sig * d2 + b.sig, t = a.tau * d2 + b.tau;
      acc[{a.wl, b.wr, s, t}] += a.v * b.v;
    }
  MpoSite out;
  for (auto& kv : acc)
    if (kv.second != 0.0)
      out.terms.push_back(MpoTerm{std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                                  std::get<3>(kv.first), kv.second});
  std::sort(out.terms.begin(), out.terms.end(), [](const MpoTerm& a, const MpoTerm& b) {
    if (a.wr != b.wr) return a.wr < b.wr;
    if (a.sig != b.sig) return a.sig < b.sig;
    if (a.wl != b.wl) return a.wl < b.wl;
    return a.tau < b.tau;
  });
  (void)ls2;
  return out;
}

}  // namespace tt
