// Host-side data model of the block-sparse tanTRG state and the device plan
// records consumed by the kernels in tt_kernels.cu.
//
// Charges are U(1) x U(1) labels q = (n, s) = (particle number, 2 Sz).  A bond
// is a sorted list of sectors (charge, dimension).  A "local space" is the set
// of d physical states of one MPO site with their charges; the super-MPS
// physical index is the pair (sigma, sigma') whose charge is q(sigma) -
// q(sigma') (Supplement, "Choi transformation": s_i = (sigma_i, sigma'_i)).
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

namespace tt {

struct Q {
  int n = 0, s = 0;
  bool operator<(const Q& o) const { return n != o.n ? n < o.n : s < o.s; }
  bool operator==(const Q& o) const { return n == o.n && s == o.s; }
  bool operator!=(const Q& o) const { return !(*this == o); }
};
inline Q operator+(Q a, Q b) { return Q{a.n + b.n, a.s + b.s}; }
inline Q operator-(Q a, Q b) { return Q{a.n - b.n, a.s - b.s}; }

// d physical states with charges; pair sectors of (sigma, sigma').
struct LocalSpace {
  int d = 0;
  std::vector<Q> q;                                   // charge of state sigma
  std::vector<Q> pq;                                  // pair-sector charges, sorted
  std::vector<std::vector<std::pair<int, int>>> pairs;  // pairs per sector, by d*sigma+sigma'
  std::vector<int> sec_of, pos_of;                    // pair index d*sigma+sigma' -> (sector, position)
  int find(Q c) const {
    for (size_t i = 0; i < pq.size(); ++i)
      if (pq[i] == c) return (int)i;
    return -1;
  }
};
LocalSpace make_local_space(const std::vector<Q>& charges);
LocalSpace hubbard_site_space();                 // d = 4
LocalSpace product_space(const LocalSpace& a, const LocalSpace& b);  // d = da * db

struct Bond {
  std::vector<Q> q;
  std::vector<int> dim;
  int find(Q c) const;  // -1 if absent
  int nsec() const { return (int)q.size(); }
  int64_t total() const {
    int64_t t = 0;
    for (int d : dim) t += d;
    return t;
  }
};

// Site tensor blocks (l, p, r): r = l + p; row-major [d_l][m_p][d_r]; ordered by
// (r, l, p) so that all blocks sharing a right sector form one contiguous
// row-major matrix of grp_rows[r] rows and d_r columns.
struct SiteBlock {
  int l, p, r;
  int dl, m, dr;
  int64_t off;
  int64_t grp_row;  // first row of this block inside its right-sector group
};
struct SiteLayout {
  const LocalSpace* ls = nullptr;
  std::vector<SiteBlock> blk;
  std::vector<int64_t> grp_off;   // per right sector
  std::vector<int64_t> grp_rows;  // per right sector
  std::vector<int> lp_index;      // [l * npq + p] -> block index or -1
  int npq = 0;
  int64_t size = 0;
  int block_of(int l, int p) const { return lp_index[(size_t)l * npq + p]; }
};
SiteLayout make_site_layout(const Bond& L, const Bond& R, const LocalSpace& ls);

// Environment layout for a bond with MPO channels of charges c[w]: for every
// ket sector b a row-major matrix with rows (w, a), a in sector b + c[w], and
// d_b columns.
struct EnvLayout {
  std::vector<int64_t> off;     // per ket sector
  std::vector<int64_t> rows;    // per ket sector
  std::vector<int> ld;          // per ket sector: row stride (d_b, or d_b rounded up to 8)
  std::vector<int64_t> rowoff;  // [b * nw + w] -> first row or -1
  std::vector<int> bra;         // [b * nw + w] -> bra sector or -1
  int nw = 0;
  int64_t size = 0;
  int64_t row_of(int b, int w) const { return rowoff[(size_t)b * nw + w]; }
};
// pad8: rows padded to a multiple of 8 elements (16-byte aligned bf16 rows,
// the alignment TMA needs for its global strides and base addresses)
EnvLayout make_env_layout(const Bond& B, const std::vector<Q>& chan, bool pad8 = false);
inline int pad8i(int x) { return (x + 7) / 8 * 8; }
inline int64_t pad8l(int64_t x) { return (x + 7) / 8 * 8; }

// Block-diagonal bond matrix (sector q -> q), row-major d_q x d_q blocks.
struct BondMatLayout {
  std::vector<int64_t> off;
  int64_t size = 0;
};
BondMatLayout make_bondmat_layout(const Bond& B);

// ---------------------------------------------------------------------------
// MPO
// ---------------------------------------------------------------------------
struct MpoTerm {
  int wl, wr;     // channel at left / right bond
  int sig, tau;   // <sig| op |tau>
  double v;
};
struct MpoSite {
  std::vector<MpoTerm> terms;  // sorted by (wr, sig, wl, tau)
};
struct Mpo {
  int N = 0;
  int Lx = 0, Wy = 0;
  std::vector<std::vector<Q>> chan;   // chan[k]: channel charges at bond k (0..N)
  std::vector<MpoSite> site;          // W_j, j = 0..N-1
  std::vector<int> start_ch, done_ch; // index of start / done channel at bond k (-1 if absent)
  LocalSpace ls;                      // d = 4
};
struct ModelSpec {
  int Lx, Wy, periodic;
  double t, U, mu;
  int form;
  double tp = 0.0;  // next-nearest (diagonal) hopping of the t-t' model
};
std::vector<std::pair<int, int>> lattice_bonds(const ModelSpec& m);
// Hopping amplitude of every pair (i < j) in 1D order: t on nearest
// neighbours, tp on the diagonals (x, y)-(x+1, y+-1) when tp != 0.
std::map<std::pair<int, int>, double> hopping_bonds(const ModelSpec& m);
Mpo build_hubbard_mpo(const ModelSpec& m);
// Two-site MPO (W_j W_{j+1} summed over the middle channel) on the product space.
MpoSite combine_two_sites(const Mpo& mpo, int j, const LocalSpace& ls2);

// ---------------------------------------------------------------------------
// Device plan records.  Pointers are encoded as slot (8 bits) | element offset
// (56 bits); the launch passes the slot base pointers.
// ---------------------------------------------------------------------------
typedef uint64_t Ref;
inline Ref mkref(int slot, int64_t off) { return ((uint64_t)slot << 56) | (uint64_t)off; }

enum Slot { S_X = 0, S_Y = 1, S_L = 2, S_R = 3, S_T1 = 4, S_T2 = 5, S_AUX = 6, S_AUX2 = 7 };

struct GGroup {
  int M, N;
  int seg0, seg1;
  Ref C;
  int ldc;
  int flags;  // bit0: accumulate into C
};
struct GSeg {
  Ref A, B;
  int lda, ldb, K;
  int tA, tB;  // tA: A stored K x M (row-major) ; tB: B stored N x K (row-major)
  // fixed-point digit operands (exact-accumulation split): the int16 row
  // exponents of A (row m at eA + m * eas) and of B (row n at eB + n * ebs)
  Ref eA = 0, eB = 0;
  int eas = 0, ebs = 0;
};
struct GTile {
  int g, m0, n0, pad;
};
struct GemmPlan {
  std::vector<GGroup> groups;
  std::vector<GSeg> segs;
  double flops = 0;  // algorithmic 2 M N K summed
  void add_group(int M, int N, Ref C, int ldc, int flags = 0) {
    groups.push_back(GGroup{M, N, (int)segs.size(), (int)segs.size(), C, ldc, flags});
  }
  void add_seg(Ref A, int lda, int tA, Ref B, int ldb, int tB, int K) {
    segs.push_back(GSeg{A, B, lda, ldb, K, tA, tB});
    GGroup& g = groups.back();
    g.seg1 = (int)segs.size();
    flops += 2.0 * g.M * (double)g.N * K;
  }
  // row exponents of the last segment's digit operands
  void set_exps(Ref eA, int eas, Ref eB, int ebs) {
    GSeg& s = segs.back();
    s.eA = eA;
    s.eas = eas;
    s.eB = eB;
    s.ebs = ebs;
  }
};

struct GItem {
  Ref dst;
  int64_t dst_rs;
  int rows, cols;
  int c0, c1;
  // digit output: the int16 exponent of item row i at e + i * e_rs
  Ref e = 0;
  int64_t e_rs = 0;
};
struct GContrib {
  Ref src;
  int64_t src_rs;
  double coef;
};
struct GatherPlan {
  std::vector<GItem> items;
  std::vector<GContrib> contribs;
  double elems = 0;
};

struct CItem {
  Ref src, dst;
  int64_t src_rs, src_cs, dst_rs, dst_cs;
  int rows, cols;
};
// FP64 -> split-bf16 copy (levels at dst + l * lo[slot(dst)]) uses CItem too.
struct CopyPlan {
  std::vector<CItem> items;
};

// FP64 rows -> fixed-point BF16 digit rows (exact-accumulation split): row r
// has cols values at src + r * s_r + k * s_k; digit level l of element k goes
// to dst + r * dst_rs + k + l * lo[slot(dst)], the row's int16 exponent to
// e + r * e_rs.
struct DItem {
  Ref src, dst, e;
  int64_t s_r, s_k, dst_rs, e_rs;
  int rows, cols;
};
struct DigitPlan {
  std::vector<DItem> items;
};

// QR job: column-major m x n matrix at ws offset `a` (ld = m); Q written to `q`
// (column-major, ld = m), R (n x n, column-major) to `r`.
struct QrJob {
  int64_t a, q, r;
  int m, n;
};
// One Cholesky + inverse: G = sum of `parts` partial Gram matrices at g + s n^2
// (upper triangles, n x n row-major) -> R (upper, row-major), R^-1.  shift: 1
// adds the CholeskyQR shift to G first; 2 marks the last pass, whose input is
// orthonormal to working accuracy (G = I + E, |E| small); 3 only flags the
// sector (m < n).  `sec` indexes the failure flag.
struct CholJob {
  int64_t g, r, ri;
  int m, n, shift, sec, parts;
  // packed upper-triangle scratch (n (n + 1) / 2 elements) for sectors too
  // large for shared memory
  int64_t pk = 0;
};

}  // namespace tt
