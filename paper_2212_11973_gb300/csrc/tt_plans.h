// Plan compilers (host).  See tt_plans.cpp for the contraction stages.
#pragma once
#include "tt_core.h"

namespace tt {

struct SitePlanHost {
  SiteLayout lay;
  GemmPlan s1, s3, s3l, r1, r3;
  GatherPlan s2, r2;
  int64_t t1_size = 0, t2_size = 0, u1_size = 0, u2_size = 0;
  int64_t lenv_size = 0, renv_size = 0;
  // split-bf16 mode: S1 reads x as per-block transposed copies [(s, a_r)][a_l]
  // with rows padded to 8 elements (K-major B operand); xsplit copies x there.
  CopyPlan xsplit;
  int64_t xt_size = 0;
  // exact mode: the same transposed x as fixed-point digits with a row
  // exponent (int16 after the four levels of the slot)
  DigitPlan xdig;
};
// FP64 environment (natural layout) -> split-bf16 copy with rows padded to 8.
CopyPlan build_env_split(const Bond& B, const std::vector<Q>& chan);
// FP64 environment -> digit rows (padded like the split copy), int16 row
// exponents after the four levels, in the layout's row order.
DigitPlan build_env_digits(const Bond& B, const std::vector<Q>& chan);
// first row of every ket sector's matrix in the environment layout
std::vector<int64_t> env_row_starts(const EnvLayout& E);

struct BondPlanHost {
  BondMatLayout mat;
  GemmPlan b1, b2;
  int64_t t_size = 0;
  // mixed precision: B1's B operand is the transposed split of x (rows padded
  // to 8), B2's A operand the split of T with rows padded to 8
  CopyPlan xsplit, tsplit;
  int64_t xt_size = 0, tp_size = 0;
  DigitPlan xdig, tdig;  // exact mode: digit copies of x (transposed) and of T
};

struct QrPlanHost {
  std::vector<QrJob> jobs;
  CopyPlan gather, scatter, rout;
  std::vector<std::pair<int, int64_t>> scatter_blocks;  // LQ: (old block, column offset in M)
  std::vector<int> lq_cols;                             // LQ: columns of M per left sector
  std::vector<int> new_dim;                             // bond dims after the move
  int64_t ws_size = 0, s_size = 0;
};

// Shifted CholeskyQR3 for the QR jobs of a gauge move (all in the workspace
// slot): G = X^T X, Cholesky (+ shift in the first pass), X <- X R^-1, three
// passes; R = R2 R1 R0 written where the Householder job puts R, Q where it
// puts Q.  Extra workspace starts at ws0.
struct CholQrPlan {
  GemmPlan gram[3], app[3], tt, rf;
  std::vector<CholJob> cj[3];
  int64_t ws_end = 0;
};
CholQrPlan build_cholqr(const std::vector<QrJob>& jobs, int64_t ws0);

// exact (with mixed): the split-BF16 layouts carry fixed-point digits; the
// GEMM segments get the operands' row exponents, the gather items the output
// exponents, S1 writes two-float pairs.
SitePlanHost build_site_plan(const Bond& BL, const Bond& BR, const LocalSpace& ls, const std::vector<MpoTerm>& terms,
                             const std::vector<Q>& chl, const std::vector<Q>& chr, bool mixed, bool exact = false);
BondPlanHost build_bond_plan(const Bond& B, const std::vector<Q>& ch, bool mixed, bool exact = false);
GemmPlan build_absorb_left(const SiteLayout& oldl, const SiteLayout& newl, const Bond& Bold, const Bond& Bnew,
                           const std::vector<int64_t>& soff, const std::vector<int>& new_of_old);
GemmPlan build_absorb_right(const SiteLayout& oldl, const SiteLayout& newl, const Bond& Bold, const Bond& Bnew,
                            const std::vector<int64_t>& soff, const std::vector<int>& new_of_old);
QrPlanHost build_qr_left(const SiteLayout& S, const Bond& BR);
QrPlanHost build_lq_right(const SiteLayout& S, const Bond& BL, bool shrink);

}  // namespace tt
