"""Host logic of the library on the CPU: the Hubbard MPO automaton and the
block plans (site H_eff, environment updates, bond H_eff) are built by the
library's own C++ host code and executed by a bounds-checked FP64 plan
executor (tests/host/plan_harness.cpp), in both the FP64 layouts and the
split-BF16 layouts (padded, transposed operands; one FP64 level stands in for
the bf16 levels).  References: the oracle's second-quantised H for the MPO,
and dense einsum contractions of the documented block layouts for the plans."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import model as om
from paper_2212_11973_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_11973_gb300", "csrc")
LOC_Q = [(0, 0), (1, 1), (1, -1), (2, 0)]  # |0>, |up>, |dn>, |updn>: (n, 2Sz)
_PI = C.POINTER(C.c_int)
_PD = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def h(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("harness") / "libplanh.so")
    srcs = [os.path.join(ROOT, "tests", "host", "plan_harness.cpp"),
            os.path.join(CSRC, "tt_model.cpp"), os.path.join(CSRC, "tt_plans.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, *srcs, "-o", out], check=True)
    lib = C.CDLL(out)
    lib.h_error.restype = C.c_char_p
    I64 = C.c_int64
    lib.h_site_op.argtypes = [_PI, _PD, C.c_int, C.c_int, C.c_int, C.c_int, _PI, _PI, _PI, _PI,
                              _PD, I64, _PD, I64, _PD, I64, _PD, I64]
    lib.h_bond_op.argtypes = [_PI, _PD, C.c_int, C.c_int, C.c_int, _PI, _PI, _PI, _PD, I64, _PD, I64, _PD, I64, _PD]
    return lib


def _ia(v):
    return (C.c_int * max(len(v), 1))(*v)


def _pd(a):
    return a.ctypes.data_as(_PD)


def _chk(lib, rc):
    assert rc == 0, lib.h_error().decode()


class Model:
    def __init__(self, lib, Lx, Wy, periodic, t, U, mu, form, tp=0.0):
        self.lib = lib
        self.geom = _ia([Lx, Wy, int(periodic), form])
        self.par = (C.c_double * 4)(t, U, mu, tp)
        N = C.c_int()
        dims = _ia([0] * 600)
        _chk(lib, lib.h_mpo_shape(self.geom, self.par, C.byref(N), dims, 600))
        self.N = N.value
        self.chi = [dims[k] for k in range(self.N + 1)]

    def W(self, j):
        W = np.zeros((self.chi[j], 4, 4, self.chi[j + 1]))
        _chk(self.lib, self.lib.h_mpo_site_dense(self.geom, self.par, j, _pd(W)))
        return W

    def chan(self, k):
        qn, qs = _ia([0] * self.chi[k]), _ia([0] * self.chi[k])
        _chk(self.lib, self.lib.h_mpo_chan(self.geom, self.par, k, qn, qs, self.chi[k]))
        return [(qn[w], qs[w]) for w in range(self.chi[k])]


# ---- the documented block layouts -> dense arrays ---------------------------

LOC_Q2 = [(a[0] + b[0], a[1] + b[1]) for a in LOC_Q for b in LOC_Q]  # sigma = 4 sigma_1 + sigma_2


def _pairs(loc=LOC_Q):
    d = len(loc)
    pq = {}
    for s in range(d):
        for sp in range(d):
            c = (loc[s][0] - loc[sp][0], loc[s][1] - loc[sp][1])
            pq.setdefault(c, []).append((s, sp))
    return [(c, sorted(v, key=lambda t: d * t[0] + t[1])) for c, v in sorted(pq.items())]


def _offsets(secs):
    o, out = 0, []
    for _, _, d in secs:
        out.append(o)
        o += d
    return out, o


def site_blocks(SL, SR, loc=LOC_Q):
    blocks, off = [], 0
    for r, (rn, rs, dr) in enumerate(SR):
        for l, (ln, ls_, dl) in enumerate(SL):
            for p, (c, prs) in enumerate(_pairs(loc)):
                if (ln + c[0], ls_ + c[1]) == (rn, rs):
                    blocks.append((l, r, prs, dl, dr, off))
                    off += dl * len(prs) * dr
    return blocks, off


def site_to_dense(v, SL, SR, loc=LOC_Q):
    ol, DL = _offsets(SL)
    orr, DR = _offsets(SR)
    d = len(loc)
    X = np.zeros((DL, d, d, DR))
    blocks, n = site_blocks(SL, SR, loc)
    assert n == v.size
    for l, r, prs, dl, dr, off in blocks:
        b = v[off:off + dl * len(prs) * dr].reshape(dl, len(prs), dr)
        for k, (s, sp) in enumerate(prs):
            X[ol[l]:ol[l] + dl, s, sp, orr[r]:orr[r] + dr] = b[:, k, :]
    return X


def env_size(S, chan):
    idx = {(n, s): i for i, (n, s, _) in enumerate(S)}
    tot = 0
    for (bn, bs, db) in S:
        for c in chan:
            a = idx.get((bn + c[0], bs + c[1]))
            if a is not None:
                tot += S[a][2] * db
    return tot


def env_to_dense(v, S, chan):
    """E[a, w, b] from the layout: per ket sector b, rows (w, a in b + c_w)."""
    o, D = _offsets(S)
    idx = {(n, s): i for i, (n, s, _) in enumerate(S)}
    E = np.zeros((D, len(chan), D))
    pos = 0
    for b, (bn, bs, db) in enumerate(S):
        for w, c in enumerate(chan):
            a = idx.get((bn + c[0], bs + c[1]))
            if a is None:
                continue
            da = S[a][2]
            E[o[a]:o[a] + da, w, o[b]:o[b] + db] = v[pos:pos + da * db].reshape(da, db)
            pos += da * db
    assert pos == v.size
    return E


def bondmat_to_dense(v, S):
    o, D = _offsets(S)
    M = np.zeros((D, D))
    pos = 0
    for i, (_, _, d) in enumerate(S):
        M[o[i]:o[i] + d, o[i]:o[i] + d] = v[pos:pos + d * d].reshape(d, d)
        pos += d * d
    assert pos == v.size
    return M


def _secs_arrays(*bonds):
    allsec = [s for b in bonds for s in b]
    return _ia([s[0] for s in allsec]), _ia([s[1] for s in allsec]), _ia([s[2] for s in allsec])


# ---- tests -------------------------------------------------------------------

@pytest.mark.parametrize("geo", [(2, 2, False, 0, 0.0), (2, 2, False, 1, 0.0), (3, 1, False, 1, 0.0),
                                 (2, 3, True, 1, 0.0), (2, 2, False, 1, -0.3), (2, 3, True, 0, 0.25),
                                 (3, 2, False, 1, -0.2)])
def test_mpo_automaton_equals_second_quantised_H(h, geo):
    """The library's compressed automaton contracts to the oracle's H (Eq. 3 /
    PH-symmetric form, with and without the t' diagonals) built from
    fermionic modes with Jordan-Wigner."""
    Lx, Wy, per, form, tp = geo
    m = Model(h, Lx, Wy, per, 1.0, 4.0, 0.3, form, tp)
    s0, dN = C.c_int(), C.c_int()
    _chk(h, h.h_mpo_boundary(m.geom, m.par, C.byref(s0), C.byref(dN)))
    T = np.zeros((1, 1, m.chi[0]))
    T[0, 0, s0.value] = 1.0
    for j in range(m.N):
        T = np.einsum("abw,wstv->asbtv", T, m.W(j)).reshape(T.shape[0] * 4, T.shape[1] * 4, m.chi[j + 1])
    H = T[:, :, dN.value]
    ref = om.dense_hamiltonian(om.Model(Lx, Wy, per, 1.0, 4.0, 0.3, form, tp)).toarray()
    assert np.abs(H - ref).max() < 1e-12


CHARGES = [(n, s) for n in range(-2, 3) for s in range(-2, 3) if (n + s) % 2 == 0]


def _random_bonds(D, seed):
    SL = wl.gaussian_sectors(D, 1.0, CHARGES, seed)
    SR = wl.gaussian_sectors(D + 3, 1.0, CHARGES, seed + 1)
    return SL, SR


# sector dimensions 1..9 (not multiples of 8: the split-BF16 layouts pad)
CASES = [((4, 2, False, 1), 3, 30), ((3, 3, True, 1), 4, 40)]
TP = {(4, 2, False, 1): 0.0, (3, 3, True, 1): -0.25}  # the cylinder case has t' diagonals


@pytest.mark.parametrize("geo,j,D", CASES)
@pytest.mark.parametrize("mixed", [0, 1])
def test_site_plans_match_dense_contractions(h, geo, j, D, mixed):
    Lx, Wy, per, form = geo
    m = Model(h, Lx, Wy, per, 1.0, 4.0, -0.3, form, TP[geo])
    SL, SR = _random_bonds(D, 7 + j)
    cl, cr = m.chan(j), m.chan(j + 1)
    W = m.W(j)
    _, nx = site_blocks(SL, SR)
    nL, nR = env_size(SL, cl), env_size(SR, cr)
    rng = np.random.default_rng(11)
    x, L, R = rng.standard_normal(nx), rng.standard_normal(nL), rng.standard_normal(nR)
    Xd, Ld, Rd = site_to_dense(x, SL, SR), env_to_dense(L, SL, cl), env_to_dense(R, SR, cr)
    qn, qs, qd = _secs_arrays(SL, SR)
    ns = _ia([len(SL), len(SR)])

    def run(op, nout):
        out = np.zeros(nout)
        _chk(h, h.h_site_op(m.geom, m.par, j, op, mixed, 0, ns, qn, qs, qd, _pd(L), nL, _pd(R), nR, _pd(x), nx,
                            _pd(out), nout))
        return out

    # H_eff apply: y[a,s,s',a'] = L[a,w,b] W[w,s,t,w'] x[b,t,s',c] R[a',w',c]
    y = site_to_dense(run(0, nx), SL, SR)
    T = np.tensordot(Ld, Xd, axes=([2], [0]))                   # a w t x c
    T = np.tensordot(T, W, axes=([1, 2], [0, 2]))               # a x c s v
    ref = np.tensordot(T, Rd, axes=([2, 4], [2, 1])).transpose(0, 2, 1, 3)  # a s x d
    assert np.abs(y - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())
    # left environment: L'[a',w',b'] = x[a,s,s',a'] L[a,w,b] W[w,s,t,w'] x[b,t,s',b']
    Ln = env_to_dense(run(1, env_size(SR, cr)), SR, cr)
    T = np.tensordot(Ld, Xd, axes=([2], [0]))                   # a w t x e
    T = np.tensordot(T, W, axes=([1, 2], [0, 2]))               # a x e s v
    ref = np.tensordot(Xd, T, axes=([0, 1, 2], [0, 3, 1]))      # d e v
    ref = ref.transpose(0, 2, 1)
    assert np.abs(Ln - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())
    # right environment: R'[a,w,b] = x[a,s,s',a'] W[w,s,t,w'] x[b,t,s',b'] R[a',w',b']
    Rn = env_to_dense(run(2, env_size(SL, cl)), SL, cl)
    T = np.tensordot(Xd, Rd, axes=([3], [2]))                   # b t x d v
    T = np.tensordot(W, T, axes=([2, 3], [1, 4]))               # w s b x d
    ref = np.tensordot(Xd, T, axes=([1, 2, 3], [1, 3, 4]))      # a w b
    assert np.abs(Rn - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("mixed", [0, 1])
def test_bond_plan_matches_dense_contraction(h, mixed):
    m = Model(h, 3, 3, True, 1.0, 4.0, -0.3, 1)
    k = 4
    S = wl.gaussian_sectors(45, 1.0, CHARGES, 5)
    ch = m.chan(k)
    n = sum(d * d for _, _, d in S)
    nE = env_size(S, ch)
    rng = np.random.default_rng(3)
    x, L, R = rng.standard_normal(n), rng.standard_normal(nE), rng.standard_normal(nE)
    qn, qs, qd = _secs_arrays(S)
    y = np.zeros(n)
    _chk(h, h.h_bond_op(m.geom, m.par, k, mixed, len(S), qn, qs, qd, _pd(L), nE, _pd(R), nE, _pd(x), n, _pd(y)))
    Ld, Rd, Sd = env_to_dense(L, S, ch), env_to_dense(R, S, ch), bondmat_to_dense(x, S)
    ref = np.tensordot(np.tensordot(Ld, Sd, axes=([2], [0])), Rd, axes=([1, 2], [1, 2]))
    assert np.abs(bondmat_to_dense(y, S) - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


def test_cholqr_gauge_plan_factorises_every_sector(h):
    """Left gauge move of a site by the library's QR and CholeskyQR3 plans
    (CPU restatement of the device Cholesky step): for every right sector with
    at least as many rows as columns, X_r = Q_r R_r with Q_r orthonormal and R_r
    upper triangular with a positive diagonal, to FP64 rounding; sectors with
    more columns than rows are flagged for the Householder kernel."""
    SL = wl.gaussian_sectors(40, 1.0, CHARGES, 21)
    SR = wl.gaussian_sectors(60, 1.0, CHARGES, 22)
    blocks, nx = site_blocks(SL, SR)
    x = np.random.default_rng(5).standard_normal(nx)
    # ill-conditioned columns (condition up to ~1e11, where unshifted CholeskyQR2
    # would break down): scale the a_r index of each right sector by 10^-k
    orr, _ = _offsets(SR)
    Xd = site_to_dense(x, SL, SR)
    for i, (_, _, d) in enumerate(SR):
        Xd[..., orr[i]:orr[i] + d] *= np.logspace(0, -11, d)
    # back to the block layout
    for l, r, prs, dl, dr, off in blocks:
        ol, _ = _offsets(SL)
        b = np.stack([Xd[ol[l]:ol[l] + dl, s, sp, orr[r]:orr[r] + dr] for s, sp in prs], axis=1)
        x[off:off + b.size] = b.ravel()
    qn, qs, qd = _secs_arrays(SL, SR)
    nrout = sum(d * d for _, _, d in SR)
    q, rr, fail = np.zeros(nx), np.zeros(nrout), (C.c_int * len(SR))()
    h.h_qr_left.argtypes = [C.c_int, C.c_int, _PI, _PI, _PI, _PD, C.c_int64, _PD, _PD, C.c_int64, _PI]
    _chk(h, h.h_qr_left(len(SL), len(SR), qn, qs, qd, _pd(x), nx, _pd(q), _pd(rr), nrout, fail))
    # group matrix of right sector r: rows (l, p, s, a_l) in block order, cols a_r
    rpos, checked = 0, 0
    for ri, (_, _, dr) in enumerate(SR):
        rows = [(off, dl * len(prs)) for l, r, prs, dl, d2, off in blocks if r == ri]
        m = sum(n for _, n in rows)
        R = rr[rpos:rpos + dr * dr].reshape(dr, dr)  # the bond matrix S, row-major
        rpos += dr * dr
        if m < dr:
            assert fail[ri] == 1
            continue
        assert fail[ri] == 0
        Xr = np.concatenate([x[o:o + n * dr].reshape(n, dr) for o, n in rows])
        Qr = np.concatenate([q[o:o + n * dr].reshape(n, dr) for o, n in rows])
        assert np.abs(Qr @ R - Xr).max() < 1e-13 * np.abs(Xr).max()
        assert np.abs(Qr.T @ Qr - np.eye(dr)).max() < 1e-13
        assert np.abs(np.tril(R, -1)).max() == 0.0 and np.all(np.diag(R) > 0)
        checked += 1
    assert checked >= len(SR) - 2


@pytest.mark.parametrize("mixed", [0, 1])
def test_two_site_plan_matches_dense_contraction(h, mixed):
    """Growth stage: W_j W_{j+1} combined over the middle channel equals the
    product of the single-site W's, and the two-site H_eff plan (product local
    space, d = 16) equals the dense contraction."""
    m = Model(h, 3, 3, True, 1.0, 4.0, -0.3, 1)
    j = 3
    W1, W2 = m.W(j), m.W(j + 1)
    W12 = np.zeros((m.chi[j], 16, 16, m.chi[j + 2]))
    _chk(h, h.h_mpo_two_site_dense(m.geom, m.par, j, _pd(W12)))
    # W12[w, (s1 s2), (t1 t2), u] = sum_v W_j[w, s1, t1, v] W_{j+1}[v, s2, t2, u]
    dense12 = np.einsum("wacv,vbdu->wabcdu", W1, W2).reshape(m.chi[j], 16, 16, m.chi[j + 2])
    assert np.abs(W12 - dense12).max() < 1e-14
    SL = wl.gaussian_sectors(12, 1.0, CHARGES, 31)
    SR = wl.gaussian_sectors(14, 1.0, CHARGES, 32)
    cl, cr = m.chan(j), m.chan(j + 2)
    _, nx = site_blocks(SL, SR, LOC_Q2)
    nL, nR = env_size(SL, cl), env_size(SR, cr)
    rng = np.random.default_rng(17)
    x, L, R = rng.standard_normal(nx), rng.standard_normal(nL), rng.standard_normal(nR)
    qn, qs, qd = _secs_arrays(SL, SR)
    y = np.zeros(nx)
    _chk(h, h.h_site_op(m.geom, m.par, j, 0, mixed, 1, _ia([len(SL), len(SR)]), qn, qs, qd, _pd(L), nL, _pd(R),
                        nR, _pd(x), nx, _pd(y), nx))
    Xd = site_to_dense(x, SL, SR, LOC_Q2)
    Ld, Rd = env_to_dense(L, SL, cl), env_to_dense(R, SR, cr)
    T = np.tensordot(Ld, Xd, axes=([2], [0]))
    T = np.tensordot(T, W12, axes=([1, 2], [0, 2]))
    refy = np.tensordot(T, Rd, axes=([2, 4], [2, 1])).transpose(0, 2, 1, 3)
    assert np.abs(site_to_dense(y, SL, SR, LOC_Q2) - refy).max() < 1e-11 * max(1.0, np.abs(refy).max())


@pytest.mark.parametrize("side", [0, 1])
def test_absorb_plans_match_dense_products(h, side):
    """A <- S A (left bond) and A <- A S (right bond) through the absorb plans."""
    SL = wl.gaussian_sectors(25, 1.0, CHARGES, 41)
    SR = wl.gaussian_sectors(28, 1.0, CHARGES, 42)
    _, nx = site_blocks(SL, SR)
    B = SL if side == 0 else SR
    ns = sum(d * d for _, _, d in B)
    rng = np.random.default_rng(9)
    x, S = rng.standard_normal(nx), rng.standard_normal(ns)
    qn, qs, qd = _secs_arrays(SL, SR)
    y = np.zeros(nx)
    h.h_absorb.argtypes = [C.c_int, C.c_int, C.c_int, _PI, _PI, _PI, _PD, C.c_int64, _PD, C.c_int64, _PD]
    _chk(h, h.h_absorb(side, len(SL), len(SR), qn, qs, qd, _pd(x), nx, _pd(S), ns, _pd(y)))
    Xd, Sd = site_to_dense(x, SL, SR), bondmat_to_dense(S, B)
    ref = np.tensordot(Sd, Xd, axes=([1], [0])) if side == 0 else np.tensordot(Xd, Sd, axes=([3], [0]))
    assert np.abs(site_to_dense(y, SL, SR) - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("geo,j,D", CASES + [((4, 2, False, 1), 3, 300)])
def test_exact_split_exponents_follow_their_rows(h, geo, j, D):
    """Exact-accumulation split plans: every digit operand row of every GEMM
    segment (S1, S3, B1, B2) reads the int16 exponent that its producer (digit
    copy of x, of T, of the environments, or the digit W-gather) wrote for
    exactly that row, and that row covers the segment's K."""
    Lx, Wy, per, form = geo
    m = Model(h, Lx, Wy, per, 1.0, 4.0, -0.3, form, TP.get(geo, 0.0))
    SL, SR = _random_bonds(D, 17 + j)
    qn, qs, qd = _secs_arrays(SL, SR)
    h.h_exact_exponents.argtypes = [_PI, _PD, C.c_int, _PI, _PI, _PI, _PI]
    _chk(h, h.h_exact_exponents(m.geom, m.par, j, _ia([len(SL), len(SR)]), qn, qs, qd))


@pytest.mark.parametrize("geo,j,D", CASES + [((6, 6, True, 1), 17, 200)])
def test_digit_gather_items_fit_the_kernel(h, geo, j, D):
    """The digit W-gather (two columns per lane, 32-bit stores of BF16 pairs,
    MPO coefficient splits in a 64-entry shared table) relies on plan
    properties the host also checks before a launch: rows of at most 256
    columns, at most 64 MPO terms per item, even BF16 offsets, disjoint items,
    and an odd row's extra column inside its own zero padding.  Includes a
    6-wide cylinder site (the widest MPO of the workloads) with odd-width
    sectors."""
    Lx, Wy, per, form = geo
    m = Model(h, Lx, Wy, per, 1.0, 8.0, -2.48, form, TP.get(geo, 0.0))
    SL, SR = _random_bonds(D, 29 + j)
    qn, qs, qd = _secs_arrays(SL, SR)
    stats = _ia([0, 0, 0])
    h.h_gather_digit_items.argtypes = [_PI, _PD, C.c_int, _PI, _PI, _PI, _PI, C.c_int, C.c_int, _PI]
    _chk(h, h.h_gather_digit_items(m.geom, m.par, j, _ia([len(SL), len(SR)]), qn, qs, qd, 256, 64, stats))
    assert 0 < stats[0] <= 256 and 0 < stats[1] <= 64
    assert stats[2] > 0  # odd widths occur, so the padding rule is exercised
