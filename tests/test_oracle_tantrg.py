"""Pins of the dense tanTRG oracle (integrator, Lanczos, gauge, truncation).

The strongest pin is tangent-space exactness (Supplement, "Splitting method"):
with bond dimensions at their maximum the 1-TDVP/2-TDVP integrators carry no
projection error, so the oracle started from the initial state padded to
maximal bonds must reproduce exact diagonalisation of the same initial
state, exp(-(beta-beta0) H/2)(I - beta0 H/2), to rounding and Krylov error.
Planted mistakes (wrong step length, wrong bond-step sign) must break it.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import model as om
from oracle import mpo as ompo
from oracle import tantrg as tt

KEYS = ("lnZ", "energy_per_site", "density", "double_occ")


def _rel(a, b):
    return abs(a - b) / max(1e-300, abs(b))


def _run_vs_ed(m, D, beta_end, tol, beta0=0.01, dtau=0.05):
    W = ompo.hubbard_mpo(m)
    st = tt.run(W, beta0, dtau, beta_end, tt.TruncOpts(D), pad_full=True)
    ob = tt.measure(st)
    ed = om.ed_thermo(m, [st.beta], beta0=beta0)[0]
    for k in KEYS:
        assert _rel(ob[k], ed[k]) < tol, (k, ob[k], ed[k])
    return st, ob


def test_full_rank_chain_matches_ed():
    """3-site open chain, bonds at their maximum (16, 16): exact up to Krylov error."""
    m = om.Model(1, 3, False, U=3.0, mu=0.4, form=0)
    st, _ = _run_vs_ed(m, 16, 1.51, 1e-10)
    assert st.bond_dims() == [16, 16]
    assert tt.hermiticity_defect(st) < 1e-7


@pytest.mark.slow
def test_full_rank_2x2_matches_ed():
    """2x2 cluster of the first workload (U=4, PH form, mu=0) untruncated (D=256)."""
    m = om.Model(2, 2, False, U=4.0, mu=0.0, form=1)
    st, ob = _run_vs_ed(m, 256, 0.51, 1e-10)
    assert st.bond_dims() == [16, 256, 16]
    assert abs(ob["density"] - 1.0) < 1e-10  # half filling at PH-symmetric mu = 0


def test_planted_wrong_step_length_is_caught(monkeypatch):
    """tau = dtau/2 per half sweep (instead of dtau/4) must break the ED pin."""
    real = tt.tdvp1_step

    def broken(st, dtau, K=8):
        tt.tdvp1_sweep_lr(st, dtau / 2, K)
        tt.tdvp1_sweep_rl(st, dtau / 2, K)
        st.beta += dtau

    monkeypatch.setattr(tt, "tdvp1_step", broken)
    m = om.Model(1, 3, False, U=3.0, mu=0.4, form=0)
    W = ompo.hubbard_mpo(m)
    st = tt.run(W, 0.01, 0.05, 0.51, tt.TruncOpts(16), pad_full=True)
    ob = tt.measure(st)
    ed = om.ed_thermo(m, [st.beta], beta0=0.01)[0]
    assert _rel(ob["lnZ"], ed["lnZ"]) > 1e-3
    monkeypatch.setattr(tt, "tdvp1_step", real)


def test_planted_wrong_bond_sign_is_caught(monkeypatch):
    """The backward bond step exp(+tau H0) taken forward breaks exactness."""
    real = tt._bond_exp

    def broken(st, k, S, t, K):
        return real(st, k, S, -t, K)

    monkeypatch.setattr(tt, "_bond_exp", broken)
    m = om.Model(1, 3, False, U=3.0, mu=0.4, form=0)
    W = ompo.hubbard_mpo(m)
    st = tt.run(W, 0.01, 0.05, 0.51, tt.TruncOpts(16), pad_full=True)
    ob = tt.measure(st)
    ed = om.ed_thermo(m, [st.beta], beta0=0.01)[0]
    assert _rel(ob["energy_per_site"], ed["energy_per_site"]) > 1e-4


def test_full_rank_two_site_growth_is_exact():
    """2-TDVP steps on the padded state (nothing truncated) are exact as well."""
    m = om.Model(1, 3, False, U=3.0, mu=0.4, form=0)
    st = tt.pad_to_full_rank(tt.init_state(ompo.hubbard_mpo(m), 0.01))
    for _ in range(3):
        tt.tdvp2_step(st, 0.05, tt.TruncOpts(16, svd_cut=0.0))
    for _ in range(3):
        tt.tdvp1_step(st, 0.05)
    ob = tt.measure(st)
    ed = om.ed_thermo(m, [st.beta], beta0=0.01)[0]
    for k in KEYS:
        assert _rel(ob[k], ed[k]) < 1e-10, (k, ob[k], ed[k])


def test_two_site_growth_on_exponential_grid_is_exact():
    """2-TDVP steps along beta_n = 2^(n/4) beta_0 (Fig. S7(b) grids) on the
    padded state: exact at full rank like the linear grid."""
    m = om.Model(1, 3, False, U=3.0, mu=0.4, form=0)
    st = tt.pad_to_full_rank(tt.init_state(ompo.hubbard_mpo(m), 0.01))
    r = 2.0 ** 0.25
    betas = []
    while st.beta < 0.3 - 1e-12:
        tt.tdvp2_step(st, min(st.beta * (r - 1.0), 0.3 - st.beta), tt.TruncOpts(16, svd_cut=0.0))
        betas.append(st.beta)
    assert len(betas) == math.ceil(math.log(0.3 / 0.01) / math.log(r))
    ob = tt.measure(st)
    ed = om.ed_thermo(m, [st.beta], beta0=0.01)[0]
    for k in KEYS:
        assert _rel(ob[k], ed[k]) < 1e-10, (k, ob[k], ed[k])


def test_run_follows_the_exponential_growth_grid():
    """run(grow_ratio=r): growth steps beta -> r beta, the last one ending at
    grow_until, then linear steps of dtau."""
    m = om.Model(2, 2, False, U=4.0, mu=0.0, form=1)
    rec = []
    r = 2.0 ** 0.5
    tt.run(ompo.hubbard_mpo(m), 0.01, 0.05, 0.25, tt.TruncOpts(8), grow_until=0.15, grow_ratio=r,
           callback=lambda st, stage: rec.append((st.beta, stage)))
    grow = [b for b, s in rec if s == "grow"]
    lin = [b for b, s in rec if s == "tdvp1"]
    want, b = [], 0.01
    while b < 0.15 - 1e-12:
        b = min(b * r, 0.15)
        want.append(b)
    assert np.allclose(grow, want, rtol=0, atol=1e-14)
    assert np.allclose(np.diff([grow[-1]] + lin), 0.05, rtol=0, atol=1e-14)


def test_compact_initial_state():
    """The compact rho_0 has the operator Schmidt ranks of I - beta0 H/2:
    2 + 4 x (distinct left ends of hopping bonds crossing the cut), minus
    dependencies (the last cut of the 2x2 cluster sees one right site)."""
    m = om.Model(2, 2, False, U=4.0, mu=0.0, form=1)
    st = tt.init_state(ompo.hubbard_mpo(m), 0.01)
    assert st.bond_dims() == [6, 10, 6]
    padded = tt.pad_to_full_rank(tt.init_state(ompo.hubbard_mpo(m), 0.01))
    assert padded.bond_dims() == [16, 256, 16]
    assert abs(tt.measure(padded)["lnZ"] - tt.measure(st)["lnZ"]) < 1e-12


def test_initial_state_is_first_order_expansion():
    """rho_h(beta0) = I - beta0 H / 2: ln Z and E at beta0 from the dense matrix."""
    m = om.Model(2, 2, False, U=4.0, mu=0.3, form=0)
    H = om.dense_hamiltonian(m).toarray()
    b0 = 0.02
    rho = np.eye(len(H)) - 0.5 * b0 * H
    st = tt.init_state(ompo.hubbard_mpo(m), b0)
    ob = tt.measure(st)
    Z = np.sum(rho * rho)
    assert abs(ob["lnZ"] - math.log(Z)) < 1e-12
    assert abs(ob["energy_per_site"] - np.trace(rho @ H @ rho) / Z / m.N) < 1e-12
    # right canonical form: sum_s A^s A^s^T = 1 on every site but the first
    for A in st.A[1:]:
        Dl = A.shape[0]
        M = A.reshape(Dl, -1)
        assert np.allclose(M @ M.T, np.eye(Dl), atol=1e-12)


def test_lanczos_full_krylov_is_exact():
    """K = dim: the Lanczos exponential equals the matrix exponential."""
    rng = np.random.default_rng(7)
    n = 12
    X = rng.standard_normal((n, n))
    H = 0.5 * (X + X.T)
    v = rng.standard_normal(n)
    for t in (-0.3, 0.2):
        y, _ = tt.lanczos_expm(lambda x: H @ x, v, t, n)
        ref = scipy.linalg.expm(t * H) @ v
        assert np.abs(y - ref).max() < 1e-11 * np.abs(ref).max()


def test_lanczos_truncated_krylov_error_and_estimate():
    """Fixed K < dim: error shrinks fast with K and the a-posteriori estimate
    bounds it within an order of magnitude."""
    rng = np.random.default_rng(3)
    n = 200
    X = rng.standard_normal((n, n)) / math.sqrt(n)
    H = X + X.T
    v = rng.standard_normal(n)
    t = -0.1
    ref = scipy.linalg.expm(t * H) @ v
    errs = []
    for K in (4, 6, 8):
        y, est = tt.lanczos_expm(lambda x: H @ x, v, t, K)
        err = np.linalg.norm(y - ref)
        errs.append(err)
        assert err < 10 * est + 1e-14
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-9 * np.linalg.norm(v)


def test_lanczos_breakdown_on_eigenvector():
    """An eigenvector spans an invariant subspace: exp(tH) v = exp(t lambda) v."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((20, 20))
    H = X + X.T
    lam, V = np.linalg.eigh(H)
    v = 3.0 * V[:, 5]
    y, _ = tt.lanczos_expm(lambda x: H @ x, v, -0.2, 8)
    assert np.abs(y - math.exp(-0.2 * lam[5]) * v).max() < 1e-12


def test_qr_and_lq_gauges():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 4, 4, 7))
    Al, S = tt.qr_left(A)
    M = Al.reshape(-1, Al.shape[3])
    assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)
    assert np.allclose(np.tensordot(Al, S, axes=([3], [0])), A, atol=1e-13)
    assert np.all(np.diag(S) >= 0)
    Ar, S2 = tt.lq_right(A)
    M = Ar.reshape(Ar.shape[0], -1)
    assert np.allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-13)
    assert np.allclose(np.tensordot(S2, Ar, axes=([1], [0])), A, atol=1e-13)
    assert np.all(np.diag(S2) >= 0)


def test_truncation_rule():
    s = np.array([1.0, 0.5, 0.5, 0.25, 0.1, 1e-15])
    assert tt.truncation_rank(s, 10, 1e-14, 1e-10) == 5       # drop below svd_cut
    assert tt.truncation_rank(s, 2, 1e-14, 1e-10) == 1        # never split 0.5, 0.5
    assert tt.truncation_rank(s, 3, 1e-14, 1e-10) == 3
    s2 = np.array([0.7, 0.7, 0.7, 0.1])
    assert tt.truncation_rank(s2, 2, 1e-14, 1e-10) == 3       # leading group kept whole
    s3 = np.array([1.0, 1e-9, 1e-9 * (1 + 1e-7), 1e-12])
    assert tt.truncation_rank(s3, 2, 0.0, 1e-10) == 1         # absolute guard groups them
    s4 = np.array([1.0, 1e-6, 1e-6 * (1 - 1e-7), 1e-12])
    assert tt.truncation_rank(s4, 2, 0.0, 1e-10) == 2         # 1e-13 apart: not grouped


def test_free_fermion_ladder_error_decreases_with_D():
    """Fig. 1(c)-style benchmark at U=0: the free-energy error against the exact
    solution is small and shrinks as D grows."""
    m = om.Model(3, 2, False, U=0.0, mu=0.0, form=1)
    W = ompo.hubbard_mpo(m)
    exact = om.ed_thermo(m, [1.01], beta0=0.01)[0]
    errs = []
    for D in (8, 24):
        st = tt.run(W, 0.01, 0.05, 1.01, tt.TruncOpts(D))
        ob = tt.measure(st)
        errs.append(_rel(ob["free_energy_per_site"], exact["free_energy_per_site"]))
    assert errs[1] < 0.5 * errs[0] < 0.05


def test_thermodynamic_invariants_along_a_truncated_run():
    """Along a truncated run: dlnZ/dbeta = -E to O(dtau^2), E non-increasing,
    f non-decreasing (df/dT = -S <= 0)."""
    m = om.Model(3, 2, False, U=4.0, mu=0.5, form=1)
    W = ompo.hubbard_mpo(m)
    rec = []
    tt.run(W, 0.01, 0.05, 0.81, tt.TruncOpts(16), callback=lambda st, _: rec.append(tt.measure(st)))
    E = np.array([r["energy_per_site"] for r in rec])
    f = np.array([r["free_energy_per_site"] for r in rec])
    lnZ = np.array([r["lnZ"] for r in rec])
    assert np.all(np.diff(E) < 1e-9)
    assert np.all(np.diff(f) > -1e-9)
    dlnz = (lnZ[2:] - lnZ[:-2]) / (2 * 0.05)
    assert np.abs(-dlnz / m.N - E[1:-1]).max() < 2e-3


def _dense_operator(st):
    """Contract the super-MPS to rho[(s_1..s_N), (s'_1..s'_N)] (small N only)."""
    T = np.ones((1, 1, 1))  # (ket configs, bra configs, bond)
    for A in st.A:
        T = np.einsum("kbl,lsxr->ksbxr", T, A).reshape(T.shape[0] * 4, T.shape[1] * 4, A.shape[3])
    return T[:, :, 0]


def test_charges_conserved_and_rho_symmetric():
    """rho_h commutes with N and S^z (no weight between ket and bra of different
    charge, beyond rounding) on the 2x2 cluster truncated to D = 12 and at full
    rank, and is symmetric (H real) at full rank; the MPO-overlap hermiticity
    monitor equals the dense operator's asymmetry."""
    m = om.Model(2, 2, False, U=4.0, mu=0.3, form=1)
    n_loc, s_loc = np.array([0, 1, 1, 2]), np.array([0, 1, -1, 0])
    conf = np.array(np.unravel_index(np.arange(4 ** m.N), (4,) * m.N)).T
    n, s = n_loc[conf].sum(1), s_loc[conf].sum(1)
    off = (n[:, None] != n[None, :]) | (s[:, None] != s[None, :])
    asyms = []
    for D, pad in ((12, False), (40, False), (256, True)):
        st = tt.run(ompo.hubbard_mpo(m), 0.01, 0.05, 0.51, tt.TruncOpts(D), pad_full=pad)
        rho = _dense_operator(st) * math.exp(st.logscale)
        if D != 40:
            assert np.sum(rho[off] ** 2) / np.sum(rho * rho) < 1e-26, D
        asym = np.linalg.norm(rho - rho.T) / np.linalg.norm(rho)
        assert abs(tt.hermiticity_defect(st) - asym) < 1e-7
        asyms.append(asym)
    # under truncation the asymmetry is a monitored number (here below 1e-2),
    # at full rank it is rounding only.  (At D = 40 the dense SVD, which sees
    # no charges, cuts inside a nearly degenerate set of singular values of
    # different sectors and mixes them at ~1e-6 in norm; the block-sparse GPU
    # path conserves both charges by construction.)
    assert asyms[2] < 1e-12 and max(asyms[:2]) < 1e-2


def test_full_rank_state_is_symmetric():
    """At full rank rho_h = exp(-(beta-beta0) H/2)(I - beta0 H/2) is a function
    of the real symmetric H, so the hermiticity defect is rounding only."""
    m = om.Model(2, 2, False, U=4.0, mu=0.0, form=1)
    st = tt.run(ompo.hubbard_mpo(m), 0.01, 0.05, 0.31, tt.TruncOpts(256), pad_full=True)
    assert tt.hermiticity_defect(st) < 1e-6


def test_lnZ_convex_in_beta():
    """d^2 lnZ / dbeta^2 = Var H >= 0 along a truncated run."""
    m = om.Model(3, 2, False, U=4.0, mu=0.5, form=1)
    rec = []
    tt.run(ompo.hubbard_mpo(m), 0.01, 0.05, 0.81, tt.TruncOpts(16), callback=lambda st, _: rec.append(tt.measure(st)))
    lnZ = np.array([r["lnZ"] for r in rec])
    assert np.all(lnZ[2:] - 2 * lnZ[1:-1] + lnZ[:-2] > -1e-9)


def test_symmetric_sweep_is_second_order_in_dtau():
    """Lie-Trotter scaling at fixed D (Supplement, "Splitting method"; Fig. S7's
    delta F against tau): from one grown state, 1-TDVP to beta = 1 with dtau =
    0.2 ... 0.025; the free-energy error against dtau = 1/160 falls by ~4 per
    halving (the L->R + R->L composition is symmetric, so second order)."""
    import copy
    m = om.Model(3, 2, False, U=4.0, mu=0.3, form=1)
    st0 = tt.run(ompo.hubbard_mpo(m), 0.01, 0.05, 0.21, tt.TruncOpts(12), grow_until=0.21)
    f = {}
    for dt in (0.2, 0.1, 0.05, 0.025, 0.00625):
        st = copy.deepcopy(st0)
        for _ in range(int(round((1.01 - st.beta) / dt))):
            tt.tdvp1_step(st, dt)
        assert abs(st.beta - 1.01) < 1e-9
        f[dt] = tt.measure(st)["free_energy_per_site"]
    e = [abs(f[dt] - f[0.00625]) for dt in (0.2, 0.1, 0.05, 0.025)]
    slopes = [math.log2(e[i] / e[i + 1]) for i in range(3)]
    assert all(1.8 < s < 2.3 for s in slopes), slopes


def test_series_initial_state_order_one_is_the_first_order_state():
    """init_state_series(order=1) (dense, SVD cut) and init_state (from the
    MPO, compressed) are the same operator I - beta0 H/2: equal observables."""
    m = om.Model(2, 2, False, U=4.0, mu=-0.3, form=1)
    W = ompo.hubbard_mpo(m)
    a, b = tt.init_state(W, 0.05), tt.init_state_series(W, 0.05, 1)
    assert a.bond_dims() == b.bond_dims()
    oa, ob = tt.measure(a), tt.measure(b)
    for k in KEYS:
        assert _rel(oa[k], ob[k]) < 1e-13, (k, oa[k], ob[k])


def test_series_initial_state_evolves_exactly_at_full_rank():
    """Third-order series state padded to maximal bonds: 1-TDVP reproduces ED
    of exp(-(beta-beta0) H/2) sum_{k<=3} (-beta0 H/2)^k/k! (exactness on the
    whole space)."""
    m = om.Model(1, 3, False, U=3.0, mu=0.4, form=0)
    W = ompo.hubbard_mpo(m)
    st = tt.run(W, 0.05, 0.05, 0.46, tt.TruncOpts(16), pad_full=True, taylor_order=3)
    ob = tt.measure(st)
    ed = om.ed_thermo(m, [st.beta], beta0=0.05, order=3)[0]
    for k in KEYS:
        assert _rel(ob[k], ed[k]) < 1e-10, (k, ob[k], ed[k])
    ed1 = om.ed_thermo(m, [st.beta], beta0=0.05, order=1)[0]
    assert _rel(ed1["lnZ"], ed["lnZ"]) > 1e-6  # the order matters at this beta0


def test_series_initial_state_converges_to_the_gibbs_state():
    """ln Z of the order-n state at beta0 approaches the exact exp(-beta0 H)
    value; the error falls by about beta0 ||H|| per order (SETTN removes the
    expansion error, Fig. S7(a))."""
    m = om.Model(1, 3, False, U=4.0, mu=-0.3, form=1)
    W = ompo.hubbard_mpo(m)
    beta0 = 0.02
    exact = om.ed_thermo(m, [beta0], beta0=0.0)[0]["lnZ"]
    errs = []
    for order in (1, 2, 3, 4, 6):
        st = tt.init_state_series(W, beta0, order)
        errs.append(abs(tt.measure(st)["lnZ"] - exact))
        ed = om.ed_thermo(m, [beta0], beta0=beta0, order=order)[0]["lnZ"]
        assert abs(tt.measure(st)["lnZ"] - ed) < 1e-12 * abs(ed)
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1] and errs[3] < 0.2 * errs[2]
    assert errs[4] < 1e-12 * abs(exact)
