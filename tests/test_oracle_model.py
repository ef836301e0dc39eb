"""Pins of the oracle's model layer against facts fixed by the physics.

Each test checks the oracle against something other than itself: an
independently built operator, a closed form, a limit, or a derivative
identity.  Two tests plant a mistake in the oracle (on the CPU) and check
that the pin catches it.
"""
import math

import numpy as np
import pytest

from oracle import model as om
from oracle import mpo as ompo


GEOMS = [
    om.Model(2, 2, False, U=4.0, mu=0.3, form=1),
    om.Model(2, 2, False, U=4.0, mu=0.3, form=0),
    om.Model(3, 2, False, U=2.0, mu=-0.5, form=1),
    om.Model(1, 3, True, U=1.0, mu=0.1, form=0),
    om.Model(2, 3, True, U=3.0, mu=0.2, form=1),
    om.Model(3, 2, False, U=2.0, mu=-0.5, form=1, tp=-0.3),   # t-t' model
    om.Model(2, 3, True, U=3.0, mu=0.2, form=0, tp=0.25),
]


def test_snake_order_is_a_path():
    """Fig. 1(a): consecutive 1D indices are lattice neighbours (the bold path)."""
    for W in (2, 3, 4, 6):
        for L in (2, 3, 5):
            m = om.Model(L, W, W > 2)
            bonds = set(om.lattice_bonds(m))
            for i in range(m.N - 1):
                assert (i, i + 1) in bonds
            # the index is a bijection
            idx = sorted(om.snake_index(x, y, W) for x in range(L) for y in range(W))
            assert idx == list(range(L * W))


def test_bond_counts_and_range():
    """CL W x L has (L-1) W + L W bonds (periodic y, W > 2); range 2W-1."""
    for W, L in ((4, 8), (6, 12), (3, 3)):
        m = om.Model(L, W, True)
        assert len(om.lattice_bonds(m)) == (L - 1) * W + L * W
        assert ompo.max_range(m) == 2 * W - 1
    lad = om.Model(8, 2, False)
    assert len(om.lattice_bonds(lad)) == 7 * 2 + 8
    assert ompo.max_range(lad) == 3


@pytest.mark.parametrize("m", GEOMS)
def test_mpo_equals_second_quantised_H(m):
    """The automaton MPO contracts to the mode-level Jordan-Wigner H (Eq. 3)."""
    H = om.dense_hamiltonian(m).toarray()
    Hm = ompo.mpo_to_dense(ompo.hubbard_mpo(m))
    assert np.abs(H - H.T).max() == 0.0
    assert np.abs(H - Hm).max() < 1e-13


def test_planted_missing_jw_sign_is_caught(monkeypatch):
    """Dropping the on-site parity in c_dn must break the MPO/H equality."""
    real = ompo.local_operators

    def broken():
        op = real()
        a_dn = np.zeros((4, 4))
        a_dn[0, 2] = 1.0
        a_dn[1, 3] = 1.0
        op["c_dn"] = a_dn
        op["cd_dn"] = a_dn.T.copy()
        return op

    monkeypatch.setattr(ompo, "local_operators", broken)
    m = om.Model(2, 2, False, U=1.0)
    H = om.dense_hamiltonian(m).toarray()
    Hm = ompo.mpo_to_dense(ompo.hubbard_mpo(m))
    assert np.abs(H - Hm).max() > 0.5


def test_planted_wrong_string_operator_is_caught(monkeypatch):
    """Using F_up instead of F on the passed-over sites must break equality."""
    real = ompo.local_operators

    def broken():
        op = real()
        op["F"] = np.diag([1.0, -1.0, 1.0, -1.0])
        return op

    monkeypatch.setattr(ompo, "local_operators", broken)
    m = om.Model(3, 2, False, U=0.0)
    H = om.dense_hamiltonian(m).toarray()
    Hm = ompo.mpo_to_dense(ompo.hubbard_mpo(m))
    assert np.abs(H - Hm).max() > 0.5


@pytest.mark.parametrize("geom,tp", [((2, 2, False), 0.0), ((4, 2, False), 0.0), ((2, 3, True), 0.0),
                                     ((3, 2, False), -0.3)])
def test_ed_matches_free_fermion_closed_form(geom, tp):
    """U = 0: ED thermodynamics equal the single-particle closed forms (also
    with the t' diagonals, whose single-particle matrix is built separately)."""
    m = om.Model(*geom, U=0.0, mu=0.37, form=1, tp=tp)
    betas = [0.1, 1.0, 4.0]
    ed = om.ed_thermo(m, betas)
    ff = om.free_fermion_thermo(m, betas)
    for a, b in zip(ed, ff):
        for k in ("lnZ", "energy_per_site", "density", "double_occ"):
            assert abs(a[k] - b[k]) <= 1e-11 * max(1.0, abs(b[k])), (k, a[k], b[k])


def _onsite_values(m):
    """The on-site term on |0>, |up>, |dn>, |up dn> (Eq. 3 or PH form)."""
    if m.form == 0:
        return np.array([0.0, -m.mu, -m.mu, m.U - 2 * m.mu])
    return np.array([m.U / 4, -m.U / 4 - m.mu, -m.U / 4 - m.mu, m.U / 4 - 2 * m.mu])


@pytest.mark.parametrize("m", GEOMS[:3])
def test_high_temperature_series(m):
    """ln Z = N ln 4 - beta <H>_0 + beta^2 Var_0(H) / 2 + O(beta^3); the infinite-T
    moments follow from the four on-site values and <K^2>_0 = t^2 N_bonds."""
    v = _onsite_values(m)
    nb = len(om.lattice_bonds(m))
    mean = m.N * v.mean()
    var = m.t ** 2 * nb + m.N * v.var()
    beta = 1e-3
    lnZ = om.ed_thermo(m, [beta])[0]["lnZ"]
    series = m.N * math.log(4.0) - beta * mean + 0.5 * beta ** 2 * var
    assert abs(lnZ - series) < 1e-7
    # infinite temperature: S -> ln 4 per site, <n> = 1, <n_up n_dn> = 1/4
    r0 = om.ed_thermo(m, [1e-9])[0]
    assert abs(r0["lnZ"] / m.N - math.log(4.0)) < 1e-8
    assert abs(r0["density"] - 1.0) < 1e-7
    assert abs(r0["double_occ"] - 0.25) < 1e-7


def test_energy_is_minus_dlnZ_dbeta():
    m = om.Model(2, 2, False, U=4.0, mu=0.2, form=0)
    h = 1e-4
    for beta in (0.5, 2.0):
        a, c, b = om.ed_thermo(m, [beta - h, beta, beta + h])
        dlnz = (b["lnZ"] - a["lnZ"]) / (2 * h)
        assert abs(-dlnz / m.N - c["energy_per_site"]) < 1e-6


def test_half_filling_at_ph_symmetric_mu0():
    """PH-symmetric form, mu = 0, bipartite lattice: n = 1 at every beta."""
    m = om.Model(2, 2, False, U=4.0, mu=0.0, form=1)
    for r in om.ed_thermo(m, [0.3, 1.0, 5.0]):
        assert abs(r["density"] - 1.0) < 1e-12


def test_ed_first_order_initial_state_limit():
    """At beta = beta0 the weights reduce to (1 - beta0 E/2)^2, i.e.
    Z = Tr (I - beta0 H/2)^2 = 4^N - beta0 Tr H + beta0^2 Tr H^2 / 4."""
    m = om.Model(2, 2, False, U=4.0, mu=0.3, form=0)
    H = om.dense_hamiltonian(m).toarray()
    b0 = 0.01
    Z = np.trace(np.eye(len(H)) - b0 * H + 0.25 * b0 ** 2 * H @ H)
    r = om.ed_thermo(m, [b0], beta0=b0)[0]
    assert abs(r["lnZ"] - math.log(Z)) < 1e-12


def test_golden_ed_values_reproduce():
    """The committed ED fixture (written by tests/golden/make_golden.py) still holds."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "ed_2x2_U4.json")
    data = json.load(open(path))
    m = om.Model(**data["model"])
    rows = om.ed_thermo(m, [r["beta"] for r in data["rows"]], beta0=data["beta0"])
    for got, want in zip(rows, data["rows"]):
        for k in ("lnZ", "energy_per_site", "density", "double_occ"):
            assert abs(got[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k]))


def test_diagonal_bonds_of_a_cylinder():
    """t' pairs: 2 per (x, y) column pair on a periodic cylinder of width W > 2
    (W (Lx - 1) each way), fewer on open edges; none for one column."""
    assert len(om.diagonal_bonds(om.Model(4, 4, True))) == 2 * 4 * 3
    assert len(om.diagonal_bonds(om.Model(4, 2, False))) == 2 * 3
    assert len(om.diagonal_bonds(om.Model(1, 4, True))) == 0
    m = om.Model(3, 3, True, tp=0.5)
    h = om.hopping_matrix(m)
    for i, j in om.diagonal_bonds(m):
        assert h[i, j] == -0.5 and h[j, i] == -0.5
