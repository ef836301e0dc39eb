"""Derived thermodynamics (post-processing of measurement series) against exact
diagonalisation: entropy, specific heat from the energy derivative and the
charge compressibility from two chemical potentials."""
import numpy as np

from oracle import model as om
from paper_2212_11973_gb300 import thermo


def _exact(m, betas):
    """S, C and the Gibbs averages from the full spectrum (beta0 = 0)."""
    blocks = om.ed_spectrum(m)
    E = np.concatenate([b[0] for b in blocks])
    S, C = [], []
    for beta in betas:
        w = np.exp(-beta * (E - E.min()))
        Z = w.sum()
        e1, e2 = (w * E).sum() / Z, (w * E * E).sum() / Z
        lnZ = np.log(Z) - beta * E.min()
        S.append((beta * e1 + lnZ) / m.N)
        C.append(beta * beta * (e2 - e1 * e1) / m.N)
    return np.array(S), np.array(C)


def test_entropy_and_specific_heat_match_ed():
    m = om.Model(2, 2, False, U=4.0, mu=0.3, form=1)
    betas = np.linspace(0.5, 2.0, 61)
    obs = om.ed_thermo(m, betas)
    S, C = _exact(m, betas)
    assert np.abs(thermo.entropy_per_site(obs) - S).max() < 1e-12
    b, c = thermo.specific_heat_per_site(obs)
    assert np.abs(c[1:-1] - C[1:-1]).max() < 2e-3 * np.abs(C).max()


def test_entropy_tends_to_ln4_at_high_temperature():
    m = om.Model(2, 2, False, U=4.0, mu=0.0, form=1)
    S = thermo.entropy_per_site(om.ed_thermo(m, [1e-4]))
    assert abs(S[0] - np.log(4.0)) < 1e-3


def test_compressibility_matches_density_derivative():
    m0 = om.Model(2, 2, False, U=4.0, mu=0.3 - 5e-5, form=1)
    m1 = om.Model(2, 2, False, U=4.0, mu=0.3 + 5e-5, form=1)
    betas = [0.5, 1.0, 2.0]
    b, chi = thermo.compressibility(om.ed_thermo(m0, betas), om.ed_thermo(m1, betas), 1e-4)
    # dn/dmu = beta (<N^2> - <N>^2) / N at fixed beta
    m = om.Model(2, 2, False, U=4.0, mu=0.3, form=1)
    nq, _, _ = om.basis_quantum_numbers(m.N)
    blocks = om.ed_spectrum(m)  # (N, Sz) blocks: every eigenstate has a definite N
    ev = np.concatenate([E for E, _, _ in blocks])
    Nn = np.concatenate([np.full(len(E), nq[idx[0]]) for E, _, idx in blocks]).astype(float)
    for beta, c in zip(b, chi):
        w = np.exp(-beta * (ev - ev.min()))
        w /= w.sum()
        exact = beta * ((w * Nn * Nn).sum() - (w * Nn).sum() ** 2) / m.N
        assert abs(c - exact) < 1e-5 * max(1.0, abs(exact))
