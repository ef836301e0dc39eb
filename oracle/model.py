"""Oracle: lattice, dense Hubbard Hamiltonian, exact diagonalisation, U=0 forms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions fixed here and restated independently by the GPU library:

* Snake order (Fig. 1(a) and its caption): site (x, y) of a W-wide lattice has
  1D index x*W + y for even x and x*W + (W-1-y) for odd x.
* Local basis sigma = n_up + 2*n_dn, i.e. {|0>, |up>, |dn>, |up dn>}, with
  |up dn> = c+_up c+_dn |0> (up before down inside a site).
* Jordan-Wigner modes are ordered site-major, up before down.

The dense Hamiltonian is built from 2N fermionic modes (a route that never
forms a site-level parity string), then permuted to the site basis, so that
it checks the automaton MPO of ``oracle.mpo`` independently.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass(frozen=True)
class Model:
    """Hubbard model on a cylinder/ladder (Eq. 3; PH form from the DQMC appendix).

    form 0: H = -t sum (c+c + h.c.) + U sum n_up n_dn - mu sum n          (Eq. 3)
    form 1: H = -t sum (c+c + h.c.) + U sum (n_up-1/2)(n_dn-1/2) - mu sum n
    tp: next-nearest (diagonal) hopping -t' of the t-t' model (Supplement,
    t-t'-U model), 0 for Eq. 3.
    """
    Lx: int
    Wy: int
    periodic_y: bool
    t: float = 1.0
    U: float = 0.0
    mu: float = 0.0
    form: int = 1
    tp: float = 0.0

    @property
    def N(self) -> int:
        return self.Lx * self.Wy


def snake_index(x: int, y: int, W: int) -> int:
    """1D position of lattice site (x, y) along the snake path of Fig. 1(a)."""
    return x * W + (y if x % 2 == 0 else W - 1 - y)


def lattice_bonds(m: Model) -> list[tuple[int, int]]:
    """Nearest-neighbour bonds (i < j in 1D order) of the CL / ladder lattice.

    Open in x; periodic in y for a cylinder (the paper's CL W x L).  A width-2
    "periodic" lattice would double the rung, so y wraps only when Wy > 2.
    """
    out = set()
    for x in range(m.Lx):
        for y in range(m.Wy):
            i = snake_index(x, y, m.Wy)
            nbrs = []
            if x + 1 < m.Lx:
                nbrs.append(snake_index(x + 1, y, m.Wy))
            if y + 1 < m.Wy:
                nbrs.append(snake_index(x, y + 1, m.Wy))
            elif m.periodic_y and m.Wy > 2:
                nbrs.append(snake_index(x, 0, m.Wy))
            for j in nbrs:
                out.add((min(i, j), max(i, j)))
    return sorted(out)


def diagonal_bonds(m: Model) -> list[tuple[int, int]]:
    """Next-nearest (diagonal) pairs (x, y)-(x+1, y+-1) in 1D order; y wraps
    under the same rule as the nearest-neighbour bonds (only when Wy > 2)."""
    out = set()
    for x in range(m.Lx - 1):
        for y in range(m.Wy):
            for dy in (1, -1):
                yy = y + dy
                if not 0 <= yy < m.Wy:
                    if not (m.periodic_y and m.Wy > 2):
                        continue
                    yy %= m.Wy
                i, j = snake_index(x, y, m.Wy), snake_index(x + 1, yy, m.Wy)
                out.add((min(i, j), max(i, j)))
    return sorted(out)


def hopping_bonds(m: Model) -> dict[tuple[int, int], float]:
    """Hopping amplitude of every pair (i < j): t on nearest neighbours, t' on
    the diagonals when t' != 0 (H contains -amp (c+_i c_j + h.c.))."""
    amp = {b: m.t for b in lattice_bonds(m)}
    if m.tp != 0.0:
        for b in diagonal_bonds(m):
            amp[b] = amp.get(b, 0.0) + m.tp
    return amp


def hopping_matrix(m: Model) -> np.ndarray:
    """Single-particle matrix of the kinetic term (no chemical potential)."""
    h = np.zeros((m.N, m.N))
    for (i, j), a in hopping_bonds(m).items():
        h[i, j] -= a
        h[j, i] -= a
    return h


# ----------------------------------------------------------------------------
# Dense second-quantised Hamiltonian (mode-level Jordan-Wigner)
# ----------------------------------------------------------------------------

def _mode_annihilators(n_modes: int) -> list[sp.csr_matrix]:
    """c_k = Z x ... x Z x b x 1 x ... x 1, mode 0 the most significant digit."""
    b = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |1> -> |0>
    z = sp.csr_matrix(np.diag([1.0, -1.0]))
    one = sp.identity(2, format="csr")
    ops = []
    for k in range(n_modes):
        mat = sp.identity(1, format="csr")
        for l in range(n_modes):
            f = z if l < k else (b if l == k else one)
            mat = sp.kron(mat, f, format="csr")
        ops.append(mat)
    return ops


def _site_basis_permutation(N: int) -> np.ndarray:
    """perm[s] = mode-basis index of site-basis state s.

    Mode basis: site j contributes digit 2*n_up + n_dn (up mode first).
    Site basis: site j contributes digit sigma = n_up + 2*n_dn.
    Site 0 is the most significant digit in both.
    """
    dim = 4 ** N
    s = np.arange(dim)
    out = np.zeros(dim, dtype=np.int64)
    for j in range(N):
        sig = (s // 4 ** (N - 1 - j)) % 4
        n_up, n_dn = sig % 2, sig // 2
        out += (2 * n_up + n_dn) * 4 ** (N - 1 - j)
    return out


def dense_hamiltonian(m: Model) -> sp.csr_matrix:
    """H of Eq. 3 (form 0) or its PH-symmetric form (form 1) in the site basis."""
    N = m.N
    c = _mode_annihilators(2 * N)
    cd = [x.T.tocsr() for x in c]
    num = [cd[k] @ c[k] for k in range(2 * N)]
    dim = 4 ** N
    H = sp.csr_matrix((dim, dim))
    for (i, j), amp in hopping_bonds(m).items():
        for s in range(2):
            a, b = 2 * i + s, 2 * j + s
            H = H - amp * (cd[a] @ c[b] + cd[b] @ c[a])
    eye = sp.identity(dim, format="csr")
    for i in range(N):
        nu, nd = num[2 * i], num[2 * i + 1]
        if m.form == 0:
            H = H + m.U * (nu @ nd)
        else:
            H = H + m.U * ((nu - 0.5 * eye) @ (nd - 0.5 * eye))
        H = H - m.mu * (nu + nd)
    perm = _site_basis_permutation(N)
    return H[perm][:, perm].tocsr()


def basis_quantum_numbers(N: int) -> tuple[np.ndarray, np.ndarray, list[np.ndarray]]:
    """Total particle number, 2*Sz and per-site (n_up, n_dn) for every site-basis state."""
    dim = 4 ** N
    s = np.arange(dim)
    ntot = np.zeros(dim, dtype=np.int64)
    sz2 = np.zeros(dim, dtype=np.int64)
    occ = []
    for j in range(N):
        sig = (s // 4 ** (N - 1 - j)) % 4
        nu, nd = sig % 2, sig // 2
        ntot += nu + nd
        sz2 += nu - nd
        occ.append(np.stack([nu, nd]))
    return ntot, sz2, occ


# ----------------------------------------------------------------------------
# Exact diagonalisation thermodynamics
# ----------------------------------------------------------------------------

def ed_spectrum(m: Model):
    """Eigenpairs of H block by block in (N, 2Sz); returns list of (E, V, idx)."""
    H = dense_hamiltonian(m)
    ntot, sz2, _ = basis_quantum_numbers(m.N)
    blocks = []
    for n in np.unique(ntot):
        for s in np.unique(sz2[ntot == n]):
            idx = np.nonzero((ntot == n) & (sz2 == s))[0]
            Hb = H[idx][:, idx].toarray()
            E, V = np.linalg.eigh(Hb)
            blocks.append((E, V, idx))
    return blocks


def ed_thermo(m: Model, betas, beta0: float = 0.0, blocks=None, order: int = 1) -> list[dict]:
    """Exact thermodynamics of rho_h = exp(-(beta-beta0) H/2) (I - beta0 H/2)
    (order = 1), or with the initial state sum_{k <= order} (-beta0 H/2)^k / k!
    (the series-expansion initialisation, Supplement "Error analysis").

    With beta0 = 0 this is the Gibbs state (rho = rho_h rho_h^T = exp(-beta H)).
    With beta0 > 0 it is the exact image of the first-order initial state
    rho_0 = 1 - tau_0 H (main text, "Benchmarks on noninteracting fermions")
    under the exact flow, which is what an untruncated tanTRG must reproduce
    (Supplement, Sec. "Splitting method": the splitting is exact on the
    tangent space).  Weights of eigenstate n: g_n^2 with
    g_n = exp(-(beta-beta0) E_n / 2) (1 - beta0 E_n / 2).
    """
    if blocks is None:
        blocks = ed_spectrum(m)
    N = m.N
    _, _, occ = basis_quantum_numbers(N)
    E_all, dens_all, dbl_all = [], [], []
    for E, V, idx in blocks:
        P = V * V  # |<basis|n>|^2, columns are eigenstates
        n_b = np.zeros(len(idx))
        d_b = np.zeros(len(idx))
        for j in range(N):
            nu, nd = occ[j][0][idx], occ[j][1][idx]
            n_b += nu + nd
            d_b += nu * nd
        E_all.append(E)
        dens_all.append(P.T @ n_b)
        dbl_all.append(P.T @ d_b)
    E = np.concatenate(E_all)
    dn = np.concatenate(dens_all)
    db = np.concatenate(dbl_all)
    out = []
    for beta in np.atleast_1d(betas):
        g = np.zeros_like(E)
        term = np.ones_like(E)
        for k in range(order + 1):
            if k:
                term = term * (-beta0 * E / 2.0) / k
            g = g + term
        logw = -(beta - beta0) * E + 2.0 * np.log(np.abs(g))
        mx = logw.max()
        w = np.exp(logw - mx)
        Zr = w.sum()
        lnZ = mx + math.log(Zr)
        out.append(dict(beta=float(beta), lnZ=lnZ,
                        energy_per_site=float((w * E).sum() / Zr / N),
                        density=float((w * dn).sum() / Zr / N),
                        double_occ=float((w * db).sum() / Zr / N),
                        free_energy_per_site=(-lnZ / (beta * N)) if beta > 0 else float("nan")))
    return out


def free_fermion_thermo(m: Model, betas) -> list[dict]:
    """U = 0 closed forms (Fig. 1(c) benchmark): both spin species independent.

    With single-particle energies e_k and modes phi_k of the hopping matrix,
    occupation f_k = 1/(exp(beta (e_k - mu)) + 1):
      ln Z = 2 sum_k ln(1 + exp(-beta (e_k - mu)))
      E    = 2 sum_k (e_k - mu) f_k
      n    = (2/N) sum_k f_k
      D_n  = (1/N) sum_i (sum_k |phi_k(i)|^2 f_k)^2      (Wick, spins independent)
    At U = 0 the PH-symmetric form adds nothing, so mu enters identically.
    """
    assert m.U == 0.0
    e, phi = np.linalg.eigh(hopping_matrix(m))
    x = e - m.mu
    N = m.N
    out = []
    for beta in np.atleast_1d(betas):
        f = 0.5 * (1.0 - np.tanh(0.5 * beta * x))  # = 1/(exp(beta x)+1), overflow-safe
        lnZ = 2.0 * np.sum(np.logaddexp(0.0, -beta * x))
        nloc = (phi * phi) @ f
        out.append(dict(beta=float(beta), lnZ=float(lnZ),
                        energy_per_site=float(2.0 * np.sum(x * f) / N),
                        density=float(2.0 * np.sum(f) / N),
                        double_occ=float(np.sum(nloc ** 2) / N),
                        free_energy_per_site=float(-lnZ / (beta * N)) if beta > 0 else float("nan")))
    return out
