"""Oracle: the Hubbard MPO W as a finite automaton, dense tensors.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper writes H as an MPO (main text, "Benchmarks on noninteracting
fermions": rho_0 is built from "the MPO representation of the Hamiltonian")
and evolves with it (Supplement, Fig. "Lanczos": L, H_i, R).  It does not
print the construction; this is the textbook automaton for a 1D chain with
long-range terms produced by the snake mapping (Fig. 1(a)):

  state 0      "start": nothing placed yet (identity so far)
  state 1      "done":  a complete term was placed
  state 2+o*R+(m-1)  channel o at distance m (1 <= m <= R), i.e. the left
               operator of a hopping term sits m sites to the left; R is the
               longest 1D bond, so D_H = 2 + 4R (no per-bond compression).

Hopping c+_{i s} c_{j s} + c+_{j s} c_{i s} with i < j in 1D order becomes,
after the Jordan-Wigner transform, (c+_s F)_i F...F (c_s)_j +
(F c_s)_i F...F (c+_s)_j with F = (-1)^n, so the four channels are

  o = 0: left c+_up F,  right c_up        o = 2: left F c_up,  right c+_up
  o = 1: left c+_dn F,  right c_dn        o = 3: left F c_dn,  right c+_dn

Tensors are W[w, sigma, tau, w'] = <sigma| op_{w w'} |tau>; bond 0 keeps only
"start", bond N only "done".
"""
from __future__ import annotations

import numpy as np

from .model import Model, hopping_bonds


def local_operators() -> dict[str, np.ndarray]:
    """4x4 operators in the basis sigma = n_up + 2 n_dn (see ``oracle.model``)."""
    nu = np.diag([0.0, 1.0, 0.0, 1.0])
    nd = np.diag([0.0, 0.0, 1.0, 1.0])
    F_up = np.diag([1.0, -1.0, 1.0, -1.0])
    F = np.diag([1.0, -1.0, -1.0, 1.0])
    # bosonic lowering operators
    a_up = np.zeros((4, 4))
    a_up[0, 1] = 1.0  # |up>    -> |0>
    a_up[2, 3] = 1.0  # |up dn> -> |dn>
    a_dn = np.zeros((4, 4))
    a_dn[0, 2] = 1.0  # |dn>    -> |0>
    a_dn[1, 3] = 1.0  # |up dn> -> |up>
    c_up = a_up
    c_dn = F_up @ a_dn  # the down electron is passed over the up electron
    return dict(I=np.eye(4), nu=nu, nd=nd, F=F, c_up=c_up, c_dn=c_dn,
                cd_up=c_up.T.copy(), cd_dn=c_dn.T.copy())


def max_range(m: Model) -> int:
    """Largest 1D distance j - i over the hopping pairs (2W-1 for a snake
    cylinder with nearest-neighbour hopping)."""
    return max((j - i for i, j in hopping_bonds(m)), default=1)


def hubbard_mpo(m: Model) -> list[np.ndarray]:
    """Dense W_j[w, sigma, tau, w'] for j = 0..N-1 (Eq. 3 / PH form)."""
    op = local_operators()
    N = m.N
    R = max_range(m)
    nch = R
    DH = 2 + 4 * nch
    bonds = hopping_bonds(m)
    lefts = [op["cd_up"] @ op["F"], op["cd_dn"] @ op["F"], op["F"] @ op["c_up"], op["F"] @ op["c_dn"]]
    rights = [op["c_up"], op["c_dn"], op["cd_up"], op["cd_dn"]]
    if m.form == 0:
        onsite = m.U * op["nu"] @ op["nd"] - m.mu * (op["nu"] + op["nd"])
    else:
        onsite = m.U * (op["nu"] - 0.5 * op["I"]) @ (op["nd"] - 0.5 * op["I"]) - m.mu * (op["nu"] + op["nd"])

    def ch(o, dist):
        return 2 + o * nch + (dist - 1)

    Ws = []
    for j in range(N):
        W = np.zeros((DH, 4, 4, DH))
        W[0, :, :, 0] = op["I"]
        W[1, :, :, 1] = op["I"]
        W[0, :, :, 1] = onsite
        for o in range(4):
            W[0, :, :, ch(o, 1)] = lefts[o]
            for dist in range(1, nch + 1):
                if dist < nch:
                    W[ch(o, dist), :, :, ch(o, dist + 1)] = op["F"]
            for dist in range(1, nch + 1):
                # the term closes here when the left operator sat at j - dist
                if (j - dist, j) in bonds:
                    W[ch(o, dist), :, :, 1] = -bonds[(j - dist, j)] * rights[o]
        if j == 0:
            W = W[0:1]
        if j == N - 1:
            W = W[..., 1:2]
        Ws.append(W)
    return Ws


def mpo_to_dense(Ws: list[np.ndarray]) -> np.ndarray:
    """Contract the MPO into the full 4^N x 4^N matrix (site 0 most significant)."""
    M = Ws[0][0]  # (4, 4, D)
    M = M.reshape(4, 4, -1)
    for W in Ws[1:]:
        # M[(a), (b), w] x W[w, s, t, w'] -> [(a s), (b t), w']
        T = np.tensordot(M, W, axes=([2], [0]))  # (A, B, s, t, w')
        A, B = T.shape[0], T.shape[1]
        T = T.transpose(0, 2, 1, 3, 4).reshape(A * 4, B * 4, -1)
        M = T
    return M[:, :, 0]
