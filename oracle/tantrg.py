"""Oracle: dense super-MPS tanTRG (1-TDVP linear stage, 2-TDVP growth stage).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Storage: the MPO rho_h is kept as its Choi super-MPS (Supplement, "Choi
transformation"): site tensors A[j] of shape (D_l, 4, 4, D_r) indexed
[a_l, sigma, sigma', a_r]; sigma is acted on by H, sigma' is a spectator
because the flow is generated by H (x) I.  rho_h = exp(logscale) * MPS.

Readings taken where the paper is silent:
* rho_h(beta) = rho_paper(beta/2) = exp(-beta H/2) (bilayer trick), so
  Z = <<rho_h|rho_h>> and E = <<rho_h|H x I|rho_h>> / Z.
* One beta-step of size dtau = a left-to-right plus a right-to-left half
  sweep, each evolving with tau = dtau/4 (rho_h -> exp(-2 tau H) rho_h =
  exp(-dtau H/2) rho_h); this is the symmetric composition of the
  Supplement's "Splitting method" section, with the main text's "4 tau = 1"
  for a unit beta-step.
* The sweep turn is literal: the last site of a half sweep is updated again
  as the first site of the next half sweep.
* Lanczos: fixed Krylov dimension K, classical Gram-Schmidt
  re-orthogonalisation applied twice, early stop only on breakdown.
* QR gauge: sign convention diag(R) >= 0.
* Growth truncation: keep at most D_max values, drop s <= svd_cut * s_max,
  never cut between s_k and s_{k+1} when s_k - s_{k+1} <= degen_tol * s_k +
  1e-14 * s_max (a degenerate group is kept or dropped whole).  svd_cut =
  1e-12 keeps the decision two orders above the rounding noise of the SVD.
* Norm tracking: after every exponential the centre tensor is normalised and
  ln(norm) is added to logscale.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .mpo import local_operators

BREAKDOWN_TOL = 1e-13
# Absolute guard of the degeneracy test, in units of the largest singular value:
# exactly degenerate pairs (spin flip) come out of any SVD split by a few ulps
# of s_max, which for small values exceeds a purely relative tolerance.
DEGEN_ABS = 1e-14


# ----------------------------------------------------------------------------
# Effective Hamiltonians and environments (Supplement, Figs. "optimalB" and
# "Lanczos": L_i . A_i first, then H_i, then R_i)
# ----------------------------------------------------------------------------

def heff_site(Lenv, W, Renv, x):
    """y = H^(1) x, y[a,s,s',a'] = sum L[a,w,b] W[w,s,t,w'] x[b,t,s',c] R[a',w',c]."""
    T1 = np.tensordot(Lenv, x, axes=([2], [0]))            # a, w, t, s', c
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 2]))        # a, s', c, s, w'
    y = np.tensordot(T2, Renv, axes=([2, 4], [2, 1]))      # a, s', s, a'
    return y.transpose(0, 2, 1, 3)


def heff_bond(Lenv, Renv, S):
    """y = H^(0) S, y[a,a'] = sum L[a,w,b] S[b,c] R[a',w,c] (Fig. optimalB(d))."""
    T = np.tensordot(Lenv, S, axes=([2], [0]))             # a, w, c
    return np.tensordot(T, Renv, axes=([1, 2], [1, 2]))    # a, a'


def heff_two(Lenv, W1, W2, Renv, C):
    """y = H^(2) C on a two-site tensor C[a, s1, s1', s2, s2', c]."""
    T1 = np.tensordot(Lenv, C, axes=([2], [0]))            # a, w, t1, s1', t2, s2', c
    T2 = np.tensordot(T1, W1, axes=([1, 2], [0, 2]))       # a, s1', t2, s2', c, s1, w1
    T3 = np.tensordot(T2, W2, axes=([6, 2], [0, 2]))       # a, s1', s2', c, s1, s2, w2
    y = np.tensordot(T3, Renv, axes=([3, 6], [2, 1]))      # a, s1', s2', s1, s2, a'
    return y.transpose(0, 3, 1, 4, 2, 5)


def left_env_update(Lenv, A, W):
    """L_{j+1}[a',w',b'] = sum A*[a,s,s',a'] L[a,w,b] W[w,s,t,w'] A[b,t,s',b']."""
    T1 = np.tensordot(Lenv, A, axes=([2], [0]))            # a, w, t, s', b'
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 2]))        # a, s', b', s, w'
    new = np.tensordot(A.conj(), T2, axes=([0, 1, 2], [0, 3, 1]))  # a', b', w'
    return new.transpose(0, 2, 1)


def right_env_update(Renv, A, W):
    """R_j[a,w,b] = sum A*[a,s,s',a'] W[w,s,t,w'] A[b,t,s',b'] R_{j+1}[a',w',b']."""
    T1 = np.tensordot(A, Renv, axes=([3], [2]))            # b, t, s', a', w'
    T2 = np.tensordot(W, T1, axes=([2, 3], [1, 4]))        # w, s, b, s', a'
    return np.tensordot(A.conj(), T2, axes=([1, 2, 3], [1, 3, 4]))  # a, w, b


# ----------------------------------------------------------------------------
# Lanczos exponential (Supplement, "Lanczos-based exponential method")
# ----------------------------------------------------------------------------

def lanczos_expm(apply, v, t, K):
    """exp(t H) v ~ ||v|| sum_i c_i q_i with c the first column of exp(t T).

    Returns (y, resid) with resid = ||v|| * beta_K * |c_K|, the usual
    a-posteriori size of the neglected Krylov direction.
    """
    nb = float(np.sqrt(np.vdot(v, v).real))
    if nb == 0.0:
        return v.copy(), 0.0
    Q = [v / nb]
    alpha, beta = [], []
    hscale = 0.0
    resid_b = 0.0
    for k in range(K):
        w = apply(Q[k])
        a = float(np.vdot(Q[k], w).real)
        w = w - a * Q[k]
        if k > 0:
            w = w - beta[k - 1] * Q[k - 1]
        for _ in range(2):  # classical Gram-Schmidt, twice
            h = [float(np.vdot(q, w).real) for q in Q]
            for q, hj in zip(Q, h):
                w = w - hj * q
        b = float(np.sqrt(np.vdot(w, w).real))
        alpha.append(a)
        hscale = max(hscale, abs(a) + b)
        if k == K - 1:
            resid_b = b
            break
        if b <= BREAKDOWN_TOL * hscale:
            break  # invariant subspace: the Krylov space is exact
        beta.append(b)
        Q.append(w / b)
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    theta, V = np.linalg.eigh(T)
    c = V @ (np.exp(t * theta) * V[0, :])
    y = nb * sum(ci * qi for ci, qi in zip(c, Q))
    return y, nb * resid_b * abs(c[-1])


# ----------------------------------------------------------------------------
# Gauge moves
# ----------------------------------------------------------------------------

def qr_signfixed(M):
    """Reduced QR M = Q R of an m x n matrix with the convention diag(R) >= 0
    (unique for full column rank)."""
    Q, R = np.linalg.qr(M)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], d[:, None] * R


def qr_left(A):
    """A = A^L S with A^L left-canonical (QR of the (D_l*16) x D_r matrix)."""
    Dl, _, _, Dr = A.shape
    Q, R = qr_signfixed(A.reshape(Dl * 16, Dr))
    return Q.reshape(Dl, 4, 4, Q.shape[1]), R


def lq_right(A):
    """A = S A^R with A^R right-canonical (QR of the transposed D_l x (16*D_r) matrix)."""
    Dl, _, _, Dr = A.shape
    Q, R = qr_signfixed(A.reshape(Dl, 16 * Dr).T)
    return Q.T.reshape(Q.shape[1], 4, 4, Dr), R.T


def truncation_rank(s, D_max, svd_cut, degen_tol):
    """Number of singular values kept by the growth-stage rule (s descending)."""
    if len(s) == 0 or s[0] <= 0.0:
        return 0
    k = int(min(D_max, np.count_nonzero(s > svd_cut * s[0])))
    if 0 < k < len(s):
        k0 = k
        tol_abs = DEGEN_ABS * s[0]
        while k > 0 and s[k - 1] - s[k] <= degen_tol * s[k - 1] + tol_abs:
            k -= 1
        if k == 0:  # the leading group itself is cut: keep the whole group
            k = k0
            while k < len(s) and s[k - 1] - s[k] <= degen_tol * s[k - 1] + tol_abs:
                k += 1
    return k


# ----------------------------------------------------------------------------
# State
# ----------------------------------------------------------------------------

@dataclass
class State:
    W: list
    A: list
    Lenv: list = field(default_factory=list)   # Lenv[k]: sites < k, bond k
    Renv: list = field(default_factory=list)   # Renv[k]: sites >= k, bond k
    logscale: float = 0.0
    beta: float = 0.0
    resid_max: float = 0.0

    @property
    def N(self):
        return len(self.A)

    def bond_dims(self):
        return [a.shape[3] for a in self.A[:-1]]


def _normalise(st: State, x):
    nu = float(np.sqrt(np.vdot(x, x).real))
    st.logscale += math.log(nu)
    return x / nu


def _right_canonicalise(st: State):
    for j in range(st.N - 1, 0, -1):
        Ar, S = lq_right(st.A[j])
        st.A[j] = Ar
        st.A[j - 1] = np.tensordot(st.A[j - 1], S, axes=([3], [0]))


def init_state(W: list, beta0: float, compress_cut: float = 1e-14) -> State:
    """rho_h(beta0) = I - beta0 H / 2 as an MPO built from the MPO of H (main
    text, "Benchmarks on noninteracting fermions": rho_0 = 1 - tau_0 H with a
    compact representation from the MPO of H, D = D_H), brought to its compact
    form and right-canonicalised (canonical centre at site 0).

    Compact form (a reading: the paper calls the representation compact but
    does not fix it): right-canonicalise by LQ, then one left-to-right SVD
    sweep that drops singular values s <= compress_cut * s_max of each bond,
    then right-canonicalise again.  The bond spaces are then the operator
    Schmidt spaces of rho_0, independent of how the MPO of H was written.
    """
    N = len(W)
    A = [w.copy() for w in W]
    last = -0.5 * beta0 * W[N - 1].copy()
    last[0, :, :, 0] += np.eye(4)  # the "start" row closed with the identity
    A[N - 1] = last
    st = State(W=W, A=A)
    _right_canonicalise(st)
    for j in range(N - 1):
        Dl, _, _, Dr = st.A[j].shape
        U, s, Vt = np.linalg.svd(st.A[j].reshape(Dl * 16, Dr), full_matrices=False)
        k = int(np.count_nonzero(s > compress_cut * s[0]))
        st.A[j] = U[:, :k].reshape(Dl, 4, 4, k)
        st.A[j + 1] = np.tensordot(s[:k, None] * Vt[:k], st.A[j + 1], axes=([1], [0]))
    _right_canonicalise(st)
    st.A[0] = _normalise(st, st.A[0])
    st.beta = beta0
    build_envs(st)
    return st


def init_state_series(W: list, beta0: float, order: int, compress_cut: float = 1e-14) -> State:
    """rho_h(beta0) = sum_{k <= order} (-beta0 H / 2)^k / k!, the series-
    expansion initial state (Supplement, "Error analysis of tanTRG": rho_0 =
    sum_n (-tau_0 H)^n / n! with the SETTN technique; here tau_0 = beta0 / 2
    because the MPO holds rho(beta/2)).  Built densely from the contracted MPO
    of H (small systems only: 4^N x 4^N), cut into the super-MPS by successive
    SVDs (singular values <= compress_cut * s_max dropped), then brought to the
    same compact right-canonical form as init_state."""
    from .mpo import mpo_to_dense
    N = len(W)
    H = mpo_to_dense(W)
    rho = np.eye(H.shape[0])
    term = np.eye(H.shape[0])
    for k in range(1, order + 1):
        term = term @ (-0.5 * beta0 * H) / k
        rho = rho + term
    # |rho>> with the pair (sigma_j, sigma'_j) per site, site 0 leftmost
    T = rho.reshape((4,) * (2 * N)).transpose([x for j in range(N) for x in (j, N + j)])
    A = []
    rest = T.reshape(1, -1)
    for j in range(N - 1):
        Dl = rest.shape[0]
        U, sv, Vt = np.linalg.svd(rest.reshape(Dl * 16, -1), full_matrices=False)
        k = int(np.count_nonzero(sv > compress_cut * sv[0]))
        A.append(U[:, :k].reshape(Dl, 4, 4, k))
        rest = sv[:k, None] * Vt[:k]
    A.append(rest.reshape(rest.shape[0], 4, 4, 1))
    st = State(W=W, A=A)
    _right_canonicalise(st)
    for j in range(N - 1):
        Dl, _, _, Dr = st.A[j].shape
        U, sv, Vt = np.linalg.svd(st.A[j].reshape(Dl * 16, Dr), full_matrices=False)
        k = int(np.count_nonzero(sv > compress_cut * sv[0]))
        st.A[j] = U[:, :k].reshape(Dl, 4, 4, k)
        st.A[j + 1] = np.tensordot(sv[:k, None] * Vt[:k], st.A[j + 1], axes=([1], [0]))
    _right_canonicalise(st)
    st.A[0] = _normalise(st, st.A[0])
    st.beta = beta0
    build_envs(st)
    return st


def pad_to_full_rank(st: State) -> State:
    """Embed the right-canonical state into bonds of the maximal dimension
    min(16^k, 16^(N-k)) by orthonormal completion (zero weight).  With every
    bond maximal the MPS manifold is the whole space, so 1-TDVP carries no
    projection error (Supplement, "Splitting method": exact on the tangent
    space); used to pin the integrator against exact diagonalisation."""
    N = st.N
    for j in range(N - 1, 0, -1):
        A = st.A[j]
        Dl, _, _, Dr = A.shape
        full = min(16 ** j, 16 ** (N - j))
        if Dl >= full:
            continue
        M = A.reshape(Dl, 16 * Dr)                  # orthonormal rows
        Qc, _ = np.linalg.qr(np.concatenate([M.T, np.eye(16 * Dr)], axis=1))
        P = Qc[:, :full].T                          # first Dl rows span M's rows
        sign = np.sign(np.sum(P[:Dl] * M, axis=1))
        P[:Dl] *= sign[:, None]
        st.A[j] = P.reshape(full, 4, 4, Dr)
        prev = st.A[j - 1]
        pad = np.zeros(prev.shape[:3] + (full - Dl,))
        st.A[j - 1] = np.concatenate([prev, pad], axis=3)
    build_envs(st)
    return st


def build_envs(st: State):
    N = st.N
    st.Lenv = [None] * (N + 1)
    st.Renv = [None] * (N + 1)
    st.Lenv[0] = np.ones((1, 1, 1))
    st.Renv[N] = np.ones((1, 1, 1))
    for j in range(N - 1, 0, -1):
        st.Renv[j] = right_env_update(st.Renv[j + 1], st.A[j], st.W[j])


# ----------------------------------------------------------------------------
# 1-TDVP: the one-site projector-splitting integrator of the tangent-space
# evolution (Supplement, "Procedure of 1-TDVP"): every site is evolved forward
# with its effective Hamiltonian, and between neighbouring sites the bond
# matrix of the gauge move is evolved backward with the zero-site one
# ----------------------------------------------------------------------------

def _site_exp(st: State, j: int, t: float, K: int):
    L, R, W = st.Lenv[j], st.Renv[j + 1], st.W[j]
    y, res = lanczos_expm(lambda x: heff_site(L, W, R, x), st.A[j], t, K)
    st.resid_max = max(st.resid_max, res)
    st.A[j] = _normalise(st, y)


def _bond_exp(st: State, k: int, S, t: float, K: int):
    L, R = st.Lenv[k], st.Renv[k]
    y, res = lanczos_expm(lambda x: heff_bond(L, R, x), S, t, K)
    st.resid_max = max(st.resid_max, res)
    return _normalise(st, y)


def tdvp1_sweep_lr(st: State, tau: float, K: int):
    N = st.N
    for j in range(N):
        _site_exp(st, j, -tau, K)                    # A_j <- exp(-tau H1) A_j
        if j == N - 1:
            break                                    # no bond update after site N
        Al, S = qr_left(st.A[j])                     # A_j = A_j^L S_j
        st.A[j] = Al
        st.Lenv[j + 1] = left_env_update(st.Lenv[j], Al, st.W[j])
        S = _bond_exp(st, j + 1, S, +tau, K)         # S_j <- exp(+tau H0) S_j
        st.A[j + 1] = np.tensordot(S, st.A[j + 1], axes=([1], [0]))


def tdvp1_sweep_rl(st: State, tau: float, K: int):
    N = st.N
    for j in range(N - 1, -1, -1):
        _site_exp(st, j, -tau, K)
        if j == 0:
            break
        Ar, S = lq_right(st.A[j])
        st.A[j] = Ar
        st.Renv[j] = right_env_update(st.Renv[j + 1], Ar, st.W[j])
        S = _bond_exp(st, j, S, +tau, K)
        st.A[j - 1] = np.tensordot(st.A[j - 1], S, axes=([3], [0]))


def tdvp1_step(st: State, dtau: float, K: int = 8):
    tau = dtau / 4.0
    tdvp1_sweep_lr(st, tau, K)
    tdvp1_sweep_rl(st, tau, K)
    st.beta += dtau


# ----------------------------------------------------------------------------
# 2-TDVP growth (Supplement, "2-TDVP in the initial stage": N-1 two-site
# updates and N-2 backward one-site updates per half sweep)
# ----------------------------------------------------------------------------

@dataclass
class TruncOpts:
    D_max: int
    svd_cut: float = 1e-12
    degen_tol: float = 1e-10


def _two_site_exp(st: State, j: int, t: float, K: int):
    C = np.tensordot(st.A[j], st.A[j + 1], axes=([3], [0]))  # a, s1, s1', s2, s2', c
    L, R, W1, W2 = st.Lenv[j], st.Renv[j + 2], st.W[j], st.W[j + 1]
    y, res = lanczos_expm(lambda x: heff_two(L, W1, W2, R, x), C, t, K)
    st.resid_max = max(st.resid_max, res)
    return _normalise(st, y)


def _split(C, opts: TruncOpts):
    Dl, Dr = C.shape[0], C.shape[5]
    U, s, Vt = np.linalg.svd(C.reshape(Dl * 16, 16 * Dr), full_matrices=False)
    k = truncation_rank(s, opts.D_max, opts.svd_cut, opts.degen_tol)
    return U[:, :k].reshape(Dl, 4, 4, k), s[:k], Vt[:k].reshape(k, 4, 4, Dr)


def tdvp2_sweep_lr(st: State, tau: float, K: int, opts: TruncOpts):
    N = st.N
    for j in range(N - 1):
        C = _two_site_exp(st, j, -tau, K)
        U, s, Vt = _split(C, opts)
        st.A[j] = U
        st.A[j + 1] = s[:, None, None, None] * Vt
        st.Lenv[j + 1] = left_env_update(st.Lenv[j], U, st.W[j])
        if j < N - 2:
            _site_exp(st, j + 1, +tau, K)            # backward one-site step


def tdvp2_sweep_rl(st: State, tau: float, K: int, opts: TruncOpts):
    for j in range(st.N - 2, -1, -1):
        C = _two_site_exp(st, j, -tau, K)
        U, s, Vt = _split(C, opts)
        st.A[j + 1] = Vt
        st.A[j] = U * s[None, None, None, :]
        st.Renv[j + 1] = right_env_update(st.Renv[j + 2], Vt, st.W[j + 1])
        if j > 0:
            _site_exp(st, j, +tau, K)


def tdvp2_step(st: State, dtau: float, opts: TruncOpts, K: int = 8):
    tau = dtau / 4.0
    tdvp2_sweep_lr(st, tau, K, opts)
    tdvp2_sweep_rl(st, tau, K, opts)
    st.beta += dtau


def bond_caps(N: int, D_max: int):
    """Largest useful dimension of bond k (1..N-1): min(D_max, 16^k, 16^(N-k))."""
    return [min(D_max, 16 ** min(k, N - k)) for k in range(1, N)]


def saturated(st: State, D_max: int) -> bool:
    return all(d == c for d, c in zip(st.bond_dims(), bond_caps(st.N, D_max)))


# ----------------------------------------------------------------------------
# Measurements (Supplement, Choi transformation: bilayer expectation values)
# ----------------------------------------------------------------------------

def measure(st: State) -> dict:
    """Full-network contractions, independent of the sweep's environments.

    lnZ = 2 logscale + ln <<psi|psi>>; eps = <<psi|H x I|psi>> / (N <<psi|psi>>);
    n and D_n are averages of local n and n_up n_dn acting on sigma.
    """
    N = st.N
    op = local_operators()
    n_op = op["nu"] + op["nd"]
    d_op = op["nu"] @ op["nd"]
    EL = [np.ones((1, 1))]
    for j in range(N):
        A = st.A[j]
        EL.append(np.einsum("ab,asxc,bsxd->cd", EL[j], A.conj(), A))
    ER = [None] * (N + 1)
    ER[N] = np.ones((1, 1))
    for j in range(N - 1, -1, -1):
        A = st.A[j]
        ER[j] = np.einsum("asxc,bsxd,cd->ab", A.conj(), A, ER[j + 1])
    nrm2 = float(EL[N][0, 0])
    dens = 0.0
    dbl = 0.0
    for j in range(N):
        A = st.A[j]
        for O, acc in ((n_op, "n"), (d_op, "d")):
            v = float(np.einsum("ab,asxc,st,btxd,cd->", EL[j], A.conj(), O, A, ER[j + 1]))
            if acc == "n":
                dens += v
            else:
                dbl += v
    L = np.ones((1, 1, 1))
    for j in range(N):
        L = left_env_update(L, st.A[j], st.W[j])
    eH = float(L[0, 0, 0])
    lnZ = 2.0 * st.logscale + math.log(nrm2)
    beta = st.beta
    return dict(beta=beta, lnZ=lnZ, energy_per_site=eH / nrm2 / N,
                density=dens / nrm2 / N, double_occ=dbl / nrm2 / N,
                free_energy_per_site=-lnZ / (beta * N),
                max_bond=max(st.bond_dims(), default=1), krylov_resid_max=st.resid_max)


def hermiticity_defect(st: State) -> float:
    """||rho_h - rho_h^T|| / ||rho_h|| from the overlaps <<rho|rho>> and <<rho|rho^T>>."""
    E1 = np.ones((1, 1))
    E2 = np.ones((1, 1))
    for A in st.A:
        E1 = np.einsum("ab,asxc,bsxd->cd", E1, A.conj(), A)
        E2 = np.einsum("ab,asxc,bxsd->cd", E2, A.conj(), A)
    n1, n2 = float(E1[0, 0]), float(E2[0, 0])
    return math.sqrt(max(2.0 * n1 - 2.0 * n2, 0.0) / n1)


# ----------------------------------------------------------------------------
# Driver
# ----------------------------------------------------------------------------

def run(W, beta0: float, dtau: float, beta_end: float, opts: TruncOpts, K: int = 8,
        grow_until: float = 1.0, callback=None, max_grow_steps=None, pad_full: bool = False,
        grow_ratio: float | None = None, taylor_order: int = 1):
    """Growth with 2-TDVP until every bond is saturated or beta >= grow_until,
    then 1-TDVP steps until beta >= beta_end (the hybrid scheme of the main
    text).  The growth grid is linear (steps of dtau) or, with grow_ratio,
    exponential: beta -> grow_ratio * beta per step, the last step ending at
    grow_until (main text, exponential grids for the two-site stage; Fig. S7
    caption: beta_n = 2^(n/m) beta_0).  ``callback(st, stage)`` runs after every
    step.  pad_full: start from the state padded to maximal bonds (no growth).
    taylor_order > 1: start from the series-expansion state (init_state_series)."""
    st = init_state(W, beta0) if taylor_order == 1 else init_state_series(W, beta0, taylor_order)
    if pad_full:
        pad_to_full_rank(st)
        max_grow_steps = 0
    n_grow = 0
    eps = 1e-12
    while st.beta < beta_end - eps:
        if saturated(st, opts.D_max) or st.beta >= grow_until - eps or (
                max_grow_steps is not None and n_grow >= max_grow_steps):
            break
        step = dtau if grow_ratio is None else min(st.beta * (grow_ratio - 1.0), grow_until - st.beta)
        tdvp2_step(st, step, opts, K)
        n_grow += 1
        if callback:
            callback(st, "grow")
    while st.beta < beta_end - eps:
        tdvp1_step(st, dtau, K)
        if callback:
            callback(st, "tdvp1")
    return st
