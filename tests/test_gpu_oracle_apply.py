"""GPU site H_eff apply against the oracle's dense definition, element-wise,
at sizes that reach the full-size kernel paths.

The library's kernel-level entry point tt_heff_apply_terms_host takes the MPO
tensor from the caller, so the test hands it the oracle's own W_j (the
uncompressed automaton of oracle/mpo.py) with channel charges derived from
W's nonzero pattern; L, R and x are seeded random block-sparse tensors in
the documented layouts.  The oracle contracts the dense forms with its
heff_site (the definition y = L W x R); the dense result must vanish outside
the charge-allowed blocks, and the GPU result must equal it block by block:

* FP64: 1e-12 of every right-sector group's largest |y| (rounding of sums of
  a few thousand products);
* split-BF16 x6: 2e-5 of the group's largest |y| (operands kept to ~2^-24,
  FP32 tensor-core accumulation folded every 128 K);
* exact-accumulation split: 1e-8 (digits to 2^-32 of each row / column bound
  per 32-wide K tile, exact tile sums).

Sizes: D = 256 with a narrow sector distribution (one sector of 172 states),
so GEMM blocks span several 128 x 128 tiles and K exceeds 128 (the TMEM fold
path); the CL4x8 MPO at its middle site (46 channels); and the CL6x12 MPO at
D = 1024 (the bench's sizes), where the oracle evaluates sampled output
fibres y[a, :, :, a'] one by one.
"""
import os
import sys

import numpy as np
import pytest

from paper_2212_11973_gb300 import workloads as wl

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import _layout as lay  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 2: 2e-5, 3: 1e-8}


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


def _oracle_mpo_site(Lx, Wy, per, U, mu, j):
    from oracle import model as om
    from oracle import mpo as ompo
    Ws = ompo.hubbard_mpo(om.Model(Lx, Wy, per, 1.0, U, mu, 1))
    return Ws[j], lay.mpo_channel_charges(Ws)


def _case(tt, Lx, Wy, per, j, D, width, seed):
    W, ch = _oracle_mpo_site(Lx, Wy, per, 8.0, wl.MU_EIGHTH_DOPING, j)
    SL = wl.gaussian_sectors(D, width, wl.SECTOR_CHARGES, seed)
    SR = wl.gaussian_sectors(D, width, wl.SECTOR_CHARGES, seed + 1)
    nx, nl, nr = tt.layout_sizes_terms(ch[j], ch[j + 1], SL, SR)
    L, R, x = (wl.random_vector(n, seed + k) for k, n in ((2, nl), (3, nr), (4, nx)))
    return W, ch[j], ch[j + 1], SL, SR, L, R, x


def _groupwise(y, y0, SL, SR):
    groups, total = lay.right_groups(SL, SR)
    assert total == y0.size
    worst = 0.0
    for off, rows, dr in groups:
        a, b = y[off:off + rows * dr], y0[off:off + rows * dr]
        s = np.abs(b).max()
        if s > 0:
            worst = max(worst, np.abs(a - b).max() / s)
    return worst


@pytest.mark.parametrize("geom", [(8, 2, False, 7), (8, 4, True, 15)])
def test_heff_apply_matches_oracle_definition(tt, geom):
    from oracle import tantrg as ot
    Lx, Wy, per, j = geom
    W, chl, chr_, SL, SR, L, R, x = _case(tt, Lx, Wy, per, j, 256, 0.6, 101 + j)
    assert max(d for _, _, d in SL) > 128 and max(d for _, _, d in SR) > 128
    Ld, Rd = lay.env_to_dense(L, SL, chl), lay.env_to_dense(R, SR, chr_)
    Y = ot.heff_site(Ld, W, Rd, lay.site_to_dense(x, SL, SR))
    y_or = lay.dense_to_site(Y, SL, SR)
    assert lay.outside_blocks_norm(Y, SL, SR) <= 1e-13 * np.linalg.norm(y_or)
    ctx = tt.Context()
    terms = lay.mpo_terms(W)
    for prec, tol in TOL.items():
        y = tt.heff_apply_terms_host(ctx, chl, chr_, terms, prec, SL, SR, L, R, x)
        err = _groupwise(y, y_or, SL, SR)
        print(f"{geom} precision {prec}: group-wise {err:.3e}")
        assert err < tol, (geom, prec, err)
    ctx.close()


def test_heff_apply_full_size_sampled_against_oracle(tt):
    """CL6x12 MPO, middle site, D = 1024 on both bonds (Gaussian sectors as in
    the kernel benchmark): 24 output fibres y[a, :, :, a'] (a, a' seeded) from
    the oracle's definition on the dense inputs, against the GPU apply."""
    from oracle import tantrg as ot
    W, chl, chr_, SL, SR, L, R, x = _case(tt, 12, 6, True, 36, 1024, 1.5, 2024)
    ctx = tt.Context()
    terms = lay.mpo_terms(W)
    ys = {p: tt.heff_apply_terms_host(ctx, chl, chr_, terms, p, SL, SR, L, R, x) for p in TOL}
    ctx.close()
    Ld, Rd, X = lay.env_to_dense(L, SL, chl), lay.env_to_dense(R, SR, chr_), lay.site_to_dense(x, SL, SR)
    Ys = {p: lay.site_to_dense(y, SL, SR) for p, y in ys.items()}
    rng = np.random.default_rng(7)
    D = X.shape[0]
    scale = np.abs(Ys[0]).max()
    for _ in range(24):
        a, ap = int(rng.integers(D)), int(rng.integers(D))
        fib = ot.heff_site(Ld[a:a + 1], W, Rd[ap:ap + 1], X)[0, :, :, 0]
        for p, tol in TOL.items():
            err = np.abs(Ys[p][a, :, :, ap] - fib).max() / scale
            assert err < tol, (p, a, ap, err)
