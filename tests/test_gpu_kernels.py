"""GPU kernel-level parity: one site H_eff apply on seeded random block-sparse
inputs (ladder MPO, Gaussian sector dimensions), split-BF16 paths against the
FP64 path of the same library call.  The FP64 apply itself is pinned to the
oracle by the sweep parity tests; here the tolerances are the split-BF16
error bounds: ~2^-16 relative for 2 levels, ~2^-24 times a small factor for 3
levels (the FP32 accumulation is folded into a two-float sum per K chunk, so
it does not grow with K)."""
import os
import sys

import numpy as np
import pytest

from paper_2212_11973_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

ALLOWED = wl.SECTOR_CHARGES


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


def _inputs(tt, mpo, site, D, seed):
    SL = wl.gaussian_sectors(D, 1.5, ALLOWED, seed)
    SR = wl.gaussian_sectors(D, 1.5, ALLOWED, seed + 1)
    nx, nl, nr = tt.layout_sizes(mpo, site, SL, SR)
    return SL, SR, wl.random_vector(nl, seed + 2), wl.random_vector(nr, seed + 3), wl.random_vector(nx, seed + 4)


def _groupwise_err(y, y0, SL, SR):
    """Largest |y - y0| of every right-sector group over that group's largest
    |y0| (the groups are the contiguous [rows x d_r] matrices of the layout)."""
    from _layout import right_groups
    groups, total = right_groups(SL, SR)
    assert total == y0.size
    worst = 0.0
    for off, rows, dr in groups:
        a, b = y[off:off + rows * dr], y0[off:off + rows * dr]
        scale = np.abs(b).max()
        if scale > 0:
            worst = max(worst, np.abs(a - b).max() / scale)
    return worst


@pytest.mark.parametrize("D", [24, 130, 300])
def test_heff_split_bf16_matches_fp64(tt, D):
    """Split-BF16 x3 / x6 and the exact-accumulation split against the FP64
    apply of the same call, element-wise per right-sector group.  Bounds: x3
    keeps ~2^-16 of every operand, x6 ~2^-24 with FP32 tensor-core
    accumulation (worst case ~gamma_K relative to sum |a_k b_k|, which for
    random-sign data stays a few times 2^-24 of the group's largest entry);
    the exact split keeps 32 bits of every row bound per GEMM segment and sums
    exactly: per product ~2^-32 max_row|a| max_col|b|, over K random-sign
    terms ~2^-32 sqrt(K) max|a| max|b| against ~sqrt(K) rms|a| rms|b| for the
    result, so (max / rms)^2 ~ 16 for Gaussian data times a few for the
    two-float intermediates: ~4e-9 relative."""
    ctx = tt.Context()
    mpo = tt.Mpo(ctx, 8, 2, False, t=1.0, U=4.0, mu=-0.3, form=1)
    SL, SR, L, R, x = _inputs(tt, mpo, 7, D, 11 * D)
    y0 = tt.heff_apply_host(ctx, mpo, 7, 0, SL, SR, L, R, x)
    assert np.isfinite(y0).all() and np.abs(y0).max() > 0
    for prec, tol_norm, tol_el in ((1, 3e-5, 3e-4), (2, 1e-6, 1e-5), (3, 5e-9, 1e-8)):
        y = tt.heff_apply_host(ctx, mpo, 7, prec, SL, SR, L, R, x)
        err = np.linalg.norm(y - y0) / np.linalg.norm(y0)
        el = _groupwise_err(y, y0, SL, SR)
        print(f"D={D} precision={prec}: normwise {err:.3e}, group-wise {el:.3e}")
        assert err < tol_norm, (D, prec, err)
        assert el < tol_el, (D, prec, el)
    mpo.close()
    ctx.close()


@pytest.mark.parametrize("m,n", [(1, 1), (40, 7), (300, 130), (2100, 200)])
def test_qr_gauge_matches_oracle(tt, m, n):
    """QR gauge kernel (FP64 Householder, diag(R) >= 0) against the oracle's QR."""
    import torch
    from oracle.tantrg import qr_signfixed
    ctx = tt.Context()
    A = wl.random_vector(m * n, 100 + m).reshape(m, n)
    Qo, Ro = qr_signfixed(A)
    Q, R = tt.qr_device(ctx, torch.from_numpy(A).cuda())
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    scale = np.abs(A).max()
    assert np.abs(Q - Qo).max() < 1e-12 * max(1.0, np.linalg.cond(A))
    assert np.abs(R - Ro).max() < 1e-12 * scale * max(1.0, np.linalg.cond(A))
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-13
    ctx.close()


def test_heff_full_size_mixed_vs_fp64(tt):
    """Bench sizes: CL6x12 MPO at the middle site, D = 1024 on both bonds.  The
    oracle cannot evaluate this apply, so the check is the property that holds
    at any size: the split-BF16 x6 apply (the timed configuration) agrees with
    the FP64 apply of the same call within the arithmetic's bound, and both are
    finite.  Bound: operands carried to ~2^-25 by three bf16 levels, six of the
    nine level products (dropped terms ~2^-25), FP32 tensor-core accumulation
    over 128-long K chunks folded into a two-float sum; the chunk sums dominate,
    worst case gamma_128 = 128 * 2^-24 ~ 7.6e-6 relative to sum |a_k b_k|, and
    with K ~ 3200 (42 channels) random-sign data stays well inside 5e-6 of
    ||y||."""
    ctx = tt.Context()
    mpo = tt.Mpo(ctx, 12, 6, True, t=1.0, U=8.0, mu=wl.MU_EIGHTH_DOPING, form=1)
    SL, SR, L, R, x = _inputs(tt, mpo, 36, 1024, 2024)
    y0 = tt.heff_apply_host(ctx, mpo, 36, 0, SL, SR, L, R, x)
    y = tt.heff_apply_host(ctx, mpo, 36, 2, SL, SR, L, R, x)
    assert np.isfinite(y0).all() and np.isfinite(y).all()
    err = np.linalg.norm(y - y0) / np.linalg.norm(y0)
    el = _groupwise_err(y, y0, SL, SR)
    print("full-size x6 relative error", err, "group-wise", el)
    assert err < 5e-6, err
    assert el < 5e-5, el
    y3 = tt.heff_apply_host(ctx, mpo, 36, 3, SL, SR, L, R, x)
    err3 = np.linalg.norm(y3 - y0) / np.linalg.norm(y0)
    el3 = _groupwise_err(y3, y0, SL, SR)
    print("full-size exact-split relative error", err3, "group-wise", el3)
    assert err3 < 5e-9 and el3 < 1e-8, (err3, el3)  # bound as in test_heff_split_bf16_matches_fp64
    mpo.close()
    ctx.close()
