"""Bounded device waits: a tcgen05 GEMM whose mbarrier wait runs out records
an error, drains its own copies and MMAs, frees its TMEM and returns; the host
reports TT_ERR_TIMEOUT, poisons the object and keeps the context usable.

The wait is made to run out by a zero time budget (one non-blocking test per
wait, issued right after the copies are started), never by a fault or an
endless loop; the copies and MMAs the aborted CTAs drain always complete."""
import numpy as np
import pytest

from paper_2212_11973_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


def _inputs(tt, mpo, site, D, seed):
    SL = wl.gaussian_sectors(D, 1.5, wl.SECTOR_CHARGES, seed)
    SR = wl.gaussian_sectors(D, 1.5, wl.SECTOR_CHARGES, seed + 1)
    nx, nl, nr = tt.layout_sizes(mpo, site, SL, SR)
    return SL, SR, wl.random_vector(nl, seed + 2), wl.random_vector(nr, seed + 3), wl.random_vector(nx, seed + 4)


def test_expired_wait_returns_timeout_and_context_survives(tt):
    ctx = tt.Context()
    mpo = tt.Mpo(ctx, 8, 2, False, t=1.0, U=4.0, mu=-0.3, form=1)
    SL, SR, L, R, x = _inputs(tt, mpo, 7, 300, 3300)
    y0 = tt.heff_apply_host(ctx, mpo, 7, 2, SL, SR, L, R, x)
    ctx.set_wait_limit(0.0)
    with pytest.raises(tt.TTError) as ei:
        tt.heff_apply_host(ctx, mpo, 7, 2, SL, SR, L, R, x)
    assert ei.value.status == 5, ei.value  # TT_ERR_TIMEOUT
    ctx.set_wait_limit(2.0)
    y1 = tt.heff_apply_host(ctx, mpo, 7, 2, SL, SR, L, R, x)
    assert np.array_equal(y0, y1)  # same kernels, same order: bitwise
    with pytest.raises(tt.TTError):
        ctx.set_wait_limit(-1.0)
    mpo.close()
    ctx.close()


def test_expired_wait_poisons_the_state(tt):
    cfg = wl.LADDER_2x4
    ctx = tt.Context()
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    rho = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, tt.TT_PREC_MIXED_BF16X6))
    rho.grow(cfg.dtau, 0.2)
    rho.step(cfg.dtau, 1)
    rho.measure()
    ctx.set_wait_limit(0.0)
    rho.step(cfg.dtau, 1)
    with pytest.raises(tt.TTError) as ei:
        rho.measure()
    assert ei.value.status == 5, ei.value
    with pytest.raises(tt.TTError) as ei:
        rho.step(cfg.dtau, 1)
    assert ei.value.status == 6, ei.value  # TT_ERR_STATE: poisoned
    ctx.set_wait_limit(2.0)
    fresh = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, tt.TT_PREC_MIXED_BF16X6))
    fresh.grow(cfg.dtau, 0.2)
    fresh.step(cfg.dtau, 1)
    o = fresh.measure()
    assert np.isfinite(o["energy_per_site"])
    fresh.close()
    rho.close()
    mpo.close()
    ctx.close()
