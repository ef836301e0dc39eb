"""Checkpoint round trip (tt_rho_save / tt_rho_load): a loaded state measures
what the saved one measured, and one beta-step from the checkpoint equals the
step of the original (FP64, bitwise up to the rebuilt environments' rounding);
a mixed-precision state loaded as FP64 then stepped in both precisions stays
within the mixed tolerance."""
import os

import pytest

from paper_2212_11973_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KEYS = ("energy_per_site", "density", "double_occ", "free_energy_per_site", "lnZ")


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("prec_saved,prec_loaded,tol", [(0, 0, 1e-11), (2, 0, 1e-6), (2, 2, 1e-6)])
def test_save_load_step(tt, tmp_path, prec_saved, prec_loaded, tol):
    cfg = wl.LADDER_2x4
    ctx = tt.Context()
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    rho = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, prec_saved, growth_precision=0))
    rho.grow(cfg.dtau, 0.2)
    rho.step(cfg.dtau, 2)
    before = rho.measure()
    path = os.path.join(str(tmp_path), "rho.ttck")
    rho.save(path)
    r2 = tt.Rho.load(ctx, mpo, path, tt.run_opts(cfg.D, cfg.krylov, prec_loaded))
    loaded = r2.measure()
    for k in KEYS:
        # a loaded state rebuilds its environments in FP64: the energy of a
        # state saved from the split-BF16 path moves by the environments'
        # mixed-precision error, everything else is a function of the tensors
        t = tol if (prec_saved and k == "energy_per_site") else 1e-12
        assert _rel(loaded[k], before[k]) < t, ("after load", k, loaded[k], before[k])
    rho.step(cfg.dtau, 1)
    r2.step(cfg.dtau, 1)
    a, b = rho.measure(), r2.measure()
    assert a["beta"] == b["beta"]
    for k in KEYS:
        assert _rel(b[k], a[k]) < tol, ("after a step", k, b[k], a[k])
    rho.close()
    r2.close()
    mpo.close()
    ctx.close()
