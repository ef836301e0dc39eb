"""The three split-BF16 GEMM kernels the tile autotuner chooses from (tcgen05
128 x 128 tiles, persistent warp-specialised tcgen05 128 x 64 tiles, mma.sync
64 x 64 tiles) compute the same contraction: a site H_eff apply at D = 300
(x6) and at the CL6x12 bench sizes (D = 1024) agree between any two of them
within the split-BF16 x6 bound, element-wise per right-sector group.  Each
kernel is forced with TT_GEMM in a child process (the choice is read once per
process); the default (autotuned) run must match as well, and a mixed sweep
records how many plans went to each kernel."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2212_11973_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from paper_2212_11973_gb300 import tantrg as tt, workloads as wl
tt.load_library()
ctx = tt.Context()
mpo = tt.Mpo(ctx, {Lx}, {Wy}, {per}, t=1.0, U=8.0, mu=wl.MU_EIGHTH_DOPING, form=1)
SL = wl.gaussian_sectors({D}, 1.5, wl.SECTOR_CHARGES, {seed})
SR = wl.gaussian_sectors({D}, 1.5, wl.SECTOR_CHARGES, {seed} + 1)
nx, nl, nr = tt.layout_sizes(mpo, {site}, SL, SR)
L, R, x = wl.random_vector(nl, {seed} + 2), wl.random_vector(nr, {seed} + 3), wl.random_vector(nx, {seed} + 4)
y = tt.heff_apply_host(ctx, mpo, {site}, 2, SL, SR, L, R, x)
np.save({out!r}, y)
"""


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


def _child(tmp_path, kernel, **kw):
    out = str(tmp_path / f"y_{kernel or 'auto'}.npy")
    env = dict(os.environ)
    env.pop("TT_GEMM", None)
    if kernel:
        env["TT_GEMM"] = kernel
    code = CHILD.format(root=ROOT, out=out, **kw)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return np.load(out)


def _groupwise(y, y0, SL, SR):
    from _layout import right_groups
    groups, total = right_groups(SL, SR)
    assert total == y0.size
    worst = 0.0
    for off, rows, dr in groups:
        a, b = y[off:off + rows * dr], y0[off:off + rows * dr]
        s = np.abs(b).max()
        if s > 0:
            worst = max(worst, np.abs(a - b).max() / s)
    return worst


@pytest.mark.parametrize("case", [dict(Lx=8, Wy=2, per=False, site=7, D=300, seed=31),
                                  dict(Lx=12, Wy=6, per=True, site=36, D=1024, seed=2024)])
def test_split_kernels_agree(tt, tmp_path, case):
    ys = {k: _child(tmp_path, k, **case) for k in ("tc", "tcp", "mma", None)}
    SL = wl.gaussian_sectors(case["D"], 1.5, wl.SECTOR_CHARGES, case["seed"])
    SR = wl.gaussian_sectors(case["D"], 1.5, wl.SECTOR_CHARGES, case["seed"] + 1)
    ref = ys["mma"]
    for k, y in ys.items():
        assert np.isfinite(y).all()
        err = _groupwise(y, ref, SL, SR)
        print(case["D"], k, "group-wise vs mma.sync", err)
        assert err < 2e-5, (k, err)


def test_mixed_sweep_reports_tuned_kernels(tt):
    import torch
    cfg = wl.LADDER_2x4
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = tt.Context(stream=stream)
        mpo = tt.Mpo(c, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
        rho = tt.Rho(c, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, 2))
        rho.grow(cfg.dtau, 0.2)
        rho.step(cfg.dtau, 2)
        s = rho.stats()
        rho.close()
        mpo.close()
        c.close()
    assert s["tuned_tc128"] + s["tuned_tcp128x64"] + s["tuned_mma64"] > 0, s
