"""Bounded device waits: a tcgen05 GEMM whose mbarrier wait runs out records
an error, drains its own copies and MMAs, frees its TMEM and returns; the host
reports TT_ERR_TIMEOUT, poisons the object and keeps the context usable.

The wait is made to run out by a zero time budget (one non-blocking test per
wait, right after the copies are started), never by a fault or an endless
loop; the copies and MMAs the aborted CTAs drain always complete.  The
three tcgen05 kernels are covered: the 128 x 128 and the persistent warp-
specialised split-BF16 ones, each forced with TT_GEMM in a child process
because the autotuner may pick the mma.sync kernel, which has no waits, and
the exact-accumulation digit kernel, which the exact split always runs."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

APPLY = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from paper_2212_11973_gb300 import tantrg as tt, workloads as wl
tt.load_library()
ctx = tt.Context()
mpo = tt.Mpo(ctx, 8, 2, False, t=1.0, U=4.0, mu=-0.3, form=1)
SL = wl.gaussian_sectors(300, 1.5, wl.SECTOR_CHARGES, 3300)
SR = wl.gaussian_sectors(300, 1.5, wl.SECTOR_CHARGES, 3301)
nx, nl, nr = tt.layout_sizes(mpo, 7, SL, SR)
L, R, x = wl.random_vector(nl, 3302), wl.random_vector(nr, 3303), wl.random_vector(nx, 3304)
y0 = tt.heff_apply_host(ctx, mpo, 7, {prec}, SL, SR, L, R, x)
ctx.set_wait_limit(0.0)
try:
    tt.heff_apply_host(ctx, mpo, 7, {prec}, SL, SR, L, R, x)
    raise SystemExit("no timeout reported")
except tt.TTError as e:
    assert e.status == 5, e  # TT_ERR_TIMEOUT
ctx.set_wait_limit(2.0)
y1 = tt.heff_apply_host(ctx, mpo, 7, {prec}, SL, SR, L, R, x)
assert np.array_equal(y0, y1)  # same kernels, same order: bitwise
try:
    ctx.set_wait_limit(-1.0)
    raise SystemExit("negative limit accepted")
except tt.TTError:
    pass
print("OK")
"""

STATE = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from paper_2212_11973_gb300 import tantrg as tt, workloads as wl
tt.load_library()
cfg = wl.LADDER_2x4
ctx = tt.Context()
mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
rho = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, {prec}))
rho.grow(cfg.dtau, 0.2)
rho.step(cfg.dtau, 1)
rho.measure()
ctx.set_wait_limit(0.0)
rho.step(cfg.dtau, 1)
try:
    rho.measure()
    raise SystemExit("no timeout reported")
except tt.TTError as e:
    assert e.status == 5, e
try:
    rho.step(cfg.dtau, 1)
    raise SystemExit("poisoned state accepted a step")
except tt.TTError as e:
    assert e.status == 6, e  # TT_ERR_STATE
ctx.set_wait_limit(2.0)
fresh = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, {prec}))
fresh.grow(cfg.dtau, 0.2)
fresh.step(cfg.dtau, 1)
assert np.isfinite(fresh.measure()["energy_per_site"])
print("OK")
"""


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# (TT_GEMM value, precision): split-BF16 x6 on a forced kernel, or the exact split
KERNELS = [("tc", 2), ("tcp", 2), ("tcz", 3)]


def _child(code, kernel, prec):
    env = dict(os.environ, TT_GEMM=kernel)
    p = subprocess.run([sys.executable, "-c", code.format(root=ROOT, prec=prec)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0 and p.stdout.strip().endswith("OK"), (kernel, p.stdout[-2000:], p.stderr[-3000:])


@pytest.mark.parametrize("kernel,prec", KERNELS)
def test_expired_wait_returns_timeout_and_context_survives(gpu, kernel, prec):
    _child(APPLY, kernel, prec)


@pytest.mark.parametrize("kernel,prec", KERNELS)
def test_expired_wait_poisons_the_state(gpu, kernel, prec):
    _child(STATE, kernel, prec)
