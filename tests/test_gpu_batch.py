"""Batch of independent instances (tt_batch_*): every instance of a batch step
must equal the same model stepped alone (same kernels and plans, so bitwise),
and the instances must really differ from each other."""
from dataclasses import replace

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


def _small_batch():
    # the batch draws (U, mu) on 2x4 ladders with D in {16, 24, 32}
    return [replace(w, Lx=4, D=(16, 24, 32)[i % 3]) for i, w in enumerate(wl.batch_ladders(4))]


def test_batch_matches_single_instances(tt):
    import torch
    ws = _small_batch()
    prec, beta0, dtau = 2, 0.01, 0.05
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = tt.Context(stream=stream)
        b = tt.Batch(c, ws, beta0, tt.run_opts(0, 8, prec, growth_precision=0))
        b.grow(dtau, 0.2)
        b.step(dtau, 3)
        got = b.measure()
        b.close()
        single = []
        for w in ws:
            mpo = tt.Mpo(c, w.Lx, w.Wy, w.periodic, t=w.t, U=w.U, mu=w.mu, form=w.form)
            rho = tt.Rho(c, mpo, beta0, tt.run_opts(w.D, 8, prec, growth_precision=0))
            rho.grow(dtau, 0.2)
            rho.step(dtau, 3)
            single.append(rho.measure())
            rho.close()
            mpo.close()
        c.close()
    for g, s in zip(got, single):
        for k in ("beta", "lnZ", "energy_per_site", "density", "double_occ", "max_bond"):
            assert g[k] == s[k], (k, g[k], s[k])
    assert len({round(g["energy_per_site"], 12) for g in got}) == len(got)
