"""Fig. 1(c) / Fig. S7 of the paper on the GPU path: free fermions (U = 0) on
the CL4x8 cylinder at half filling, where the free energy has a closed form.

* Growth on an exponential grid beta_n = 2^(n/2) beta_0 (2-TDVP) from
  beta_0 = 1e-4 to beta = 1, then 1-TDVP with 4 tau = 1/4 to beta = 9: the
  relative free-energy error delta F against the closed form is recorded at
  every integer beta.  At D = 128 the one-site projection error dominates
  (free fermions at half filling carry a large operator entanglement across a
  width-4 cut; the paper needs D ~ 1000 for its small errors), so only a loose
  bound is asserted.
* Lie-Trotter scaling (Fig. S7(c)): from the same state at beta = 1, evolve to
  beta = 9 with 4 tau = 1, 1/2, 1/4 and with the reference 4 tau = 1/16;
  delta F_LT = |F(tau) - F_ref| / |F_ref| follows c tau^alpha with alpha ~ 2
  (fitted slope between 1.5 and 2.7: the reference's own error, a quarter of
  the smallest step's, flattens the fit a little).
The linear stage runs in split-BF16 x6 with FP64-class environment updates on
a side stream (graph-replayed steps).
"""
import os
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


def test_free_fermion_cylinder_errors_and_lie_trotter_slope(tt):
    import torch
    from oracle import model as om
    Lx, Wy, mu, D = 8, 4, 0.0, 128
    m = om.Model(Lx, Wy, True, 1.0, 0.0, mu, 1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = tt.Context(stream=stream)
        mpo = tt.Mpo(ctx, Lx, Wy, True, t=1.0, U=0.0, mu=mu, form=1)
        rho = tt.Rho(ctx, mpo, 1e-4, tt.run_opts(D, 8, 2, growth_precision=0))
        rho.grow_exp(2.0 ** 0.5, 1.0)
        b = rho.measure()["beta"]
        if b < 1.0 - 1e-9:
            rho.step(1.0 - b, 1)
        path = os.path.join(tempfile.mkdtemp(), "beta1.ttck")
        rho.save(path)

        def dF(o):
            ex = om.free_fermion_thermo(m, [o["beta"]])[0]["free_energy_per_site"]
            return abs(o["free_energy_per_site"] - ex) / abs(ex)

        errs = {1: dF(rho.measure())}
        for _ in range(32):
            rho.step(0.25, 1)
            o = rho.measure()
            if abs(o["beta"] - round(o["beta"])) < 1e-9:
                errs[int(round(o["beta"]))] = dF(o)
        rho.close()
        print("delta F vs beta (D=128):", {k: f"{v:.2e}" for k, v in sorted(errs.items())})
        assert len(errs) == 9 and max(errs.values()) < 0.2, errs

        def f_at_9(dtau):
            r = tt.Rho.load(ctx, mpo, path, tt.run_opts(D, 8, 2))
            r.step(dtau, int(round(8.0 / dtau)))
            o = r.measure()
            r.close()
            assert abs(o["beta"] - 9.0) < 1e-9
            return o["free_energy_per_site"]

        f_ref = f_at_9(1.0 / 16)
        taus, lt = [], []
        for dtau in (1.0, 0.5, 0.25):
            taus.append(dtau / 4.0)
            lt.append(abs(f_at_9(dtau) - f_ref) / abs(f_ref))
        alpha = np.polyfit(np.log(taus), np.log(lt), 1)[0]
        print("Lie-Trotter delta F at beta=9:", [f"{e:.2e}" for e in lt], "slope", round(float(alpha), 3))
        assert 1.5 < alpha < 2.7, (lt, alpha)
        mpo.close()
        ctx.close()
