"""GPU parity: the CUDA tanTRG path against the CPU oracle on the same inputs.

FP64 path: relative difference <= 1e-10 in energy and free energy per site
(and density, double occupancy).  Mixed path (split-BF16 x6): <= 1e-6 in
energy and double occupancy.  Both sides run the same algorithm (growth with
2-TDVP, then 1-TDVP, K = 8, tau = dtau / 4 per half sweep).
"""
import pytest

from paper_2212_11973_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KEYS_FP64 = ("energy_per_site", "free_energy_per_site", "density", "double_occ", "lnZ")


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def tt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg
    tantrg.load_library()
    return tantrg


@pytest.fixture(scope="module")
def ctx(tt):
    c = tt.Context()
    yield c
    c.close()


def _gpu_run(tt, ctx, cfg, beta_end, precision=None, D=None, grow_until=1.0, env_precision=0):
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    D = D or cfg.D
    prec = cfg.precision if precision is None else precision
    rho = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(D, cfg.krylov, prec, env_precision=env_precision))
    rho.grow(cfg.dtau, min(grow_until, beta_end))  # the oracle's switch rule, same grow_until
    obs = [rho.measure()]
    while obs[-1]["beta"] < beta_end - 1e-9:
        rho.step(cfg.dtau, 1)
        obs.append(rho.measure())
    dims = rho.bond_dims()
    rho.close()
    mpo.close()
    return obs, dims


def _oracle_run(cfg, beta_end, D=None, grow_until=1.0):
    from oracle import model as om
    from oracle import mpo as ompo
    from oracle import tantrg as ot
    m = om.Model(cfg.Lx, cfg.Wy, cfg.periodic, cfg.t, cfg.U, cfg.mu, cfg.form)
    rec = {}

    def cb(st, stage):
        rec[round(st.beta, 9)] = ot.measure(st)

    st = ot.run(ompo.hubbard_mpo(m), cfg.beta0, cfg.dtau, beta_end, ot.TruncOpts(D or cfg.D), K=cfg.krylov,
                grow_until=grow_until, callback=cb)
    return rec, st


def test_cluster_2x2_fp64_matches_oracle(tt, ctx):
    cfg = wl.CLUSTER_2x2
    gpu, dims = _gpu_run(tt, ctx, cfg, 1.01)
    ref, st = _oracle_run(cfg, 1.01)
    assert dims[1:-1] == st.bond_dims()
    for o in gpu:
        r = ref[round(o["beta"], 9)]
        for k in KEYS_FP64:
            assert _rel(o[k], r[k]) < 1e-10, (o["beta"], k, o[k], r[k])


def test_cluster_2x2_untruncated_matches_oracle(tt, ctx):
    """Full rank (D = 256, bonds 16/256/16): GPU FP64 against the oracle."""
    cfg = wl.CLUSTER_2x2_FULL
    gpu, dims = _gpu_run(tt, ctx, cfg, 0.51)
    ref, st = _oracle_run(cfg, 0.51)
    assert dims == [1, 16, 256, 16, 1] and st.bond_dims() == [16, 256, 16]
    for o in gpu:
        r = ref[round(o["beta"], 9)]
        for k in KEYS_FP64:
            assert _rel(o[k], r[k]) < 1e-10, (o["beta"], k, o[k], r[k])


def test_ladder_fp64_matches_oracle(tt, ctx):
    """2x4 ladder at D = 32: several sectors per bond, truncated growth to
    beta = 0.2, then 1-TDVP steps to 0.51 on both sides."""
    cfg = wl.LADDER_2x4
    gpu, dims = _gpu_run(tt, ctx, cfg, 0.51, grow_until=0.2)
    ref, st = _oracle_run(cfg, 0.51, grow_until=0.2)
    assert len(gpu) >= 6  # the linear stage ran
    assert dims[1:-1] == st.bond_dims()
    for o in gpu:
        r = ref[round(o["beta"], 9)]
        for k in KEYS_FP64:
            assert _rel(o[k], r[k]) < 1e-10, (o["beta"], k, o[k], r[k])


@pytest.mark.parametrize("prec,env,tol", [(2, 0, 1e-6), (3, 0, 1e-8), (3, 2, 1e-8)])
def test_ladder_mixed_matches_oracle(tt, ctx, prec, env, tol):
    """Split-BF16 x6 applies (environment updates on the exact-accumulation
    split, the default) at 1e-6; every contraction on the exact split
    (~2^-32 per GEMM) at 1e-8, also with the environment updates in
    double-float (env_precision 2, ~2^-46 per operation)."""
    cfg = wl.LADDER_2x4
    gpu, dims = _gpu_run(tt, ctx, cfg, 0.51, precision=prec, grow_until=0.2, env_precision=env)
    ref, st = _oracle_run(cfg, 0.51, grow_until=0.2)
    assert len(gpu) >= 6  # the linear stage ran in split-BF16
    assert dims[1:-1] == st.bond_dims()
    for o in gpu:
        r = ref[round(o["beta"], 9)]
        for k in ("energy_per_site", "double_occ", "free_energy_per_site"):
            assert _rel(o[k], r[k]) < tol, (o["beta"], k, o[k], r[k])


def test_graph_replay_matches_direct_launches(tt):
    """On a non-default stream a beta-step is captured once as a CUDA graph and
    replayed; the kernels are deterministic, so the observables must be
    bitwise equal to the per-launch path (legacy default stream)."""
    import torch
    cfg = wl.LADDER_2x4
    out = []
    for use_stream in (False, True):
        stream = torch.cuda.Stream() if use_stream else torch.cuda.default_stream()
        with torch.cuda.stream(stream):
            c = tt.Context(stream=stream)
            mpo = tt.Mpo(c, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
            rho = tt.Rho(c, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, 2))
            rho.grow(cfg.dtau, 0.2)
            rho.step(cfg.dtau, 3)
            out.append(rho.measure())
            rho.close()
            mpo.close()
            c.close()
    for k in ("lnZ", "energy_per_site", "density", "double_occ"):
        assert out[0][k] == out[1][k], (k, out[0][k], out[1][k])


def _steps_with_qr(tt, monkeypatch, mode, cfg, D, steps, prec):
    if mode:
        monkeypatch.setenv("TT_QR", mode)
    else:
        monkeypatch.delenv("TT_QR", raising=False)
    c = tt.Context()
    mpo = tt.Mpo(c, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    rho = tt.Rho(c, mpo, cfg.beta0, tt.run_opts(D, cfg.krylov, prec))
    rho.grow(cfg.dtau, 0.2)
    obs = []
    for _ in range(steps):
        rho.step(cfg.dtau, 1)
        obs.append(rho.measure())
    rho.close()
    mpo.close()
    c.close()
    return obs


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (3, 1e-8)])
def test_cholqr_gauge_matches_householder(tt, monkeypatch, prec, tol):
    """4x8 cylinder at D = 128 (tall sector blocks up to a few hundred rows):
    the CholeskyQR3 gauge and the Householder-only gauge give the same state
    up to rounding.  FP64 mode factorises in FP64 (observables agree to
    1e-10); the exact split factorises in double-float (~2^-46, orthogonality
    ~1e-12 per gauge move, far inside its 1e-8 budget)."""
    cfg = wl.CYL_4x8_D256
    a = _steps_with_qr(tt, monkeypatch, "householder", cfg, 128, 3, prec)
    b = _steps_with_qr(tt, monkeypatch, None, cfg, 128, 3, prec)
    for oa, ob in zip(a, b):
        for k in KEYS_FP64:
            assert _rel(ob[k], oa[k]) < tol, (prec, oa["beta"], k, ob[k], oa[k])


def test_profiled_graph_replay_reports_times(tt):
    """Profiling events inside the captured beta-step are record nodes: after
    replays every kernel class reports a positive device time."""
    import torch
    cfg = wl.LADDER_2x4
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = tt.Context(stream=stream)
        mpo = tt.Mpo(c, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
        rho = tt.Rho(c, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, 2))
        rho.grow(cfg.dtau, 0.2)
        rho.set_profiling(True)
        rho.step(cfg.dtau, 3)
        s = rho.stats()
        rho.close()
        mpo.close()
        c.close()
    assert s["step_ms"] > 0 and s["heff_ms"] > 0 and s["env_ms"] > 0 and s["qr_ms"] > 0
    assert s["heff_ms"] + s["env_ms"] + s["qr_ms"] < s["step_ms"]


def test_cluster_2x2_t_prime_fp64_matches_oracle(tt, ctx):
    """t-t' model (diagonal hopping t' = -0.3) on the 2x2 cluster: GPU FP64
    against the oracle, growth and 1-TDVP steps."""
    from oracle import model as om
    from oracle import mpo as ompo
    from oracle import tantrg as ot
    cfg = wl.CLUSTER_2x2
    tp = -0.3
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form, tp=tp)
    rho = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, 0))
    rho.grow(cfg.dtau, 0.3)
    rho.step(cfg.dtau, 4)
    got = rho.measure()
    rho.close()
    mpo.close()
    m = om.Model(cfg.Lx, cfg.Wy, cfg.periodic, cfg.t, cfg.U, cfg.mu, cfg.form, tp)
    st = ot.run(ompo.hubbard_mpo(m), cfg.beta0, cfg.dtau, got["beta"] - 1e-9, ot.TruncOpts(cfg.D), K=cfg.krylov,
                grow_until=0.3)
    want = ot.measure(st)
    for k in KEYS_FP64:
        assert _rel(got[k], want[k]) < 1e-10, (k, got[k], want[k])


def test_exponential_growth_grid_matches_oracle(tt, ctx):
    """Growth on beta_n = 2^(n/4) beta_0 (tt_rho_grow_exp) to beta = 0.3, then
    linear 1-TDVP steps: GPU FP64 against the oracle on the same grid."""
    from oracle import model as om
    from oracle import mpo as ompo
    from oracle import tantrg as ot
    cfg = wl.CLUSTER_2x2
    r = 2.0 ** 0.25
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    rho = tt.Rho(ctx, mpo, cfg.beta0, tt.run_opts(cfg.D, cfg.krylov, 0))
    rho.grow_exp(r, 0.3)  # stops at 0.3 or when every bond is saturated
    obs = [rho.measure()]
    for _ in range(4):
        rho.step(cfg.dtau, 1)
        obs.append(rho.measure())
    rho.close()
    mpo.close()
    m = om.Model(cfg.Lx, cfg.Wy, cfg.periodic, cfg.t, cfg.U, cfg.mu, cfg.form)
    rec = {}
    ot.run(ompo.hubbard_mpo(m), cfg.beta0, cfg.dtau, obs[-1]["beta"] - 1e-9, ot.TruncOpts(cfg.D), K=cfg.krylov,
           grow_until=0.3, grow_ratio=r, callback=lambda st, stage: rec.__setitem__(round(st.beta, 9), ot.measure(st)))
    for o in obs:
        want = rec[round(o["beta"], 9)]
        for k in KEYS_FP64:
            assert _rel(o[k], want[k]) < 1e-10, (o["beta"], k, o[k], want[k])


def test_series_initial_state_matches_oracle_and_ed(tt, ctx):
    """SETTN initialisation of order 3 (Supplement, "Error analysis"): at beta0
    the state is sum_{k<=3} (-beta0 H/2)^k/k! (ED with that initial state);
    after growth (D = 256 on the 2x2 cluster) and 1-TDVP steps the GPU matches
    the oracle's run from its own series state."""
    from oracle import model as om
    from oracle import mpo as ompo
    from oracle import tantrg as ot
    cfg = wl.CLUSTER_2x2_FULL
    beta0, order = 0.05, 3
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    rho = tt.Rho(ctx, mpo, beta0, tt.run_opts(cfg.D, cfg.krylov, 0), taylor_order=order)
    obs = [rho.measure()]
    rho.grow(cfg.dtau, 0.2)
    obs.append(rho.measure())
    while obs[-1]["beta"] < 0.4 - 1e-9:
        rho.step(cfg.dtau, 1)
        obs.append(rho.measure())
    dims = rho.bond_dims()
    rho.close()
    mpo.close()
    m = om.Model(cfg.Lx, cfg.Wy, cfg.periodic, cfg.t, cfg.U, cfg.mu, cfg.form)
    rec = {}
    st = ot.run(ompo.hubbard_mpo(m), beta0, cfg.dtau, obs[-1]["beta"] - 1e-9, ot.TruncOpts(cfg.D), K=cfg.krylov,
                grow_until=0.2, taylor_order=order,
                callback=lambda s, stage: rec.__setitem__(round(s.beta, 9), ot.measure(s)))
    assert dims[1:-1] == st.bond_dims() == [16, 256, 16]
    ed = om.ed_thermo(m, [beta0], beta0=beta0, order=order)[0]
    for k in KEYS_FP64:
        assert _rel(obs[0][k], ed[k]) < 1e-12, ("ED at beta0", k, obs[0][k], ed[k])
    for o in obs[1:]:
        r = rec[round(o["beta"], 9)]
        for k in KEYS_FP64:
            assert _rel(o[k], r[k]) < 1e-10, ("oracle", o["beta"], k, o[k], r[k])
