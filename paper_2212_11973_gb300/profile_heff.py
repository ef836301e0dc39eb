"""One site H_eff apply at the bench sizes, for profilers.

CL6x12 Hubbard MPO (U = 8, 1/8-doping mu) at the middle site, Gaussian sector
tables of total dimension D on both bonds, seeded standard-normal L, R and x,
applied through the kernel-level entry point tt_heff_apply_host (split-BF16
x6 by default: split copies, S1 and S3 on the tcgen05 kernel, the W-gather).
Small on the device (well under 1 GB at D = 1024), no CUDA graph, no
profiler start/stop: suited to `ncu -k ... -c ...` captures.

    python -m paper_2212_11973_gb300.profile_heff --D 1024 --repeat 2
"""
from __future__ import annotations

import argparse
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--D", type=int, default=1024)
    ap.add_argument("--precision", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()
    from paper_2212_11973_gb300 import tantrg as tt
    from paper_2212_11973_gb300 import workloads as wl
    cfg = wl.CYL_6x12_D1024
    ctx = tt.Context()
    mpo = tt.Mpo(ctx, cfg.Lx, cfg.Wy, cfg.periodic, t=cfg.t, U=cfg.U, mu=cfg.mu, form=cfg.form)
    site = cfg.N // 2
    SL = wl.gaussian_sectors(args.D, 1.5, wl.SECTOR_CHARGES, 2024)
    SR = wl.gaussian_sectors(args.D, 1.5, wl.SECTOR_CHARGES, 2025)
    nx, nl, nr = tt.layout_sizes(mpo, site, SL, SR)
    L, R, x = wl.random_vector(nl, 2026), wl.random_vector(nr, 2027), wl.random_vector(nx, 2028)
    for i in range(args.repeat):
        t0 = time.perf_counter()
        y = tt.heff_apply_host(ctx, mpo, site, args.precision, SL, SR, L, R, x)
        print(f"apply {i}: {time.perf_counter() - t0:.4f} s (host arrays, copies included), "
              f"|x| = {nx}, |L| = {nl}, |R| = {nr}, |y| = {float((y * y).sum()) ** 0.5:.6e}", flush=True)
    mpo.close()
    ctx.close()


if __name__ == "__main__":
    main()
