"""Chemical potential for 1/8 hole doping on the CL4x8 cylinder.

The grand-canonical density depends on temperature, so mu is fixed once: the
value that gives n = 7/8 (within 0.005) at the final beta = 10 of the CL4x8
runs (U = 8, particle-hole symmetric form), found by bracketing with the FP64
path at D = 128.  n(mu) is increasing, so the Illinois variant of regula falsi
on n(mu) - 7/8 converges from any bracket [mu_lo, mu_hi] with n(mu_lo) < 7/8 <
n(mu_hi).

    python -m paper_2212_11973_gb300.tune_mu --lo -3.5 --hi 0.0
"""
from __future__ import annotations

import argparse
import json
import time


def density_at(mu: float, beta_end: float = 10.0, D: int = 128, U: float = 8.0) -> dict:
    import torch
    from paper_2212_11973_gb300 import tantrg as tt
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = tt.Context(stream=stream)
        mpo = tt.Mpo(ctx, 8, 4, True, t=1.0, U=U, mu=mu, form=1)
        rho = tt.Rho(ctx, mpo, 0.01, tt.run_opts(D, 8, 0))
        dtau = 0.05
        rho.grow(dtau, 1.0)
        beta = rho.measure()["beta"]
        n = int(round((beta_end - beta) / dtau))
        rho.step(dtau, n)
        o = rho.measure()
        rho.close()
        mpo.close()
        ctx.close()
    return o


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lo", type=float, default=-3.5)
    ap.add_argument("--hi", type=float, default=0.0)
    ap.add_argument("--target", type=float, default=0.875)
    ap.add_argument("--tol", type=float, default=0.005)
    ap.add_argument("--max-iter", type=int, default=12)
    args = ap.parse_args()
    t0 = time.time()
    lo, hi = args.lo, args.hi
    flo = density_at(lo)["density"] - args.target
    fhi = density_at(hi)["density"] - args.target
    print(json.dumps({"mu": lo, "n_minus_target": flo}), flush=True)
    print(json.dumps({"mu": hi, "n_minus_target": fhi}), flush=True)
    if not (flo < 0 < fhi):
        raise SystemExit("bracket does not contain the target density")
    side = 0
    best = (lo, flo) if abs(flo) < abs(fhi) else (hi, fhi)
    for _ in range(args.max_iter):
        if abs(best[1]) <= args.tol / 2:
            break
        mu = (lo * fhi - hi * flo) / (fhi - flo)
        o = density_at(mu)
        f = o["density"] - args.target
        print(json.dumps({"mu": mu, "n_minus_target": f, "beta": o["beta"], "energy_per_site": o["energy_per_site"]}),
              flush=True)
        if abs(f) < abs(best[1]):
            best = (mu, f)
        if f < 0:
            lo, flo = mu, f
            if side == -1:
                fhi /= 2
            side = -1
        else:
            hi, fhi = mu, f
            if side == 1:
                flo /= 2
            side = 1
    print(json.dumps({"mu_frozen": best[0], "n": best[1] + args.target, "seconds": time.time() - t0}), flush=True)


if __name__ == "__main__":
    main()
