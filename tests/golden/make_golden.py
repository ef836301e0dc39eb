"""Write the stored expected values under tests/golden/ by calling only oracle/.

Run from the repository root:  python tests/golden/make_golden.py

ed_2x2_U4.json   exact diagonalisation of the 2x2 open Hubbard cluster (t=1,
                 U=4, mu=0, particle-hole symmetric form) for the state
                 exp(-(beta-beta0) H/2) (I - beta0 H/2), beta0 = 0.01, on the
                 beta grid beta0 + n * 0.05 used by the 80-step run to beta ~ 4.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import model as om  # noqa: E402


def main():
    spec = dict(Lx=2, Wy=2, periodic_y=False, t=1.0, U=4.0, mu=0.0, form=1)
    m = om.Model(**spec)
    beta0 = 0.01
    betas = [beta0 + 0.05 * n for n in (0, 1, 2, 10, 20, 40, 80)]
    rows = om.ed_thermo(m, betas, beta0=beta0)
    out = dict(model=spec, beta0=beta0, source="oracle.model.ed_thermo", rows=rows)
    with open(os.path.join(HERE, "ed_2x2_U4.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
