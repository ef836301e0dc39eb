"""Derived thermodynamics from a series of measurements (post-processing).

tanTRG yields ln Z, the energy, density and double occupancy per site on a
beta grid (main text: thermodynamics from the partition function; Fig. 3 /
Supplement t-t'-U results show the entropy, specific heat and charge
compressibility derived from them).  These helpers take the `measure()`
dictionaries of one or two runs:

  S/N   = beta (e - f)                      entropy per site (f = -ln Z/(beta N))
  C/N   = -beta^2 de/dbeta                  specific heat per site
  chi_c = dn/dmu                            charge compressibility
"""
from __future__ import annotations

import numpy as np


def entropy_per_site(obs: list[dict]) -> np.ndarray:
    """S/N = beta (e - f) at every point of the series."""
    return np.array([o["beta"] * (o["energy_per_site"] - o["free_energy_per_site"]) for o in obs])


def specific_heat_per_site(obs: list[dict]) -> tuple[np.ndarray, np.ndarray]:
    """C/N = -beta^2 de/dbeta by second-order finite differences on the
    (possibly non-uniform) beta grid of the series; returns (betas, C)."""
    b = np.array([o["beta"] for o in obs])
    e = np.array([o["energy_per_site"] for o in obs])
    if b.size < 3:
        raise ValueError("need at least three points")
    return b, -b * b * np.gradient(e, b, edge_order=2)


def compressibility(obs_minus: list[dict], obs_plus: list[dict], dmu: float) -> tuple[np.ndarray, np.ndarray]:
    """chi_c = dn/dmu by a central difference of two runs at mu -+ dmu/2 on
    the same beta grid; returns (betas, chi)."""
    b = np.array([o["beta"] for o in obs_minus])
    if not np.allclose(b, [o["beta"] for o in obs_plus]):
        raise ValueError("the two runs must share the beta grid")
    n0 = np.array([o["density"] for o in obs_minus])
    n1 = np.array([o["density"] for o in obs_plus])
    return b, (n1 - n0) / dmu
