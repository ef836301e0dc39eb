"""The test-side layout bookkeeping (tests/_layout.py) agrees with the
library's own element counts (tt_layout_sizes_terms needs no GPU), and the
dense conversions round-trip."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import _layout as lay  # noqa: E402

from paper_2212_11973_gb300 import workloads as wl  # noqa: E402


def _oracle_site(Lx, Wy, per, j):
    from oracle import model as om
    from oracle import mpo as ompo
    Ws = ompo.hubbard_mpo(om.Model(Lx, Wy, per, 1.0, 8.0, -0.5, 1))
    return Ws[j], lay.mpo_channel_charges(Ws)


def test_layout_counts_match_the_library():
    from paper_2212_11973_gb300 import build
    build.build()
    from paper_2212_11973_gb300 import tantrg as tt
    tt.load_library()
    for (Lx, Wy, per, j, D, w) in ((8, 2, False, 7, 130, 1.5), (4, 4, True, 6, 256, 0.6)):
        W, ch = _oracle_site(Lx, Wy, per, j)
        SL = wl.gaussian_sectors(D, w, wl.SECTOR_CHARGES, 5)
        SR = wl.gaussian_sectors(D, w, wl.SECTOR_CHARGES, 6)
        nx, nl, nr = tt.layout_sizes_terms(ch[j], ch[j + 1], SL, SR)
        assert nx == lay.site_blocks(SL, SR)[1]
        assert nl == lay.env_rows(SL, ch[j])[1]
        assert nr == lay.env_rows(SR, ch[j + 1])[1]


def test_dense_round_trip():
    SL = wl.gaussian_sectors(40, 1.0, wl.SECTOR_CHARGES, 1)
    SR = wl.gaussian_sectors(50, 1.0, wl.SECTOR_CHARGES, 2)
    n = lay.site_blocks(SL, SR)[1]
    x = wl.random_vector(n, 3)
    X = lay.site_to_dense(x, SL, SR)
    assert np.array_equal(lay.dense_to_site(X, SL, SR), x)
    assert lay.outside_blocks_norm(X, SL, SR) < 1e-12
    assert np.isclose((X * X).sum(), (x * x).sum())


def test_channel_charges_conserve_on_every_term():
    W, ch = _oracle_site(4, 4, True, 6)
    for (wl_, wr, s, t, v) in lay.mpo_terms(W):
        ql, qr = ch[6][wl_], ch[7][wr]
        assert qr == (ql[0] + lay.LOCAL_Q[s][0] - lay.LOCAL_Q[t][0], ql[1] + lay.LOCAL_Q[s][1] - lay.LOCAL_Q[t][1])
