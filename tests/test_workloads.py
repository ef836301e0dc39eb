"""Seeded input generators: splitmix64 against its published outputs and the
batch parameter draws (U in [2, 10], mu in [-2, 0], D cycling 64/96/128)."""
from paper_2212_11973_gb300 import workloads as wl


def test_splitmix64_reference_outputs():
    # first outputs for seed 0 of the reference splitmix64 (Steele, Lea, Flood,
    # OOPSLA 2014; the public-domain C version by Vigna)
    g = wl.splitmix64(0)
    assert [next(g) for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_batch_ladders_draws():
    b = wl.batch_ladders()
    assert len(b) == 64
    assert all(2.0 <= w.U < 10.0 and -2.0 <= w.mu < 0.0 for w in b)
    assert [w.D for w in b[:6]] == [64, 96, 128, 64, 96, 128]
    assert all((w.Lx, w.Wy, w.periodic, w.N) == (8, 2, False, 16) for w in b)
    # the draws are the stated function of the generator's stream
    g = wl.splitmix64(wl.BATCH_SEED)
    u1, u2 = (next(g) >> 11) * 2.0 ** -53, (next(g) >> 11) * 2.0 ** -53
    assert b[0].U == 2.0 + 8.0 * u1 and b[0].mu == -2.0 + 2.0 * u2
    assert len({w.U for w in b}) == 64
