"""The seeded workload generator shared by the tests, the oracle runs and the
benchmark (ffe_workloads): splitmix64 against its published test vector, and
the draws of the batched pulsar workload."""
import math

import ffe_workloads as W

# Vigna's splitmix64 reference output for seed 1234567 (the first five 64-bit words)
SPLITMIX64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                      4593380528125082431, 16408922859458223821]


def test_splitmix64_published_vector():
    g = W.splitmix64(1234567)
    got = [next(g) for _ in range(5)]
    want = [(w >> 11) * 2.0 ** -53 for w in SPLITMIX64_1234567]
    assert got == want


def test_pulsar_draws_ranges_and_size():
    """32 instances from seed 1531: R_LC in [3, 8), chi in [0, 60 deg), 4-8
    angular and 8-16 radial elements per wedge, P in {4, 5}; 99,990 elements in
    all (six wedges each), the same draws on every call."""
    d = W.pulsar_draws()
    assert d == W.pulsar_draws()
    assert len(d) == 32
    for x in d:
        assert 3.0 <= x["r_lc"] < 8.0
        assert 0.0 <= x["chi"] < math.radians(60.0)
        assert 4 <= x["n_ang"] <= 8 and 8 <= x["n_rad"] <= 16
        assert x["P"] in (4, 5)
    assert sum(6 * x["n_ang"] ** 2 * x["n_rad"] for x in d) == 99990
    cfgs = W.pulsars()
    assert [c["P"] for c in cfgs] == [x["P"] for x in d]
    assert all(c["r_out"] == 4.0 * x["r_lc"] for c, x in zip(cfgs, d))
