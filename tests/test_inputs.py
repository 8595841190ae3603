"""The seeded input generators: the counter-based generator against the published SplitMix64
outputs, its streams, and the Fe-C recipe (0.1 % C on distinct octahedral sites of bcc Fe)."""
import os

import numpy as np

from paper_1107_2619_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _hex_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = int(v, 16)
    return vals


def test_mixer_reproduces_the_published_splitmix64_outputs():
    g = _hex_golden("splitmix64.txt")
    with np.errstate(over="ignore"):
        states = np.arange(1, 5, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        out = I._mix64(states)
    assert [int(x) for x in out] == [g[f"out{k}"] for k in range(1, 5)]


def test_streams_are_reproducible_prefix_stable_and_distinct():
    a = I.random_u64(7, 3, 1000)
    assert np.array_equal(a, I.random_u64(7, 3, 1000))
    assert np.array_equal(a[:10], I.random_u64(7, 3, 10))        # word k depends on k only
    assert not np.any(a == I.random_u64(7, 4, 1000))            # another stream
    assert not np.any(a == I.random_u64(8, 3, 1000))            # another seed
    assert len(np.unique(a)) == a.size


def test_uniforms_carry_53_bits_in_the_unit_interval():
    u = I.random_uniform(11, 1, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    m = u * 2.0 ** 53
    assert np.array_equal(m, np.floor(m))
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002


def test_fe_c_carbon_sits_on_distinct_octahedral_sites():
    n = 20
    w = I.bcc_fe_c(n, seed=4)
    n_fe = 2 * n ** 3
    assert (w.species == 0).sum() == n_fe
    c = w.pos[w.species == 1]
    assert c.shape[0] == round(0.001 * n_fe)
    # in units of a/2 an octahedral site has one or two odd coordinates (edge midpoints, face
    # centres); bcc Fe sites have none or three
    x = c / (2.8665 / 2.0)
    q = np.rint(x).astype(int)
    assert np.abs(x - q).max() < 0.35                            # within the 0.05 Å displacements
    odd = (q % 2 != 0).sum(axis=1)
    assert np.all((odd == 1) | (odd == 2))
    assert len({tuple(v) for v in q % (2 * n)}) == c.shape[0]   # distinct sites
    other = I.bcc_fe_c(n, seed=5)
    assert not np.array_equal(c, other.pos[other.species == 1])   # the sites follow the seed
