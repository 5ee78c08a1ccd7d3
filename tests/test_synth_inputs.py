"""The seeded input generators (synth/): the counter-based generator against
the published SplitMix64 sequence, the statistics of its normal deviates,
addressability of any block, and the 500-atom disordered cluster of the
learned-screening workload (0.1 atoms per cubic Angstrom, 1.0 A minimum
separation, two thirds carbon)."""

import numpy as np
import pytest

from synth import rng
from synth.systems import random_cluster


def test_splitmix64_reference_sequence():
    """SplitMix64 from state 0: the first three outputs of the published
    generator (state advanced by the golden-ratio constant, then mixed)."""
    g = 0x9E3779B97F4A7C15
    states = np.array([0, g, (2 * g) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    out = rng._mix(states)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_deviates_have_unit_moments():
    z = rng.normal_stream(7, 3, 0, 1_000_000)
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 3)) < 5 * np.sqrt(15.0 / n)           # odd moment
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)    # kurtosis of N(0,1)


def test_any_block_regenerates_alone_and_threads_do_not_matter():
    full = rng.normal_stream(11, 5, 0, 3 << 22)
    part = rng.normal_stream(11, 5, 5_000_000, 1000)
    np.testing.assert_array_equal(part, full[5_000_000:5_001_000])
    again = rng.normal_stream(11, 5, 0, 3 << 22, threads=1)
    np.testing.assert_array_equal(again, full)
    other = rng.normal_stream(11, 6, 5_000_000, 1000)
    assert not np.allclose(other, part)


@pytest.fixture(scope="module")
def cluster():
    return random_cluster(500, 0.1, 1.0, 20210428)


def test_cluster_geometry(cluster):
    xyz = cluster.xyz
    assert xyz.shape == (500, 3)
    box = (500 / 0.1) ** (1.0 / 3.0)
    assert np.all(xyz >= 0.0) and np.all(xyz <= box)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)
    d[np.diag_indices(500)] = np.inf
    assert d.min() >= 1.0
    n_c = sum(s == "C" for s in cluster.species)
    assert abs(n_c - 500 * 2 / 3) < 4 * np.sqrt(500 * 2 / 9)        # binomial spread
    assert cluster.n_ao.sum() == 13 * n_c + 5 * (500 - n_c)
    assert cluster.n_ri.sum() == 30 * n_c + 12 * (500 - n_c)


def test_cluster_is_seeded(cluster):
    again = random_cluster(500, 0.1, 1.0, 20210428)
    np.testing.assert_array_equal(again.xyz, cluster.xyz)
    assert again.species == cluster.species
    other = random_cluster(500, 0.1, 1.0, 20210429)
    assert not np.allclose(other.xyz, cluster.xyz)
