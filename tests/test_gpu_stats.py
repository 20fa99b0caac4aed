"""Pair-separation histogram / radial distribution function (needs a GPU).

Integer counts must equal the oracle's brute-force count over all pairs of
the positions lcs_get_state returns (same FP64 separation arithmetic).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import L, gpu_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("N,n,P,nbins", [(16, 20000, (2, 2, 2), 16), (12, 30000, (3, 1, 2), 7),
                                         (3, 2000, (1, 1, 1), 50)])
def test_pair_histogram_equals_brute_force(lcs, N, n, P, nbins):
    # the histogram does not depend on the field: particles and velocities
    # of a 16^3 case, the field of the grid under test (N = 3 has no room
    # for several Fourier modes, so a uniform flow there)
    field, _, x, v, tau = synth.small_case(300 + N, 16, 8, 4.0, n, 0.05, dt=0.01)
    field = field if N == 16 else np.full((3, N, N, N), 0.3)
    sim = lcs.Simulator(field, x, v, 0.01, tau=tau, sub=P, sort_every=3)
    sim.step(4)   # moved, migrated and sorted state
    st = gpu_state(sim)
    r_max = L / N
    got = sim.pair_histogram(r_max, nbins)
    want = oracle.pair_hist(st["x"], L, r_max, nbins)
    assert got.sum() > 0
    assert np.array_equal(got, want), (got, want)


def test_pair_histogram_of_a_cubic_lattice(lcs):
    m = 6
    a = L / m
    g = np.arange(m) * a + 0.1 * a
    x = np.stack([c.ravel() for c in np.meshgrid(g, g, g, indexing="ij")])
    n = x.shape[1]
    field = np.zeros((3, 3, 3, 3))
    sim = lcs.Simulator(field, x, np.zeros_like(x), 0.01, tau_const=0.1)
    r_max, nbins = 0.99 * (L / 3), 11    # L/N = 2a; bins of 0.18 a
    got = sim.pair_histogram(r_max, nbins)
    want = np.zeros(nbins, np.int64)
    for k, mult in ((1.0, 3), (math.sqrt(2), 6), (math.sqrt(3), 4)):
        want[int(k * a / (r_max / nbins))] += mult * n
    assert np.array_equal(got, want), (got, want)
    assert np.array_equal(got, oracle.pair_hist(gpu_state(sim)["x"], L, r_max, nbins))


def test_uniform_particles_are_not_clustered(lcs):
    N, n = 32, 300000
    field, _, x, v, _ = synth.small_case(320, N, 8, 4.0, n, None)
    sim = lcs.Simulator(field, x, v, 0.01, tau_const=0.1, sub=(2, 2, 2))
    r, g, counts = sim.rdf(L / N, 8)
    assert counts[1:].min() > 1000
    assert np.all(np.abs(g[1:] - 1) < 0.05), g
    # g is the counts over the pair count of an ideal gas in each shell
    edges = np.linspace(0.0, L / N, 9)
    expected = n * (n - 1) / 2 * (4 / 3 * math.pi * np.diff(edges ** 3)) / L ** 3
    assert np.allclose(g, counts / expected, rtol=1e-12, atol=0)
    assert np.allclose(r, 0.5 * (edges[1:] + edges[:-1]), rtol=1e-15)
    assert np.array_equal(counts, sim.pair_histogram(L / N, 8))


def test_pair_histogram_arguments_and_tiny_sets(lcs):
    field, _, x, v, _ = synth.small_case(330, 8, 8, 2.0, 2, None)
    for n in (0, 1):
        sim = lcs.Simulator(field, x[:, :n], v[:, :n], 0.01, tau_const=0.1)
        assert np.array_equal(sim.pair_histogram(L / 8, 4), np.zeros(4, np.int64))
    sim = lcs.Simulator(field, x, v, 0.01, tau_const=0.1)
    for r_max, nbins in ((L / 8 * 1.01, 4), (0.0, 4), (L / 16, 0), (L / 16, 5000)):
        with pytest.raises(lcs.LcsError) as e:
            sim.pair_histogram(r_max, nbins)
        assert e.value.status == lcs.LCS_ERR_ARG
    small = lcs.Simulator(np.zeros((3, 2, 2, 2)), x, v, 0.01, tau_const=0.1)
    with pytest.raises(lcs.LcsError) as e:
        small.pair_histogram(0.1, 4)   # N = 2: neighbouring cells coincide
    assert e.value.status == lcs.LCS_ERR_ARG
