"""The seeded input generator (no solver arithmetic here)."""

import numpy as np

from synth import dirichlet_design, load_right_edge, load_top_edge, splitmix64


def test_splitmix64_published_outputs():
    # SplitMix64 started from state 0 emits 0xE220A8397B1DCDAF first; its
    # second output is the hash of one golden-ratio increment.
    assert int(splitmix64(0)) == 0xE220A8397B1DCDAF
    assert int(splitmix64(0x9E3779B97F4A7C15)) == 0x6E789E6AA1B965F4


def test_dirichlet_design_properties():
    x = dirichlet_design(33, 17, 4, seed=0)
    assert x.shape == (4, 17, 33)
    np.testing.assert_allclose(x.sum(axis=0), 1.0, rtol=1e-15)
    assert x.min() > 0.0 and x.max() < 1.0
    # Each fraction of a flat Dirichlet over 4 phases has mean 1/4 and
    # variance (1/4)(3/4)/5.
    big = dirichlet_design(256, 256, 4, seed=1)
    assert abs(big.mean() - 0.25) < 1e-3
    assert abs(big[0].var() - 0.0375) < 2e-3
    np.testing.assert_array_equal(dirichlet_design(33, 17, 4, seed=0), x)
    assert not np.array_equal(dirichlet_design(33, 17, 4, seed=2), x)
    # Chunking does not change the stream.
    np.testing.assert_array_equal(dirichlet_design(33, 17, 4, seed=0, chunk=100), x)


def test_loads():
    f = load_top_edge(4, 3)
    assert f.shape == (4, 5, 2) and f[3, :, 1].sum() == -5 and np.count_nonzero(f) == 5
    g = load_right_edge(4, 3)
    assert g[:, 4, 0].sum() == 4 and np.count_nonzero(g) == 4


def test_torch_generator_matches_numpy():
    # The device version of the design generator (for designs too large to
    # build on the host), run here on CPU tensors: the same fractions up to
    # the rounding of the logarithm and of the normalising sum (a few ulps;
    # a wrong bit in the integer hash would change a fraction by O(1)), for
    # several phase counts, chunkings and seeds, including seeds above 2^63.
    import torch
    from synth import dirichlet_design_torch
    for nelx, nely, n_phase, seed, chunk in ((33, 17, 4, 0, 1 << 22), (40, 24, 16, 9, 100),
                                            (16, 8, 3, (1 << 63) + 12345, 7)):
        ref = dirichlet_design(nelx, nely, n_phase, seed)
        got = dirichlet_design_torch(nelx, nely, n_phase, seed, torch.device("cpu"), chunk=chunk).numpy()
        np.testing.assert_allclose(got, ref, rtol=2e-15, atol=0)
