"""The seeded input recipe (Sec. 4.2 shapes): each generator produces what its
description states.  CPU only; no step of the method is involved."""
import numpy as np
import pytest

import gen


@pytest.mark.parametrize("kind", ["gaussian", "pnoise", "ar1"])
def test_dictionaries_are_seeded_unit_norm_column_major(kind):
    make = {"gaussian": lambda g: gen.gaussian_dict(64, 300, g),
            "pnoise": lambda g: gen.pnoise_dict(64, 300, g),
            "ar1": lambda g: gen.ar1_dict(64, 300, 0.9, g)}[kind]
    D = make(gen.rng(5))
    assert D.dtype == np.float64 and D.flags.f_contiguous and D.shape == (64, 300)
    np.testing.assert_allclose(np.linalg.norm(D, axis=0), 1.0, rtol=1e-13)
    np.testing.assert_array_equal(D, make(gen.rng(5)))
    assert not np.array_equal(D, make(gen.rng(6)))


def test_pnoise_atoms_cluster_around_the_first_axis():
    """Pnoise atoms are e_1 plus small noise: every atom has a positive first
    entry and the dictionary is far more coherent than a Gaussian one."""
    g = gen.rng(8)
    P = gen.pnoise_dict(64, 400, g)
    G = gen.gaussian_dict(64, 400, g)
    assert np.all(P[0] > 0)
    coh = lambda D: np.abs(D.T @ D - np.eye(D.shape[1])).mean()
    assert coh(P) > 5 * coh(G)


def test_ar1_columns_have_lag_one_correlation_rho():
    D = gen.ar1_dict(4096, 64, 0.9, gen.rng(9))
    lag1 = np.sum(D[1:] * D[:-1]) / np.sum(D[:-1] * D[:-1])
    assert abs(lag1 - 0.9) < 0.01


def test_observation_has_the_exact_snr():
    g = gen.rng(10)
    D = gen.gaussian_dict(200, 500, g)
    x0 = gen.bernoulli_gaussian_x0(500, 0.05, g)
    for snr in (20.0, 10.0, 35.0):
        y = gen.observe(D, x0, g, snr_db=snr)
        s = D @ x0
        assert abs(10 * np.log10(np.sum(s * s) / np.sum((y - s) ** 2)) - snr) < 1e-10


def test_sparse_and_group_coefficients():
    g = gen.rng(11)
    x = gen.bernoulli_gaussian_x0(100000, 0.01, g)
    assert abs(np.count_nonzero(x) - 1000) < 4 * np.sqrt(100000 * 0.01 * 0.99)
    x = gen.sparse_x0(500, 10, g)
    assert np.count_nonzero(x) == 10
    goff = gen.contiguous_groups(1000, 10)
    assert goff[0] == 0 and goff[-1] == 1000 and np.all(np.diff(goff) == 10)
    x = gen.group_x0(goff, 7, g)
    active = [np.any(x[goff[i]:goff[i + 1]] != 0) for i in range(goff.size - 1)]
    assert sum(active) == 7
    for i in np.flatnonzero(active):
        assert np.all(x[goff[i]:goff[i + 1]] != 0)


@pytest.mark.parametrize("kind", ["gaussian", "pnoise"])
def test_atom_like_observation_is_unit(kind):
    y = gen.atom_like_y(300, kind, gen.rng(12))
    assert abs(np.linalg.norm(y) - 1.0) < 1e-14


def test_named_workload_shapes():
    D, y, x0 = gen.config1()
    assert D.shape == (100, 500) and y.shape == (100,) and np.count_nonzero(x0) == 10
    D, y, x0, goff, w = gen.config3(N=200, K=1000)
    assert goff.size - 1 == 100 and np.allclose(w, np.sqrt(10))
    assert sum(np.any(x0[goff[i]:goff[i + 1]] != 0) for i in range(100)) == 10


def test_paper_group_problem_bernoulli_groups():
    """Sec. 4.2: groups active with probability 0.05, N(0,1) coefficients in active
    groups only, unit-norm observation, Pnoise atoms, w_g = sqrt(group size)."""
    D, y, x0, goff, w = gen.paper_group_problem(5, seed=7, N=200, K=4000)
    assert D.shape == (200, 4000) and np.allclose(np.linalg.norm(D, axis=0), 1.0)
    assert abs(np.linalg.norm(y) - 1.0) < 1e-12
    assert np.allclose(w, np.sqrt(5.0)) and goff[-1] == 4000 and np.all(np.diff(goff) == 5)
    act = np.array([np.any(x0[goff[i]:goff[i + 1]] != 0) for i in range(goff.size - 1)])
    assert all(np.all(x0[goff[i]:goff[i + 1]] != 0) for i in np.flatnonzero(act))
    assert 0.03 < act.mean() < 0.07  # 800 groups, Bernoulli(0.05)
    assert np.median(D[0]) > 0.5  # Pnoise atoms cluster around e_1 (Gaussian atoms: about 0)
