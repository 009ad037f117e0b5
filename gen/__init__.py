"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4.2).

Shared by the tests, the benchmark and the smoke check; it holds no step of
the method (no correlation, threshold, screening or lambda_* computation),
only random draws and the normalisations that define the data:

- ``gaussian_dict``: atoms i.i.d. uniform on the unit sphere (normalised
  N(0, I_N) columns), Sec. 4.2.1.
- ``pnoise_dict``: atoms e_1 + 0.1 kappa g, kappa ~ U(0, 1), g ~ N(0, I_N),
  normalised, Sec. 4.2.1.
- ``ar1_dict``: columns following an AR(1) process along the signal axis
  (d[0] = e_0, d[n] = rho d[n-1] + sqrt(1 - rho^2) e_n), normalised.
- ``observe``: y = D x0 + e with e Gaussian scaled to an exact SNR in dB
  (10 log10(||D x0||^2 / ||e||^2) = snr_db), or with a given noise sigma.

Every array is float64 and column-major (Fortran order), atom i being the
contiguous column D[:, i].
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _normalise(D):
    return np.asfortranarray(D / np.linalg.norm(D, axis=0, keepdims=True))


def gaussian_dict(N: int, K: int, g: np.random.Generator) -> np.ndarray:
    return _normalise(np.asfortranarray(g.standard_normal((N, K))))


def pnoise_dict(N: int, K: int, g: np.random.Generator) -> np.ndarray:
    D = 0.1 * g.uniform(0.0, 1.0, size=(1, K)) * g.standard_normal((N, K))
    D[0, :] += 1.0
    return _normalise(np.asfortranarray(D))


def ar1_dict(N: int, K: int, rho: float, g: np.random.Generator) -> np.ndarray:
    e = g.standard_normal((N, K))
    D = np.empty((N, K))
    D[0] = e[0]
    s = np.sqrt(1.0 - rho * rho)
    for n in range(1, N):
        D[n] = rho * D[n - 1] + s * e[n]
    return _normalise(np.asfortranarray(D))


def orthonormal_dict(N: int, g: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(g.standard_normal((N, N)))
    return np.asfortranarray(q * np.sign(np.diag(r)))


def sparse_x0(K: int, k: int, g: np.random.Generator) -> np.ndarray:
    """k nonzeros at uniform random positions, N(0, 1) values."""
    x = np.zeros(K)
    idx = g.choice(K, size=k, replace=False)
    x[idx] = g.standard_normal(k)
    return x


def bernoulli_gaussian_x0(K: int, p: float, g: np.random.Generator) -> np.ndarray:
    mask = g.uniform(size=K) < p
    x = np.zeros(K)
    x[mask] = g.standard_normal(int(mask.sum()))
    return x


def group_x0(goff: np.ndarray, n_active: int, g: np.random.Generator) -> np.ndarray:
    """n_active groups chosen uniformly, N(0, 1) entries in each."""
    nG = goff.size - 1
    x = np.zeros(int(goff[-1]))
    for gi in g.choice(nG, size=n_active, replace=False):
        x[goff[gi]:goff[gi + 1]] = g.standard_normal(int(goff[gi + 1] - goff[gi]))
    return x


def bernoulli_group_x0(goff: np.ndarray, p: float, g: np.random.Generator) -> np.ndarray:
    """Each group active independently with probability p (at least one active), N(0, 1)
    entries in the active groups (the paper's Group-Lasso data, Sec. 4.2)."""
    nG = goff.size - 1
    act = g.uniform(size=nG) < p
    if not act.any():
        act[g.integers(nG)] = True
    x = np.zeros(int(goff[-1]))
    for gi in np.flatnonzero(act):
        x[goff[gi]:goff[gi + 1]] = g.standard_normal(int(goff[gi + 1] - goff[gi]))
    return x


def observe(D, x0, g: np.random.Generator, snr_db: float | None = 20.0, sigma: float | None = None):
    s = D @ x0
    e = g.standard_normal(D.shape[0])
    if sigma is not None:
        return s + sigma * e
    ns = np.linalg.norm(s)
    if ns == 0.0:
        return e
    return s + e * (ns / np.linalg.norm(e)) * 10.0 ** (-snr_db / 20.0)


def atom_like_y(N: int, kind: str, g: np.random.Generator) -> np.ndarray:
    """An observation drawn from the same distribution as the atoms (the paper's Lasso
    experiments, Sec. 4.2): uniform on the unit sphere, or a normalised Pnoise draw."""
    if kind == "gaussian":
        v = g.standard_normal(N)
    elif kind == "pnoise":
        v = 0.1 * g.uniform(0.0, 1.0) * g.standard_normal(N)
        v[0] += 1.0
    else:
        raise ValueError(kind)
    return v / np.linalg.norm(v)


def contiguous_groups(K: int, size: int) -> np.ndarray:
    return np.arange(0, K + 1, size, dtype=np.int64)


# ------------------------------------------------------------ named workloads

def lasso_problem(N: int, K: int, seed: int, p: float = 0.01, snr_db: float = 20.0, kind: str = "gaussian"):
    """Gaussian (or Pnoise / AR(1)) unit-norm D, Bernoulli(p)-Gaussian x0, y at snr_db."""
    g = rng(seed)
    if kind == "gaussian":
        D = gaussian_dict(N, K, g)
    elif kind == "pnoise":
        D = pnoise_dict(N, K, g)
    elif kind == "ar1":
        D = ar1_dict(N, K, 0.9, g)
    else:
        raise ValueError(kind)
    x0 = bernoulli_gaussian_x0(K, p, g)
    if not x0.any():
        x0[g.integers(K)] = 1.0
    y = observe(D, x0, g, snr_db=snr_db)
    return D, y, x0


def config1(seed: int = 1001):
    """100 x 500 Gaussian unit-norm D, 10 nonzeros N(0,1), y = D x0 + N(0, 0.01^2)."""
    g = rng(seed)
    D = gaussian_dict(100, 500, g)
    x0 = sparse_x0(500, 10, g)
    y = observe(D, x0, g, sigma=0.01)
    return D, y, x0


def config2(seed: int = 1002, N: int = 2000, K: int = 10000):
    """N x K Gaussian unit-norm D, Bernoulli(0.01)-Gaussian x0, 20 dB."""
    return lasso_problem(N, K, seed)


CONFIG2_RATIOS = (0.1, 0.3, 0.5, 0.7, 0.9)
CONFIG3_RATIOS = (0.2, 0.5, 0.8)


def config3(seed: int = 1003, N: int = 2000, K: int = 10000, gsize: int = 10, n_active: int = 10):
    """N x K Gaussian unit-norm D, contiguous groups of gsize with w_g = sqrt(gsize),
    n_active groups of N(0,1) entries, 20 dB."""
    g = rng(seed)
    D = gaussian_dict(N, K, g)
    goff = contiguous_groups(K, gsize)
    w = np.full(goff.size - 1, np.sqrt(gsize))
    x0 = group_x0(goff, n_active, g)
    y = observe(D, x0, g, snr_db=20.0)
    return D, y, x0, goff, w


def paper_group_problem(gsize: int, seed: int, N: int = 2000, K: int = 10000, kind: str = "pnoise",
                        p: float = 0.05):
    """The paper's Group-Lasso experiment (Sec. 4.2, Sec. 4.4): a Pnoise (or Gaussian)
    dictionary, groups of gsize atoms, each group active with probability p, N(0,1)
    coefficients, y the l2-normalised sum of D x0 and a 20 dB Gaussian noise; weights
    w_g = sqrt(gsize).  The paper draws random groups of equal size; the atoms are
    i.i.d., so contiguous groups of a freshly drawn dictionary have the same law."""
    g = rng(seed)
    D = pnoise_dict(N, K, g) if kind == "pnoise" else gaussian_dict(N, K, g)
    goff = contiguous_groups(K, gsize)
    w = np.full(goff.size - 1, np.sqrt(gsize))
    x0 = bernoulli_group_x0(goff, p, g)
    y = observe(D, x0, g, snr_db=20.0)
    return D, y / np.linalg.norm(y), x0, goff, w
