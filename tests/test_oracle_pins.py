"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a brute-force enumeration, a printed formula of the paper, the KKT
conditions, an independent library routine, or an invariance.  All run on
the CPU (no GPU marker).
"""
import itertools

import numpy as np
import pytest

import gen
import oracle


def _small_lasso(seed, N=30, K=80, k=4, sigma=0.01):
    g = gen.rng(seed)
    D = gen.gaussian_dict(N, K, g)
    x0 = gen.sparse_x0(K, k, g)
    y = gen.observe(D, x0, g, sigma=sigma)
    return D, y


# ---------------------------------------------------------------- lambda_*

@pytest.mark.parametrize("groups", [False, True])
def test_lambda_max_is_the_zero_threshold(groups):
    """Sec. 2.2.2 / eq. (gstar): x = 0 iff lambda >= lambda_*."""
    D, y = _small_lasso(1)
    goff = gen.contiguous_groups(D.shape[1], 4) if groups else None
    w = np.full(goff.size - 1, 2.0) if groups else None
    lm, star, _ = oracle.lambda_max(D, y, goff, w)
    test = "gsafe" if groups else "safe"
    r = oracle.solve(D, y, lm * (1 + 1e-9), goff, w, test=test, tol=1e-12, max_iter=50)
    assert r["iters"] == 0 and not r["x"].any() and r["gap"] == 0.0
    lam = lm * (1 - 1e-3)
    r = oracle.solve(D, y, lam, goff, w, test="none", tol=0, max_iter=5000)
    nz = np.flatnonzero(r["x"])
    if groups:
        assert set(nz) <= set(range(goff[star], goff[star + 1])) and nz.size > 0
    else:
        # one active atom: x_* = sign(b_*) (lambda_* - lambda) / ||d_*||^2 (KKT with support {i_*})
        b = D.T @ y
        assert list(nz) == [star]
        assert np.isclose(r["x"][star], np.sign(b[star]) * (lm - lam) / (D[:, star] @ D[:, star]), rtol=1e-8)


# ----------------------------------------------------- closed forms (prox)

def test_orthonormal_dictionary_soft_threshold():
    """D^T D = I: the Lasso solution is soft(D^T y, lambda) (eq. softTh)."""
    g = gen.rng(2)
    D = gen.orthonormal_dict(64, g)
    y = g.standard_normal(64)
    b = D.T @ y
    lam = 0.6 * np.abs(b).max()
    want = np.sign(b) * np.maximum(np.abs(b) - lam, 0)
    for alg in ("ista", "fista"):
        for test in ("none", "safe", "dst3", "dome"):
            r = oracle.solve(D, y, lam, alg=alg, test=test, tol=1e-15, max_iter=400, L=1.0)
            np.testing.assert_allclose(r["x"], want, atol=1e-12)


def test_orthonormal_dictionary_group_soft_threshold():
    """D^T D = I: the Group-Lasso solution is the group soft threshold of D_g^T y
    with threshold lambda w_g (eq. gr_softTh)."""
    g = gen.rng(3)
    D = gen.orthonormal_dict(60, g)
    y = g.standard_normal(60)
    goff = gen.contiguous_groups(60, 5)
    w = np.sqrt(np.diff(goff).astype(float))
    b = D.T @ y
    lm = max(np.linalg.norm(b[goff[i]:goff[i + 1]]) / w[i] for i in range(goff.size - 1))
    lam = 0.5 * lm
    want = np.zeros(60)
    for i in range(goff.size - 1):
        bg = b[goff[i]:goff[i + 1]]
        nb = np.linalg.norm(bg)
        want[goff[i]:goff[i + 1]] = max(0.0, (nb - lam * w[i]) / nb) * bg
    for test in ("none", "gsafe", "dgst3"):
        r = oracle.solve(D, y, lam, goff, w, test=test, tol=1e-15, max_iter=400, L=1.0)
        np.testing.assert_allclose(r["x"], want, atol=1e-12)


# ------------------------------------------------- brute force (tiny Lasso)

def _lasso_bruteforce(D, y, lam):
    """Exact Lasso minimiser by enumerating supports and signs: on support S with
    signs s, D_S^T D_S x_S = D_S^T y - lam s; accept when sign(x_S) = s and
    |d_j^T (y - D_S x_S)| <= lam off the support (eq. primaldual)."""
    N, K = D.shape
    best = None
    for size in range(0, min(N, K) + 1):
        for S in itertools.combinations(range(K), size):
            S = list(S)
            for s in itertools.product((-1.0, 1.0), repeat=size):
                s = np.array(s)
                if size:
                    A = D[:, S]
                    xs = np.linalg.solve(A.T @ A, A.T @ y - lam * s)
                    if np.any(np.sign(xs) != s):
                        continue
                    r = y - A @ xs
                else:
                    xs = np.zeros(0)
                    r = y
                c = D.T @ r
                if np.all(np.abs(np.delete(c, S)) <= lam * (1 + 1e-12)):
                    x = np.zeros(K)
                    x[S] = xs
                    return x
        if best is not None:
            break
    raise AssertionError("no KKT point found")


@pytest.mark.parametrize("seed", [11, 12, 13])
@pytest.mark.parametrize("test", ["safe", "dst3", "dome"])
@pytest.mark.parametrize("dynamic", [True, False])
def test_bruteforce_and_safety_tiny(seed, test, dynamic):
    """Definition 1 and Theorem 1: the screened solver returns the exact minimiser,
    and no screened atom is nonzero in it."""
    g = gen.rng(seed)
    N, K = 6, 9
    D = gen.gaussian_dict(N, K, g)
    y = D @ gen.sparse_x0(K, 2, g) + 0.05 * g.standard_normal(N)
    lm, _, _ = oracle.lambda_max(D, y)
    for ratio in (0.3, 0.6, 0.9):
        lam = ratio * lm
        xbf = _lasso_bruteforce(D, y, lam)
        for alg in ("ista", "fista", "cp"):
            r = oracle.solve(D, y, lam, alg=alg, test=test, dynamic=dynamic, tol=0, max_iter=20000)
            np.testing.assert_allclose(r["x"], xbf, atol=1e-8)
            screened = r["scr_iter"] != 0
            assert not np.any(xbf[screened] != 0), (test, ratio, alg)


# ------------------------------------------------------------------- KKT

def test_kkt_lasso_config1_shape():
    """eq. (primaldual): |d_i^T (y - D x)| <= lambda, = lambda sign(x_i) on the support."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    r = oracle.solve(D, y, lam, alg="ista", test="dst3", tol=1e-13, max_iter=200000)
    assert r["status"] == 0
    c = D.T @ (y - D @ r["x"])
    assert np.all(np.abs(c) <= lam * (1 + 1e-5))
    S = r["x"] != 0
    np.testing.assert_allclose(c[S], lam * np.sign(r["x"][S]), rtol=1e-5)


def test_kkt_group_lasso():
    """eq. (primaldualKKT_glasso): ||D_g^T r|| <= lambda w_g, with D_g^T r =
    lambda w_g x_g/||x_g|| on active groups."""
    D, y, _, goff, w = gen.config3(1003, N=60, K=200, gsize=5, n_active=3)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.4 * lm
    r = oracle.solve(D, y, lam, goff, w, test="dgst3", tol=1e-14, max_iter=100000)
    res = y - D @ r["x"]
    for i in range(goff.size - 1):
        sl = slice(goff[i], goff[i + 1])
        cg = D[:, sl].T @ res
        xg = r["x"][sl]
        assert np.linalg.norm(cg) <= lam * w[i] * (1 + 1e-5)
        if np.any(xg != 0):
            np.testing.assert_allclose(cg, lam * w[i] * xg / np.linalg.norm(xg), atol=1e-5 * lam * w[i])


def test_matches_independent_coordinate_descent():
    """An independent solver (scikit-learn coordinate descent) agrees on the minimiser."""
    sk = pytest.importorskip("sklearn.linear_model")
    D, y = _small_lasso(4, N=40, K=120, k=5)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.3 * lm
    m = sk.Lasso(alpha=lam / D.shape[0], fit_intercept=False, tol=1e-14, max_iter=200000).fit(D, y)
    r = oracle.solve(D, y, lam, test="dst3", tol=1e-15, max_iter=100000)
    np.testing.assert_allclose(r["x"], m.coef_, atol=1e-7)


# ------------------------------------------------------- gap / trajectories

@pytest.mark.parametrize("test", ["none", "safe", "dst3", "dome"])
def test_gap_nonnegative_and_sets_nested(test):
    """A duality gap is >= 0 at every iteration; screened sets only grow (Alg. 3)."""
    D, y = _small_lasso(5, N=50, K=300, k=5)
    lm, _, _ = oracle.lambda_max(D, y)
    r = oracle.solve(D, y, 0.5 * lm, test=test, tol=1e-12, max_iter=5000)
    h = r["hist"]
    assert np.all(h[:, 4] >= -1e-12 * 0.5 * (y @ y))
    assert np.all(np.diff(h[:, 0]) <= 0)
    assert r["status"] == 0 and r["gap"] <= 1e-12 * 0.5 * (y @ y)
    # each atom is screened once, at the first test that removes it: the atoms
    # recorded as screened by iteration t are exactly those gone from A_t
    s = r["scr_iter"]
    for t in range(1, r["iters"] + 1):
        assert np.count_nonzero((s != 0) & (s <= t)) == 300 - h[t - 1, 0]


@pytest.mark.parametrize("alg", ["ista", "fista"])
@pytest.mark.parametrize("test", ["none", "dst3", "dgst3"])
def test_warm_start_at_the_minimiser_stays_there(alg, test):
    """The minimiser is a fixed point of the proximal gradient step of Table 1
    (ISTA; FISTA's extrapolation of two equal iterates is zero), so a solve
    warm-started there (x_0 = u_0 = x*) has a zero gap from its first iteration."""
    if test == "dgst3":
        D, y, _, goff, w = gen.config3(1007, N=50, K=200, gsize=4, n_active=3)
    else:
        (D, y), goff, w = _small_lasso(6, N=50, K=200, k=5), None, None
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.4 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    xs = oracle.solve(D, y, lam, goff, w, test="none", tol=1e-15, max_iter=200000, L=L)["x"]
    r = oracle.solve(D, y, lam, goff, w, alg=alg, test=test, tol=0, max_iter=3, L=L, x0=xs)
    assert np.all(r["hist"][:, 4] <= 1e-11 * 0.5 * (y @ y))
    np.testing.assert_allclose(r["x"], xs, atol=1e-9 * np.abs(xs).max())


@pytest.mark.parametrize("alg", ["ista", "fista", "cp"])
@pytest.mark.parametrize("test", ["dst3", "dgst3"])
def test_gap_certifies_the_distance_to_the_minimiser(alg, test):
    """For any x, P(x) - P* >= 1/2 ||D (x - x~)||^2 (the quadratic term of P is
    exact and x~ minimises the convex rest), and the duality gap (Sec. 2.2)
    bounds P(x_t) - P*, so 1/2 ||D (x_t - x~)||^2 <= gap_t for the iterate the
    solver returns after t iterations."""
    if test == "dgst3":
        D, y, _, goff, w = gen.config3(1009, N=40, K=160, gsize=4, n_active=3)
    else:
        (D, y), goff, w = _small_lasso(8, N=40, K=160, k=5), None, None
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.3 * lm
    xs = oracle.solve(D, y, lam, goff, w, test="none", tol=1e-15, max_iter=200000)["x"]
    yy = y @ y
    for t in (1, 2, 3, 5, 10, 30, 100):
        r = oracle.solve(D, y, lam, goff, w, alg=alg, test=test, tol=0, max_iter=t)
        e = D @ (r["x"] - xs)
        assert 0.5 * (e @ e) <= r["hist"][t - 1, 4] + 1e-12 * yy


@pytest.mark.parametrize("groups", [False, True])
def test_history_counts_atoms_and_nonzeros(groups):
    """The per-iteration history holds the quantities of the paper's flops
    accounting (Sec. 4.1): |A_t| counts atoms (not groups) still active after
    the test of iteration t, i.e. K minus the atoms recorded as screened by t,
    and ||x_t||_0 counts the nonzeros of the iterate returned after t iterations."""
    if groups:
        D, y, _, goff, w = gen.config3(1011, N=50, K=240, gsize=6, n_active=3)
        test = "dgst3"
    else:
        (D, y), goff, w, test = _small_lasso(9, N=50, K=240, k=5), None, None, "dst3"
    K = D.shape[1]
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.3 * lm  # small enough that atoms leave the support in the first iterations
    r = oracle.solve(D, y, lam, goff, w, test=test, tol=1e-10, max_iter=3000)
    h, s = r["hist"], r["scr_iter"]
    assert r["n_active"] == K - np.count_nonzero(s) == h[r["iters"] - 1, 0]
    assert r["nnz"] == np.count_nonzero(r["x"]) == h[r["iters"] - 1, 1]
    for t in list(range(1, 21)) + [r["iters"]]:
        assert h[t - 1, 0] == K - np.count_nonzero((s != 0) & (s <= t))
        rt = oracle.solve(D, y, lam, goff, w, test=test, tol=0, max_iter=t)
        assert h[t - 1, 1] == np.count_nonzero(rt["x"])


def test_scale_covariance():
    """P(a lambda, D, a y) has solution a x(lambda, D, y)."""
    D, y = _small_lasso(6)
    lm, _, _ = oracle.lambda_max(D, y)
    r1 = oracle.solve(D, y, 0.4 * lm, tol=1e-15, max_iter=50000)
    r2 = oracle.solve(D, 3.0 * y, 1.2 * lm, tol=1e-15, max_iter=50000)
    np.testing.assert_allclose(r2["x"], 3.0 * r1["x"], atol=1e-9)


# ---------------------------------------------- static tests vs the paper

def _unit_y_problem(seed, N=40, K=400, kind="gaussian"):
    g = gen.rng(seed)
    D = gen.pnoise_dict(N, K, g) if kind == "pnoise" else gen.gaussian_dict(N, K, g)
    y = D @ gen.sparse_x0(K, 4, g) + 0.3 * g.standard_normal(N)
    return D, y / np.linalg.norm(y)


@pytest.mark.parametrize("ratio", [0.5, 0.7, 0.9])
def test_static_safe_is_algorithm4_formula(ratio):
    """Algorithm 4 (||y|| = 1): screen i iff |d_i^T y| < lambda - 1 + lambda/lambda_*;
    the dynamic test at the first ISTA iteration from 0 screens the same set."""
    D, y = _unit_y_problem(7)
    lm, _, b = oracle.lambda_max(D, y)
    lam = ratio * lm
    want = np.abs(b) < lam - 1 + lam / lm
    rs = oracle.solve(D, y, lam, alg="ista", test="safe", dynamic=False, max_iter=1, tol=0)
    rd = oracle.solve(D, y, lam, alg="ista", test="safe", dynamic=True, max_iter=1, tol=0)
    np.testing.assert_array_equal(rs["scr_iter"] != 0, want)
    np.testing.assert_array_equal(rd["scr_iter"] != 0, want)


@pytest.mark.parametrize("kind", ["gaussian", "pnoise"])
@pytest.mark.parametrize("ratio", [0.6, 0.8, 0.95])
def test_static_dome_is_printed_lemma(ratio, kind):
    """Lemma 4 with theta = y, ||y|| = 1, unit atoms, in the printed form:
    Q^l(t) < y^T d_i < Q^u(t), t = d_*^T d_i, with the printed constants."""
    D, y = _unit_y_problem(8, kind=kind)
    lm, star, b = oracle.lambda_max(D, y)
    lam = ratio * lm
    dstar = np.sign(b[star]) * D[:, star]
    t = D.T @ dstar
    r = np.sqrt((1 / lam - 1 / lm) ** 2 - (lm / lam - 1) ** 2)  # printed r_theta at theta = y
    const = lam - 1 + lam / lm
    Ql = np.where(t <= lm, (lm - lam) * t - lam + lam * r * np.sqrt(1 - t * t), -const)
    Qu = np.where(t < -lm, const, (lm - lam) * t + lam - lam * r * np.sqrt(1 - t * t))
    want = (Ql < b) & (b < Qu)
    rs = oracle.solve(D, y, lam, alg="ista", test="dome", dynamic=False, max_iter=1, tol=0)
    got = rs["scr_iter"] != 0
    # an atom may sit on a boundary within rounding; there must be none in these draws
    assert np.array_equal(got, want), np.flatnonzero(got != want)
    if kind == "pnoise" or ratio > 0.9:
        assert want.sum() > 0


@pytest.mark.parametrize("kind", ["gaussian", "pnoise"])
@pytest.mark.parametrize("ratio", [0.6, 0.8, 0.95])
def test_static_dst3_is_printed_lemma(ratio, kind):
    """Lemma 3 with theta = y (the ST3 test): screen iff 1 - |d_i^T c| > r with
    c = y/lambda - (lambda_*/lambda - 1) d_*, r = sqrt(||mu y - y/lambda||^2 - (lambda_*/lambda - 1)^2),
    mu = 1/lambda_* for ||y|| = 1."""
    D, y = _unit_y_problem(9, kind=kind)
    lm, star, b = oracle.lambda_max(D, y)
    lam = ratio * lm
    dstar = np.sign(b[star]) * D[:, star]
    c = y / lam - (lm / lam - 1) * dstar
    r = np.sqrt(np.linalg.norm(y / lm - y / lam) ** 2 - (lm / lam - 1) ** 2)
    want = 1 - np.abs(D.T @ c) > r
    rs = oracle.solve(D, y, lam, alg="ista", test="dst3", dynamic=False, max_iter=1, tol=0)
    np.testing.assert_array_equal(rs["scr_iter"] != 0, want)


# ------------------------------------------- Lasso = singleton Group-Lasso

@pytest.mark.parametrize("pair", [("safe", "gsafe"), ("dst3", "dgst3")])
def test_lasso_tests_are_singleton_group_tests(pair):
    """Appendix: Lemmas 2/3 are Lemmas 5/6 with groups of size one and w = 1."""
    D, y = _small_lasso(10, N=40, K=200)
    lm, _, _ = oracle.lambda_max(D, y)
    goff = gen.contiguous_groups(200, 1)
    w = np.ones(200)
    a = oracle.solve(D, y, 0.5 * lm, test=pair[0], tol=1e-12, max_iter=3000)
    b = oracle.solve(D, y, 0.5 * lm, goff, w, test=pair[1], tol=1e-12, max_iter=3000)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-12)
    np.testing.assert_array_equal(a["scr_iter"], b["scr_iter"])
    assert a["iters"] == b["iters"]


# -------------------------------------------------- regions contain theta~

@pytest.mark.parametrize("test", ["safe", "dst3", "dome"])
def test_regions_contain_dual_optimum(test):
    """Each iteration's sphere (or dome) contains theta~ = (y - D x~)/lambda."""
    D, y = _small_lasso(14, N=40, K=300, k=4)
    lm, star, b = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    ref = oracle.solve(D, y, lam, test="none", tol=1e-15, max_iter=100000)
    th = (y - D @ ref["x"]) / lam
    r = oracle.solve(D, y, lam, test=test, tol=1e-10, max_iter=5000)
    h = r["hist"]
    dstar = np.sign(b[star]) * D[:, star]
    if test == "safe":
        dist = np.linalg.norm(th - y / lam)
        assert np.all(dist <= h[:, 3] + 1e-9)
    elif test == "dst3":
        c = y / lam - (lm / lam - 1) * dstar / (dstar @ dstar)
        assert np.all(np.linalg.norm(th - c) <= h[:, 3] + 1e-9)
    else:
        assert np.all(np.linalg.norm(th - y / lam) <= h[:, 2] + 1e-9)
        assert dstar @ th <= 1 + 1e-9


def test_group_regions_contain_dual_optimum():
    D, y, _, goff, w = gen.config3(15, N=50, K=200, gsize=4, n_active=3)
    lm, star, b = oracle.lambda_max(D, y, goff, w)
    lam = 0.5 * lm
    ref = oracle.solve(D, y, lam, goff, w, test="none", tol=1e-15, max_iter=100000)
    th = (y - D @ ref["x"]) / lam
    # every group constraint of Lemma 5's feasible set holds at theta~
    for i in range(goff.size - 1):
        assert np.linalg.norm(D[:, goff[i]:goff[i + 1]].T @ th) <= w[i] * (1 + 1e-8)
    r = oracle.solve(D, y, lam, goff, w, test="gsafe", tol=1e-10, max_iter=5000)
    assert np.all(np.linalg.norm(th - y / lam) <= r["hist"][:, 3] + 1e-9)
    # DGST3 ball: bounding sphere of the half-space cap; containment of theta~
    r = oracle.solve(D, y, lam, goff, w, test="dgst3", tol=1e-10, max_iter=5000)
    Dg = D[:, goff[star]:goff[star + 1]]
    n = Dg @ (Dg.T @ y) / lm
    c = y / lam - (n @ y / lam - w[star] ** 2) * n / (n @ n)
    assert np.all(np.linalg.norm(th - c) <= r["hist"][:, 3] + 1e-9)


@pytest.mark.parametrize("test", ["gsafe", "dgst3"])
def test_group_weights_are_a_change_of_variables(test):
    """Eq. (1) with weights w: substituting x_g = z_g / w_g turns (D, w) into
    (D_g / w_g, unit weights) with the same objective, so lambda_*, the static
    screened set (Lemmas 5 and 6 through Lemma 7) and the minimiser (x = z / w)
    must all agree between the two problems."""
    g = gen.rng(21)
    D = gen.gaussian_dict(50, 200, g)
    goff = gen.contiguous_groups(200, 4)
    G = goff.size - 1
    w = 0.5 + 1.5 * g.random(G)
    y = gen.observe(D, gen.group_x0(goff, 3, g), g, snr_db=20.0)
    wcol = np.repeat(w, np.diff(goff))
    Dz = D / wcol
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lz, _, _ = oracle.lambda_max(Dz, y, goff, np.ones(G))
    np.testing.assert_allclose(lz, lm, rtol=1e-13)
    partial = 0
    for ratio in (0.6, 0.8, 0.9, 0.95):
        lam = ratio * lm
        rx = oracle.solve(D, y, lam, goff, w, alg="ista", test=test, dynamic=False, max_iter=1, tol=0)
        rz = oracle.solve(Dz, y, lam, goff, np.ones(G), alg="ista", test=test, dynamic=False, max_iter=1, tol=0)
        np.testing.assert_array_equal(rx["scr_iter"] != 0, rz["scr_iter"] != 0)
        partial += 0 < np.count_nonzero(rx["scr_iter"]) < 200
    assert partial >= 2
    lam = 0.5 * lm
    rx = oracle.solve(D, y, lam, goff, w, test=test, tol=1e-14, max_iter=100000)
    rz = oracle.solve(Dz, y, lam, goff, np.ones(G), test=test, tol=1e-14, max_iter=100000)
    np.testing.assert_allclose(rx["x"], rz["x"] / wcol, atol=1e-6 * np.abs(rx["x"]).max())


# ----------------------------------------------------- Lemma 8 and Lemma 4

def test_dual_scaling_is_optimal_feasible_scaling():
    """Lemma 8: mu minimises ||s theta - y/lambda|| over feasible s (|s| m <= 1);
    checked against a fine 1-D scan."""
    g = gen.rng(16)
    for _ in range(20):
        D = gen.gaussian_dict(20, 60, g)
        y = g.standard_normal(20)
        theta = g.standard_normal(20)
        lam = g.uniform(0.1, 2.0)
        m = np.abs(D.T @ theta).max()
        mu = oracle.dual_scaling(theta, y, lam, m)
        assert abs(mu) * m <= 1 + 1e-12
        s = np.linspace(-1 / m, 1 / m, 200001)
        f = np.linalg.norm(s[:, None] * theta[None, :] - y[None, :] / lam, axis=1)
        assert np.linalg.norm(mu * theta - y / lam) <= f.min() + 1e-12


def test_dome_max_matches_numeric_maximum():
    """Lemma 4's region: the closed-form max of d^T theta over the dome agrees with
    a brute-force maximisation over the plane spanned by n and d."""
    g = gen.rng(17)
    for _ in range(200):
        t = g.uniform(-0.99, 0.99)
        R = g.uniform(0.1, 2.0)
        psi = g.uniform(0.0, R)
        dc0 = g.uniform(-1, 1)
        # coordinates: n = (1, 0), d = (t, sqrt(1 - t^2)); theta = c0 + (a, c); n^T c0 - off = psi
        ang = np.linspace(0, 2 * np.pi, 4001)
        rad = np.linspace(0, R, 801)
        A = rad[:, None] * np.cos(ang)[None, :]
        C = rad[:, None] * np.sin(ang)[None, :]
        ok = A <= -psi
        val = t * A + np.sqrt(1 - t * t) * C
        num = dc0 + val[ok].max()
        got = oracle.dome_max(dc0, t, psi, R)
        assert got >= num - 1e-9
        assert got <= num + 5e-3 * R


# ---------------------------------------------------------- spectral norms

def test_spectral_norms_match_library():
    g = gen.rng(18)
    D = gen.gaussian_dict(30, 90, g)
    L = oracle.spectral_norm_sq(D, tol=1e-14)
    assert np.isclose(L, np.linalg.norm(D, 2) ** 2, rtol=1e-9)
    # the default step constant of a solve is an upper bound of ||D||_2^2
    # (the premise of the descent lemma behind every row of Table 1)
    r = oracle.solve(D, gen.rng(19).standard_normal(30), 0.1, test="none", max_iter=1)
    assert np.linalg.norm(D, 2) ** 2 <= r["L"] <= np.linalg.norm(D, 2) ** 2 * (1 + 1e-5)
    for c0, c1 in ((0, 1), (0, 5), (10, 30), (40, 73)):
        s = oracle.group_spec_norm(D, c0, c1)
        assert np.isclose(s, np.linalg.norm(D[:, c0:c1], 2), rtol=1e-12)


def test_group_spectral_norms_of_large_groups_match_library():
    """Groups of 50 to 128 columns (the paper's group-size sweep goes to 100): the Jacobi
    value is an upper bound of ||D_g||_2 and agrees with LAPACK."""
    g = gen.rng(21)
    D = gen.gaussian_dict(200, 300, g)
    for c0, c1 in ((0, 50), (50, 150), (150, 278)):
        s = oracle.group_spec_norm(D, c0, c1)
        ref = np.linalg.norm(D[:, c0:c1], 2)
        assert s >= ref * (1 - 1e-14) and np.isclose(s, ref, rtol=1e-10)


@pytest.mark.parametrize("pair", [("safe", "gsafe"), ("dst3", "dgst3")])
def test_singleton_groups_with_unequal_norms(pair):
    """The singleton-group identity also holds for atoms of unequal norms (Lemma 7's
    sphere test with ||D_g|| = ||d_i||, Lemma 6's n = sign(b_*) d_*)."""
    D, y = _small_lasso(19, N=40, K=200)
    D = D * gen.rng(20).uniform(0.5, 2.0, size=(1, 200))
    lm, _, _ = oracle.lambda_max(D, y)
    goff = gen.contiguous_groups(200, 1)
    a = oracle.solve(D, y, 0.5 * lm, test=pair[0], tol=1e-12, max_iter=5000)
    b = oracle.solve(D, y, 0.5 * lm, goff, np.ones(200), test=pair[1], tol=1e-12, max_iter=5000)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-11)
    np.testing.assert_array_equal(a["scr_iter"], b["scr_iter"])
    assert (a["scr_iter"] != 0).sum() > 0


def test_fista_rate_bound():
    """FISTA (Table 1, l_0 = 1) satisfies Beck and Teboulle's bound
    F(x_t) - F* <= 2 L ||x_0 - x*||^2 / (t + 1)^2 at every iteration, and its first
    extrapolation is zero, so its first two iterates are ISTA's."""
    D, y = _small_lasso(21, N=60, K=150, k=6)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.1 * lm
    ref = oracle.solve(D, y, lam, test="none", tol=0, max_iter=60000)
    Fs = 0.5 * np.sum((D @ ref["x"] - y) ** 2) + lam * np.abs(ref["x"]).sum()
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    r = oracle.solve(D, y, lam, alg="fista", test="none", tol=0, max_iter=400, L=L)
    h = r["hist"]
    yy = y @ y
    F = h[:, 4] + 0.5 * yy - 0.5 * lam * lam * h[:, 2] ** 2  # primal = gap + dual
    t = np.arange(1, F.size + 1)
    assert np.all(F - Fs <= 2 * L * np.sum(ref["x"] ** 2) / (t + 1) ** 2 + 1e-12)
    ri = oracle.solve(D, y, lam, alg="ista", test="none", tol=0, max_iter=3, L=L)
    np.testing.assert_allclose(h[:2, 4], ri["hist"][:2, 4], rtol=1e-13)
    assert abs(h[2, 4] - ri["hist"][2, 4]) > 1e-10 * yy


def test_fista_rate_bound_on_the_worst_case_quadratic():
    """Beck and Teboulle's bound on Nesterov's worst-case least-squares instance,
    where it is nearly tight: D = B/2 with B the (n+1) x n first-difference
    matrix (D^T D = tridiag(-1, 2, -1)/4, ||D||^2 < 1 = L), y = e_1/2, and a
    lambda small enough that x* keeps the all-positive support, so x* solves
    D^T D x = D^T y - lambda 1 (KKT).  FISTA stays within the bound up to
    t = n/2; ISTA, whose rate is only O(1/t), exceeds it there, so a FISTA that
    lost its acceleration fails this pin."""
    n = 600
    B = np.zeros((n + 1, n))
    B[np.arange(n), np.arange(n)] = 1.0
    B[np.arange(1, n + 1), np.arange(n)] = -1.0
    D = np.asfortranarray(0.5 * B)
    y = np.zeros(n + 1)
    y[0] = 0.5
    lam = 1e-7
    xs = np.linalg.solve(D.T @ D, D.T @ y - lam)
    assert np.all(xs > 0)
    Fs = 0.5 * np.sum((D @ xs - y) ** 2) + lam * xs.sum()
    T = n // 2 - 1
    t = np.arange(1, T + 1)
    bound = 2 * 1.0 * np.sum(xs ** 2) / (t + 1) ** 2

    def excess(alg):
        h = oracle.solve(D, y, lam, alg=alg, test="none", tol=0, max_iter=T, L=1.0)["hist"]
        F = h[:, 4] + 0.5 * (y @ y) - 0.5 * lam * lam * h[:, 2] ** 2  # primal = gap + dual
        return (F - Fs) / bound

    assert np.all(excess("fista") <= 1.0)
    assert excess("ista").max() > 1.1


def _region_max(D, y, lam, lstar, star_sign_col, R, dome):
    """max_i |d_i^T theta| over {||theta - y/lambda|| <= R} (intersected with
    {d_*^T theta <= 1} for the dome) by enumerating the region's boundary in the
    plane of d_* and d_i: a linear function is maximised at an extreme point,
    i.e. on the feasible arc of the circle or at an end of the chord."""
    c0 = y / lam
    ds = star_sign_col
    e1 = ds / np.linalg.norm(ds)
    ga = D.T @ e1                                    # component of d_i along e1
    gb = np.sqrt(np.maximum(np.sum(D * D, axis=0) - ga * ga, 0.0))  # along e2(i)
    dc = D.T @ c0
    phi = np.linspace(0.0, 2 * np.pi, 40001)
    a, b = R * np.cos(phi), R * np.sin(phi)
    if dome:
        amax = (1.0 - ds @ c0) / np.linalg.norm(ds)
        keep = a <= amax
        a, b = a[keep], b[keep]
        if R * R >= amax * amax:
            h = np.sqrt(R * R - amax * amax)
            a = np.concatenate([a, [amax, amax]])
            b = np.concatenate([b, [h, -h]])
    val = dc[:, None] + ga[:, None] * a[None, :] + gb[:, None] * b[None, :]
    return np.maximum(val.max(axis=1), (-val).max(axis=1))


@pytest.mark.parametrize("test", ["safe", "dome"])
def test_static_screen_equals_brute_force_region_maximum(test):
    """Atoms of unequal norms: the static test (Sec. 2.2.2, theta = -y, so
    mu theta = y / lambda_* and R = ||y/lambda - y/lambda_*||) screens exactly
    the atoms whose maximum of |d_i^T theta| over the test region is below 1
    (SAFE: the ball, Lemma 2; Dome: the ball cut by d_*^T theta <= 1, Lemma 4),
    the maximum found by brute force; atoms within 1e-6 of 1 are not judged."""
    g = gen.rng(41)
    D = np.asfortranarray(gen.gaussian_dict(40, 300, g) * (0.5 + 1.5 * g.random(300)))
    y = g.standard_normal(40)
    lm, star, b = oracle.lambda_max(D, y)
    ds = np.sign(b[star]) * D[:, star]
    screened_any = 0
    for ratio in (0.5, 0.7, 0.85, 0.95):
        lam = ratio * lm
        R = np.linalg.norm(y / lam - y / lm)
        M = _region_max(D, y, lam, lm, ds, R, dome=test == "dome")
        r = oracle.solve(D, y, lam, alg="ista", test=test, dynamic=False, max_iter=1, tol=0)
        clear = np.abs(M - 1.0) > 1e-6
        np.testing.assert_array_equal((r["scr_iter"] == -1)[clear], (M < 1.0)[clear])
        screened_any += 0 < np.count_nonzero(M < 1.0) < 300
    assert screened_any >= 2


@pytest.mark.parametrize("alg", ["ista", "fista", "cp"])
@pytest.mark.parametrize("test", ["safe", "dst3", "dome", "gsafe", "dgst3"])
def test_every_dual_point_obeys_weak_duality(alg, test):
    """Lemma 8 makes mu_t theta_t dual feasible, so its dual value
    1/2 ||y||^2 - lambda^2/2 R_t^2 (R_t = ||y/lambda - mu_t theta_t||) never
    exceeds the primal optimum, at any iteration; atoms of unequal norms, group
    weights on both sides of 1."""
    g = gen.rng(43)
    D = np.asfortranarray(gen.gaussian_dict(40, 160, g) * (0.5 + 1.5 * g.random(160)))
    goff, w = None, None
    if test in ("gsafe", "dgst3"):
        goff = gen.contiguous_groups(160, 4)
        w = 0.5 + 1.5 * g.random(40)
        x0 = gen.group_x0(goff, 3, g)
    else:
        x0 = gen.sparse_x0(160, 5, g)
    y = gen.observe(D, x0, g, snr_db=20.0)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    yy = y @ y
    for ratio in (0.3, 0.7):
        lam = ratio * lm
        ref = oracle.solve(D, y, lam, goff, w, alg="fista", test="none", tol=1e-14, max_iter=100000)
        P_ub = ref["primal"]  # an upper bound of the optimum
        h = oracle.solve(D, y, lam, goff, w, alg=alg, test=test, tol=0, max_iter=300)["hist"]
        dual = 0.5 * yy - 0.5 * lam * lam * h[:, 2] ** 2
        assert np.all(dual <= P_ub + 1e-13 * yy)


@pytest.mark.parametrize("test", ["safe", "dst3", "dome"])
def test_chambolle_pock_first_test_is_the_static_test(test):
    """Chambolle-Pock (Table 1) starts from theta_0 = 0, so theta_1 = -sigma y / (1 + sigma) is a
    positive multiple of -y: after the dual scaling of Lemma 8 its first dynamic test is the
    static test of Algorithm 1, whatever sigma_0."""
    D, y = _small_lasso(23, N=40, K=300, k=4)
    lm, _, _ = oracle.lambda_max(D, y)
    for ratio in (0.5, 0.8):
        rs = oracle.solve(D, y, ratio * lm, alg="ista", test=test, dynamic=False, max_iter=1, tol=0)
        for sig in (0.0, 0.3, 5.0):
            rc = oracle.solve(D, y, ratio * lm, alg="cp", test=test, dynamic=True, max_iter=1, tol=0, cp_sigma=sig)
            np.testing.assert_array_equal(rc["scr_iter"] != 0, rs["scr_iter"] != 0)


def test_chambolle_pock_reaches_the_pinned_solution_and_gamma_stalls_it():
    """With gamma = 0 (phi_t = 1) Chambolle-Pock converges to the minimiser pinned by the
    KKT and brute-force tests; a positive gamma shrinks tau_t towards 0 on the Lasso (its
    penalty is not strongly convex) and the same iteration budget no longer suffices."""
    D, y = _small_lasso(24, N=60, K=200, k=5)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.3 * lm
    ref = oracle.solve(D, y, lam, alg="fista", test="none", tol=1e-14, max_iter=200000)
    r0 = oracle.solve(D, y, lam, alg="cp", test="dst3", tol=1e-12, max_iter=20000)
    assert r0["status"] == 0
    np.testing.assert_allclose(r0["x"], ref["x"], atol=1e-6 * np.abs(ref["x"]).max())
    r1 = oracle.solve(D, y, lam, alg="cp", test="dst3", tol=1e-12, max_iter=20000, cp_gamma=1.0)
    assert r1["status"] == 1
    # with tau_0 != sigma_0 (tau_0 sigma_0 ||D||^2 < 1) the fixed point is still the minimiser,
    # which fixes where each of the two steps enters the primal and the dual updates
    Ln = np.linalg.norm(D, 2) ** 2
    for tau, sigma in ((0.3, 3.0), (3.0, 0.3)):
        r2 = oracle.solve(D, y, lam, alg="cp", test="dst3", tol=1e-12, max_iter=50000,
                          cp_tau=tau / np.sqrt(Ln), cp_sigma=sigma / np.sqrt(Ln))
        assert r2["status"] == 0
        np.testing.assert_allclose(r2["x"], ref["x"], atol=1e-6 * np.abs(ref["x"]).max())


@pytest.mark.parametrize("steps", [(0.35, 2.2), (2.2, 0.35), (0.99, 0.99)])
def test_chambolle_pock_iterates_are_fejer_monotone(steps):
    """With gamma = 0, Chambolle-Pock is a proximal point method in the metric
    M = [[I/tau, -D^T], [-D, I/sigma]] (positive definite when tau sigma ||D||^2 < 1):
    for z_k = (x_{t-1}, theta_t) and the saddle point z* = (x*, D x* - y) of
    min_x max_theta theta^T D x - 1/2 ||theta||^2 - theta^T y + lambda ||x||_1,
    every step obeys ||z_{k+1} - z*||_M^2 + ||z_{k+1} - z_k||_M^2 <= ||z_k - z*||_M^2
    (firm nonexpansiveness of the resolvent), a property of every intermediate iterate."""
    g = gen.rng(51)
    D = gen.gaussian_dict(30, 90, g)
    y = gen.observe(D, gen.sparse_x0(90, 4, g), g, sigma=0.05)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.4 * lm
    Ln = np.linalg.norm(D, 2) ** 2
    tau, sigma = steps[0] / np.sqrt(Ln), steps[1] / np.sqrt(Ln)
    assert tau * sigma * Ln < 1
    xs = oracle.solve(D, y, lam, alg="fista", test="none", tol=1e-15, max_iter=200000)["x"]
    ts = D @ xs - y

    def m2(dx, dt):
        return dx @ dx / tau + dt @ dt / sigma - 2.0 * dt @ (D @ dx)

    z = [(np.zeros(90), None)]
    for t in range(1, 61):
        r = oracle.solve(D, y, lam, alg="cp", test="none", tol=0, max_iter=t, cp_tau=tau, cp_sigma=sigma)
        z[-1] = (z[-1][0], r["theta"])      # z_{t-1} = (x_{t-1}, theta_t)
        z.append((r["x"], None))
    z = z[:-1]
    d0 = m2(z[0][0] - xs, z[0][1] - ts)
    for a, b in zip(z[:-1], z[1:]):
        lhs = m2(b[0] - xs, b[1] - ts) + m2(b[0] - a[0], b[1] - a[1])
        assert lhs <= m2(a[0] - xs, a[1] - ts) + 1e-10 * d0


# ------------------------------------------------- per-atom test margins

def _unequal_norm_problem(seed, N=40, K=300):
    g = gen.rng(seed)
    D = np.asfortranarray(gen.gaussian_dict(N, K, g) * (0.5 + 1.5 * g.random(K)))
    y = D @ gen.sparse_x0(K, 4, g) + 0.05 * g.standard_normal(N)
    return D, y


@pytest.mark.parametrize("test", ["safe", "dome"])
def test_logged_margins_are_the_region_maximum(test):
    """Dynamic tests, atoms of unequal norms: the margin logged for atom i at iteration
    t is (1 - max |d_i^T theta| over the region of iteration t) / ||d_i|| (SAFE: the
    ball of radius R_t about y/lambda, Lemma 2; Dome: that ball cut by
    d_*^T theta <= 1, Lemma 4), the maximum found by brute force in the plane of d_*
    and d_i; and an atom is screened at the first iteration whose margin is positive."""
    D, y = _unequal_norm_problem(43)
    K = D.shape[1]
    lm, star, b = oracle.lambda_max(D, y)
    ds = np.sign(b[star]) * D[:, star]
    nrm = np.linalg.norm(D, axis=0)
    T = 30
    compared = screened = 0
    for ratio in (0.5, 0.8):
        lam = ratio * lm
        r = oracle.solve(D, y, lam, alg="fista", test=test, tol=0, max_iter=T, margins=T)
        M = r["margins"]
        assert M.shape == (T + 1, K) and np.all(np.isnan(M[0]))  # no static test
        for t in (1, 2, 5, 12, 30):
            mx = _region_max(D, y, lam, lm, ds, r["hist"][t - 1, 2], dome=test == "dome")
            tested = ~np.isnan(M[t])
            np.testing.assert_allclose(M[t][tested] * nrm[tested], 1.0 - mx[tested], atol=1e-6)
            compared += int(tested.sum())
        s = r["scr_iter"]
        for i in range(K):
            pos = np.flatnonzero(~np.isnan(M[1:, i]) & (M[1:, i] > 1e-12)) + 1
            if s[i] > 0:
                assert pos.size == 1 and pos[0] == s[i] and np.all(np.isnan(M[s[i] + 1:, i]))
                screened += 1
            else:
                assert pos.size == 0 and not np.any(np.isnan(M[1:, i]))
    assert compared > 1000 and screened > 10


@pytest.mark.parametrize("ratio", [0.8, 0.9])
def test_dst3_ball_lies_between_the_dome_and_its_half_space_cut(ratio):
    """Lemma 3 vs Lemma 4 from the same dual point: the DST3 sphere contains the dome
    (ball cut by d_*^T theta <= 1), so every DST3 margin is at most the dome margin;
    the dome lies in the SAFE ball, so every SAFE margin is at most the dome margin."""
    D, y = _unequal_norm_problem(44)
    D = gen._normalise(D)  # the dome needs unit atoms
    lm, _, _ = oracle.lambda_max(D, y)
    theta = D @ oracle.solve(D, y, 0.95 * lm, test="none", tol=1e-12, max_iter=50000)["x"] - y
    m = {t: oracle.sequential_screen(D, y, ratio * lm, theta, test=t) for t in ("safe", "dst3", "dome")}
    assert np.all(m["dst3"]["margins"] <= m["dome"]["margins"] + 1e-12)
    assert np.all(m["safe"]["margins"] <= m["dome"]["margins"] + 1e-12)
    assert m["dome"]["screened"].sum() >= max(m["safe"]["screened"].sum(), m["dst3"]["screened"].sum(), 1)


# ------------------------------------- sequential screening (lambda paths)

@pytest.mark.parametrize("test", ["safe", "dst3", "dome"])
def test_sequential_screen_is_safe_from_any_dual_point(test):
    """Discussion (Sec. 5), regularization paths: the dual feasible set does not
    depend on lambda, so Lemma 8's scaling of any theta over the whole dictionary
    gives a safe region at any lambda.  Tiny problems: atoms screened from the
    residual of the brute-force solution at the previous lambda, and from random
    theta, are zero in the brute-force minimiser at the next lambda."""
    screened = 0
    for seed in (61, 62, 63):
        g = gen.rng(seed)
        N, K = 6, 9
        D = gen.gaussian_dict(N, K, g)
        y = D @ gen.sparse_x0(K, 2, g) + 0.05 * g.standard_normal(N)
        lm, _, _ = oracle.lambda_max(D, y)
        ratios = (0.95, 0.8, 0.6, 0.4)
        xs = [_lasso_bruteforce(D, y, r * lm) for r in ratios]
        for k in range(1, len(ratios)):
            for theta in (D @ xs[k - 1] - y, g.standard_normal(N)):
                s = oracle.sequential_screen(D, y, ratios[k] * lm, theta, test=test)
                assert not np.any(xs[k][s["screened"]] != 0), (seed, k, test)
                screened += int(s["screened"].sum())
    assert screened > 5


@pytest.mark.parametrize("test", ["safe", "dome"])
def test_sequential_margins_are_the_region_maximum(test):
    """The sequential test's margins equal (1 - the brute-force maximum of |d_i^T theta|
    over its region) / ||d_i||, with R = ||y/lambda - mu theta||, where mu is no worse
    than any feasible scaling found by a 1-D scan (Lemma 8)."""
    D, y = _unequal_norm_problem(45)
    if test == "dome":
        D = gen._normalise(D)
    lm, star, b = oracle.lambda_max(D, y)
    ds = np.sign(b[star]) * D[:, star]
    nrm = np.linalg.norm(D, axis=0)
    theta = D @ oracle.solve(D, y, 0.9 * lm, test="none", tol=1e-12, max_iter=50000)["x"] - y
    lam = 0.7 * lm
    s = oracle.sequential_screen(D, y, lam, theta, test=test)
    m = np.abs(D.T @ theta).max()
    grid = np.linspace(-1 / m, 1 / m, 200001)
    best = np.linalg.norm(grid[:, None] * theta[None, :] - y[None, :] / lam, axis=1).min()
    assert abs(s["mu"]) * m <= 1 + 1e-12
    assert abs(s["R"] - np.linalg.norm(s["mu"] * theta - y / lam)) <= 1e-12 * s["R"]
    assert s["R"] <= best + 1e-12
    mx = _region_max(D, y, lam, lm, ds, s["R"], dome=test == "dome")
    np.testing.assert_allclose(s["margins"] * nrm, 1.0 - mx, atol=1e-6)
    assert 0 < s["screened"].sum() < D.shape[1]


@pytest.mark.parametrize("test", ["safe", "dst3", "dome", "gsafe", "dgst3"])
def test_warm_started_first_test_is_the_sequential_test(test):
    """With a warm start x_0 = u_0 = x_k (the solution at lambda_k), iteration 1's dual
    point is theta_1 = D x_k - y and its correlations cover every atom, so the test of
    iteration 1 at lambda_{k+1} screens exactly the atoms of the sequential test."""
    g = gen.rng(46)
    N, K = 50, 400
    D = gen.gaussian_dict(N, K, g)
    y = D @ gen.sparse_x0(K, 5, g) + 0.05 * g.standard_normal(N)
    goff = w = None
    if test in ("gsafe", "dgst3"):
        goff = gen.contiguous_groups(K, 4)
        w = np.full(goff.size - 1, 2.0)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    xk = oracle.solve(D, y, 0.9 * lm, goff, w, test="none", tol=1e-13, max_iter=100000)["x"]
    lam = 0.8 * lm
    r = oracle.solve(D, y, lam, goff, w, alg="fista", test=test, tol=0, max_iter=1, x0=xk, margins=1)
    s = oracle.sequential_screen(D, y, lam, D @ xk - y, goff, w, test=test)
    np.testing.assert_array_equal(r["scr_iter"] == 1, s["screened"])
    np.testing.assert_allclose(r["margins"][1], s["margins"], rtol=0, atol=1e-12)
    assert 0 < s["screened"].sum() < K


# ------------------------------------- Table 1 updates worked by hand (1 x 1)

def _soft(v, t):
    return np.sign(v) * max(abs(v) - t, 0.0)


def test_fista_first_iterates_follow_the_printed_sequence():
    """Table 1 FISTA on the 1 x 1 problem D = [d]: l_0 = 1 and
    l_t = (1 + sqrt(1 + 4 l_{t-1}^2)) / 2 give l_1 = the golden ratio, l_2 and l_3
    below; the iterates x_1 .. x_5 worked by hand from these values equal the
    oracle's.  Another O(1/t^2) momentum sequence changes x_3 onwards."""
    d, yv, lam, L = 1.3, 0.9, 0.05, 4.0
    l = [1.0, (1 + np.sqrt(5.0)) / 2, 2.193527085331, 2.749791340120]
    for t in range(1, 4):  # the printed recurrence, checked against the values above
        assert abs(l[t] - (1 + np.sqrt(1 + 4 * l[t - 1] ** 2)) / 2) < 1e-11
    l = [1.0]
    for t in range(1, 6):
        l.append((1 + np.sqrt(1 + 4 * l[-1] ** 2)) / 2)
    x_prev, u, want = 0.0, 0.0, []
    for t in range(1, 6):
        x = _soft(u - d * (d * u - yv) / L, lam / L)
        u = x + (l[t - 1] - 1) / l[t] * (x - x_prev)
        x_prev = x
        want.append(x)
    D = np.array([[d]])
    for t in range(1, 6):
        got = oracle.solve(D, np.array([yv]), lam, alg="fista", test="none", tol=0, max_iter=t, L=L)["x"][0]
        assert abs(got - want[t - 1]) <= 1e-14, (t, got, want[t - 1])


@pytest.mark.parametrize("steps", [(0.3, 0.9, 0.5), (0.0, 0.0, 0.0), (0.0, 0.0, 2.0)])
def test_chambolle_pock_first_iterates_follow_table_1(steps):
    """Table 1 Chambolle-Pock on the 1 x 1 problem D = [d], worked by hand:
    theta_t = (theta_{t-1} + sigma_{t-1} (d u_{t-1} - y)) / (1 + sigma_{t-1}),
    x_t = prox_{lambda tau_{t-1}}(x_{t-1} - tau_{t-1} d theta_t),
    phi_t = 1 / sqrt(1 + 2 gamma tau_{t-1}), tau_t = phi_t tau_{t-1},
    sigma_t = sigma_{t-1} / phi_t, u_t = x_t + phi_t (x_t - x_{t-1}), with the readings
    of the constants the paper leaves open: theta_0 = 0 and, when not given,
    tau_0 = sigma_0 = 0.99 / sqrt(L)."""
    tau0, sigma0, gamma = steps
    d, yv, lam, L = 1.3, 0.9, 0.05, 1.69 * (1 + 1e-6)
    tau = tau0 if tau0 > 0 else 0.99 / np.sqrt(L)
    sigma = sigma0 if sigma0 > 0 else 0.99 / np.sqrt(L)
    theta, x, u, want = 0.0, 0.0, 0.0, []
    for t in range(1, 6):
        theta = (theta + sigma * (d * u - yv)) / (1 + sigma)
        xn = _soft(x - tau * d * theta, lam * tau)
        phi = 1 / np.sqrt(1 + 2 * gamma * tau)
        tau, sigma = phi * tau, sigma / phi
        u = xn + phi * (xn - x)
        x = xn
        want.append((x, theta))
    D = np.array([[d]])
    for t in range(1, 6):
        r = oracle.solve(D, np.array([yv]), lam, alg="cp", test="none", tol=0, max_iter=t, L=L,
                         cp_tau=tau0, cp_sigma=sigma0, cp_gamma=gamma)
        assert abs(r["x"][0] - want[t - 1][0]) <= 1e-14, (t, r["x"][0], want[t - 1])
        assert abs(r["theta"][0] - want[t - 1][1]) <= 1e-14


# ------------------------------- adaptive steps: backtracking, SpaRSA, TwIST

ADAPTIVE = [("ista", True), ("fista", True), ("sparsa", False), ("twist", False)]


@pytest.mark.parametrize("alg,bt", ADAPTIVE)
@pytest.mark.parametrize("test", ["none", "safe", "dst3", "dome"])
def test_adaptive_steps_reach_the_brute_force_minimiser(alg, bt, test):
    """Definition 1 and Theorem 1 for the Table 1 rows whose step adapts (ISTA / FISTA with
    backtracking, SpaRSA, TwIST): the exact minimiser, and no screened atom in its support."""
    for seed in (71, 72):
        g = gen.rng(seed)
        N, K = 6, 9
        D = gen.gaussian_dict(N, K, g)
        y = D @ gen.sparse_x0(K, 2, g) + 0.05 * g.standard_normal(N)
        lm, _, _ = oracle.lambda_max(D, y)
        for ratio in (0.3, 0.7):
            xbf = _lasso_bruteforce(D, y, ratio * lm)
            r = oracle.solve(D, y, ratio * lm, alg=alg, backtracking=bt, test=test, tol=1e-16, max_iter=500000)
            np.testing.assert_allclose(r["x"], xbf, atol=1e-8)
            assert not np.any(xbf[r["scr_iter"] != 0] != 0)


@pytest.mark.parametrize("alg,bt", ADAPTIVE)
def test_adaptive_steps_group_lasso_kkt(alg, bt):
    """Group-Lasso (eq. group-lasso) with DGST3: the adaptive rows reach a point satisfying
    eq. primaldualKKT_glasso."""
    g = gen.rng(73)
    N, K = 40, 120
    D = gen.gaussian_dict(N, K, g)
    goff = gen.contiguous_groups(K, 4)
    w = g.uniform(1.0, 2.5, size=goff.size - 1)
    y = gen.observe(D, gen.group_x0(goff, 3, g), g)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.4 * lm
    r = oracle.solve(D, y, lam, goff, w, alg=alg, backtracking=bt, test="dgst3", tol=1e-14, max_iter=200000)
    c = D.T @ (y - D @ r["x"])
    for k in range(goff.size - 1):
        xs, cs = r["x"][goff[k]:goff[k + 1]], c[goff[k]:goff[k + 1]]
        if np.linalg.norm(xs) > 0:
            np.testing.assert_allclose(cs, lam * w[k] * xs / np.linalg.norm(xs), atol=1e-6 * lam)
        else:
            assert np.linalg.norm(cs) <= lam * w[k] * (1 + 1e-6)


def test_sparsa_first_iterate_is_istas_and_bb_steps_beat_ista():
    """SpaRSA (Table 1: ISTA with the Barzilai-Borwein rule): with alpha_1 = L its first
    iterate is ISTA's; on the ill-conditioned Pnoise dictionary of Sec. 4.2 its BB steps
    reach the gap tolerance in far fewer iterations than ISTA; its objective obeys the
    nonmonotone acceptance rule F(x_t) <= max of the previous 5."""
    D, y, _ = gen.lasso_problem(200, 800, seed=74, p=0.02, kind="pnoise")
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    a = oracle.solve(D, y, lam, alg="sparsa", test="none", tol=0, max_iter=1, L=L)
    b = oracle.solve(D, y, lam, alg="ista", test="none", tol=0, max_iter=1, L=L)
    np.testing.assert_allclose(a["x"], b["x"], rtol=0, atol=1e-15)
    s = oracle.solve(D, y, lam, alg="sparsa", test="dst3", tol=1e-9, max_iter=200000, L=L)
    i = oracle.solve(D, y, lam, alg="ista", test="dst3", tol=1e-9, max_iter=200000, L=L)
    assert s["status"] == 0 and 20 * s["iters"] < i["iters"]
    yy = y @ y
    h = s["hist"]
    F = np.concatenate([[0.5 * yy], h[:, 4] + 0.5 * yy - 0.5 * lam * lam * h[:, 2] ** 2])
    for t in range(1, F.size):
        assert F[t] <= F[max(0, t - 5):t].max() + 1e-12 * yy


def test_twist_is_monotone_and_fista_backtracking_obeys_its_rate():
    """TwIST with its monotone safeguard never increases F; FISTA with backtracking (eta = 2)
    satisfies Beck-Teboulle's bound F(x_t) - F* <= 2 eta L_f ||x_0 - x*||^2 / (t + 1)^2."""
    D, y = _small_lasso(75, N=60, K=150, k=6)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.2 * lm
    yy = y @ y
    ref = oracle.solve(D, y, lam, test="none", tol=1e-14, max_iter=200000)
    Fs = 0.5 * np.sum((D @ ref["x"] - y) ** 2) + lam * np.abs(ref["x"]).sum()
    tw = oracle.solve(D, y, lam, alg="twist", test="none", tol=0, max_iter=400)["hist"]
    F = tw[:, 4] + 0.5 * yy - 0.5 * lam * lam * tw[:, 2] ** 2
    assert np.all(np.diff(F) <= 1e-12 * yy) and F[-1] - Fs < 1e-6 * yy
    bt = oracle.solve(D, y, lam, alg="fista", backtracking=True, test="none", tol=0, max_iter=400)["hist"]
    F = bt[:, 4] + 0.5 * yy - 0.5 * lam * lam * bt[:, 2] ** 2
    Lf = np.linalg.norm(D, 2) ** 2
    t = np.arange(1, F.size + 1)
    assert np.all(F - Fs <= 2 * 2.0 * Lf * np.sum(ref["x"] ** 2) / (t + 1) ** 2 + 1e-12)


def test_adaptive_first_iterates_follow_the_cited_rules():
    """1 x 1 problem D = [d], worked by hand from the rules the paper cites (Table 1):
    backtracking doubles L from 1 until the quadratic model holds (for a 1 x 1 least
    squares the model is exact, so L_1 = 2 >= d^2 = 1.69); TwIST's a = rho^2 + 1,
    b = 2a / (1 + xi_1) with rho = (1 - sqrt(xi_1)) / (1 + sqrt(xi_1)) and its first step the
    shrinkage step; SpaRSA's BB value on a 1 x 1 problem is d^2."""
    d, yv, lam = 1.3, 0.9, 0.05
    D, Y = np.array([[d]]), np.array([yv])
    F = lambda x: 0.5 * (d * x - yv) ** 2 + lam * abs(x)
    # FISTA with backtracking: L_1 = 2 (1 -> 2), then fixed
    x_prev, u, l, want = 0.0, 0.0, 1.0, []
    for t in range(1, 5):
        xx = _soft(u - d * (d * u - yv) / 2.0, lam / 2.0)
        ln = (1 + np.sqrt(1 + 4 * l * l)) / 2
        u, x_prev, l = xx + (l - 1) / ln * (xx - x_prev), xx, ln
        want.append(xx)
    for t in range(1, 5):
        got = oracle.solve(D, Y, lam, alg="fista", backtracking=True, test="none", tol=0, max_iter=t)["x"][0]
        assert abs(got - want[t - 1]) <= 1e-14, (t, got, want)
    # TwIST, xi_1 = 0.1, L = d^2 (1 + 1e-6)
    L = d * d * (1 + 1e-6)
    xi = 0.1
    rho = (1 - np.sqrt(xi)) / (1 + np.sqrt(xi))
    a, b = rho * rho + 1, 2 * (rho * rho + 1) / (1 + xi)
    x2, x1 = 0.0, 0.0
    want = []
    for t in range(1, 7):
        p = _soft(x1 - d * (d * x1 - yv) / L, lam / L)
        xn = p if t == 1 else (1 - a) * x2 + (a - b) * x1 + b * p
        if t > 1 and F(xn) > F(x1):
            xn = p
        x2, x1 = x1, xn
        want.append(xn)
    for t in range(1, 7):
        got = oracle.solve(D, Y, lam, alg="twist", twist_xi1=xi, test="none", tol=0, max_iter=t, L=L)["x"][0]
        assert abs(got - want[t - 1]) <= 1e-14, (t, got, want)
    # SpaRSA: alpha_1 = L, then the BB value d^2 (accepted: the 1 x 1 model is exact)
    x, want = 0.0, []
    for t in range(1, 5):
        al = L if t == 1 else d * d
        x = _soft(x - d * (d * x - yv) / al, lam / al)
        want.append(x)
    for t in range(1, 5):
        got = oracle.solve(D, Y, lam, alg="sparsa", test="none", tol=0, max_iter=t, L=L)["x"][0]
        assert abs(got - want[t - 1]) <= 1e-14, (t, got, want)


def test_gap_every_checks_the_stopping_rule_every_k_iterations():
    D, y = _small_lasso(76)
    lm, _, _ = oracle.lambda_max(D, y)
    a = oracle.solve(D, y, 0.3 * lm, alg="fista", test="dst3", tol=1e-8, max_iter=100000)
    b = oracle.solve(D, y, 0.3 * lm, alg="fista", test="dst3", tol=1e-8, max_iter=100000, gap_every=7)
    assert b["iters"] % 7 == 0 and a["iters"] <= b["iters"] < a["iters"] + 7


@pytest.mark.parametrize("kind,seed,ratio", [("pnoise", 76, 0.3), ("ar1", 75, 0.1), ("pnoise", 77, 0.1)])
def test_sparsa_objective_obeys_the_nonmonotone_rule(kind, seed, ratio):
    """SpaRSA's acceptance test (Wright-Nowak-Figueiredo): every accepted iterate satisfies
    F(x_t) <= max of the 5 previous accepted F, over 3000 iterations on ill-conditioned
    dictionaries (Pnoise, AR(1)) where the Barzilai-Borwein step often overshoots."""
    D, y, _ = gen.lasso_problem(200, 800, seed=seed, p=0.02, kind=kind)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    yy = y @ y
    h = oracle.solve(D, y, lam, alg="sparsa", test="none", tol=0, max_iter=3000)["hist"]
    F = np.concatenate([[0.5 * yy], h[:, 4] + 0.5 * yy - 0.5 * lam * lam * h[:, 2] ** 2])
    for t in range(1, F.size):
        assert F[t] <= F[max(0, t - 5):t].max() + 1e-12 * yy, t
