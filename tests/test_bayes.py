"""The surrogate of the tuner's Bayesian optimisation (strategy=bayes; the paper
tunes with Bayesian optimisation next to random search, Sec. 5.3), host only.

Pinned against things other than the library's own formulas: an independent
Gaussian-process implementation (scikit-learn, where installed), interpolation
and prior limits that any GP regression must meet, expected improvement by
numerical integration of its definition, and search behaviour on a synthetic
discrete space whose optimum is known."""

from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_2303_12374_gb300 import kl

LENGTHS = [0.05, 0.1, 0.2, 0.3, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0]


def _data(n=15, d=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d))
    y = np.sin(3 * X[:, 0]) + X[:, 1] ** 2 - X[:, 2]
    return X, y, rng.random((9, d))


@pytest.mark.parametrize("ls,noise", [(0.4, 1e-3), (1.5, 1e-6), (0.1, 1e-2)])
def test_posterior_matches_scikit_learn(ls, noise):
    gp_mod = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    X, y, Xq = _data()
    gp = gp_mod.GaussianProcessRegressor(
        kernel=kern.Matern(length_scale=ls, length_scale_bounds="fixed", nu=2.5),
        alpha=noise, normalize_y=True, optimizer=None).fit(X, y)
    m_ref, s_ref = gp.predict(Xq, return_std=True)
    m, v, used = kl.kl_bo_posterior(X, y, Xq, ls, noise)
    assert used == ls
    np.testing.assert_allclose(m, m_ref, rtol=0, atol=1e-10)
    np.testing.assert_allclose(np.sqrt(v), s_ref, rtol=0, atol=1e-7)


def test_length_scale_maximises_marginal_likelihood():
    gp_mod = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    for seed in range(3):
        X, y, Xq = _data(n=20, seed=seed)
        lml = []
        for ls in LENGTHS:
            gp = gp_mod.GaussianProcessRegressor(
                kernel=kern.Matern(length_scale=ls, length_scale_bounds="fixed", nu=2.5),
                alpha=1e-4, normalize_y=True, optimizer=None).fit(X, y)
            lml.append(gp.log_marginal_likelihood_value_)
        _, _, used = kl.kl_bo_posterior(X, y, Xq)
        assert used == LENGTHS[int(np.argmax(lml))]


def test_interpolates_observations_without_noise():
    X, y, _ = _data()
    m, v, _ = kl.kl_bo_posterior(X, y, X, 0.3, 1e-12)
    np.testing.assert_allclose(m, y, atol=1e-6)
    assert np.all(v < 1e-8 * y.var())


def test_far_from_data_is_the_prior():
    X, y, _ = _data()
    far = np.full((2, 3), 1e3)
    m, v, _ = kl.kl_bo_posterior(X, y, far, 0.3, 1e-4)
    np.testing.assert_allclose(m, y.mean(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(v, y.var(), rtol=1e-12)


def test_constant_observations():
    X, _, Xq = _data()
    y = np.full(len(X), 2.5)
    m, v, _ = kl.kl_bo_posterior(X, y, Xq, 0.5, 1e-4)
    np.testing.assert_allclose(m, 2.5, atol=1e-12)


def test_expected_improvement_is_its_integral():
    integrate = pytest.importorskip("scipy.integrate")
    X, y, C = _data()
    xi = 0.05
    m, v, ls = kl.kl_bo_posterior(X, y, C)
    choice, ei = kl.kl_bo_suggest(X, y, C, xi=xi)
    b = y.min()
    for q in range(len(C)):
        s = np.sqrt(v[q])
        dens = lambda f: np.exp(-0.5 * ((f - m[q]) / s) ** 2) / (s * np.sqrt(2 * np.pi))
        ref, _ = integrate.quad(lambda f: (b - xi - f) * dens(f), m[q] - 12 * s, b - xi)
        ref = max(ref, 0.0)
        assert abs(ei[q] - ref) <= 1e-7 * max(1.0, abs(ref)) + 1e-12, q
    assert choice == int(np.argmax(ei))


def test_expected_improvement_without_variance():
    # at an observation with (almost) no noise the variance vanishes and EI is
    # the plain improvement max(b - m - xi, 0): zero at the best observation
    X, y, _ = _data()
    _, ei = kl.kl_bo_suggest(X, y, X, xi=0.0, length_scale=0.3, noise=1e-12)
    assert np.all(ei < 1e-6)


def test_pending_points_spread_a_batch():
    X, y, C = _data(n=12, seed=4)
    first, ei0 = kl.kl_bo_suggest(X, y, C)
    second, ei1 = kl.kl_bo_suggest(X, y, C, pending=C[first:first + 1])
    assert second != first
    assert ei1[first] < 0.5 * ei0[first]


def test_invalid_arguments():
    X, y, C = _data()
    bad = y.copy()
    bad[3] = np.nan
    with pytest.raises(kl.KLError) as e:
        kl.kl_bo_posterior(X, bad, C)
    assert e.value.status == -1
    with pytest.raises(kl.KLError):
        kl.kl_bo_suggest(X, y, C[:0])
    with pytest.raises(kl.KLError):
        kl.kl_bo_posterior(X[:0], y[:0], C)
    # two identical rows with no noise: not positive definite
    X2 = np.vstack([X, X[:1]])
    y2 = np.append(y, y[0])
    with pytest.raises(kl.KLError):
        kl.kl_bo_posterior(X2, y2, C, 0.3, 1e-300)


def _grid_problem():
    g = np.array(list(itertools.product(range(8), repeat=4)), float) / 7.0
    c = np.array([0.71, 0.28, 0.43, 0.86])
    w = np.array([3.0, 1.0, 2.0, 0.5])
    f = np.log(1.0 + 10 * ((g - c) ** 2 * w).sum(1)) + 0.05 * np.sin(9 * g[:, 0] + 4 * g[:, 2])
    return g, f


@pytest.mark.parametrize("batch", [1, 4])
def test_search_finds_the_optimum_of_a_grid(batch):
    """8^4 = 4096 settings with one best: random search needs 2048 draws on
    average, the surrogate-guided search (with `batch` candidates chosen
    before their values are known) a few dozen."""
    g, f = _grid_problem()
    best = int(f.argmin())
    counts = []
    for seed in range(5):
        rng = np.random.default_rng(seed)
        seen = [int(i) for i in rng.choice(len(g), 8, replace=False)]
        while best not in seen and len(seen) < 200:
            pend = []
            for _ in range(batch):
                mask = np.ones(len(g), bool)
                mask[seen + pend] = False
                cand = np.nonzero(mask)[0]
                ch, _ = kl.kl_bo_suggest(g[seen], f[seen], g[cand],
                                         pending=g[pend] if pend else None)
                pend.append(int(cand[ch]))
            seen += pend
        counts.append(len(seen))
    assert max(counts) <= 80 * batch ** 0.5, counts
    assert np.median(counts) <= 40 * batch ** 0.5, counts


def test_convergence_summary():
    from paper_2303_12374_gb300 import tune_compare as tc
    inf = float("inf")
    runs = {("bayes", 1): [(0.5, 300.0), (0.9, inf), (1.2, 215.0), (2.0, 205.0)],
            ("random", 1): [(0.4, 250.0), (0.8, 260.0)]}
    rows = {r["strategy"]: r for r in tc.summarise(runs, 200.0)}
    b, r = rows["bayes"], rows["random"]
    assert (b["evals_to_10pct"], b["s_to_10pct"]) == (3, 1.2)
    assert (b["evals_to_5pct"], b["s_to_5pct"]) == (4, 2.0)
    assert b["evals_to_2pct"] is None and b["ok"] == 3 and b["best_us"] == 205.0
    assert r["evals_to_10pct"] is None and r["median_eval_us"] == 260.0
    assert "| bayes | 1 | 4 | 205.0 | 3 / 1.2 |" in tc.markdown(tc.summarise(runs, 200.0), 200.0)
