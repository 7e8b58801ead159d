"""Pins for the oracle's Algorithm 1 with per-point penalties mu_k = mu w_k (em_admm_wpen):
hand-worked iterations, steps from the augmented Lagrangian with per-constraint penalties, the
reduction to Algorithm 1 for equal weights, and the optimum of problem (1) at convergence
(CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_wpen_hand_worked_example():
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "wpen_worked_example.txt"))
            if l.strip() and not l.startswith("#")]
    pts = np.array([[0.0], [4.0]])
    w = np.array([1.0, 3.0])
    for it, z_ref, rp_ref, rd_ref in rows:
        z, used, rp, rd = oracle.em_admm_wpen(pts, w, -10.0, 4.0, 0.5, int(it))
        assert used == int(it)
        assert abs(z[0] - z_ref) < 1e-14
        assert abs(rp - rp_ref) < 1e-14
        assert abs(rd - rd_ref) < 1e-14


def _lagrangian_steps_perk(pts, w, lo, hi, mu, z, y, steps):
    """Steps of ADMM on the augmented Lagrangian with penalty mu_k = mu w_k on constraint k,
    each by numerical minimisation (x_k, then z over the box, then y_k += mu_k (x_k - z))."""
    n, d = pts.shape
    muk = mu * w
    for _ in range(steps):
        x = np.zeros_like(pts)
        for k in range(n):
            f = lambda xx: (w[k] * np.linalg.norm(xx - pts[k]) + (xx - z) @ y[k]
                            + 0.5 * muk[k] * np.sum((xx - z) ** 2))
            best = None
            for x0 in (z, pts[k], z - y[k] / muk[k]):
                r = minimize(f, x0, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-15, "maxiter": 40000})
                if best is None or r.fun < best.fun:
                    best = r
            x[k] = best.x
        g = lambda zz: sum(y[k] @ (x[k] - zz) + 0.5 * muk[k] * np.sum((x[k] - zz) ** 2) for k in range(n))
        r = minimize(g, np.clip(z, lo, hi), method="L-BFGS-B", bounds=[(lo, hi)] * d,
                     options={"ftol": 1e-16, "gtol": 1e-12})
        z = r.x
        y = y + muk[:, None] * (x - z)
    return z


def test_wpen_steps_match_augmented_lagrangian():
    pts = np.array([[0.0, 0.0], [4.0, 1.0], [1.0, 5.0], [6.0, 6.0]])
    w = np.array([1.0, 0.7, 1.3, 0.4])
    lo, hi, mu = 0.5, 5.0, 0.8
    z0 = oracle.weighted_mean_start(pts, w, lo, hi)
    for steps in (1, 2, 3):
        z_ref = _lagrangian_steps_perk(pts, w, lo, hi, mu, z0.copy(), np.zeros_like(pts), steps)
        z, *_ = oracle.em_admm_wpen(pts, w, lo, hi, mu, steps)
        assert np.linalg.norm(z - z_ref) < 1e-5, (steps, z, z_ref)


def test_wpen_equal_weights_is_algorithm_1():
    # w_k = c for every k: mu_k = mu c, the radius w_k / mu_k = 1/mu equals Algorithm 1's c/(mu c),
    # and the weighted mean is the plain mean, so the iterates are Algorithm 1's at penalty mu c
    # (the residual norms differ only by the common factor c, which cancels in each ratio)
    rng = np.random.default_rng(31)
    pts = rng.uniform(0, 255, (25, 6))
    for c in (1.0, 0.37):
        w = np.full(25, c)
        for T, tol in ((1, 0.0), (17, 0.0), (300, 1e-5)):
            za, ua, rpa, rda = oracle.em_admm(pts, w, 20.0, 230.0, 0.05 * c, T, tol=tol, check_every=3)
            zw, uw, rpw, rdw = oracle.em_admm_wpen(pts, w, 20.0, 230.0, 0.05, T, tol=tol, check_every=3)
            assert ua == uw
            assert np.max(np.abs(za - zw)) <= 1e-10 * 255
            assert rpw == pytest.approx(rpa, rel=1e-8) and rdw == pytest.approx(rda, rel=1e-8)


def test_wpen_zero_weight_point_changes_nothing():
    # a point with w = 0 has no penalty and no say in z; its terms carry weight 0 in the residuals
    rng = np.random.default_rng(32)
    pts = rng.uniform(0, 255, (12, 4))
    w = rng.exponential(1.0, 12)
    z1, u1, rp1, rd1 = oracle.em_admm_wpen(pts, w, 0.0, 255.0, 0.1, 200, tol=1e-4, check_every=5)
    pts2 = np.vstack([pts, [[999.0, -5.0, 3.0, 600.0]]])
    w2 = np.append(w, 0.0)
    z2, u2, rp2, rd2 = oracle.em_admm_wpen(pts2, w2, 0.0, 255.0, 0.1, 200, tol=1e-4, check_every=5)
    assert np.array_equal(z1, z2) and u1 == u2 and rp1 == rp2 and rd1 == rd2


def test_wpen_converges_to_the_optimum_of_problem_1():
    rng = np.random.default_rng(33)
    for d, n in ((2, 5), (7, 30), (49, 60)):
        pts = rng.uniform(0, 255, (n, d))
        w = rng.exponential(1.0, n)
        z, used, *_ = oracle.em_admm_wpen(pts, w, 0.0, 255.0, 0.01, 20000, tol=1e-13, check_every=10)
        assert oracle.kkt_residual(z, pts, w, 0.0, 255.0) < 1e-6
        za, *_ = oracle.em_admm(pts, w, 0.0, 255.0, 0.005 * w.mean(), 20000)
        Fz, Fa = oracle.objective(z, pts, w), oracle.objective(za, pts, w)
        assert Fz <= Fa * (1 + 1e-9)
    # d = 1: the weighted scalar median, clamped to C
    v = rng.uniform(0, 10, 11)
    wv = rng.uniform(0.1, 1, 11)
    order = np.argsort(v)
    cum = np.cumsum(wv[order])
    med = v[order][np.searchsorted(cum, 0.5 * cum[-1])]
    z, *_ = oracle.em_admm_wpen(v[:, None], wv, -1e6, 1e6, 0.05, 5000)
    assert abs(z[0] - med) < 1e-7
    z, *_ = oracle.em_admm_wpen(v[:, None], wv, -1e6, med - 1.0, 0.05, 5000)
    assert abs(z[0] - (med - 1.0)) < 1e-9
    # the planar Fermat point (all angles below 120 degrees), embedded in R^3
    A = np.array([[0.0, 0.0, 5.0], [4.0, 0.0, 5.0], [1.0, 3.0, 5.0]])
    z, *_ = oracle.em_admm_wpen(A, np.ones(3), -1e6, 1e6, 0.5, 5000)
    u = (A - z) / np.linalg.norm(A - z, axis=1)[:, None]
    assert np.linalg.norm(u.sum(0)) <= 1e-6
    # an obtuse triangle: the minimiser is the obtuse vertex
    B = np.array([[0.0, 0.0], [10.0, 0.0], [5.0, 0.5]])
    z, *_ = oracle.em_admm_wpen(B, np.ones(3), -1e6, 1e6, 0.5, 5000)
    assert np.linalg.norm(z - B[2]) < 1e-6


def test_wpen_bruteforce_grid():
    rng = np.random.default_rng(34)
    for trial in range(3):
        pts = rng.uniform(0, 10, (5, 2))
        w = rng.uniform(0.2, 2.0, 5)
        lo, hi = 2.0, 8.0
        z, *_ = oracle.em_admm_wpen(pts, w, lo, hi, 0.2, 20000, tol=1e-13, check_every=10)
        delta = 0.01
        g = np.arange(lo, hi + delta / 2, delta)
        X, Y = np.meshgrid(g, g, indexing="ij")
        F = sum(w[k] * np.sqrt((X - pts[k, 0]) ** 2 + (Y - pts[k, 1]) ** 2) for k in range(5))
        fmin = F.min()
        Fz = oracle.objective(z, pts, w)
        assert Fz <= fmin + 1e-12
        assert Fz >= fmin - w.sum() * delta * math.sqrt(2) / 2


def test_wpen_stops_sooner_than_algorithm_1_on_nlem_problems():
    """On NLEM problems of a synthetic image at mu = 0.01 (stopping rule at 1e-4 checked every
    10 iterations, cap 300) the per-point penalties stop sooner on average than Algorithm 1."""
    g, _ = synth.noisy_image(9001, 64, 64, 20.0)
    rng = np.random.default_rng(35)
    plain, wpen = [], []
    for lin in rng.choice(64 * 64, 12, replace=False):
        pts, w, _ = oracle.nlem_problem(g, 7, 21, 200.0, int(lin))
        plain.append(oracle.em_admm(pts, w, 0.0, 255.0, 0.01, 300, tol=1e-4, check_every=10)[1])
        wpen.append(oracle.em_admm_wpen(pts, w, 0.0, 255.0, 0.01, 300, tol=1e-4, check_every=10)[1])
    assert np.mean(wpen) < 0.6 * np.mean(plain), (np.mean(wpen), np.mean(plain))


def test_wpen_batch_and_nlem_drivers():
    # the threaded drivers with penalty 1 equal em_admm_wpen per problem, bit for bit
    rng = np.random.default_rng(36)
    B, n, d = 7, 9, 4
    pts = rng.uniform(0, 255, (B, n, d)).astype(np.float32)
    w = rng.exponential(1.0, (B, n)).astype(np.float32)
    z, used, rp, rd = oracle.em_admm_batch(pts, w, 10.0, 240.0, 0.05, 200, tol=1e-4, check_every=4, nthreads=3,
                                           penalty=1)
    for b in range(B):
        zb, ub, rpb, rdb = oracle.em_admm_wpen(pts[b].astype(np.float64), w[b].astype(np.float64), 10.0, 240.0, 0.05,
                                               200, tol=1e-4, check_every=4)
        assert np.array_equal(z[b], zb) and used[b] == ub and rp[b] == rpb and rd[b] == rdb
    g, _ = synth.noisy_image(9002, 20, 17, 20.0)
    res = oracle.nlem(g, 5, 7, 200.0, 0.02, 40, tol=1e-4, check_every=5, pixels=[0, 50, 339], penalty=1)
    for i, lin in enumerate((0, 50, 339)):
        P, W_, pc = oracle.nlem_problem(g, 5, 7, 200.0, lin)
        zb, ub, *_ = oracle.em_admm_wpen(P, W_, 0.0, 255.0, 0.02, 40, tol=1e-4, check_every=5)
        assert res["out"][i] == zb[12] and res["iters_used"][i] == ub
