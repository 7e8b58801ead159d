"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics, independent of the
oracle's own code (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# prox map (Sec. 2, Eqs. defprox, closed-form, proxfstar, MD)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("lam", [0.0, 0.3, 1.0, 2.5, 7.0])
def test_prox_matches_argmin_1d(lam):
    rng = np.random.default_rng(1)
    for _ in range(10):
        v, u = rng.normal(size=1) * 3, rng.normal(size=1) * 3
        res = minimize_scalar(lambda x: lam * abs(x - u[0]) + 0.5 * (x - v[0]) ** 2,
                              bounds=(-50, 50), method="bounded", options={"xatol": 1e-12})
        assert abs(oracle.prox(v, u, lam)[0] - res.x) < 1e-7


@pytest.mark.parametrize("lam", [0.2, 1.0, 4.0])
def test_prox_matches_argmin_2d(lam):
    rng = np.random.default_rng(2)
    for _ in range(8):
        v, u = rng.normal(size=2) * 2, rng.normal(size=2) * 2
        obj = lambda x: lam * np.linalg.norm(x - u) + 0.5 * np.sum((x - v) ** 2)
        best = None
        for x0 in (v, u, 0.5 * (u + v)):
            r = minimize(obj, x0, method="Nelder-Mead", options={"xatol": 1e-11, "fatol": 1e-14, "maxiter": 20000})
            if best is None or r.fun < best.fun:
                best = r
        p = oracle.prox(v, u, lam)
        assert obj(p) <= best.fun + 1e-10
        assert np.linalg.norm(p - best.x) < 1e-5


def test_prox_limits_and_moreau():
    rng = np.random.default_rng(3)
    for d in (1, 3, 49):
        v, u = rng.normal(size=d) * 5, rng.normal(size=d) * 5
        assert np.allclose(oracle.prox(v, u, 0.0), v)                 # lam = 0 gives v
        assert np.allclose(oracle.prox(v, u, 1e300), u)               # lam = inf gives u
        for lam in (0.1, 1.0, 10.0, 100.0):
            p, pc = oracle.prox(v, u, lam), oracle.prox_conj(v, u, lam)
            assert np.allclose(p + pc, v, atol=1e-12)                 # Moreau decomposition (MD)
            assert np.linalg.norm(pc) <= lam * (1 + 1e-12)            # inside the lam-ball (CF)
    # zero distance: the argmin is v itself
    v = np.array([1.0, 2.0])
    assert np.array_equal(oracle.prox(v, v, 3.0), v)


def test_box_projection():
    rng = np.random.default_rng(4)
    x = rng.normal(size=100) * 200 + 100
    p = oracle.project_box(x, 0.0, 255.0)
    assert np.array_equal(p, np.clip(x, 0.0, 255.0))
    assert np.array_equal(oracle.project_box(p, 0.0, 255.0), p)       # idempotent
    y = rng.normal(size=100) * 200 + 100
    assert np.linalg.norm(oracle.project_box(y, 0, 255) - p) <= np.linalg.norm(y - x) + 1e-12


# ---------------------------------------------------------------------------------------
# Algorithm 1: hand-worked iterations, and one step from the augmented Lagrangian
# ---------------------------------------------------------------------------------------

def test_alg1_hand_worked_example():
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "alg1_worked_example.txt"))
            if l.strip() and not l.startswith("#")]
    pts = np.array([[0.0], [10.0]])
    w = np.array([3.0, 1.0])
    for it, z_ref, rp_ref, rd_ref in rows:
        z, used, rp, rd = oracle.em_admm(pts, w, 0.0, 10.0, 1.0, int(it))
        assert used == int(it)
        assert abs(z[0] - z_ref) < 1e-14
        assert abs(rp - rp_ref) < 1e-14
        assert abs(rd - rd_ref) < 1e-14


def _lagrangian_steps(pts, w, lo, hi, mu, z, y, steps):
    """ADMM steps taken directly from the augmented Lagrangian of Sec. 2 by numerical
    minimisation (Gauss-Seidel over x_k then z, then the multiplier rule)."""
    n, d = pts.shape
    for _ in range(steps):
        x = np.zeros_like(pts)
        for k in range(n):
            f = lambda xx: (w[k] * np.linalg.norm(xx - pts[k]) + (xx - z) @ y[k]
                            + 0.5 * mu * np.sum((xx - z) ** 2))
            best = None
            for x0 in (z, pts[k], z - y[k] / mu):
                r = minimize(f, x0, method="Nelder-Mead",
                             options={"xatol": 1e-12, "fatol": 1e-15, "maxiter": 40000})
                if best is None or r.fun < best.fun:
                    best = r
            x[k] = best.x
        g = lambda zz: sum(y[k] @ (x[k] - zz) + 0.5 * mu * np.sum((x[k] - zz) ** 2) for k in range(n))
        r = minimize(g, np.clip(z, lo, hi), method="L-BFGS-B", bounds=[(lo, hi)] * d,
                     options={"ftol": 1e-16, "gtol": 1e-12})
        z = r.x
        y = y + mu * (x - z)
    return z


def test_alg1_steps_match_augmented_lagrangian():
    pts = np.array([[0.0, 0.0], [4.0, 1.0], [1.0, 5.0], [6.0, 6.0]])
    w = np.array([1.0, 0.7, 1.3, 0.4])
    lo, hi, mu = 0.5, 5.0, 0.8
    z0 = oracle.weighted_mean_start(pts, w, lo, hi)
    for steps in (1, 2, 3):
        z_ref = _lagrangian_steps(pts, w, lo, hi, mu, z0.copy(), np.zeros_like(pts), steps)
        z, *_ = oracle.em_admm(pts, w, lo, hi, mu, steps)
        assert np.linalg.norm(z - z_ref) < 1e-5, (steps, z, z_ref)


# ---------------------------------------------------------------------------------------
# closed forms of problem (1)
# ---------------------------------------------------------------------------------------

def _converged(pts, w, lo, hi, mu=None, iters=20000):
    if mu is None:
        mu = 1e-2 * max(np.sum(w), 1e-12) / len(w)
    return oracle.em_admm(pts, w, lo, hi, mu, iters)[0]


def test_single_point_is_its_projection():
    rng = np.random.default_rng(6)
    for d in (1, 4, 49):
        a = rng.uniform(-100, 400, size=(1, d))
        z = _converged(a, np.array([2.0]), 0.0, 255.0, mu=1.0, iters=200)
        assert np.allclose(z, np.clip(a[0], 0, 255), atol=1e-9)


def test_two_points_heavier_wins():
    rng = np.random.default_rng(7)
    for d in (1, 3, 25):
        a = rng.uniform(10, 240, size=(2, d))
        z = _converged(a, np.array([1.5, 1.0]), 0.0, 255.0, mu=0.05, iters=5000)
        assert np.linalg.norm(z - a[0]) < 1e-7


def _weighted_median_interval(x, w):
    o = np.argsort(x)
    xs, ws = x[o], w[o]
    c = np.cumsum(ws)
    half = 0.5 * c[-1]
    i = int(np.searchsorted(c, half - 1e-15 * c[-1]))
    if abs(c[i] - half) <= 1e-12 * c[-1] and i + 1 < len(xs):
        return xs[i], xs[i + 1]
    return xs[i], xs[i]


def test_d1_is_weighted_scalar_median():
    rng = np.random.default_rng(8)
    for trial in range(20):
        n = int(rng.integers(1, 12))
        x = rng.uniform(-50, 300, n)
        w = rng.uniform(0.1, 3.0, n)
        lo, hi = 0.0, 255.0
        z = _converged(x[:, None], w, lo, hi, mu=0.01 * w.mean(), iters=20000)[0]
        a, b = _weighted_median_interval(x, w)
        a, b = min(max(a, lo), hi), min(max(b, lo), hi)
        F = lambda t: float(np.sum(w * np.abs(t - x)))
        assert a - 1e-6 <= z <= b + 1e-6, (z, a, b)
        assert F(z) <= F(a) + 1e-7 * F(a)


def _fermat_point(A, B, C):
    """Fermat point of a triangle with all angles < 120 deg: intersection of the lines joining
    each vertex to the apex of the equilateral triangle erected outward on the opposite side."""
    def apex(P, Q, R):   # apex on side PQ, away from R
        m = 0.5 * (P + Q)
        t = np.array([-(Q - P)[1], (Q - P)[0]]) * (math.sqrt(3) / 2)
        c1, c2 = m + t, m - t
        return c1 if np.linalg.norm(c1 - R) > np.linalg.norm(c2 - R) else c2
    A1, B1 = apex(B, C, A), apex(C, A, B)
    M = np.array([A1 - A, -(B1 - B)]).T
    s = np.linalg.solve(M, B - A)
    return A + s[0] * (A1 - A)


def test_planar_fermat_point_embedded():
    rng = np.random.default_rng(9)
    found = 0
    while found < 6:
        T = rng.uniform(-5, 5, size=(3, 2))
        angs = []
        for i in range(3):
            u, v = T[(i + 1) % 3] - T[i], T[(i + 2) % 3] - T[i]
            angs.append(math.degrees(math.acos(u @ v / np.linalg.norm(u) / np.linalg.norm(v))))
        if max(angs) >= 115:
            continue
        found += 1
        F2 = _fermat_point(*T)
        d = 6
        Q, _ = np.linalg.qr(rng.normal(size=(d, 2)))        # random orthonormal 2-frame in R^6
        off = rng.uniform(-1, 1, d)
        pts = T @ Q.T + off
        z = _converged(pts, np.ones(3), -1e3, 1e3, mu=0.02, iters=20000)
        assert np.linalg.norm(z - (F2 @ Q.T + off)) < 1e-6


def test_obtuse_triangle_gives_vertex():
    T = np.array([[0.0, 0.0], [10.0, 0.0], [5.0, 0.8]])      # angle at the third vertex > 120 deg
    z = _converged(T, np.ones(3), -1e3, 1e3, mu=0.02, iters=20000)
    assert np.linalg.norm(z - T[2]) < 1e-7


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_grid(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 7))
    d = 1 + seed % 2
    pts = rng.uniform(-2, 12, (n, d))
    w = rng.uniform(0.2, 2.0, n)
    lo, hi = 0.0, 10.0
    z = _converged(pts, w, lo, hi, mu=0.02, iters=30000)
    delta = 0.01 if d == 2 else 0.0005
    g = np.arange(lo, hi + delta / 2, delta)
    grid = np.stack(np.meshgrid(*([g] * d), indexing="ij"), -1).reshape(-1, d)
    F = np.sum(w[None, :] * np.linalg.norm(grid[:, None, :] - pts[None, :, :], axis=2), axis=1)
    fmin = F.min()
    fz = oracle.objective(z, pts, w)
    assert fmin - w.sum() * delta * math.sqrt(d) / 2 - 1e-9 <= fz <= fmin + 1e-9
    assert np.all(z >= lo - 1e-12) and np.all(z <= hi + 1e-12)


# ---------------------------------------------------------------------------------------
# "minimiser = projection of the EM" (Sec. 1) holds in d = 1 and when the EM is in C, and
# fails in general for d >= 2
# ---------------------------------------------------------------------------------------

def test_projection_claim_d1():
    rng = np.random.default_rng(11)
    for _ in range(10):
        n = int(rng.integers(2, 9))
        x = rng.uniform(-100, 400, (n, 1))
        w = rng.uniform(0.1, 2, n)
        em = _converged(x, w, -1e4, 1e4, mu=0.01 * w.mean(), iters=20000)
        zc = _converged(x, w, 0.0, 255.0, mu=0.01 * w.mean(), iters=20000)
        F = lambda t: oracle.objective(t, x, w)
        assert F(zc) <= F(np.clip(em, 0, 255)) + 1e-7 * F(zc)
        assert F(np.clip(em, 0, 255)) <= F(zc) + 1e-6 * F(zc)


def test_projection_claim_interior():
    rng = np.random.default_rng(12)
    pts = rng.uniform(50, 200, (9, 5))
    w = rng.uniform(0.5, 1.5, 9)
    em = _converged(pts, w, -1e4, 1e4, mu=0.05, iters=20000)
    assert np.all((em > 0) & (em < 255))
    zc = _converged(pts, w, 0.0, 255.0, mu=0.05, iters=20000)
    assert np.linalg.norm(zc - em) < 1e-6


def test_projection_claim_counterexample():
    pts = np.array([[-1.4, 0.5], [1.3, -2.5], [3.6, 1.2]])
    w = np.array([0.7, 1.3, 1.9])
    em = _converged(pts, w, -1e6, 1e6, mu=1e-3, iters=40000)
    zc = _converged(pts, w, 0.0, 1.0, mu=1e-3, iters=40000)
    assert np.allclose(em, [3.6, 1.2], atol=1e-7)          # the EM sits on the heaviest point
    Fp = oracle.objective(np.clip(em, 0, 1), pts, w)
    Fc = oracle.objective(zc, pts, w)
    assert Fc < Fp - 0.5                                    # projecting the EM is not optimal
    assert oracle.kkt_residual(zc, pts, w, 0.0, 1.0) < 1e-8


# ---------------------------------------------------------------------------------------
# optimality and comparison with Weiszfeld / IRLS
# ---------------------------------------------------------------------------------------

def test_kkt_at_converged_solution():
    rng = np.random.default_rng(13)
    for d, n in ((2, 5), (7, 30), (49, 60)):
        pts = rng.uniform(0, 255, (n, d))
        w = rng.exponential(1.0, n)
        z = _converged(pts, w, 0.0, 255.0, mu=0.005 * w.mean(), iters=20000)
        assert oracle.kkt_residual(z, pts, w, 0.0, 255.0) < 1e-6


def test_weiszfeld_monotone_and_admm_not_worse():
    rng = np.random.default_rng(14)
    for d, n in ((2, 6), (5, 12), (25, 40)):
        pts = rng.normal(size=(n, d)) * 10
        w = rng.uniform(0.2, 2, n)
        x0 = pts.mean(0) + 0.37
        xw, F = oracle.weiszfeld(pts, w, x0, 400)
        assert np.all(np.diff(F) <= 1e-12 * F[0])           # Weiszfeld never increases F
        z = _converged(pts, w, -1e6, 1e6, mu=0.01, iters=20000)
        Fz = oracle.objective(z, pts, w)
        assert Fz <= F[-1] + 1e-9 * Fz
        assert np.linalg.norm(z - xw) < 1e-4 * (1 + np.linalg.norm(z))


def test_irls_surrogate_close_to_em():
    rng = np.random.default_rng(15)
    pts = rng.uniform(0, 255, (30, 9))
    w = rng.uniform(0.1, 1, 30)
    eps = 1e-6
    x, F = oracle.irls(pts, w, -1e6, 1e6, pts.mean(0), eps, 3000)
    z = _converged(pts, w, -1e6, 1e6, mu=0.01, iters=20000)
    Fz = oracle.objective(z, pts, w)
    assert abs(F[-1] - Fz) <= math.sqrt(eps) * w.sum() + 1e-9 * Fz
    # the surrogate (2) decreases along the IRLS iterates (majorise-minimise)
    xs = pts.mean(0)
    prev = np.inf
    for it in range(20):
        xs, _ = oracle.irls(pts, w, -1e6, 1e6, xs, eps, 1)
        Fe = float(np.sum(w * np.sqrt(np.sum((xs - pts) ** 2, 1) + eps)))
        assert Fe <= prev + 1e-9 * Fe
        prev = Fe


# ---------------------------------------------------------------------------------------
# invariances of Algorithm 1 (iterates, not only the limit)
# ---------------------------------------------------------------------------------------

def test_invariances():
    rng = np.random.default_rng(16)
    pts = rng.uniform(0, 255, (40, 9))
    w = rng.exponential(1.0, 40)
    mu, T = 0.7, 37
    z, *_ = oracle.em_admm(pts, w, 0.0, 255.0, mu, T)
    perm = rng.permutation(40)
    zp, *_ = oracle.em_admm(pts[perm], w[perm], 0.0, 255.0, mu, T)
    assert np.allclose(z, zp, rtol=0, atol=1e-9)
    za, *_ = oracle.em_admm(pts, 3.0 * w, 0.0, 255.0, 3.0 * mu, T)       # (w, mu) -> (aw, a mu)
    assert np.allclose(z, za, rtol=0, atol=1e-9)
    zs, *_ = oracle.em_admm(2.0 * pts, w, 0.0, 510.0, mu / 2.0, T)       # (a, C, mu) -> (sa, sC, mu/s)
    assert np.allclose(2.0 * z, zs, rtol=0, atol=1e-9)


def test_iters_zero_returns_projected_weighted_mean():
    rng = np.random.default_rng(17)
    pts = rng.uniform(-50, 300, (11, 4))
    w = rng.uniform(0.1, 1, 11)
    z, used, rp, rd = oracle.em_admm(pts, w, 0.0, 255.0, 1.0, 0)
    assert used == 0
    assert np.allclose(z, np.clip((w[:, None] * pts).sum(0) / w.sum(), 0, 255), atol=1e-12)


def test_tolerance_stopping_rule():
    rng = np.random.default_rng(18)
    pts = rng.uniform(0, 255, (50, 9))
    w = rng.exponential(1.0, 50)
    z, used, rp, rd = oracle.em_admm(pts, w, 0.0, 255.0, 0.01, 500, tol=1e-4, check_every=5)
    assert used % 5 == 0 and used < 500
    assert rp < 1e-4 and rd < 1e-4
    # the previous check point had not met the rule
    _, _, rp0, rd0 = oracle.em_admm(pts, w, 0.0, 255.0, 0.01, used - 5)
    assert not (rp0 < 1e-4 and rd0 < 1e-4)
    # fixed count: same iterate as tol-mode at that count
    zf, usedf, _, _ = oracle.em_admm(pts, w, 0.0, 255.0, 0.01, used)
    assert usedf == used and np.array_equal(zf, z)


# ---------------------------------------------------------------------------------------
# constraint sets beyond the box (Sec. 2 needs only a closed convex C with a simple projection)
# ---------------------------------------------------------------------------------------

def test_project_set_ball_and_boxes():
    rng = np.random.default_rng(40)
    c = np.array([3.0, -1.0])
    r = 2.5
    gx, gy = np.meshgrid(np.linspace(c[0] - r, c[0] + r, 801), np.linspace(c[1] - r, c[1] + r, 801))
    grid = np.stack([gx.ravel(), gy.ravel()], 1)
    grid = grid[np.sum((grid - c) ** 2, 1) <= r * r]
    for _ in range(20):
        x = rng.uniform(-6, 10, 2)
        p = oracle.project_set(x, oracle.SET_BALL, c, r=r)
        dmin = np.sqrt(np.min(np.sum((grid - x) ** 2, 1)))           # brute-force distance to the ball
        assert np.linalg.norm(p - c) <= r + 1e-12
        assert dmin - 2 * (2 * r / 800) <= np.linalg.norm(x - p) <= dmin + 1e-12
        assert np.allclose(oracle.project_set(p, oracle.SET_BALL, c, r=r), p, atol=1e-12)
    inside = c + np.array([0.3, -0.7])
    assert np.array_equal(oracle.project_set(inside, oracle.SET_BALL, c, r=r), inside)
    assert np.array_equal(oracle.project_set(np.array([5.0, 1.0]), oracle.SET_BALL, c, r=0.0), c)
    lo, hi = np.array([0.0, -2.0, 5.0]), np.array([1.0, 2.0, 5.0])
    x = np.array([-3.0, 0.5, 9.0])
    assert np.array_equal(oracle.project_set(x, oracle.SET_COORD_BOXES, lo, hi), np.array([0.0, 0.5, 5.0]))


def test_em_admm_set_reduces_to_known_cases():
    rng = np.random.default_rng(41)
    pts = rng.uniform(0, 255, (25, 4))
    w = rng.uniform(0.2, 1, 25)
    # equal per-coordinate bounds are the scalar box: the same iterates as em_admm
    za, ua, rpa, rda = oracle.em_admm(pts, w, 20.0, 200.0, 0.5, 60, tol=1e-6, check_every=3)
    zb, ub, rpb, rdb = oracle.em_admm_set(pts, w, oracle.SET_COORD_BOXES, np.full(4, 20.0), np.full(4, 200.0),
                                          mu=0.5, iters=60, tol=1e-6, check_every=3)
    assert np.array_equal(za, zb) and ua == ub and rpa == rpb and rda == rdb
    # a ball that holds every point changes nothing; radius 0 pins the centre
    zu, *_ = oracle.em_admm(pts, w, -1e9, 1e9, 0.5, 400)
    zl, *_ = oracle.em_admm_set(pts, w, oracle.SET_BALL, pts.mean(0), r=1e6, mu=0.5, iters=400)
    assert np.allclose(zl, zu, atol=1e-9)
    c = np.array([1.0, 2.0, 3.0, 4.0])
    z0, *_ = oracle.em_admm_set(pts, w, oracle.SET_BALL, c, r=0.0, mu=0.5, iters=30)
    assert np.allclose(z0, c, atol=1e-12)
    # d = 1 boxes: the weighted median clamped to [lo, hi]
    v = rng.uniform(0, 10, 9)
    wv = rng.uniform(0.1, 1, 9)
    order = np.argsort(v)
    cum = np.cumsum(wv[order])
    med = v[order][np.searchsorted(cum, 0.5 * cum[-1])]
    for lo, hi in ((0.0, 10.0), (med + 0.5, 12.0), (-1.0, med - 0.7)):
        z, *_ = oracle.em_admm_set(v[:, None], wv, oracle.SET_COORD_BOXES, np.array([lo]), np.array([hi]), mu=0.05,
                                   iters=4000)
        F = lambda t: float(np.sum(wv * np.abs(t - v)))
        assert F(z[0]) <= F(min(max(med, lo), hi)) * (1 + 1e-7) + 1e-9
        assert lo - 1e-12 <= z[0] <= hi + 1e-12


def test_em_admm_set_two_dimensional_brute_force():
    """d = 2: the converged objective is the minimum over a fine grid of the set, up to the grid's
    Lipschitz bound (sum w times half a grid diagonal)."""
    rng = np.random.default_rng(42)
    pts = rng.uniform(0, 10, (12, 2))
    w = rng.uniform(0.2, 1, 12)
    F = lambda Z: np.sum(w[None, :] * np.linalg.norm(Z[:, None, :] - pts[None, :, :], axis=2), axis=1)
    c, r = np.array([1.0, 1.0]), 2.0                                  # a ball away from the points
    z, *_ = oracle.em_admm_set(pts, w, oracle.SET_BALL, c, r=r, mu=0.1, iters=6000)
    gx, gy = np.meshgrid(np.linspace(-1, 3, 401), np.linspace(-1, 3, 401))
    grid = np.stack([gx.ravel(), gy.ravel()], 1)
    grid = grid[np.sum((grid - c) ** 2, 1) <= r * r]
    step = 4.0 / 400
    assert np.linalg.norm(z - c) <= r + 1e-9
    assert F(z[None])[0] <= F(grid).min() + w.sum() * step + 1e-9
    lo, hi = np.array([6.0, 0.0]), np.array([9.0, 2.0])                # a box on one side of the points
    z, *_ = oracle.em_admm_set(pts, w, oracle.SET_COORD_BOXES, lo, hi, mu=0.1, iters=6000)
    gx, gy = np.meshgrid(np.linspace(6, 9, 301), np.linspace(0, 2, 201))
    grid = np.stack([gx.ravel(), gy.ravel()], 1)
    assert np.all(z >= lo - 1e-12) and np.all(z <= hi + 1e-12)
    assert F(z[None])[0] <= F(grid).min() + w.sum() * 0.01 + 1e-9


# ---------------------------------------------------------------------------------------
# accelerated Algorithm 1 (fast ADMM with restart; Sec. 4 names accelerated ADMM as future work)
# ---------------------------------------------------------------------------------------

def test_fast_admm_starts_as_algorithm_1():
    """alpha starts at 1, so the first extrapolation has weight 0: iterations 1 and 2 are
    Algorithm 1's, bit for bit; the third differs."""
    rng = np.random.default_rng(50)
    pts = rng.uniform(0, 255, (30, 5))
    w = rng.uniform(0.1, 1, 30)
    for T in (1, 2):
        za, *_ = oracle.em_admm(pts, w, 0.0, 255.0, 0.3, T)
        zf, *_ = oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.3, T)
        assert np.array_equal(za, zf)
    za, *_ = oracle.em_admm(pts, w, 0.0, 255.0, 0.3, 3)
    zf, *_ = oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.3, 3)
    assert not np.array_equal(za, zf)


def test_fast_admm_converges_to_the_optimum():
    rng = np.random.default_rng(51)
    for trial in range(4):
        pts = rng.uniform(0, 255, (25, 6))
        w = rng.uniform(0.1, 1, 25)
        z_ref = _converged(pts, w, 20.0, 230.0, mu=0.05, iters=20000)
        zf, used, *_ = oracle.em_admm_fast(pts, w, 20.0, 230.0, 0.05, 20000, tol=1e-12, check_every=10)
        F_ref, F_f = oracle.objective(z_ref, pts, w), oracle.objective(zf, pts, w)
        assert F_f <= F_ref * (1 + 1e-9)
    # d = 1: the weighted median
    v = rng.uniform(0, 10, 11)
    wv = rng.uniform(0.1, 1, 11)
    order = np.argsort(v)
    cum = np.cumsum(wv[order])
    med = v[order][np.searchsorted(cum, 0.5 * cum[-1])]
    z, *_ = oracle.em_admm_fast(v[:, None], wv, -1e6, 1e6, 0.05, 5000)
    F = lambda t: float(np.sum(wv * np.abs(t - v)))
    assert F(z[0]) <= F(med) * (1 + 1e-9) + 1e-12
    # planar Fermat point of a triangle with all angles below 120 degrees, embedded in R^3
    A = np.array([[0.0, 0.0, 5.0], [4.0, 0.0, 5.0], [1.0, 3.0, 5.0]])
    z, *_ = oracle.em_admm_fast(A, np.ones(3), -1e6, 1e6, 0.5, 5000)
    u = (A - z) / np.linalg.norm(A - z, axis=1)[:, None]
    assert np.linalg.norm(u.sum(0)) <= 1e-6                 # unit vectors to the vertices sum to zero


def test_fast_admm_needs_fewer_iterations_at_large_mu():
    """On NLEM problems of a synthetic image at mu = 1 (the stopping rule at 1e-4, checked every 10
    iterations, cap 300) the accelerated variant stops sooner on average than Algorithm 1."""
    g, _ = synth.noisy_image(9001, 64, 64, 20.0)
    rng = np.random.default_rng(52)
    plain, fast = [], []
    for lin in rng.choice(64 * 64, 16, replace=False):
        pts, w, _ = oracle.nlem_problem(g, 7, 21, 200.0, int(lin))
        plain.append(oracle.em_admm(pts, w, 0.0, 255.0, 1.0, 300, tol=1e-4, check_every=10)[1])
        fast.append(oracle.em_admm_fast(pts, w, 0.0, 255.0, 1.0, 300, tol=1e-4, check_every=10)[1])
    assert np.mean(fast) < 0.75 * np.mean(plain), (np.mean(fast), np.mean(plain))


def test_fast_admm_fixed_restart_periods_1_and_2_replay_algorithm_1():
    """With a fixed restart period the schedule is known in closed form.  A restart sets alpha = 1,
    and the momentum weight (alpha - 1) / alpha+ is 0 at alpha = 1, so with periods 1 and 2 no step
    ever extrapolates: period 1 redoes every step once from the previous iterate, so iteration 2m
    ends at Algorithm 1's iterate m; period 2 ends iteration 2m at Algorithm 1's iterate m + 1.
    Both hold bit for bit and count one restart per period."""
    rng = np.random.default_rng(53)
    pts = rng.uniform(0, 255, (40, 6))
    w = rng.uniform(0.05, 1, 40)
    for m in (1, 2, 5, 9):
        za, *_ = oracle.em_admm(pts, w, 10.0, 240.0, 0.2, m)
        z1, used, _, _, rest = oracle.em_admm_fast(pts, w, 10.0, 240.0, 0.2, 2 * m, restart_every=1)
        assert np.array_equal(z1, za) and used == 2 * m and rest == 2 * m
        za1, *_ = oracle.em_admm(pts, w, 10.0, 240.0, 0.2, m + 1)
        z2, _, _, _, rest2 = oracle.em_admm_fast(pts, w, 10.0, 240.0, 0.2, 2 * m, restart_every=2)
        assert np.array_equal(z2, za1) and rest2 == m
    # period 3 is the first that extrapolates: it leaves Algorithm 1 at iteration 3
    za, *_ = oracle.em_admm(pts, w, 10.0, 240.0, 0.2, 3)
    z3, *_ = oracle.em_admm_fast(pts, w, 10.0, 240.0, 0.2, 3, restart_every=3)
    assert not np.array_equal(z3, za)


def test_fast_admm_period_beyond_the_run_never_restarts():
    """A period longer than the run takes the momentum at every step, as the residual test does
    when it can never fail (eta so large that c < eta c_prev always holds)."""
    rng = np.random.default_rng(54)
    pts = rng.uniform(0, 255, (30, 4))
    w = rng.uniform(0.1, 1, 30)
    zk, _, _, _, rk = oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.5, 40, restart_every=41)
    ze, _, _, _, re_ = oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.5, 40, eta=1e300)
    assert rk == 0 and re_ == 0 and np.array_equal(zk, ze)


def test_fast_admm_hand_worked_example():
    """Iterates of the accelerated method worked by hand (derivation in the golden file): with a fixed
    period of 3 the first extrapolated step puts z at -0.125 - 0.625 beta, beta = (phi - 1) / alpha+,
    which pins the momentum weight; under the residual rule the restarts at iterations 2-5 pin that c
    is measured against the step's start z^ and that a restart resumes from the previous iterate."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fast_admm_worked_example.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 11
    pts = np.array([[0.0], [10.0]])
    w = np.array([3.0, 1.0])
    for period, it, z_ref, rest_ref in rows:
        z, used, _, _, rest = oracle.em_admm_fast(pts, w, -10.0, 20.0, 1.0, int(it), restart_every=int(period))
        assert used == int(it)
        assert abs(z[0] - float(z_ref)) < 1e-14, (period, it, z[0], z_ref)
        assert rest == int(rest_ref), (period, it, rest, rest_ref)


def test_fast_admm_decision_margin_limits():
    """The decision margin (a diagnostic of how near the run came to deciding the other way) is
    +inf where no decision compares two finite residuals: one iteration, or a fixed period."""
    rng = np.random.default_rng(55)
    pts = rng.uniform(0, 255, (20, 3))
    w = rng.uniform(0.1, 1, 20)
    assert oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.1, 1, with_margin=True)[5] == np.inf
    assert oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.1, 30, restart_every=4, with_margin=True)[5] == np.inf
    m = oracle.em_admm_fast(pts, w, 0.0, 255.0, 0.1, 30, with_margin=True)[5]
    assert 0.0 <= m < np.inf


# ---------------------------------------------------------------------------------------
# the optimality residual at points that are NOT optimal (reading C7), worked by hand
# ---------------------------------------------------------------------------------------

def test_kkt_residual_interior_point_by_hand():
    # z = 0, a_1 = (3, 0), a_2 = (0, 4), a_3 = (-5, 0), w = (1, 1, 3): the unit vectors
    # (z - a_k)/||z - a_k|| are (-1, 0), (0, -1), (1, 0), so g = (2, -1) and sum w = 5.
    # z - g / sum w = (-0.4, 0.2); inside the box nothing clamps and R = sqrt(0.2).
    z = np.zeros(2)
    pts = np.array([[3.0, 0.0], [0.0, 4.0], [-5.0, 0.0]])
    w = np.array([1.0, 1.0, 3.0])
    assert oracle.kkt_residual(z, pts, w, -10.0, 10.0) == pytest.approx(math.sqrt(0.2), rel=1e-14)
    # dropping the division by sum w would give ||g|| = sqrt(5); the scale is fixed by the
    # gradient of problem (1): its central finite difference has the same norm as g here
    h = 1e-6
    grad = np.array([(oracle.objective(z + h * e, pts, w) - oracle.objective(z - h * e, pts, w)) / (2 * h)
                     for e in np.eye(2)])
    assert np.allclose(grad, [2.0, -1.0], atol=1e-8)
    assert oracle.kkt_residual(z, pts, w, -10.0, 10.0) == pytest.approx(np.linalg.norm(grad) / 5.0, rel=1e-7)


def test_kkt_residual_with_active_bound_by_hand():
    # the same points with z on the lower face of C = [0, 10]^2: z - g / sum w = (-0.4, 0.2)
    # clamps to (0, 0.2), so R = 0.2.  A flipped sign of g would step to (0.4, -0.2), clamp to
    # (0.4, 0) and give 0.4; the lower bound only blocks the descent direction -g.
    z = np.zeros(2)
    pts = np.array([[3.0, 0.0], [0.0, 4.0], [-5.0, 0.0]])
    w = np.array([1.0, 1.0, 3.0])
    assert oracle.kkt_residual(z, pts, w, 0.0, 10.0) == pytest.approx(0.2, rel=1e-14)
    # on the upper face C = [-10, 0]^2 the step clamps to (-0.4, 0): R = 0.4
    assert oracle.kkt_residual(z, pts, w, -10.0, 0.0) == pytest.approx(0.4, rel=1e-14)
    # d = 1: points -2, -1, 5 with unit weights give g = 1 + 1 - 1 = 1 at z = 0, so the step
    # z - g / 3 = -1/3 leaves [0, 10] and clamps back to z: the clamped median 0 is optimal, R = 0
    assert oracle.kkt_residual(np.array([0.0]), np.array([[-2.0], [-1.0], [5.0]]), np.array([1.0, 1.0, 1.0]),
                               0.0, 10.0) == 0.0


def test_kkt_residual_at_a_data_point_by_hand():
    # z coincides with a_1 (weight w_1): the subgradient of w_1 ||z - a_1|| at z is the ball of
    # radius w_1, so the residual uses g reduced in norm by w_1.  With a_2 = (4, 0), w_2 = 1 and
    # a_3 = (0, -2), w_3 = 2, the other points give g = (-1, 0) + 2 (0, 1) = (-1, 2), ||g|| = sqrt 5.
    z = np.zeros(2)
    pts = np.array([[0.0, 0.0], [4.0, 0.0], [0.0, -2.0]])
    # w_1 = 1.5 < sqrt 5: R = (sqrt 5 - 1.5) / (1.5 + 1 + 2) inside the box
    w = np.array([1.5, 1.0, 2.0])
    assert oracle.kkt_residual(z, pts, w, -10.0, 10.0) == pytest.approx((math.sqrt(5) - 1.5) / 4.5, rel=1e-14)
    # w_1 = 3 >= sqrt 5: the data point is the minimiser (the vertex condition of the Fermat-Weber
    # problem), so the residual is exactly 0; the objective confirms it is no worse than nearby points
    w = np.array([3.0, 1.0, 2.0])
    assert oracle.kkt_residual(z, pts, w, -10.0, 10.0) == 0.0
    F0 = oracle.objective(z, pts, w)
    rng = np.random.default_rng(3)
    for _ in range(50):
        assert oracle.objective(rng.normal(size=2) * 0.05, pts, w) >= F0
    # just above the vertex threshold the point stops being optimal
    w = np.array([math.sqrt(5) - 0.01, 1.0, 2.0])
    assert oracle.kkt_residual(z, pts, w, -10.0, 10.0) == pytest.approx(0.01 / (math.sqrt(5) + 2.99), rel=1e-12)


# ---------------------------------------------------------------------------------------
# the threaded batch driver against the single-problem solver
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("nthreads", [1, 4, 5])
def test_em_admm_batch_equals_single_problem_runs(nthreads):
    # B = 13 problems (not a multiple of the thread count), a start point per problem, the
    # tolerance rule and a box other than [0, 255]: every output equals Algorithm 1 run on that
    # problem alone from its float32 inputs widened to double, bit for bit.
    rng = np.random.default_rng(21)
    B, n, d = 13, 9, 4
    pts = rng.uniform(0, 255, (B, n, d)).astype(np.float32)
    w = rng.exponential(1.0, (B, n)).astype(np.float32)
    z0 = rng.uniform(0, 255, (B, d)).astype(np.float32)
    lo, hi, mu = 20.0, 190.0, 0.05
    z, used, rp, rd = oracle.em_admm_batch(pts, w, lo, hi, mu, 400, z0=z0, tol=1e-3, check_every=3,
                                           nthreads=nthreads)
    stopped_early = 0
    for b in range(B):
        zb, ub, rpb, rdb = oracle.em_admm(pts[b].astype(np.float64), w[b].astype(np.float64), lo, hi, mu, 400,
                                          z0=z0[b].astype(np.float64), tol=1e-3, check_every=3)
        assert np.array_equal(z[b], zb)
        assert used[b] == ub and rp[b] == rpb and rd[b] == rdb
        stopped_early += ub < 400
    assert stopped_early >= B // 2          # the tolerance path is exercised
    # without a start point the batch starts from the projected weighted mean, as em_admm does
    z, used, _, _ = oracle.em_admm_batch(pts, w, lo, hi, mu, 7, nthreads=nthreads)
    for b in range(B):
        zb, ub, _, _ = oracle.em_admm(pts[b].astype(np.float64), w[b].astype(np.float64), lo, hi, mu, 7)
        assert np.array_equal(z[b], zb) and used[b] == ub
