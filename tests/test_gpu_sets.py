"""Standalone batches over constraint sets beyond the box (Algorithm 1 with another projection,
Sec. 2): per-coordinate boxes and Euclidean balls, against the FP64 oracle's em_admm_set.
Tolerance as for every FP32 path: |x_gpu - x_oracle| <= 1e-4 * max(|x_oracle|, 1)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
DEV = "cuda:0"


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_03879_gb300 as m
    m.load_library()
    return m


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


# every runtime-dimension shape (d <= 28, 60, 120, 148), sizes up to each one's capacity
@pytest.mark.parametrize("n,d", [(500, 9), (441, 25), (256, 49), (441, 49), (800, 49), (200, 100), (256, 147),
                                 (33, 2)])
def test_coordinate_boxes_against_oracle(nl, n, d):
    B = 12
    pts = synth.em_points(7100 + d, np.arange(B), n, d)
    w = synth.em_weights(7100 + d, np.arange(B), n)
    rng = np.random.default_rng(7100 + d)
    lo = rng.uniform(0, 120, d).astype(np.float32)
    hi = (lo + rng.uniform(5, 120, d)).astype(np.float32)
    r = nl.em_solve_batch_set(_t(pts), _t(w), lo=_t(lo), hi=_t(hi), rho=1.0, iters=50)
    x = r["x"].cpu().numpy()
    assert np.all(x >= lo - 1e-6) and np.all(x <= hi + 1e-6)
    for b in range(0, B, 3):
        z, *_ = oracle.em_admm_set(pts[b], w[b], oracle.SET_COORD_BOXES, lo, hi, mu=1.0, iters=50)
        assert rel_err(x[b], z).max() <= TOL
    assert np.all(r["iters_used"].cpu().numpy() == 50)


@pytest.mark.parametrize("n,d,radius", [(256, 49, 40.0), (441, 49, 40.0), (256, 147, 150.0), (100, 5, 0.0),
                                        (250, 60, 1e4)])
def test_ball_against_oracle(nl, n, d, radius):
    """A ball centred away from the points (the solution on its sphere), a zero radius (the centre)
    and a radius holding every point (the unconstrained median)."""
    B = 10
    pts = synth.em_points(7200 + d, np.arange(B), n, d)
    w = synth.em_weights(7200 + d, np.arange(B), n)
    c = np.full(d, 40.0, np.float32)
    r = nl.em_solve_batch_set(_t(pts), _t(w), center=_t(c), radius=radius, rho=1.0, iters=60)
    x = r["x"].cpu().numpy()
    assert np.all(np.linalg.norm(x - c, axis=1) <= radius * (1 + 1e-6) + 1e-4)
    for b in range(0, B, 3):
        z, *_ = oracle.em_admm_set(pts[b], w[b], oracle.SET_BALL, c, r=radius, mu=1.0, iters=60)
        assert rel_err(x[b], z).max() <= TOL


def test_sets_tolerance_mode_and_start_points(nl):
    """Tolerance mode (each problem stops at its own check) and caller start points, projected onto
    the set before the first iteration."""
    B, n, d = 16, 200, 30
    pts = synth.em_points(7300, np.arange(B), n, d)
    w = synth.em_weights(7300, np.arange(B), n)
    c = np.full(d, 120.0, np.float32)
    x0 = (pts[:, 0, :] + 50.0).astype(np.float32)
    r = nl.em_solve_batch_set(_t(pts), _t(w), center=_t(c), radius=60.0, rho=1e-2, iters=400, x0=_t(x0), tol=1e-4,
                              check_every=5)
    used = r["iters_used"].cpu().numpy()
    x = r["x"].cpu().numpy()
    for b in range(0, B, 4):
        z0 = oracle.project_set(x0[b], oracle.SET_BALL, c, r=60.0)
        z, u, *_ = oracle.em_admm_set(pts[b], w[b], oracle.SET_BALL, c, r=60.0, mu=1e-2, iters=int(used[b]), z0=z0)
        assert rel_err(x[b], z).max() <= TOL
    assert np.all(used % 5 == 0) and np.all(used >= 5)
    lo = np.zeros(d, np.float32)
    hi = np.full(d, 100.0, np.float32)
    s = nl.em_solve_batch_set(_t(pts), _t(w), lo=_t(lo), hi=_t(hi), rho=1.0, iters=20, x0=_t(x0))
    for b in range(0, B, 5):
        z, *_ = oracle.em_admm_set(pts[b], w[b], oracle.SET_COORD_BOXES, lo, hi, mu=1.0, iters=20,
                                   z0=np.clip(x0[b], 0.0, 100.0))
        assert rel_err(s["x"][b].cpu().numpy(), z).max() <= TOL


def test_sets_equal_bounds_match_the_box_kernel(nl):
    """Per-coordinate bounds all equal to [lo, hi] are the paper's box: the same problem through
    em_solve_batch agrees up to FP32 rounding order."""
    B, n, d = 8, 256, 49
    pts = synth.em_points(7400, np.arange(B), n, d)
    w = synth.em_weights(7400, np.arange(B), n)
    a = nl.em_solve_batch_set(_t(pts), _t(w), lo=_t(np.full(d, 10.0)), hi=_t(np.full(d, 200.0)), rho=1.0, iters=80)
    b = nl.em_solve_batch(_t(pts), _t(w), box=(10.0, 200.0), rho=1.0, iters=80)
    assert rel_err(a["x"].cpu().numpy(), b["x"].cpu().numpy()).max() <= TOL


def test_sets_argument_errors(nl):
    pts = torch.zeros((2, 5, 3), device=DEV)
    w = torch.ones((2, 5), device=DEV)
    c = torch.zeros(3, device=DEV)
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch_set(pts, w, center=c, radius=-1.0)
    assert e.value.code == -1
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch_set(pts, w, center=c, radius=float("inf"))
    assert e.value.code == -1
    with pytest.raises(nl.NlemError) as e:          # above the 256 points of the d = 29..148 shapes
        nl.em_solve_batch_set(torch.zeros((1, 300, 40), device=DEV), torch.ones((1, 300), device=DEV),
                              center=torch.zeros(40, device=DEV), radius=1.0)
    assert e.value.code == -5
    r = nl.em_solve_batch_set(pts[:0], w[:0], center=c, radius=1.0)
    assert r["x"].shape == (0, 3)
