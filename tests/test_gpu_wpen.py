"""GPU parity of EM-ADMM with per-point penalties mu_k = rho w_k (options.penalty =
NLEM_PENALTY_WEIGHTED) against the oracle's em_admm_wpen, through the C ABI.  Tolerance as for
Algorithm 1: |z_gpu - z_oracle| <= 1e-4 * max(|z_oracle|, 1) after the same iteration count."""
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_03879_gb300 as m
    m.load_library()
    return m


@pytest.mark.parametrize("n,rho", [(1, 0.05), (100, 0.05), (200, 0.01), (441, 0.05), (441, 1.0), (896, 0.02)])
def test_wpen_batch_fixed_iters(nl, n, rho):
    # every compiled shape for d = 49 (up to 128, 192, 448 and 896 points)
    B, d, T = 6, 49, 50
    pts = synth.em_points(300 + n, np.arange(B), n, d)
    w = synth.em_weights(300 + n, np.arange(B), n)
    r = nl.em_solve_batch(_t(pts), _t(w), rho=rho, iters=T, penalty=nl.PENALTY_WEIGHTED)
    zo, used, rp, rd = oracle.em_admm_batch(pts, w, 0.0, 255.0, rho, T, penalty=1)
    assert np.all(r["iters_used"].cpu().numpy() == T)
    assert rel_err(r["x"].cpu().numpy(), zo).max() <= TOL
    assert np.allclose(r["residual"].cpu().numpy(), np.maximum(rp, rd), rtol=2e-2, atol=1e-6)


def test_wpen_batch_start_point_box_and_zero_weights(nl):
    B, n, d = 5, 150, 49
    rng = np.random.default_rng(41)
    pts = synth.em_points(41, np.arange(B), n, d)
    w = synth.em_weights(41, np.arange(B), n)
    w[:, ::7] = 0.0                        # points with no penalty and no say in z
    w[4, :] = 0.0                          # every weight zero: the weights are taken as 1
    x0 = rng.uniform(-20, 300, (B, d)).astype(np.float32)
    r = nl.em_solve_batch(_t(pts), _t(w), box=(10.0, 200.0), rho=0.1, iters=30, x0=_t(x0),
                          penalty=nl.PENALTY_WEIGHTED)
    zo, *_ = oracle.em_admm_batch(pts, w, 10.0, 200.0, 0.1, 30, z0=np.clip(x0, 10, 200), penalty=1)
    assert rel_err(r["x"].cpu().numpy(), zo).max() <= TOL


def test_wpen_batch_tolerance_mode_and_fp64_check(nl):
    B, n, d = 16, 441, 49
    pts = synth.em_points(42, np.arange(B), n, d)
    w = synth.em_weights(42, np.arange(B), n)
    rho, m = 0.05, 5
    r = nl.em_solve_batch(_t(pts), _t(w), rho=rho, iters=300, tol=1e-4, check_every=m, fp64_check=True,
                          penalty=nl.PENALTY_WEIGHTED)
    used = r["iters_used"].cpu().numpy()
    x = r["x"].cpu().numpy()
    zo, uo, *_ = oracle.em_admm_batch(pts, w, 0.0, 255.0, rho, 300, tol=1e-4, check_every=m, penalty=1)
    assert np.all((used % m == 0) | (used == 300))
    assert np.mean(used == uo) >= 0.9
    assert np.mean(used < 300) >= 0.9          # the rule, not the cap, stops them
    for b in range(B):
        z, _, rp, rd = oracle.em_admm_wpen(pts[b], w[b], 0.0, 255.0, rho, int(used[b]))
        assert rel_err(x[b], z).max() <= TOL
        if used[b] < 300:
            assert max(rp, rd) < 1e-4 * 1.05
        xb = x[b].astype(np.float64)
        assert abs(r["obj64"][b].item() - oracle.objective(xb, pts[b], w[b])) <= 1e-10 * oracle.objective(xb, pts[b], w[b])
        assert abs(r["kkt64"][b].item() - oracle.kkt_residual(xb, pts[b], w[b], 0.0, 255.0)) <= 1e-6


@pytest.mark.parametrize("H,W,S", [(40, 36, 11), (29, 33, 21), (24, 17, 15)])
def test_wpen_nlem_all_pixels(nl, H, W, S):
    g, _ = synth.noisy_image(4000 + S, H, W, 20.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=S, h=200.0, rho=0.02, iters=40, penalty=nl.PENALTY_WEIGHTED)
    ref = oracle.nlem(g, 7, S, 200.0, 0.02, 40, penalty=1)
    err = rel_err(r["out"].cpu().numpy(), ref["out"])
    assert err.max() <= TOL, err.max()


def test_wpen_nlem_noisy_patch_start_and_tolerance_replay(nl):
    g, _ = synth.noisy_image(4100, 36, 44, 30.0)
    m = 5
    r = nl.nlem_denoise(_t(g), patch=7, window=21, h=300.0, rho=0.01, iters=300, tol=1e-4, check_every=m,
                        init=nl.INIT_NOISY_PATCH, penalty=nl.PENALTY_WEIGHTED)
    used = r["iters_used"].cpu().numpy().reshape(-1)
    out = r["out"].cpu().numpy().reshape(-1)
    ref = oracle.nlem(g, 7, 21, 300.0, 0.01, 300, tol=1e-4, check_every=m, init_mode=1, penalty=1)
    assert np.mean(used == ref["iters_used"].reshape(-1)) >= 0.9
    assert np.mean(used < 300) >= 0.95
    for p in np.arange(0, 36 * 44, 29):
        rr = oracle.nlem(g, 7, 21, 300.0, 0.01, int(used[p]), init_mode=1, pixels=[p], penalty=1)
        assert rel_err(out[p], rr["out"][0]) <= TOL
        if used[p] < 300:
            assert max(rr["r_pri"][0], rr["r_dual"][0]) < 1e-4 * 1.05


def test_wpen_full_size_sampled(nl):
    """512x512, 21x21 window, 7x7 patches, tolerance 1e-4 every 10 iterations, cap 300, at the
    launch the benchmark row times: sampled pixels against the oracle replayed at the GPU's count."""
    g, _ = synth.noisy_image(2001, 512, 512, 20.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=21, h=200.0, rho=0.01, iters=300, tol=1e-4, check_every=10,
                        penalty=nl.PENALTY_WEIGHTED)
    out = r["out"].cpu().numpy().reshape(-1)
    used = r["iters_used"].cpu().numpy().reshape(-1)
    assert np.mean(used < 300) > 0.95
    rng = np.random.default_rng(5)
    pix = np.concatenate([[0, 511, 512 * 511, 512 * 512 - 1, 512 * 256 + 256], rng.choice(512 * 512, 11, False)])
    for p in pix:
        rr = oracle.nlem(g, 7, 21, 200.0, 0.01, int(used[p]), pixels=[p], penalty=1)
        assert rel_err(out[p], rr["out"][0]) <= TOL, (p, out[p], rr["out"][0])


def test_wpen_unsupported_combinations(nl):
    g = _t(np.zeros((16, 16), dtype=np.float32))
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(g, patch=5, window=5, h=100.0, penalty=nl.PENALTY_WEIGHTED)
    assert e.value.code == -5
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(g, patch=7, window=7, h=100.0, layout=nl.LAYOUT_PAIR, penalty=nl.PENALTY_WEIGHTED)
    assert e.value.code == -5
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(g, patch=7, window=7, h=100.0, iters=4, solver=nl.SOLVER_IRLS, penalty=nl.PENALTY_WEIGHTED)
    assert e.value.code == -1
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(g, patch=7, window=7, h=100.0, penalty=7)
    assert e.value.code == -1
    pts = _t(synth.em_points(1, np.arange(2), 30, 25))
    w = _t(synth.em_weights(1, np.arange(2), 30))
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch(pts, w, penalty=nl.PENALTY_WEIGHTED)
    assert e.value.code == -5
