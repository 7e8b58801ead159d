"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerance for the FP32 path after a fixed iteration count:
|z_gpu - z_oracle| <= 1e-4 * max(|z_oracle|, 1) per output coordinate / pixel."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


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


DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# ---------------------------------------------------------------------------------------
# standalone batches
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,d", [(1, 1), (2, 3), (7, 1), (33, 2), (121, 49), (441, 49), (700, 49), (64, 25),
                                 (441, 25), (300, 81), (441, 81), (50, 10), (200, 60), (90, 100), (128, 120)])
def test_em_batch_fixed_iters(nl, n, d):
    B = 6
    pts = synth.em_points(100 + n, np.arange(B), n, d)
    w = synth.em_weights(100 + n, np.arange(B), n)
    T = 40
    r = nl.em_solve_batch(_t(pts), _t(w), rho=1.0, iters=T)
    zo, used, rp, rd = oracle.em_admm_batch(pts, w, 0.0, 255.0, 1.0, T)
    assert np.all(r["iters_used"].cpu().numpy() == T)
    assert rel_err(r["x"].cpu().numpy(), zo).max() <= TOL
    # residual output = max(r_pri, r_dual) of the last iteration
    ro = np.maximum(rp, rd)
    assert np.allclose(r["residual"].cpu().numpy(), ro, rtol=2e-2, atol=1e-6)


@pytest.mark.parametrize("rho", [1e-3, 0.05, 1.0, 20.0])
def test_em_batch_rho_range(nl, rho):
    B, n, d = 5, 441, 49
    pts = synth.em_points(7, np.arange(B), n, d)
    w = synth.em_weights(7, np.arange(B), n)
    r = nl.em_solve_batch(_t(pts), _t(w), rho=rho, iters=60)
    zo, *_ = oracle.em_admm_batch(pts, w, 0.0, 255.0, rho, 60)
    assert rel_err(r["x"].cpu().numpy(), zo).max() <= TOL


def test_em_batch_start_point_and_box(nl):
    B, n, d = 4, 100, 49
    rng = np.random.default_rng(3)
    pts = synth.em_points(8, np.arange(B), n, d)
    w = synth.em_weights(8, np.arange(B), n)
    x0 = rng.uniform(-20, 300, (B, d)).astype(np.float32)
    r = nl.em_solve_batch(_t(pts), _t(w), box=(10.0, 200.0), rho=0.3, iters=25, x0=_t(x0))
    zo, *_ = oracle.em_admm_batch(pts, w, 10.0, 200.0, 0.3, 25, z0=np.clip(x0, 10, 200))
    assert rel_err(r["x"].cpu().numpy(), zo).max() <= TOL


def test_em_iters_zero_and_single(nl):
    B, n, d = 3, 41, 49
    pts = synth.em_points(9, np.arange(B), n, d)
    w = synth.em_weights(9, np.arange(B), n)
    r = nl.em_solve_batch(_t(pts), _t(w), iters=0)
    zo, *_ = oracle.em_admm_batch(pts, w, 0.0, 255.0, 1.0, 0)
    assert rel_err(r["x"].cpu().numpy(), zo).max() <= 1e-6
    x = nl.em_solve(_t(pts[1]), _t(w[1]), rho=0.5, iters=33)
    z1, *_ = oracle.em_admm(pts[1], w[1], 0.0, 255.0, 0.5, 33)
    assert rel_err(x.cpu().numpy(), z1).max() <= TOL


def test_em_zero_weights_and_invalid_inputs(nl):
    B, n, d = 3, 20, 49
    pts = synth.em_points(10, np.arange(B), n, d)
    w = synth.em_weights(10, np.arange(B), n)
    w[0] = 0.0                    # all weights zero: plain-mean start, lam = 0
    pts[1, 3, 5] = np.nan         # non-finite point
    w[2, 4] = -1.0                # negative weight
    r = nl.em_solve_batch(_t(pts), _t(w), iters=10)
    used = r["iters_used"].cpu().numpy()
    x = r["x"].cpu().numpy()
    assert used[0] == 10 and used[1] == -1 and used[2] == -1
    assert np.all(np.isnan(x[1])) and np.all(np.isnan(x[2]))
    zo, *_ = oracle.em_admm_batch(pts[:1], w[:1], 0.0, 255.0, 1.0, 10)
    assert rel_err(x[0], zo[0]).max() <= TOL


def test_em_tolerance_mode(nl):
    B, n, d = 16, 441, 49
    pts = synth.em_points(11, np.arange(B), n, d)
    w = synth.em_weights(11, np.arange(B), n)
    rho, m = 0.02, 5
    r = nl.em_solve_batch(_t(pts), _t(w), rho=rho, iters=300, tol=1e-4, check_every=m)
    used = r["iters_used"].cpu().numpy()
    x = r["x"].cpu().numpy()
    zo, uo, rpo, rdo = oracle.em_admm_batch(pts, w, 0.0, 255.0, rho, 300, tol=1e-4, check_every=m)
    assert np.all((used % m == 0) | (used == 300))
    assert np.mean(used == uo) >= 0.9
    for b in range(B):
        # replay the oracle for exactly the GPU's iteration count
        z, _, rp, rd = oracle.em_admm(pts[b], w[b], 0.0, 255.0, rho, int(used[b]))
        assert rel_err(x[b], z).max() <= TOL
        if used[b] < 300:
            assert max(rp, rd) < 1e-4 * 1.05


def test_em_fp64_check(nl):
    B, n, d = 4, 200, 49
    pts = synth.em_points(12, np.arange(B), n, d)
    w = synth.em_weights(12, np.arange(B), n)
    r = nl.em_solve_batch(_t(pts), _t(w), rho=0.01, iters=200, fp64_check=True)
    x = r["x"].cpu().numpy().astype(np.float64)
    for b in range(B):
        F = oracle.objective(x[b], pts[b], w[b])
        R = oracle.kkt_residual(x[b], pts[b], w[b], 0.0, 255.0)
        assert abs(r["obj64"][b].item() - F) <= 1e-10 * F
        assert abs(r["kkt64"][b].item() - R) <= 1e-8 * max(R, 1.0)


def test_em_permutation_invariance(nl):
    B, n, d = 2, 300, 49
    pts = synth.em_points(13, np.arange(B), n, d)
    w = synth.em_weights(13, np.arange(B), n)
    perm = np.random.default_rng(0).permutation(n)
    a = nl.em_solve_batch(_t(pts), _t(w), iters=50)["x"].cpu().numpy()
    b = nl.em_solve_batch(_t(pts[:, perm]), _t(w[:, perm]), iters=50)["x"].cpu().numpy()
    assert rel_err(a, b).max() <= TOL


# ---------------------------------------------------------------------------------------
# NLEM
# ---------------------------------------------------------------------------------------

def test_nlem_64x64_all_pixels(nl):
    """64x64, sigma=20, 7x7 patches, 11x11 window, h=200, rho=1, 100 iterations, weighted-
    mean start: every one of the 4096 pixels against the oracle."""
    g, f = synth.noisy_image(1001, 64, 64, 20.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=11, h=200.0, rho=1.0, iters=100)
    ref = oracle.nlem(g, 7, 11, 200.0, 1.0, 100)
    err = rel_err(r["out"].cpu().numpy(), ref["out"])
    assert err.max() <= TOL, err.max()
    assert np.all(r["iters_used"].cpu().numpy() == 100)
    assert synth.psnr(r["out"].cpu().numpy(), f) > synth.psnr(g, f) + 4


@pytest.mark.parametrize("H,W,k,S,init", [(23, 31, 5, 9, 0), (17, 13, 7, 21, 0), (30, 30, 9, 11, 1),
                                          (40, 37, 7, 15, 1), (20, 26, 5, 21, 0), (12, 12, 9, 21, 0)])
def test_nlem_shapes_and_borders(nl, H, W, k, S, init):
    g, _ = synth.noisy_image(1100 + H + W, H, W, 25.0)
    h = 250.0
    r = nl.nlem_denoise(_t(g), patch=k, window=S, h=h, rho=0.5, iters=30, init=init)
    ref = oracle.nlem(g, k, S, h, 0.5, 30, init_mode=init)
    err = rel_err(r["out"].cpu().numpy(), ref["out"])
    assert err.max() <= TOL, err.max()


def test_nlem_tolerance_mode_replay(nl):
    g, _ = synth.noisy_image(1201, 48, 40, 20.0)
    m = 5
    r = nl.nlem_denoise(_t(g), patch=7, window=21, h=200.0, rho=1e-3, iters=300, tol=1e-4, check_every=m)
    used = r["iters_used"].cpu().numpy().reshape(-1)
    out = r["out"].cpu().numpy().reshape(-1)
    ref = oracle.nlem(g, 7, 21, 200.0, 1e-3, 300, tol=1e-4, check_every=m)
    assert np.mean(used == ref["iters_used"].reshape(-1)) >= 0.9
    pix = np.arange(0, 48 * 40, 37)
    resid = r["residual"].cpu().numpy().reshape(-1)
    for p in pix:
        rr = oracle.nlem(g, 7, 21, 200.0, 1e-3, int(used[p]), pixels=[p])
        assert rel_err(out[p], rr["out"][0]) <= TOL
        ro = max(rr["r_pri"][0], rr["r_dual"][0])
        if used[p] < 300:             # stopped by the rule: the oracle agrees it had converged
            assert ro < 1e-4 * 1.05
        else:                         # stopped by the cap: same residual as the oracle's
            assert abs(resid[p] - ro) <= 2e-2 * ro


def test_nlem_fp64_check_and_invariants(nl):
    g = np.full((16, 18), 77.25, dtype=np.float32)
    r = nl.nlem_denoise(_t(g), patch=5, window=7, h=100.0, iters=20, fp64_check=True)
    assert np.allclose(r["out"].cpu().numpy(), 77.25, atol=1e-4)
    assert np.all(r["kkt64"].cpu().numpy() < 1e-3)
    g2, _ = synth.noisy_image(1301, 14, 15, 30.0)
    r2 = nl.nlem_denoise(_t(g2), patch=7, window=1, h=300.0, iters=10)
    assert np.allclose(r2["out"].cpu().numpy(), np.clip(g2, 0, 255), atol=1e-3)


def test_nlem_full_size_sampled(nl):
    """512x512, 21x21 window, 7x7 patches, rho=1, tolerance 1e-4 with the 300 cap (the
    production workload): sampled pixels against the oracle replayed at the GPU's count."""
    for sigma in (10.0, 40.0):
        g, _ = synth.noisy_image(2001, 512, 512, sigma)
        r = nl.nlem_denoise(_t(g), patch=7, window=21, h=10 * sigma, rho=1.0, iters=300, tol=1e-4,
                            check_every=10)
        out = r["out"].cpu().numpy().reshape(-1)
        used = r["iters_used"].cpu().numpy().reshape(-1)
        rng = np.random.default_rng(int(sigma))
        pix = np.concatenate([[0, 511, 512 * 511, 512 * 512 - 1, 512 * 256 + 256], rng.choice(512 * 512, 11, False)])
        for p in pix:
            rr = oracle.nlem(g, 7, 21, 10 * sigma, 1.0, int(used[p]), pixels=[p])
            assert rel_err(out[p], rr["out"][0]) <= TOL, (p, out[p], rr["out"][0])


def test_em_full_size_sampled(nl):
    """262144 problems of n=441, d=49 (points from the device generator, 22.6 GB), rho=1,
    tolerance 1e-4 with the 300 cap: sampled problems against the oracle."""
    B, n, d = 262144, 441, 49
    dev = torch.device(DEV)
    synth.build_device_generator() if not __import__("os").path.exists(synth.SYNTH_LIB) else None
    pts = torch.empty((B, n, d), dtype=torch.float32, device=dev)
    synth.device_em_points(2002, B, n, d, pts.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    w = _t(synth.em_weights(2002, np.arange(B), n))
    r = nl.em_solve_batch(pts, w, rho=1.0, iters=300, tol=1e-4, check_every=10)
    x = r["x"]
    used = r["iters_used"].cpu().numpy()
    sample = np.array([0, 1, B // 2, B - 1, 77777, 123456])
    host_pts = synth.em_points(2002, sample, n, d)
    assert np.array_equal(pts[torch.from_numpy(sample).to(dev)].cpu().numpy(), host_pts)
    wh = synth.em_weights(2002, sample, n)
    for i, b in enumerate(sample):
        z, *_ = oracle.em_admm(host_pts[i], wh[i], 0.0, 255.0, 1.0, int(used[b]))
        assert rel_err(x[b].cpu().numpy(), z).max() <= TOL
    del pts
    torch.cuda.empty_cache()


def test_invalid_arguments(nl):
    g = _t(np.zeros((10, 10), np.float32))
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(g, patch=4)
    assert e.value.code == -1
    with pytest.raises(nl.NlemError):
        nl.nlem_denoise(g, patch=11)
    with pytest.raises(nl.NlemError):
        nl.nlem_denoise(g, patch=3, window=5, h=-1.0)
    with pytest.raises(nl.NlemError):
        nl.nlem_denoise(g, patch=3, rho=0.0)
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(_t(np.zeros((40, 40), np.float32)), patch=7, window=41)
    assert e.value.code == -5
    pts = _t(np.zeros((1, 5, 3), np.float32))
    w = _t(np.ones((1, 5), np.float32))
    with pytest.raises(nl.NlemError):
        nl.em_solve_batch(pts, w, box=(5.0, 1.0))
    with pytest.raises(nl.NlemError):
        nl.em_solve_batch(pts, w, iters=-1)


def test_pitched_image_views_match_contiguous(nl):
    """Images are read through their row pitch: a column slice of a wider array (rows 57 floats
    apart, starting 5 floats in) gives bitwise the same result as its contiguous copy, for a
    single image and inside a batch."""
    g, _ = synth.noisy_image(1300, 36, 44, 20.0)
    wide = torch.zeros((36, 44 + 13), dtype=torch.float32, device=DEV)
    wide[:, 5:49] = _t(g)
    view = wide[:, 5:49]
    assert not view.is_contiguous()
    kw = dict(patch=7, window=11, h=200.0, rho=1.0, iters=25)
    a = nl.nlem_denoise(view, **kw)
    b = nl.nlem_denoise(view.contiguous(), **kw)
    assert torch.equal(a["out"], b["out"])
    outs = nl.nlem_denoise_batch([view, view.contiguous()], [7, 7], [11, 11], [200.0, 200.0], rho=1.0, iters=25)
    assert torch.equal(outs[0]["out"], outs[1]["out"])
    with pytest.raises(ValueError):
        nl.nlem_denoise(view.t(), **kw)      # columns are not contiguous
