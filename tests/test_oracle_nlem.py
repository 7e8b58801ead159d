"""Pins for the oracle's NLEM driver (Sec. 3) and for the seeded input generators (CPU only)."""
import numpy as np
import pytest

import oracle
import synth


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 1234567 (reference output of the published generator)
    got = synth.draw_u64(np.uint64(1234567), np.arange(5))
    assert got.tolist() == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                            4593380528125082431, 16408922859458223821]


def test_generators_are_counter_based():
    full = synth.em_points(7, np.arange(6), 13, 5)
    part = synth.em_points(7, [4, 1], 13, 5)
    assert np.array_equal(full[[4, 1]], part)
    w = synth.em_weights(7, np.arange(6), 13)
    assert np.array_equal(w[[5, 2]], synth.em_weights(7, [5, 2], 13))
    assert np.all(w > 0)
    pts = synth.em_points(3, np.arange(200), 50, 7)
    out = np.all((pts == 0) | (pts == 255), axis=2)
    assert 0.07 < out.mean() < 0.13                      # ~10% whole-point outliers
    assert pts.min() >= 0 and pts.max() <= 255
    g1, f1 = synth.noisy_image(5, 40, 30, 20.0)
    g2, _ = synth.noisy_image(5, 40, 30, 20.0)
    assert np.array_equal(g1, g2) and g1.dtype == np.float32
    assert 15 < np.std(g1 - f1) < 25


def _reflect_patches(img, k):
    r = (k - 1) // 2
    P = np.pad(img.astype(np.float64), r, mode="reflect")
    H, W = img.shape
    return lambda i, j: P[i:i + k, j:j + k].reshape(-1)


@pytest.mark.parametrize("k,S", [(3, 5), (7, 11), (5, 7)])
def test_problem_assembly(k, S):
    g, _ = synth.noisy_image(21, 23, 19, 20.0)
    H, W = g.shape
    patch = _reflect_patches(g, k)
    h = 200.0
    R = (S - 1) // 2
    for lin in (0, W - 1, (H // 2) * W + W // 2, H * W - 1, 3 * W + 1):
        pts, w, pc = oracle.nlem_problem(g, k, S, h, lin)
        i, j = divmod(lin, W)
        assert np.array_equal(pc, patch(i, j))
        exp_pts = [patch(a, b) for a in range(max(0, i - R), min(H, i + R + 1))
                   for b in range(max(0, j - R), min(W, j + R + 1))]
        assert len(pts) == len(exp_pts)
        assert np.array_equal(pts, np.array(exp_pts))
        self_idx = [t for t, p in enumerate(pts) if np.array_equal(p, pc)]
        assert any(abs(w[t] - 1.0) < 1e-15 for t in self_idx)        # w_ii = exp(0) = 1
        assert np.all((w > 0) & (w <= 1))
    # corner window holds ((S+1)/2)^2 centres, interior S^2
    assert len(oracle.nlem_problem(g, k, S, h, 0)[1]) == ((S + 1) // 2) ** 2


def test_bf16_weight_model_error_bound():
    g, _ = synth.noisy_image(22, 30, 30, 30.0, salt_pepper=0.05)
    for lin in (0, 455, 899):
        p0, w0, pc = oracle.nlem_problem(g, 9, 7, 300.0, lin, weight_mode=0)
        p1, w1, _ = oracle.nlem_problem(g, 9, 7, 300.0, lin, weight_mode=1)
        D0 = -np.log(w0) * 300.0 ** 2
        D1 = -np.log(w1) * 300.0 ** 2
        # bf16 keeps 8 significant bits: each product is off by at most ~2^-8 relative
        bound = 2 * np.sum(np.abs(pc)[None, :] * np.abs(p0), axis=1) * 2.0 ** -7 + 1e-6
        assert np.all(np.abs(D1 - D0) <= bound)


def test_constant_image():
    for c in (0.0, 37.5, 255.0):
        g = np.full((12, 13), c, dtype=np.float32)
        r = oracle.nlem(g, 3, 5, 100.0, 1.0, 20)
        assert np.allclose(r["out"], c, atol=1e-12)
    g = np.full((9, 9), 300.0, dtype=np.float32)
    assert np.allclose(oracle.nlem(g, 3, 5, 100.0, 1.0, 20)["out"], 255.0)


def test_window_one_gives_clamped_input():
    g, _ = synth.noisy_image(23, 15, 17, 40.0)
    r = oracle.nlem(g, 5, 1, 400.0, 1.0, 10)
    assert np.allclose(r["out"], np.clip(g, 0, 255), atol=1e-12)
    assert np.all(r["n"] == 1)


def test_patch_one_is_weighted_scalar_median():
    g, _ = synth.noisy_image(24, 14, 11, 20.0)
    H, W = g.shape
    S, h = 5, 60.0
    r = oracle.nlem(g, 1, S, h, 0.02, 6000)
    R = 2
    for lin in range(0, H * W, 7):
        i, j = divmod(lin, W)
        vals = g[max(0, i - R):i + R + 1, max(0, j - R):j + R + 1].astype(np.float64).reshape(-1)
        w = np.exp(-(vals - float(g[i, j])) ** 2 / h ** 2)
        F = lambda t: float(np.sum(w * np.abs(t - vals)))
        cand = np.clip(vals, 0, 255)
        Fstar = min(F(t) for t in cand)                   # a weighted median is a data point
        assert F(r["out"][i, j]) <= Fstar * (1 + 1e-9) + 1e-9


def test_nlem_denoises_synthetic_image():
    g, f = synth.noisy_image(25, 48, 48, 20.0)
    r = oracle.nlem(g, 7, 11, 200.0, 1e-3, 4, init_mode=1)
    assert synth.psnr(r["out"], f) > synth.psnr(g, f) + 4.0


def test_pixel_subset_matches_full():
    g, _ = synth.noisy_image(26, 20, 20, 20.0)
    full = oracle.nlem(g, 5, 7, 200.0, 1.0, 15)
    pix = [0, 21, 399, 200]
    sub = oracle.nlem(g, 5, 7, 200.0, 1.0, 15, pixels=pix)
    assert np.array_equal(sub["out"], full["out"].reshape(-1)[pix])


# ---------------------------------------------------------------------------------------
# NLEM-IRLS (the comparison method of Sec. 3): IRLS on the surrogate of Eq. 2 per pixel
# ---------------------------------------------------------------------------------------

def test_nlem_irls_patch_one_reaches_weighted_median():
    """k = 1: each problem is a weighted scalar median of the window's pixel values.  The
    surrogate's minimiser is within sum_k w_k sqrt(eps) of problem (1)'s optimum in objective."""
    g, _ = synth.noisy_image(27, 12, 11, 20.0)
    H, W = g.shape
    S, h, eps = 5, 60.0, 1e-6
    pix = list(range(0, H * W, 5))
    r = oracle.nlem_irls(g, 1, S, h, eps, 3000, pixels=pix)
    R = 2
    for m, lin in enumerate(pix):
        i, j = divmod(lin, W)
        vals = g[max(0, i - R):i + R + 1, max(0, j - R):j + R + 1].astype(np.float64).reshape(-1)
        w = np.exp(-(vals - float(g[i, j])) ** 2 / h ** 2)
        F = lambda t: float(np.sum(w * np.abs(t - vals)))
        Fstar = min(F(t) for t in np.clip(vals, 0, 255))
        assert F(r["out"][m]) <= Fstar + w.sum() * np.sqrt(eps) + 1e-9 * Fstar
        assert abs(r["obj"][m] - F(r["out"][m])) <= 1e-9 * max(1.0, Fstar)


def test_nlem_irls_constant_image_and_zero_steps():
    for c in (0.0, 91.0, 255.0):
        g = np.full((9, 10), c, dtype=np.float32)
        assert np.allclose(oracle.nlem_irls(g, 3, 5, 100.0, 1e-6, 6)["out"], c, atol=1e-9)
    g = np.full((9, 9), 300.0, dtype=np.float32)
    assert np.allclose(oracle.nlem_irls(g, 3, 5, 100.0, 1e-6, 6)["out"], 255.0)
    # zero steps: the start point of the NLEM driver (weighted mean, or the clamped noisy pixel)
    g, _ = synth.noisy_image(28, 13, 12, 30.0)
    r0 = oracle.nlem_irls(g, 5, 7, 300.0, 1e-6, 0)
    assert np.allclose(r0["out"], oracle.nlem(g, 5, 7, 300.0, 1.0, 0)["out"], rtol=0, atol=1e-9)
    assert np.all(r0["step"] == 0.0)
    r1 = oracle.nlem_irls(g, 5, 7, 300.0, 1e-6, 0, init_mode=1)
    assert np.allclose(r1["out"], np.clip(g, 0, 255), atol=0)


def test_nlem_irls_last_step_and_monotone_surrogate():
    """The reported step is ||x(T) - x(T-1)|| / ||x(T)|| of the T-step run, and the surrogate of
    Eq. 2 does not increase from T-1 to T steps (IRLS is a majorise-minimise scheme; the box
    projection keeps that because the quadratic majoriser is separable per coordinate)."""
    g, _ = synth.noisy_image(29, 14, 14, 40.0)
    k, S, h, eps = 5, 9, 400.0, 1e-6
    lin = 5 * 14 + 8
    pts, w, pc = oracle.nlem_problem(g, k, S, h, lin)
    x0 = oracle.project_box(pc, 0.0, 255.0)
    sur = lambda x: float(np.sum(w * np.sqrt(np.sum((x - pts) ** 2, 1) + eps)))
    prev = sur(x0)
    for T in (1, 2, 3, 5):
        r = oracle.nlem_irls(g, k, S, h, eps, T, init_mode=1, pixels=[lin])
        xa, _ = oracle.irls(pts, w, 0.0, 255.0, x0, eps, T - 1)
        xb, _ = oracle.irls(pts, w, 0.0, 255.0, x0, eps, T)
        assert r["out"][0] == xb[(k * k - 1) // 2]
        assert np.isclose(r["step"][0], np.linalg.norm(xb - xa) / np.linalg.norm(xb), rtol=1e-12)
        assert sur(xb) <= prev + 1e-12 * prev
        prev = sur(xb)


# ---------------------------------------------------------------------------------------
# multichannel NLEM: stacked channel patches (Sec. 3 with colour patches)
# ---------------------------------------------------------------------------------------

def test_nlem_color_identical_channels_is_grayscale_rescaled():
    """With C identical channels every distance is C times the grayscale one (w = exp(-D/(h/sqrt C)^2))
    and every shrink step of Algorithm 1 sees sqrt(C) times the grayscale norm, so the iterates are
    the grayscale ones at h/sqrt(C) and mu*sqrt(C), block by block (residuals included)."""
    g, _ = synth.noisy_image(31, 11, 12, 25.0)
    for C, init, T in ((3, 0, 25), (2, 1, 12)):
        col = oracle.nlem_color(np.stack([g] * C), 3, 5, 250.0, 0.7, T, init_mode=init, tol=1e-3, check_every=4)
        gray = oracle.nlem(g, 3, 5, 250.0 / np.sqrt(C), 0.7 * np.sqrt(C), T, init_mode=init, tol=1e-3, check_every=4)
        for c in range(C):
            assert np.allclose(col["out"][c], gray["out"], rtol=0, atol=1e-8)
        assert np.array_equal(col["iters_used"], gray["iters_used"])
        assert np.allclose(col["r_pri"], gray["r_pri"], rtol=1e-7, atol=1e-12)


def test_nlem_color_one_varying_channel_and_permutation():
    """Constant channels add nothing to the distances, and the solution keeps them at their (in-box)
    value, so the varying channel's output is grayscale NLEM with the same h and mu.  Permuting the
    input channels permutes the outputs."""
    g, _ = synth.noisy_image(32, 10, 13, 20.0)
    img = np.stack([np.full_like(g, 40.0), g, np.full_like(g, 200.0)])
    r = oracle.nlem_color(img, 3, 5, 200.0, 1.0, 20)
    ref = oracle.nlem(g, 3, 5, 200.0, 1.0, 20)
    assert np.allclose(r["out"][1], ref["out"], rtol=0, atol=1e-8)
    assert np.allclose(r["out"][0], 40.0, atol=1e-9) and np.allclose(r["out"][2], 200.0, atol=1e-9)
    h2, _ = synth.noisy_image(33, 10, 13, 30.0)
    img2 = np.stack([g, h2, np.clip(g + h2 - 100.0, -20.0, 300.0).astype(np.float32)])
    a = oracle.nlem_color(img2, 3, 5, 300.0, 1.0, 15, pixels=[0, 17, 64, 129])
    b = oracle.nlem_color(img2[[2, 0, 1]], 3, 5, 300.0, 1.0, 15, pixels=[0, 17, 64, 129])
    assert np.allclose(b["out"], a["out"][[2, 0, 1]], rtol=0, atol=1e-9)
    const = oracle.nlem_color(np.stack([np.full_like(g, 7.0), np.full_like(g, 300.0)]), 3, 5, 100.0, 1.0, 10)
    assert np.allclose(const["out"][0], 7.0) and np.allclose(const["out"][1], 255.0)
