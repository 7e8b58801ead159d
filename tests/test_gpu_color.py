"""GPU multichannel NLEM (stacked channel patches, Sec. 3) against the FP64 oracle's composition,
and standalone problems of dimension 121..148.  Tolerance as for every FP32 path:
|z_gpu - z_oracle| <= 1e-4 * max(|z_oracle|, 1) per output value."""
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


def _rgb(seed, H, W, sigma):
    """Three correlated channels: one clean image per channel plus independent noise."""
    return np.stack([synth.noisy_image(seed + c, H, W, sigma)[0] for c in range(3)])


# patch 5 up to the 21x21 window (d = 75, 441 points), patch 7 up to 15x15 (d = 147, 225 points) in
# one CTA and at 17x17 and 21x21 over a two-CTA cluster (border pixels whose clipped window fits the
# first CTA leave the second one without points); both start points; the tolerance mode, where both
# CTAs of a cluster must stop at the same check
@pytest.mark.parametrize("k,S,H,W,init,T,tol", [(5, 21, 24, 23, 0, 30, 0.0), (5, 11, 17, 20, 1, 20, 0.0),
                                                (5, 3, 9, 8, 0, 10, 0.0), (7, 15, 21, 19, 0, 25, 0.0),
                                                (7, 9, 16, 15, 1, 12, 0.0), (5, 21, 22, 21, 0, 300, 1e-4),
                                                (7, 21, 25, 24, 0, 20, 0.0), (7, 17, 20, 22, 1, 15, 0.0),
                                                (7, 21, 23, 22, 0, 300, 1e-4)])
def test_color_all_pixels_against_oracle(nl, k, S, H, W, init, T, tol):
    img = _rgb(6100 + 10 * k + S, H, W, 20.0)
    h = 10 * 20.0 * np.sqrt(3.0)
    kw = dict(tol=tol, check_every=10) if tol > 0 else {}
    split = k == 7 and S * S > 256          # the FP64 check needs the window in one CTA
    r = nl.nlem_denoise_color(torch.from_numpy(img).to(DEV), patch=k, window=S, h=h, rho=1.0, iters=T, init=init,
                              fp64_check=not split, **kw)
    if tol > 0:
        # tolerance mode: each pixel against the oracle at the count the GPU reports
        used = r["iters_used"].cpu().numpy().reshape(-1)
        got = r["out"].cpu().numpy().reshape(3, -1)
        pix = np.arange(0, H * W, 7)
        for p in pix:
            ref = oracle.nlem_color(img, k, S, h, 1.0, int(used[p]), init_mode=init, pixels=[p])
            assert rel_err(got[:, p], ref["out"][:, 0]).max() <= TOL
        assert np.all(used >= 10) and np.all(used <= T)
        return
    ref = oracle.nlem_color(img, k, S, h, 1.0, T, init_mode=init)
    err = rel_err(r["out"].cpu().numpy(), ref["out"])
    assert err.max() <= TOL, err.max()
    assert np.all(r["iters_used"].cpu().numpy() == T)
    if not split:
        assert np.all(np.isfinite(r["obj64"].cpu().numpy())) and np.all(r["kkt64"].cpu().numpy() >= 0)


def test_color_identical_channels_match_grayscale(nl):
    """Three copies of one image at h and rho are grayscale NLEM at h/sqrt(3) and rho*sqrt(3)."""
    g, _ = synth.noisy_image(6201, 30, 28, 25.0)
    img = torch.from_numpy(np.stack([g, g, g])).to(DEV)
    a = nl.nlem_denoise_color(img, patch=5, window=15, h=250.0, rho=0.5, iters=40)
    b = nl.nlem_denoise(torch.from_numpy(g).to(DEV), patch=5, window=15, h=250.0 / np.sqrt(3.0),
                        rho=0.5 * np.sqrt(3.0), iters=40)
    for c in range(3):
        assert rel_err(a["out"][c].cpu().numpy(), b["out"].cpu().numpy()).max() <= TOL


def test_color_full_size_sampled(nl):
    """512 x 512, 5x5 colour patches, 21x21 window, the paper's 4 iterations at mu = 1e-3 from the noisy
    patch: sampled pixels (corners, borders, interior) against the oracle."""
    H = W = 512
    img = _rgb(6301, H, W, 20.0)
    h = 200.0 * np.sqrt(3.0)
    r = nl.nlem_denoise_color(torch.from_numpy(img).to(DEV), patch=5, window=21, h=h, rho=1e-3, iters=4, init=1)
    rng = np.random.default_rng(6301)
    pix = np.unique(np.concatenate([[0, W - 1, (H - 1) * W, H * W - 1, 5 * W + 300], rng.integers(0, H * W, 40)]))
    ref = oracle.nlem_color(img, 5, 21, h, 1e-3, 4, init_mode=1, pixels=pix)
    got = r["out"].cpu().numpy().reshape(3, -1)[:, pix]
    assert rel_err(got, ref["out"]).max() <= TOL


def test_color_argument_errors(nl):
    img = torch.zeros((3, 16, 16), device=DEV)
    for kw, code in ((dict(patch=7, window=23), -5), (dict(patch=9, window=5), -5), (dict(patch=4), -1),
                     (dict(patch=5, window=23), -5), (dict(patch=7, window=17, fp64_check=True), -5)):
        with pytest.raises(nl.NlemError) as e:
            nl.nlem_denoise_color(img, **kw)
        assert e.value.code == code, kw
    with pytest.raises(nl.NlemError) as e:       # two channels are not compiled
        nl.nlem_denoise_color(torch.zeros((2, 16, 16), device=DEV), patch=5, window=5)
    assert e.value.code == -5


@pytest.mark.parametrize("n,d", [(100, 121), (256, 147), (30, 148), (129, 130)])
def test_em_batch_dimensions_above_120(nl, n, d):
    """Standalone problems with d in 121..148 (the runtime-dimension shapes of 37 slots per lane)."""
    B = 24
    pts = synth.em_points(6400 + d, np.arange(B), n, d)
    w = synth.em_weights(6400 + d, np.arange(B), n)
    r = nl.em_solve_batch(torch.from_numpy(pts).to(DEV), torch.from_numpy(w).to(DEV), rho=1.0, iters=40)
    for b in range(0, B, 5):
        z, *_ = oracle.em_admm(pts[b].astype(np.float64), w[b].astype(np.float64), 0.0, 255.0, 1.0, 40)
        assert rel_err(r["x"][b].cpu().numpy(), z).max() <= TOL
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch(torch.zeros((1, 257, 140), device=DEV), torch.ones((1, 257), device=DEV))
    assert e.value.code == -5
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch(torch.zeros((1, 5, 149), device=DEV), torch.ones((1, 5), device=DEV))
    assert e.value.code == -1
