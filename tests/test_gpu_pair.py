"""GPU parity of the pixel-pair NLEM layout (two horizontally adjacent pixels per CTA, one
shared-memory copy of the points their windows share) against the FP64 oracle, and against
the one-pixel-per-CTA layout.  Tolerance as for every FP32 path:
|z_gpu - z_oracle| <= 1e-4 * max(|z_oracle|, 1) per pixel."""
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
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# Widths odd and even (an odd width leaves the last pixel of a row without a partner),
# windows from 1 (no shared points) to 21 (441 points, both exclusive columns), clipped
# windows on every border, both start points.
@pytest.mark.parametrize("H,W,S,init", [(24, 25, 21, 0), (20, 16, 17, 1), (15, 9, 11, 0), (9, 8, 3, 1),
                                        (7, 7, 1, 0), (30, 31, 19, 0), (11, 40, 21, 1), (28, 7, 21, 0)])
def test_pair_layout_all_pixels_against_oracle(nl, H, W, S, init):
    g, _ = synth.noisy_image(3100 + 7 * H + W + S, H, W, 20.0)
    T = 40
    r = nl.nlem_denoise(_t(g), patch=7, window=S, h=200.0, rho=1.0, iters=T, init=init, layout=nl.LAYOUT_PAIR)
    ref = oracle.nlem(g, 7, S, 200.0, 1.0, T, init_mode=init)
    err = rel_err(r["out"].cpu().numpy(), ref["out"])
    assert err.max() <= TOL, err.max()
    assert np.all(r["iters_used"].cpu().numpy() == T)
    # the residual output is the one-pixel layout's quantity, up to FP32 rounding order.  Where
    # ||z - z_prev|| is a few FP32 ulps of z the dual residual is rounding noise in both layouts
    # (and against the FP64 oracle), so the check is on nearly all pixels and on the median.
    q = nl.nlem_denoise(_t(g), patch=7, window=S, h=200.0, rho=1.0, iters=T, init=init, layout=nl.LAYOUT_PIXEL)
    ra, rb = r["residual"].cpu().numpy().astype(np.float64), q["residual"].cpu().numpy().astype(np.float64)
    rel = np.abs(ra - rb) / np.maximum(rb, 1e-7)
    assert np.mean(rel <= 1e-2) >= 0.97 and np.median(rel) <= 1e-4, (np.mean(rel <= 1e-2), np.median(rel))


def test_pair_and_pixel_layouts_agree(nl):
    """The same 64x64 image through both layouts (window 21, 60 iterations): equal up to FP32
    rounding order, and the automatic choice for window 21 is the pair layout (for window 15
    the one-pixel layout)."""
    g, _ = synth.noisy_image(3201, 64, 64, 25.0)
    kw = dict(patch=7, window=21, h=250.0, rho=1.0, iters=60)
    a = nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PAIR, **kw)
    b = nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PIXEL, **kw)
    c = nl.nlem_denoise(_t(g), **kw)
    assert rel_err(a["out"].cpu().numpy(), b["out"].cpu().numpy()).max() <= TOL
    assert torch.equal(a["out"], c["out"])
    kw15 = dict(kw, window=15)
    assert torch.equal(nl.nlem_denoise(_t(g), **kw15)["out"], nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PIXEL, **kw15)["out"])


def test_pair_layout_stops_each_pixel_on_its_own(nl):
    """Tolerance mode: the two pixels of a pair may stop at different checks.  Each pixel's
    output is the oracle's at the count the GPU reports; the counts match the one-pixel layout's
    for nearly all pixels, and pairs with unequal counts occur."""
    g, _ = synth.noisy_image(3301, 40, 46, 20.0)
    m = 5
    kw = dict(patch=7, window=21, h=200.0, rho=1e-3, iters=300, tol=1e-4, check_every=m)
    r = nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PAIR, **kw)
    q = nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PIXEL, **kw)
    used = r["iters_used"].cpu().numpy()
    assert np.mean(used == q["iters_used"].cpu().numpy()) >= 0.9
    assert np.any(used[:, 0::2] != used[:, 1::2])
    out = r["out"].cpu().numpy().reshape(-1)
    resid = r["residual"].cpu().numpy().reshape(-1)
    flat = used.reshape(-1)
    # pixels whose partner stopped at a different count, plus a spread of others
    diff = np.flatnonzero((used[:, 0::2] != used[:, 1::2]).reshape(-1))
    rows, pairs = np.divmod(diff, 46 // 2)
    pix = np.unique(np.concatenate([(rows * 46 + 2 * pairs)[:6], (rows * 46 + 2 * pairs + 1)[:6],
                                    np.arange(0, 40 * 46, 97)]))
    for p in pix:
        rr = oracle.nlem(g, 7, 21, 200.0, 1e-3, int(flat[p]), pixels=[p])
        assert rel_err(out[p], rr["out"][0]) <= TOL, (p, flat[p])
        ro = max(rr["r_pri"][0], rr["r_dual"][0])
        if flat[p] < 300:
            assert ro < 1e-4 * 1.05
        else:
            assert abs(resid[p] - ro) <= 2e-2 * ro


def test_pair_layout_fp64_check(nl):
    """The FP64 objective and optimality residual of each pixel of a pair match the one-pixel
    layout's (both evaluated in double at nearly the same z), and a constant image is a fixed
    point with a zero optimality residual."""
    g, _ = synth.noisy_image(3401, 18, 21, 30.0)
    kw = dict(patch=7, window=13, h=300.0, rho=1.0, iters=50, fp64_check=True)
    a = nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PAIR, **kw)
    b = nl.nlem_denoise(_t(g), layout=nl.LAYOUT_PIXEL, **kw)
    fa, fb = a["obj64"].cpu().numpy(), b["obj64"].cpu().numpy()
    assert np.allclose(fa, fb, rtol=1e-6)
    ka, kb = a["kkt64"].cpu().numpy(), b["kkt64"].cpu().numpy()
    assert np.allclose(ka, kb, rtol=0.05, atol=1e-3 * np.abs(fb).max())
    c = np.full((12, 15), 91.5, dtype=np.float32)
    rc = nl.nlem_denoise(_t(c), patch=7, window=9, h=100.0, iters=20, fp64_check=True, layout=nl.LAYOUT_PAIR)
    assert np.allclose(rc["out"].cpu().numpy(), 91.5, atol=1e-4)
    assert np.all(rc["kkt64"].cpu().numpy() < 1e-3)


def test_pair_layout_full_size_sampled(nl):
    """512x512, sigma 20, window 21, rho 1, tolerance 1e-4 with the 300 cap (the production
    workload) through the pair layout: sampled pixels, both members of their pairs, against the
    oracle replayed at the GPU's count."""
    g, _ = synth.noisy_image(3501, 512, 512, 20.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=21, h=200.0, rho=1.0, iters=300, tol=1e-4, check_every=10,
                        layout=nl.LAYOUT_PAIR)
    out = r["out"].cpu().numpy().reshape(-1)
    used = r["iters_used"].cpu().numpy().reshape(-1)
    rng = np.random.default_rng(35)
    base = np.concatenate([[0, 510, 512 * 511, 512 * 512 - 2, 512 * 256 + 256], 2 * rng.choice(512 * 256, 5, False)])
    for p in np.concatenate([base, base + 1]):
        rr = oracle.nlem(g, 7, 21, 200.0, 1.0, int(used[p]), pixels=[int(p)])
        assert rel_err(out[p], rr["out"][0]) <= TOL, (p, out[p], rr["out"][0])


def test_pair_layout_rejects_what_it_does_not_cover(nl):
    g = _t(np.zeros((40, 40), np.float32))
    for kw in (dict(patch=5, window=11), dict(patch=7, window=23), dict(patch=7, window=21, precision=nl.PREC_BF16)):
        with pytest.raises(nl.NlemError) as e:
            nl.nlem_denoise(g, layout=nl.LAYOUT_PAIR, iters=2, **kw)
        assert e.value.code == -5
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise(g, patch=7, window=21, iters=2, layout=7)
    assert e.value.code == -1


def test_pair_layout_pitched_view_matches_contiguous(nl):
    """The pair kernel reads the image through its row pitch: a column slice of a wider array
    gives bitwise the result of its contiguous copy (odd width, window 21)."""
    g, _ = synth.noisy_image(3601, 30, 37, 20.0)
    wide = torch.zeros((30, 37 + 11), dtype=torch.float32, device=DEV)
    wide[:, 3:40] = _t(g)
    view = wide[:, 3:40]
    assert not view.is_contiguous()
    kw = dict(patch=7, window=21, h=200.0, rho=1.0, iters=25, layout=nl.LAYOUT_PAIR)
    a = nl.nlem_denoise(view, **kw)
    b = nl.nlem_denoise(view.contiguous(), **kw)
    assert torch.equal(a["out"], b["out"]) and torch.equal(a["iters_used"], b["iters_used"])
