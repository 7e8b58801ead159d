"""GPU tests of the learned warm start: features against the oracle, forward / backward of the
MLP against the CPU FP64 model at FP16 tolerance, Adam, checkpoints, the per-pixel start /
penalty path, and what a trained network gains over plain EM-ADMM."""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
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


def test_features_match_oracle(nl):
    g, _ = synth.noisy_image(8000, 40, 44, 25.0)
    h = 250.0
    pix = np.array([0, 43, 44 * 20 + 21, 40 * 44 - 1, 44 * 7 + 3, 44 * 33 + 40], dtype=np.int32)
    feats = nl.nlem_features(torch.from_numpy(g).to(DEV), 7, 21, h, pixels=torch.from_numpy(pix).to(DEV)).cpu().numpy()
    for row, lin in zip(feats, pix):
        pts, w, _ = oracle.nlem_problem(g, 7, 21, h, int(lin))
        f = oracle.features(pts, w.astype(np.float32).astype(np.float64))
        d = 49
        assert rel_err(row[:d], f[:d]).max() <= 1e-4                      # weighted mean
        assert abs(row[2 * d] - f[2 * d]) <= 1e-4 * max(1.0, f[2 * d])     # entropy
        assert abs(row[2 * d + 1] - f[2 * d + 1]) <= 1e-5                 # largest weight
        # weighted medians are data values; a mismatch is only allowed where the cumulative
        # weight sits at half the total to within FP32 weight rounding
        for c in range(d):
            if row[d + c] != f[d + c]:
                vals = pts[:, c]
                cum_at = np.sum(w[vals <= row[d + c]])
                assert abs(cum_at - 0.5 * w.sum()) <= 1e-5 * w.sum(), (lin, c)


@pytest.mark.parametrize("k,S", [(5, 15), (9, 21), (7, 25)])
def test_features_other_patches_and_windows(nl, k, S):
    """Patch 5 and 9 and the largest 7x7 window (a 31 x 31 tile): the same checks as above."""
    g, _ = synth.noisy_image(8100 + k + S, 36, 33, 25.0)
    h = 250.0
    d = k * k
    pix = np.array([0, 32, 33 * 18 + 17, 36 * 33 - 1, 33 * 5 + 30], dtype=np.int32)
    feats = nl.nlem_features(torch.from_numpy(g).to(DEV), k, S, h, pixels=torch.from_numpy(pix).to(DEV)).cpu().numpy()
    for row, lin in zip(feats, pix):
        pts, w, _ = oracle.nlem_problem(g, k, S, h, int(lin))
        f = oracle.features(pts, w.astype(np.float32).astype(np.float64))
        assert rel_err(row[:d], f[:d]).max() <= 1e-4
        assert abs(row[2 * d] - f[2 * d]) <= 1e-4 * max(1.0, f[2 * d])
        assert abs(row[2 * d + 1] - f[2 * d + 1]) <= 1e-5
        for c in range(d):
            if row[d + c] != f[d + c]:
                vals = pts[:, c]
                cum_at = np.sum(w[vals <= row[d + c]])
                assert abs(cum_at - 0.5 * w.sum()) <= 1e-5 * w.sum(), (lin, c)


def test_features_list_matches_image_and_rejects_outside_indices(nl):
    """Rows of a pixel list equal the rows of the whole-image pass bitwise; listed indices outside
    the image give NaN rows and leave the other rows unchanged."""
    g, _ = synth.noisy_image(8200, 24, 29, 20.0)
    gi = torch.from_numpy(g).to(DEV)
    full = nl.nlem_features(gi, 7, 21, 200.0)
    pix = torch.tensor([5, 24 * 29, 100, -3, 24 * 29 - 1], dtype=torch.int32, device=DEV)
    rows = nl.nlem_features(gi, 7, 21, 200.0, pixels=pix)
    for i, p in enumerate(pix.tolist()):
        if 0 <= p < 24 * 29:
            assert torch.equal(rows[i], full[p])
        else:
            assert torch.isnan(rows[i]).all()


def _fp16_params(ws, seed):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=ws.num_params) * 0.05).astype(np.float16).astype(np.float32)
    ws.set_params(p)
    return p.astype(np.float64)


def test_mlp_forward_and_gradient_against_cpu(nl):
    d = 49
    ws = nl.WarmStart(d, nref=441.0, seed=3)
    p = _fp16_params(ws, 1)
    rng = np.random.default_rng(2)
    Bn = 70
    feats = np.concatenate([rng.uniform(0, 255, (Bn, 2 * d)), rng.uniform(3, 6, (Bn, 1)), rng.uniform(0, 0.3, (Bn, 1))],
                           axis=1).astype(np.float32)
    tgt = rng.normal(size=(Bn, d + 1)).astype(np.float32)
    ft, tt = torch.from_numpy(feats).to(DEV), torch.from_numpy(tgt).to(DEV)
    y = ws.forward(ft).cpu().numpy()
    yref = oracle.mlp_forward(p, d, feats.astype(np.float64), nref=441.0)
    assert np.max(np.abs(y - yref)) <= 1e-3 * max(1.0, np.max(np.abs(yref)))
    loss, grad = ws.loss_grad(ft, tt)
    Lref, gref = oracle.mlp_loss_grad(p, d, feats.astype(np.float64), tgt.astype(np.float64), nref=441.0)
    assert abs(loss.item() - Lref) <= 1e-3 * Lref
    g = grad.cpu().numpy()
    assert np.max(np.abs(g - gref)) <= 1e-3 * np.max(np.abs(gref))
    assert np.linalg.norm(g - gref) <= 1e-3 * np.linalg.norm(gref)
    ws.close()


def test_adam_step_and_checkpoint(nl):
    d = 25
    ws = nl.WarmStart(d, seed=4)
    p0 = ws.get_params().astype(np.float64)
    rng = np.random.default_rng(5)
    feats = torch.from_numpy(np.concatenate([rng.uniform(0, 255, (64, 2 * d)), rng.uniform(3, 6, (64, 1)),
                                             rng.uniform(0, 0.3, (64, 1))], axis=1).astype(np.float32)).to(DEV)
    tgt = torch.from_numpy(rng.normal(size=(64, d + 1)).astype(np.float32)).to(DEV)
    _, g = ws.loss_grad(feats, tgt)
    g = g.cpu().numpy().astype(np.float64)
    lr = 1e-2
    ws.train_step(feats, tgt, lr)
    p1 = ws.get_params().astype(np.float64)
    # first Adam step: m = (1-b1) g, v = (1-b2) g^2, bias-corrected -> p - lr * g / (|g| + eps)
    expect = p0 - lr * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p1 - expect)) <= 1e-5
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "ws.bin")
        ws.save(path)
        ws2 = nl.WarmStart(d, seed=99)
        ws2.load(path)
        assert np.array_equal(ws2.get_params(), ws.get_params())
        y1 = ws.forward(feats)
        y2 = ws2.forward(feats)
        assert torch.equal(y1, y2)
        ws2.close()
    ws.close()


def test_per_pixel_start_and_penalty(nl):
    """nlem_denoise_ex with per-pixel x0 and rho equals the oracle started from the same point
    with the same penalty."""
    g, _ = synth.noisy_image(8100, 30, 28, 20.0)
    H, W = g.shape
    h = 200.0
    img = torch.from_numpy(g).to(DEV)
    rng = np.random.default_rng(6)
    x0 = rng.uniform(-10, 265, (H * W, 49)).astype(np.float32)
    rho = np.exp(rng.uniform(np.log(1e-3), 0, H * W)).astype(np.float32)
    pix = np.array([0, 5, 100, 451, H * W - 1], dtype=np.int32)
    r = nl.nlem_denoise_ex(img, 7, 11, h, iters=40, pixels=torch.from_numpy(pix).to(DEV), x0=torch.from_numpy(x0).to(DEV),
                           rho_pix=torch.from_numpy(rho).to(DEV), z_out=True)
    out = r["out"].cpu().numpy().reshape(-1)
    z = r["z"].cpu().numpy()
    for lin in pix:
        pts, w, _ = oracle.nlem_problem(g, 7, 11, h, int(lin))
        zo, *_ = oracle.em_admm(pts, w, 0.0, 255.0, float(rho[lin]), 40, z0=np.clip(x0[lin], 0, 255))
        assert rel_err(z[lin], zo).max() <= TOL
        assert rel_err(out[lin], zo[24]) <= TOL


def test_per_pixel_start_and_penalty_on_pixel_pairs(nl):
    """Every pixel of an image with per-pixel x0 and rho and a 21x21 window (7x7 patches: the pixel-pair
    kernel, which also writes the whole solution patches) equals the oracle started from the same point
    with the same penalty; odd width, so the last pair has no second pixel."""
    g, _ = synth.noisy_image(8110, 26, 31, 25.0)
    H, W = g.shape
    h = 250.0
    img = torch.from_numpy(g).to(DEV)
    rng = np.random.default_rng(7)
    x0 = rng.uniform(-10, 265, (H * W, 49)).astype(np.float32)
    rho = np.exp(rng.uniform(np.log(1e-3), 0, H * W)).astype(np.float32)
    r = nl.nlem_denoise_ex(img, 7, 21, h, iters=40, x0=torch.from_numpy(x0).to(DEV),
                           rho_pix=torch.from_numpy(rho).to(DEV), z_out=True)
    out = r["out"].cpu().numpy().reshape(-1)
    z = r["z"].cpu().numpy()
    worst = 0.0
    for lin in range(H * W):
        pts, w, _ = oracle.nlem_problem(g, 7, 21, h, lin)
        zo, *_ = oracle.em_admm(pts, w, 0.0, 255.0, float(rho[lin]), 40, z0=np.clip(x0[lin], 0, 255))
        worst = max(worst, rel_err(z[lin], zo).max(), rel_err(out[lin], zo[24]))
    assert worst <= TOL, worst


def test_pixel_list_entries_outside_the_image_are_skipped(nl):
    """A pixel list with entries outside [0, H*W) (negative, past the end) and a duplicate: the valid
    pixels get the same values as the whole-image solve, the other outputs keep what they held."""
    g, _ = synth.noisy_image(8150, 20, 23, 20.0)
    H, W = g.shape
    img = torch.from_numpy(g).to(DEV)
    full = nl.nlem_denoise(img, patch=7, window=11, h=200.0, rho=1.0, iters=30, layout=nl.LAYOUT_PIXEL)
    pix = torch.tensor([-1, 7, H * W, 200, 7, 2 ** 30, H * W - 1], dtype=torch.int32, device=DEV)
    sentinel = -12345.0
    o = dict(out=torch.full((H, W), sentinel, device=DEV), iters_used=torch.full((H, W), -7, dtype=torch.int32, device=DEV),
             residual=torch.zeros((H, W), device=DEV))
    nl.nlem_denoise_ex(img, 7, 11, 200.0, rho=1.0, iters=30, pixels=pix, out=o)
    got = o["out"].reshape(-1).cpu()
    ref = full["out"].reshape(-1).cpu()
    valid = [7, 200, H * W - 1]
    for p in valid:
        assert got[p] == ref[p]
    mask = torch.ones(H * W, dtype=torch.bool)
    mask[valid] = False
    assert torch.all(got[mask] == sentinel)
    assert torch.all(o["iters_used"].reshape(-1).cpu()[mask] == -7)


def test_ws_labels_match_their_definition(nl):
    """nlem_ws_labels against its definition composed on the host from nlem_denoise_ex runs: the
    grid penalty that reaches the tolerance first (ties to the earlier one), its win counts, and the
    targets [(z* - m) / 16, ln rho*] from the tight solve at that penalty; an entry outside the image
    gets NaN targets."""
    from paper_1501_03879_gb300 import warmstart as wst
    H, W = 40, 44
    g, _ = synth.noisy_image(8150, H, W, 25.0)
    img = torch.from_numpy(g).to(DEV)
    rng = np.random.default_rng(3)
    pix_np = np.sort(rng.choice(H * W, 300, replace=False)).astype(np.int32)
    pix = torch.from_numpy(pix_np).to(DEV)
    feats = nl.nlem_features(img, 7, 21, 250.0, pixels=pix)
    grid = (1e-3, 1e-2, 0.1, 1.0)
    tgt, counts = nl.nlem_ws_labels(img, pix, feats, grid, h=250.0, tol=1e-4, check_every=5, cap=300,
                                    tight_tol=1e-6, tight_cap=1000)
    its = []
    for rho in grid:
        r = nl.nlem_denoise_ex(img, 7, 21, 250.0, rho=rho, iters=300, tol=1e-4, check_every=5, pixels=pix)
        its.append(r["iters_used"].reshape(-1).cpu().numpy()[pix_np])
    its = np.stack(its)                              # [grid, n]
    best = np.argmin(its, axis=0)                    # first minimum: the earlier penalty on ties
    rho_star = np.asarray(grid, dtype=np.float32)[best]
    assert counts == [int(np.sum(best == j)) for j in range(len(grid))]
    rho_map = np.ones(H * W, dtype=np.float32)
    rho_map[pix_np] = rho_star
    r = nl.nlem_denoise_ex(img, 7, 21, 250.0, rho=1.0, iters=1000, tol=1e-6, check_every=5, pixels=pix,
                           rho_pix=torch.from_numpy(rho_map).to(DEV), z_out=True)
    z = r["z"].cpu().numpy()[pix_np]
    m = feats.cpu().numpy()[:, :49]
    got = tgt.cpu().numpy()
    assert np.allclose(got[:, :49], (z - m) / wst.DELTA_SCALE, rtol=0, atol=1e-6)
    assert np.allclose(got[:, 49], np.log(rho_star.astype(np.float64)), rtol=0, atol=1e-6)
    # an index outside the image
    bad = torch.tensor([5, H * W + 3], dtype=torch.int32, device=DEV)
    fb = nl.nlem_features(img, 7, 21, 250.0, pixels=bad)
    tb, cb = nl.nlem_ws_labels(img, bad, fb, grid, h=250.0, tight_cap=50)
    tb = tb.cpu().numpy()
    assert np.all(np.isfinite(tb[0])) and np.all(np.isnan(tb[1])) and sum(cb) == 1


def test_trained_warm_start_gains_over_plain_admm(nl):
    """Train on solves of two synthetic images, evaluate on a held-out one: the learned start and
    penalty reach the 1e-4 residual in far fewer iterations than plain EM-ADMM (rho = 1) and
    than the best single penalty of the grid, with few fallbacks, and its answers are those of
    the oracle replayed from the same start."""
    from paper_1501_03879_gb300 import warmstart as wst
    train_imgs = [torch.from_numpy(synth.noisy_image(8200 + i, 72, 72, s)[0]).to(DEV) for i, s in enumerate((15.0, 35.0))]
    feats, tgt, info = wst.make_training_set(train_imgs, [150.0, 350.0], per_image=2048, seed=1)
    ws = nl.WarmStart(49, seed=7)
    hist = wst.train(ws, feats, tgt, epochs=40, batch=512, lr=2e-3, seed=1)
    assert hist[-1] < hist[0]
    gt, _ = synth.noisy_image(8300, 64, 64, 25.0)
    img = torch.from_numpy(gt).to(DEV)
    ev = wst.evaluate(ws, img, 250.0)
    best_rho = wst.RHO_GRID[int(np.argmax(info["best_rho_counts"]))]
    plain_best = nl.nlem_denoise(img, 7, 21, 250.0, rho=best_rho, iters=300, tol=1e-4, check_every=10)
    it_best = float(plain_best["iters_used"].float().mean().item())
    n = 64 * 64
    warm_work = ev["warm_iters"] + 300.0 * ev["fallback"] / n
    print(f"warm {ev['warm_iters']:.1f} it (+{ev['fallback']} fallbacks, work {warm_work:.2f}), plain rho=1 "
          f"{ev['plain_iters']:.1f}, plain rho={best_rho} {it_best:.1f}")
    assert warm_work < 0.25 * ev["plain_iters"]
    assert warm_work <= 1.25 * it_best
    assert ev["fallback"] <= 0.05 * n
    # replay a few pixels in the oracle from the network's start and penalty
    feats_img = nl.nlem_features(img, 7, 21, 250.0)
    _, x0, rho = ws.predict(feats_img)
    x0, rho = x0.cpu().numpy(), rho.cpu().numpy()
    used = ev["warm"]["iters_used"].cpu().numpy().reshape(-1)
    out = ev["warm"]["out"].cpu().numpy().reshape(-1)
    for lin in (0, 777, 2080, 4095):
        if used[lin] >= 300:
            continue   # fell back
        pts, w, _ = oracle.nlem_problem(gt, 7, 21, 250.0, lin)
        zo, *_ = oracle.em_admm(pts, w, 0.0, 255.0, float(rho[lin]), int(used[lin]), z0=np.clip(x0[lin], 0, 255))
        assert rel_err(out[lin], zo[24]) <= TOL
    ws.close()


def test_warm_start_full_size_sampled(nl):
    """The learned-start path at the benchmark's size (2048x2048, sigma 25, 7x7 patches, 21x21
    window, tol 1e-4 every 10, cap 300): each sampled pixel equals the oracle replayed for the
    iterations the GPU ran, from the network's start and penalty, or, where the warm-started
    solve reached the cap, from the weighted mean at rho = 1 (the fallback)."""
    from paper_1501_03879_gb300 import warmstart as wst
    train = [torch.from_numpy(synth.noisy_image(8400, 96, 96, 25.0)[0]).to(DEV)]
    feats, tgt, _ = wst.make_training_set(train, [250.0], per_image=4096, seed=2)
    ws = nl.WarmStart(49, seed=11)
    wst.train(ws, feats, tgt, epochs=10, batch=512, lr=2e-3, seed=2)
    Hs = Ws = 2048
    g, _ = synth.noisy_image(8500, Hs, Ws, 25.0)
    img = torch.from_numpy(g).to(DEV)
    kw = dict(iters=300, tol=1e-4, check_every=10)
    r = nl.nlem_denoise_warm(ws, img, 7, 21, 250.0, rho_fallback=1.0, **kw)
    out = r["out"].cpu().numpy().reshape(-1)
    used = r["iters_used"].cpu().numpy().reshape(-1)
    rng = np.random.default_rng(12)
    pix = np.unique(np.concatenate([[0, Ws - 1, Ws * (Hs - 1), Hs * Ws - 1, 1000 * Ws + 5, 7 * Ws + 2040],
                                    rng.integers(0, Hs * Ws, 6)])).astype(np.int32)
    _, x0, rho = ws.predict(nl.nlem_features(img, 7, 21, 250.0))
    x0, rho = x0.cpu().numpy(), rho.cpu().numpy()
    # the warm-started solve alone, on the sampled pixels: which of them fell back
    ex = nl.nlem_denoise_ex(img, 7, 21, 250.0, rho=1.0, pixels=torch.from_numpy(pix).to(DEV),
                            x0=torch.from_numpy(x0).to(DEV), rho_pix=torch.from_numpy(rho).to(DEV), **kw)
    used_ex = ex["iters_used"].cpu().numpy().reshape(-1)[pix]
    for lin, uex in zip(pix, used_ex):
        pts, w, _ = oracle.nlem_problem(g, 7, 21, 250.0, int(lin))
        if uex < 300:
            assert used[lin] == uex
            zo, *_ = oracle.em_admm(pts, w, 0.0, 255.0, float(rho[lin]), int(uex), z0=np.clip(x0[lin], 0, 255))
        else:
            zo, *_ = oracle.em_admm(pts, w, 0.0, 255.0, 1.0, int(used[lin]))
        assert rel_err(out[lin], zo[24]) <= TOL, (int(lin), int(uex), int(used[lin]))
    ws.close()


def test_ws_train_matches_steps_and_is_seeded(nl):
    """nlem_ws_train: one epoch with the whole set as the minibatch equals one Adam step on the
    set (the order only changes the summation order), its reported loss is the set's loss, the
    same seed reproduces the same parameters and another seed orders the minibatches
    differently."""
    d = 25
    rng = np.random.default_rng(21)
    N = 96
    feats = torch.from_numpy(np.concatenate([rng.uniform(0, 255, (N, 2 * d)), rng.uniform(3, 6, (N, 1)),
                                             rng.uniform(0, 0.3, (N, 1))], axis=1).astype(np.float32)).to(DEV)
    tgt = torch.from_numpy(rng.normal(size=(N, d + 1)).astype(np.float32)).to(DEV)
    lr = 1e-3
    a, b = nl.WarmStart(d, seed=4), nl.WarmStart(d, seed=4)
    loss0, _ = a.loss_grad(feats, tgt)
    a.train_step(feats, tgt, lr)
    hist = b.train(feats, tgt, epochs=1, batch=N, lr=lr, seed=9)
    assert abs(hist[0] - loss0.item()) <= 1e-5 * loss0.item()
    pa, pb = a.get_params(), b.get_params()
    close = np.abs(pa - pb) <= 1e-6 * np.maximum(1.0, np.abs(pa)) + 1e-3 * lr
    assert close.mean() >= 0.999      # a first Adam step is lr*sign(g): gradients at rounding level may flip
    c1, c2, c3 = nl.WarmStart(d, seed=5), nl.WarmStart(d, seed=5), nl.WarmStart(d, seed=5)
    h1 = c1.train(feats, tgt, epochs=3, batch=16, lr=lr, seed=1)
    c2.train(feats, tgt, epochs=3, batch=16, lr=lr, seed=1)
    c3.train(feats, tgt, epochs=3, batch=16, lr=lr, seed=2)
    assert np.array_equal(c1.get_params(), c2.get_params())
    assert not np.array_equal(c1.get_params(), c3.get_params())
    assert len(h1) == 3 and all(np.isfinite(h1))
    with pytest.raises(nl.NlemError):
        c1.train(feats, tgt, epochs=1, batch=0, lr=lr)
    for m in (a, b, c1, c2, c3):
        m.close()
