"""GPU parity of the batched persistent launch (uneven image sizes, mixed 5x5 / 7x7 patches,
mixed windows, one graph-captured launch) against the FP64 oracle, plus graph replay."""
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


def _specs():
    # (H, W, sigma, patch, window): uneven sizes and aspect ratios, borders larger than windows
    return [(23, 40, 10.0, 5, 11), (37, 29, 20.0, 7, 21), (16, 16, 30.0, 7, 13), (50, 18, 40.0, 5, 21),
            (31, 33, 20.0, 7, 15), (12, 45, 10.0, 5, 9), (41, 41, 30.0, 5, 17)]


@pytest.mark.parametrize("forced", [None, 0, 1])
def test_batch_matches_oracle_every_pixel(nl, forced):
    """Every pixel of seven uneven images against the oracle, with the autotuner's launch shape and
    with each shape variant pinned (one solver shape per patch size; one per window-size class)."""
    specs = _specs()
    imgs_h = [synth.noisy_image(3000 + i, H, W, s)[0] for i, (H, W, s, k, S) in enumerate(specs)]
    imgs = [torch.from_numpy(g).to(DEV) for g in imgs_h]
    ctx = nl.Context(0)
    if forced is not None:
        nl.nlem_batch_force_config(forced, fetch=4, ctas_per_sm=2, ctx=ctx)
    T = 25
    outs = nl.nlem_denoise_batch(imgs, [k for *_, k, S in specs], [S for *_, S in specs],
                                 [10 * s for _, _, s, _, _ in specs], rho=0.7, iters=T, ctx=ctx)
    cfg = nl.nlem_batch_config(ctx)
    assert "CTA/SM" in cfg
    if forced == 1:
        assert cfg.startswith("by window")
    for i, ((H, W, s, k, S), g) in enumerate(zip(specs, imgs_h)):
        ref = oracle.nlem(g, k, S, 10 * s, 0.7, T)
        err = rel_err(outs[i]["out"].cpu().numpy(), ref["out"])
        assert err.max() <= TOL, (i, err.max())
        assert np.all(outs[i]["iters_used"].cpu().numpy() == T)


def test_batch_graph_replay_and_new_contents(nl):
    specs = _specs()[:4]
    imgs_h = [synth.noisy_image(3100 + i, H, W, s)[0] for i, (H, W, s, k, S) in enumerate(specs)]
    imgs = [torch.from_numpy(g).to(DEV) for g in imgs_h]
    ctx = nl.Context(0)
    args = ([k for *_, k, S in specs], [S for *_, S in specs], [10 * s for _, _, s, _, _ in specs])
    o1 = nl.nlem_denoise_batch(imgs, *args, rho=1.0, iters=15, ctx=ctx)
    first = [o["out"].clone() for o in o1]
    o2 = nl.nlem_denoise_batch(imgs, *args, rho=1.0, iters=15, ctx=ctx, outs=o1)   # replays the graph
    for a, b in zip(first, o2):
        assert torch.equal(a, b["out"])
    # same pointers, new pixel values: the replayed graph reads the new contents
    new_h = [synth.noisy_image(3200 + i, H, W, s)[0] for i, (H, W, s, k, S) in enumerate(specs)]
    for t, g in zip(imgs, new_h):
        t.copy_(torch.from_numpy(g))
    o3 = nl.nlem_denoise_batch(imgs, *args, rho=1.0, iters=15, ctx=ctx, outs=o1)
    for i, ((H, W, s, k, S), g) in enumerate(zip(specs, new_h)):
        ref = oracle.nlem(g, k, S, 10 * s, 1.0, 15)
        assert rel_err(o3[i]["out"].cpu().numpy(), ref["out"]).max() <= TOL


def test_batch_tolerance_mode(nl):
    specs = _specs()[:3]
    imgs_h = [synth.noisy_image(3300 + i, H, W, s)[0] for i, (H, W, s, k, S) in enumerate(specs)]
    imgs = [torch.from_numpy(g).to(DEV) for g in imgs_h]
    outs = nl.nlem_denoise_batch(imgs, [k for *_, k, S in specs], [S for *_, S in specs],
                                 [10 * s for _, _, s, _, _ in specs], rho=1e-3, iters=300, tol=1e-4, check_every=5)
    for i, ((H, W, s, k, S), g) in enumerate(zip(specs, imgs_h)):
        used = outs[i]["iters_used"].cpu().numpy().reshape(-1)
        out = outs[i]["out"].cpu().numpy().reshape(-1)
        for p in range(0, H * W, 17):
            rr = oracle.nlem(g, k, S, 10 * s, 1e-3, int(used[p]), pixels=[p])
            assert rel_err(out[p], rr["out"][0]) <= TOL


def test_batch_uneven_64_images_sampled(nl):
    """The 64-image batch (sides uniform on 128..1024, sigma in {10,20,30,40}, search radius
    5..10, 5x5 or 7x7 patches) in one persistent launch; 20 iterations; sampled pixels of every
    image against the oracle."""
    specs = synth.batch_specs(1004, 64)
    imgs_h = [sp.make()[0] for sp in specs]
    imgs = [torch.from_numpy(g).to(DEV) for g in imgs_h]
    outs = nl.nlem_denoise_batch(imgs, [sp.patch for sp in specs], [sp.window for sp in specs],
                                 [sp.h for sp in specs], rho=1.0, iters=20)
    rng = np.random.default_rng(5)
    for sp, g, o in zip(specs, imgs_h, outs):
        pix = np.concatenate([[0, sp.H * sp.W - 1], rng.choice(sp.H * sp.W, 3, replace=False)])
        ref = oracle.nlem(g, sp.patch, sp.window, sp.h, 1.0, 20, pixels=pix)
        got = o["out"].cpu().numpy().reshape(-1)[pix]
        assert rel_err(got, ref["out"]).max() <= TOL


@pytest.mark.parametrize("forced", [None, 0, 1])
def test_batch_accelerated_fixed_period_every_pixel(nl, forced):
    """The accelerated solver in the persistent launch, on a fixed restart period (its schedule does
    not depend on rounding): every pixel of the seven uneven images against the oracle's
    em_admm_fast, with the autotuner's shape and with each variant pinned."""
    specs = _specs()
    imgs_h = [synth.noisy_image(3500 + i, H, W, s)[0] for i, (H, W, s, k, S) in enumerate(specs)]
    imgs = [torch.from_numpy(g).to(DEV) for g in imgs_h]
    ctx = nl.Context(0)
    if forced is not None:
        nl.nlem_batch_force_config(forced, fetch=4, ctas_per_sm=1, ctx=ctx)
    T, k_r = 40, 6
    outs = nl.nlem_denoise_batch(imgs, [k for *_, k, S in specs], [S for *_, S in specs],
                                 [10 * s for _, _, s, _, _ in specs], rho=0.7, iters=T, ctx=ctx,
                                 solver=nl.SOLVER_FAST, restart_every=k_r)
    cfg = nl.nlem_batch_config(ctx)
    assert cfg.startswith("accelerated")
    if forced == 1:
        assert "by window" in cfg
    for i, ((H, W, s, k, S), g) in enumerate(zip(specs, imgs_h)):
        ref = oracle.nlem(g, k, S, 10 * s, 0.7, T, fast=True, restart_every=k_r)
        err = rel_err(outs[i]["out"].cpu().numpy(), ref["out"])
        assert err.max() <= TOL, (i, err.max())
        assert np.all(outs[i]["iters_used"].cpu().numpy() == T)


def test_batch_accelerated_rho1_stops_by_the_rule(nl):
    """At rho = 1 (tolerance 1e-4 every 10 iterations, cap 300) Algorithm 1 reaches the cap on almost
    every pixel.  The accelerated batch stops pixels by the rule, each at a check point with its
    residual below the tolerance, as often as the oracle's accelerated solver does on a sample of the
    same pixels (these small images are hard: the oracle stops 53-72% of them)."""
    specs = [(48, 64, 20.0, 7, 21), (40, 40, 10.0, 5, 15), (56, 32, 40.0, 7, 11)]
    imgs_h = [synth.noisy_image(3700 + i, H, W, s)[0] for i, (H, W, s, k, S) in enumerate(specs)]
    imgs = [torch.from_numpy(g).to(DEV) for g in imgs_h]
    args = ([k for *_, k, S in specs], [S for *_, S in specs], [10 * s for _, _, s, _, _ in specs])
    fast = nl.nlem_denoise_batch(imgs, *args, rho=1.0, iters=300, tol=1e-4, check_every=10, solver=nl.SOLVER_FAST)
    plain = nl.nlem_denoise_batch(imgs, *args, rho=1.0, iters=300, tol=1e-4, check_every=10)
    used = np.concatenate([o["iters_used"].cpu().numpy().reshape(-1) for o in fast])
    res = np.concatenate([o["residual"].cpu().numpy().reshape(-1) for o in fast])
    used_plain = np.concatenate([o["iters_used"].cpu().numpy().reshape(-1) for o in plain])
    assert np.all((used % 10 == 0) | (used == 300))
    assert np.all(res[used < 300] < 1e-4)
    got, ref = [], []
    for (H, W, s, k, S), g, o in zip(specs, imgs_h, fast):
        pix = np.arange(0, H * W, 5)
        r = oracle.nlem(g, k, S, 10 * s, 1.0, 300, tol=1e-4, check_every=10, pixels=pix, fast=True)
        ref.append(r["iters_used"] < 300)
        got.append(o["iters_used"].cpu().numpy().reshape(-1)[pix] < 300)
    got, ref = np.concatenate(got), np.concatenate(ref)
    assert abs(got.mean() - ref.mean()) <= 0.1, (got.mean(), ref.mean())
    assert got.mean() >= np.mean(used_plain < 300) + 0.4


def test_batch_rejects_unsupported(nl):
    g = torch.zeros((20, 20), device=DEV)
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise_batch([g], [9], [11], [100.0])
    assert e.value.code == -5
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise_batch([g], [7], [23], [100.0])
    assert e.value.code == -5
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise_batch([g], [4], [11], [100.0])
    assert e.value.code == -1
    with pytest.raises(nl.NlemError) as e:   # IRLS is nlem_denoise's only
        nl.nlem_denoise_batch([g], [7], [11], [100.0], solver=nl.SOLVER_IRLS)
    assert e.value.code == -1
