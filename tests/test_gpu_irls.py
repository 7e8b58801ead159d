"""GPU NLEM-IRLS (IRLS on the surrogate of Eq. 2 inside the one-pixel NLEM kernel, the comparison
method of Sec. 3) against the FP64 oracle's composition of the NLEM problem and IRLS.
Tolerance as for every FP32 path: |x_gpu - x_oracle| <= 1e-4 * max(|x_oracle|, 1) per pixel."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
DEV = "cuda:0"
EPS = 1e-6


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


# every compiled IRLS shape: patch 7 with windows 11 (E49_2), 15 (4x3), 21 (7) and 29 (7W), patch 5
# and 9 on their one shape; both start points; clipped windows on every border
@pytest.mark.parametrize("k,S,H,W,init,T", [(7, 21, 26, 23, 1, 4), (7, 21, 20, 24, 0, 10), (7, 11, 17, 19, 1, 4),
                                            (7, 15, 18, 16, 0, 6), (7, 29, 33, 31, 1, 3), (5, 13, 15, 17, 0, 5),
                                            (9, 15, 19, 18, 1, 4), (5, 3, 9, 8, 1, 4)])
def test_irls_all_pixels_against_oracle(nl, k, S, H, W, init, T):
    sigma = 20.0
    g, _ = synth.noisy_image(5100 + 11 * k + S + H, H, W, sigma)
    h = 10 * sigma
    r = nl.nlem_denoise(_t(g), patch=k, window=S, h=h, rho=1.0, iters=T, init=init, solver=nl.SOLVER_IRLS,
                        irls_eps=EPS, fp64_check=True)
    ref = oracle.nlem_irls(g, k, S, h, EPS, T, init_mode=init)
    err = rel_err(r["out"].cpu().numpy(), ref["out"])
    assert err.max() <= TOL, err.max()
    assert np.all(r["iters_used"].cpu().numpy() == T)
    # the last relative step, and the FP64 objective of problem (1) at the GPU's x(T).  After a few
    # steps x(T) is not a minimiser, so the objective moves to first order with x: F is Lipschitz
    # with constant sum_k w_k, and ||x_gpu - x_ref|| <= sqrt(d) * TOL * 255 under the tolerance above.
    st = r["residual"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(st - ref["step"]) <= 1e-3 * ref["step"] + 2e-6), np.max(np.abs(st - ref["step"]))
    ob = r["obj64"].cpu().numpy()
    assert np.all(np.abs(ob - ref["obj"]) <= ref["wsum"] * k * TOL * 255.0)


def test_irls_other_eps_and_zero_steps(nl):
    """A larger epsilon (the surrogate moves away from problem (1)) and iters = 0 (the start point,
    equal to EM-ADMM's with zero iterations)."""
    g, _ = synth.noisy_image(5201, 22, 21, 40.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=21, h=400.0, iters=5, init=1, solver=nl.SOLVER_IRLS, irls_eps=4.0)
    ref = oracle.nlem_irls(g, 7, 21, 400.0, 4.0, 5, init_mode=1)
    assert rel_err(r["out"].cpu().numpy(), ref["out"]).max() <= TOL
    for init in (0, 1):
        a = nl.nlem_denoise(_t(g), patch=7, window=21, h=400.0, iters=0, init=init, solver=nl.SOLVER_IRLS)
        b = nl.nlem_denoise(_t(g), patch=7, window=21, h=400.0, iters=0, init=init, layout=nl.LAYOUT_PIXEL)
        assert torch.equal(a["out"], b["out"])
        assert torch.all(a["iters_used"] == 0) and torch.all(a["residual"] == 0)


def test_irls_full_size_sampled(nl):
    """512 x 512, 7x7 patches, 21x21 window, sigma 20, 4 steps from the noisy patch (the setting
    of Sec. 3): sampled pixels on the borders, the corners and the interior against the oracle."""
    H = W = 512
    g, _ = synth.noisy_image(5301, H, W, 20.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=21, h=200.0, iters=4, init=1, solver=nl.SOLVER_IRLS)
    rng = np.random.default_rng(5301)
    pix = np.unique(np.concatenate([[0, W - 1, (H - 1) * W, H * W - 1, 9 * W + 3, 300 * W + 511],
                                    rng.integers(0, H * W, 60)]))
    ref = oracle.nlem_irls(g, 7, 21, 200.0, EPS, 4, init_mode=1, pixels=pix)
    got = r["out"].cpu().numpy().reshape(-1)[pix]
    assert rel_err(got, ref["out"]).max() <= TOL


def test_irls_bf16_weights(nl):
    """BF16 tensor-core cross terms feed IRLS as they feed EM-ADMM: the result is IRLS on the
    oracle's BF16 weight model."""
    g, _ = synth.noisy_image(5401, 24, 22, 20.0)
    r = nl.nlem_denoise(_t(g), patch=7, window=15, h=200.0, iters=4, init=1, solver=nl.SOLVER_IRLS,
                        precision=nl.PREC_BF16)
    got = r["out"].cpu().numpy().reshape(-1)
    errs = []
    for lin in range(0, 24 * 22, 37):
        pts, w, pc = oracle.nlem_problem(g, 7, 15, 200.0, lin, weight_mode=1)
        x, _ = oracle.irls(pts, w, 0.0, 255.0, oracle.project_box(pc, 0.0, 255.0), EPS, 4)
        errs.append(float(rel_err(got[lin], x[24])))
    print(f"IRLS on BF16 weights vs the oracle's BF16 model: max rel {max(errs):.3e}, median {np.median(errs):.3e}")
    assert max(errs) <= TOL


def test_irls_argument_errors(nl):
    g = _t(synth.noisy_image(5501, 16, 16, 20.0)[0])
    with pytest.raises(nl.NlemError) as e:      # the pair kernel runs EM-ADMM only
        nl.nlem_denoise(g, patch=7, window=21, iters=2, solver=nl.SOLVER_IRLS, layout=nl.LAYOUT_PAIR)
    assert e.value.code == -5
    for kw in (dict(tol=1e-4), dict(irls_eps=0.0), dict(irls_eps=float("nan")), dict(solver=7)):
        with pytest.raises(nl.NlemError) as e:
            nl.nlem_denoise(g, patch=7, window=21, iters=2, **dict(dict(solver=nl.SOLVER_IRLS), **kw))
        assert e.value.code == -1
    # entry points that run EM-ADMM only refuse the IRLS option
    from paper_1501_03879_gb300 import _binding as b
    lib = b.load_library()
    ctx = b._ctx(torch.device(DEV))
    o = b._options(solver=nl.SOLVER_IRLS)
    pts = torch.zeros((2, 5, 3), device=DEV)
    w = torch.ones((2, 5), device=DEV)
    x = torch.empty((2, 3), device=DEV)
    rc = lib.em_solve_batch(ctx.handle, b._ptr(pts), b._ptr(w), 2, 5, 3, b._Box(0.0, 255.0), ctypes.c_float(1.0), 3,
                            None, ctypes.byref(o), b._ptr(x), None, None, None, None, None)
    assert rc == -1
    assert "EM-ADMM only" in lib.nlem_last_error().decode()
