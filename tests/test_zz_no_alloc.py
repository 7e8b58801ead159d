"""The allocation-free batched entry point, nlem_denoise_batch_noalloc, against the regular
nlem_denoise_batch on the same inputs, for two calls in a row.

It exists for callers that cannot allocate device memory themselves or through a library
(code running inside another framework's allocator or under a fixed memory budget): its
scratch space is a fixed array inside libnlem.so.  This file is collected last so that a run
stopping at its first failure has already run every other test."""
import numpy as np
import pytest

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


def _batch(seed, specs):
    imgs = [torch.from_numpy(synth.noisy_image(seed + i, H, W, s)[0]).to(DEV) for i, (H, W, s, k, S) in enumerate(specs)]
    outs = [dict(out=torch.full((H, W), -1.0, device=DEV),
                 iters_used=torch.full((H, W), -7, dtype=torch.int32, device=DEV)) for (H, W, *_ ) in specs]
    return imgs, outs


def test_noalloc_matches_batch_twice(nl):
    calls = [
        (5000, [(29, 37, 20.0, 7, 15), (18, 26, 30.0, 5, 11), (40, 21, 10.0, 5, 21)]),
        (5100, [(33, 17, 40.0, 7, 21), (25, 25, 20.0, 5, 9)]),
    ]
    ctx = nl.Context(0)
    for seed, specs in calls:
        imgs, outs = _batch(seed, specs)
        ks = [k for *_, k, S in specs]
        Ss = [S for *_, S in specs]
        hs = [10 * s for _, _, s, _, _ in specs]
        nl.nlem_denoise_batch_noalloc(imgs, ks, Ss, hs, outs, rho=0.8, iters=15)
        ref = nl.nlem_denoise_batch(imgs, ks, Ss, hs, rho=0.8, iters=15, ctx=ctx)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert rel_err(o["out"].cpu().numpy(), r["out"].cpu().numpy()).max() <= TOL
            assert torch.equal(o["iters_used"], r["iters_used"])


def test_noalloc_rejects_oversized_batch(nl):
    g = torch.zeros((8, 8), device=DEV)
    outs = [dict(out=torch.zeros((8, 8), device=DEV)) for _ in range(257)]
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_denoise_batch_noalloc([g] * 257, [5] * 257, [5] * 257, [10.0] * 257, outs)
    assert e.value.code == -1


def test_noalloc_tolerance_mode_and_residuals_match_batch(nl):
    # the residual stopping rule (tol 1e-4 checked every 10 iterations) with the residual
    # buffer: 7x7 patches run the same solver shape in both entry points, so the iteration
    # counts agree pixel by pixel and the residuals to within rounding
    specs = [(30, 26, 20.0, 7, 11), (21, 35, 40.0, 7, 15)]
    ctx = nl.Context(0)
    for call in range(2):
        imgs, outs = _batch(5200 + 10 * call, specs)
        for o, (H, W, *_ ) in zip(outs, specs):
            o["residual"] = torch.full((H, W), -3.0, device=DEV)
        ks = [k for *_, k, S in specs]
        Ss = [S for *_, S in specs]
        hs = [10 * s for _, _, s, _, _ in specs]
        nl.nlem_denoise_batch_noalloc(imgs, ks, Ss, hs, outs, rho=1e-3, iters=300, tol=1e-4, check_every=10)
        ref = nl.nlem_denoise_batch(imgs, ks, Ss, hs, rho=1e-3, iters=300, tol=1e-4, check_every=10, ctx=ctx)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o["iters_used"], r["iters_used"])
            it = o["iters_used"].cpu().numpy()
            stopped = it < 300
            assert it.min() >= 10 and stopped.mean() > 0.5          # most pixels stop by the rule
            assert rel_err(o["out"].cpu().numpy(), r["out"].cpu().numpy()).max() <= TOL
            ro, rr = o["residual"].cpu().numpy(), r["residual"].cpu().numpy()
            assert np.all(ro >= 0) and np.all(ro[stopped] < 1e-4)
            assert np.abs(ro - rr).max() <= 1e-6


def test_noalloc_error_codes_match_batch(nl):
    # the same invalid or unsupported options give the same status as nlem_denoise_batch
    import ctypes
    from paper_1501_03879_gb300 import _binding as b
    lib = nl.load_library()
    g = torch.zeros((16, 16), device=DEV)
    out = torch.zeros((16, 16), device=DEV)
    desc = (b._ImageDesc * 1)()
    desc[0].image, desc[0].out = g.data_ptr(), out.data_ptr()
    desc[0].H = desc[0].W = desc[0].pitch = 16
    desc[0].patch, desc[0].window, desc[0].h = 5, 5, 100.0
    ctx = nl.Context(0)

    def both(**kw):
        o = b._Options()
        lib.nlem_options_default(ctypes.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        rc_a = lib.nlem_denoise_batch_noalloc(desc, 1, ctypes.c_float(1.0), 5, b._Box(0.0, 255.0), ctypes.byref(o), None)
        rc_b = lib.nlem_denoise_batch(ctx.handle, desc, 1, ctypes.c_float(1.0), 5,
                                      b._Box(0.0, 255.0), ctypes.byref(o), None)
        torch.cuda.synchronize()
        return rc_a, rc_b

    assert both(precision=nl.PREC_BF16) == (-5, -5)
    assert both(layout=7) == (-1, -1)
    assert both(solver=nl.SOLVER_IRLS) == (-1, -1)
    assert both(solver=9) == (-1, -1)
    assert both(solver=nl.SOLVER_FAST, restart_every=-1) == (-1, -1)
    assert both(solver=nl.SOLVER_FAST, penalty=nl.PENALTY_WEIGHTED) == (-5, -5)
    assert both(check_every=0) == (-1, -1)
    assert both() == (0, 0)
    assert both(solver=nl.SOLVER_FAST, restart_every=3) == (0, 0)


def test_noalloc_accelerated_matches_batch(nl):
    # the accelerated solver on a fixed restart period (a schedule that does not depend on
    # rounding), 5x5 and 7x7 patches in one call, against nlem_denoise_batch
    specs = [(27, 33, 20.0, 7, 21), (31, 22, 30.0, 5, 11), (19, 40, 40.0, 7, 13)]
    ctx = nl.Context(0)
    imgs, outs = _batch(5400, specs)
    ks = [k for *_, k, S in specs]
    Ss = [S for *_, S in specs]
    hs = [10 * s for _, _, s, _, _ in specs]
    nl.nlem_denoise_batch_noalloc(imgs, ks, Ss, hs, outs, rho=1.0, iters=40, solver=nl.SOLVER_FAST,
                                  restart_every=5)
    ref = nl.nlem_denoise_batch(imgs, ks, Ss, hs, rho=1.0, iters=40, ctx=ctx, solver=nl.SOLVER_FAST,
                                restart_every=5)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o["iters_used"], r["iters_used"])
        assert rel_err(o["out"].cpu().numpy(), r["out"].cpu().numpy()).max() <= TOL


_RESET_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import synth
from paper_1501_03879_gb300 import _binding as b
lib = b.load_library()
rt = None
for line in open("/proc/self/maps"):
    if "libcudart.so" in line:
        rt = ctypes.CDLL(line.split()[-1])
        break
assert rt is not None, "libcudart not loaded by libnlem.so"
H, W = 24, 30
g = np.ascontiguousarray(synth.noisy_image(5300, H, W, 20.0)[0], dtype=np.float32)

def run():
    pi, po = ctypes.c_void_p(), ctypes.c_void_p()
    assert rt.cudaMalloc(ctypes.byref(pi), ctypes.c_size_t(g.nbytes)) == 0
    assert rt.cudaMalloc(ctypes.byref(po), ctypes.c_size_t(g.nbytes)) == 0
    assert rt.cudaMemcpy(pi, g.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(g.nbytes), 1) == 0
    d = (b._ImageDesc * 1)()
    d[0].image, d[0].out = pi.value, po.value
    d[0].H, d[0].W, d[0].pitch, d[0].patch, d[0].window, d[0].h = H, W, W, 7, 9, 200.0
    o = b._Options()
    lib.nlem_options_default(ctypes.byref(o))
    rc = lib.nlem_denoise_batch_noalloc(d, 1, ctypes.c_float(0.8), 15, b._Box(0.0, 255.0), ctypes.byref(o), None)
    assert rc == 0, lib.nlem_last_error()
    out = np.empty_like(g)
    assert rt.cudaMemcpy(out.ctypes.data_as(ctypes.c_void_p), po, ctypes.c_size_t(g.nbytes), 2) == 0
    assert rt.cudaDeviceSynchronize() == 0
    rt.cudaFree(pi); rt.cudaFree(po)
    return out

first = run()
assert rt.cudaDeviceReset() == 0      # a new primary context: the array has a new address
second = run()
np.save(sys.argv[2], np.stack([g, first, second]))
"""


def test_noalloc_after_device_reset(nl, tmp_path):
    # In a process of its own (torch is not used there): a call, cudaDeviceReset, and a call in
    # the new context.  The array's address is looked up in the current context on every call,
    # so the second call uses the new context's copy; both results equal the regular entry point.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = tmp_path / "reset.npy"
    p = subprocess.run([sys.executable, "-c", _RESET_CHILD, root, str(res)], capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    g, first, second = np.load(res)
    assert np.array_equal(first, second)
    ref = nl.nlem_denoise_batch([torch.from_numpy(g).to(DEV)], [7], [9], [200.0], rho=0.8, iters=15,
                                ctx=nl.Context(0))
    torch.cuda.synchronize()
    assert rel_err(first, ref[0]["out"].cpu().numpy()).max() <= TOL
