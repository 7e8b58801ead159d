"""The debug build (libnlem_debug.so: -DNLEM_DEBUG, bounds-checked tile, image, point-row,
work-item and accelerated-solver indices) on small cases of every NLEM kernel family and of the
accelerated solver against the FP64 oracle, with its
bounds-check record read back: no index may leave what it indexes.  It runs in a process of its
own, which loads the debug library in place of the release one."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import torch
import oracle, synth
from paper_1501_03879_gb300 import _binding as b, build
b._LIB_PATH = build.LIB_DEBUG
import paper_1501_03879_gb300 as nl
nl.load_library()
assert nl.nlem_debug_status()["count"] == 0
dev = "cuda:0"
def rel(a, r):
    return float(np.max(np.abs(np.asarray(a, np.float64) - r) / np.maximum(np.abs(r), 1.0)))
worst = 0.0
# one pixel per CTA and pixel pairs, borders wider than the window, odd sizes
for (H, W, k, S, layout) in ((23, 31, 7, 21, nl.LAYOUT_PAIR), (23, 31, 7, 21, nl.LAYOUT_PIXEL), (9, 40, 5, 11, 0),
                             (17, 12, 9, 13, 0), (8, 8, 7, 9, nl.LAYOUT_PAIR)):
    g, _ = synth.noisy_image(6000 + H + W, H, W, 20.0)
    r = nl.nlem_denoise(torch.from_numpy(g).to(dev), patch=k, window=S, h=200.0, rho=0.5, iters=12, layout=layout)
    worst = max(worst, rel(r["out"].cpu().numpy(), oracle.nlem(g, k, S, 200.0, 0.5, 12)["out"]))
# the batched launch (both shape variants) and a standalone batch
specs = [(21, 30, 5, 11), (26, 19, 7, 21), (12, 33, 7, 13)]
imgs = [synth.noisy_image(6100 + i, H, W, 30.0)[0] for i, (H, W, k, S) in enumerate(specs)]
for v in (0, 1):
    ctx = nl.Context(0)
    nl.nlem_batch_force_config(v, fetch=4, ctas_per_sm=2, ctx=ctx)
    outs = nl.nlem_denoise_batch([torch.from_numpy(g).to(dev) for g in imgs], [k for *_, k, S in specs],
                                 [S for *_, S in specs], [300.0] * 3, rho=0.5, iters=10, ctx=ctx)
    for (H, W, k, S), g, o in zip(specs, imgs, outs):
        worst = max(worst, rel(o["out"].cpu().numpy(), oracle.nlem(g, k, S, 300.0, 0.5, 10)["out"]))
pts = synth.em_points(61, np.arange(3), 300, 49)
w = synth.em_weights(61, np.arange(3), 300)
x = nl.em_solve_batch(torch.from_numpy(pts).to(dev), torch.from_numpy(w).to(dev), rho=0.5, iters=15)["x"]
worst = max(worst, rel(x.cpu().numpy(), oracle.em_admm_batch(pts, w, 0.0, 255.0, 0.5, 15)[0]))
# the accelerated solver on a fixed restart period (its schedule does not depend on rounding): NLEM one
# pixel per CTA, both batch variants (5x5 and 7x7) and a standalone batch
g, _ = synth.noisy_image(6200, 23, 31, 20.0)
r = nl.nlem_denoise(torch.from_numpy(g).to(dev), patch=7, window=21, h=200.0, rho=0.5, iters=12,
                    solver=nl.SOLVER_FAST, restart_every=4)
worst = max(worst, rel(r["out"].cpu().numpy(), oracle.nlem(g, 7, 21, 200.0, 0.5, 12, fast=True, restart_every=4)["out"]))
for v in (0, 1):
    ctx = nl.Context(0)
    nl.nlem_batch_force_config(v, fetch=4, ctas_per_sm=1, ctx=ctx)
    outs = nl.nlem_denoise_batch([torch.from_numpy(g).to(dev) for g in imgs], [k for *_, k, S in specs],
                                 [S for *_, S in specs], [300.0] * 3, rho=0.5, iters=10, ctx=ctx,
                                 solver=nl.SOLVER_FAST, restart_every=3)
    for (H, W, k, S), g, o in zip(specs, imgs, outs):
        ref = oracle.nlem(g, k, S, 300.0, 0.5, 10, fast=True, restart_every=3)["out"]
        worst = max(worst, rel(o["out"].cpu().numpy(), ref))
x = nl.em_solve_batch(torch.from_numpy(pts).to(dev), torch.from_numpy(w).to(dev), rho=0.5, iters=15,
                      solver=nl.SOLVER_FAST, restart_every=5)["x"]
worst = max(worst, rel(x.cpu().numpy(), oracle.em_admm_batch(pts, w, 0.0, 255.0, 0.5, 15, fast=True,
                                                             restart_every=5)[0]))
st = nl.nlem_debug_status()
print("DEBUG", st["count"], st["site"], st["index"], st["limit"], worst)
"""


def test_debug_build_bounds_checks_and_parity():
    from paper_1501_03879_gb300 import build
    build.build(debug=True)
    p = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout + p.stderr
    line = [l for l in p.stdout.splitlines() if l.startswith("DEBUG")][-1].split()
    count, site, index, limit, worst = int(line[1]), int(line[2]), int(line[3]), int(line[4]), float(line[5])
    assert count == 0, f"bounds check failed at site {site}: index {index} of {limit}"
    assert worst <= 1e-4


def test_release_build_has_no_debug_record():
    import paper_1501_03879_gb300 as nl
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nl.load_library()
    with pytest.raises(nl.NlemError) as e:
        nl.nlem_debug_status()
    assert e.value.code == -5
