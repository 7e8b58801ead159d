"""em_solve_batch_host: the batch solve on host buffers with chunked, double-buffered copies that
overlap the solves.  Every problem is solved by one CTA on its own, so the results must equal
em_solve_batch's on the same inputs bit for bit, whatever the chunking."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_03879_gb300 as m
    m.load_library()
    return m


def _inputs(seed, B, n, d, pinned):
    pts = torch.from_numpy(synth.em_points(seed, np.arange(B), n, d))
    w = torch.from_numpy(synth.em_weights(seed, np.arange(B), n))
    if pinned:
        pts, w = pts.pin_memory(), w.pin_memory()
    return pts, w


@pytest.mark.parametrize("chunk", [300, 1000, 0])
def test_host_batch_equals_device_batch(nl, chunk):
    """1000 problems of 441 x 49 in chunks of 300 (four chunks, the last one ragged), one chunk, and
    the automatic size; tolerance mode, so the iteration counts and residuals are compared too."""
    B, n, d = 1000, 441, 49
    pts, w = _inputs(4100, B, n, d, pinned=True)
    kw = dict(rho=1e-3, iters=60, tol=1e-4, check_every=5)
    h = nl.em_solve_batch_host(pts, w, chunk=chunk, **kw)
    g = nl.em_solve_batch(pts.to(DEV), w.to(DEV), **kw)
    assert torch.equal(h["x"], g["x"].cpu())
    assert torch.equal(h["iters_used"], g["iters_used"].cpu())
    assert torch.equal(h["residual"], g["residual"].cpu())


def test_host_batch_many_chunks_start_points_and_pageable_memory(nl):
    """714 chunks of 7 problems (each double buffer reused hundreds of times), caller start points,
    pageable host memory: still equal to the device call, and a few problems against the oracle."""
    B, n, d = 5000, 33, 2
    pts, w = _inputs(4200, B, n, d, pinned=False)
    x0 = torch.from_numpy(np.ascontiguousarray(pts.numpy()[:, 0, :] * 0.5 + 10.0))
    kw = dict(rho=1.0, iters=25)
    h = nl.em_solve_batch_host(pts, w, x0=x0, chunk=7, **kw)
    g = nl.em_solve_batch(pts.to(DEV), w.to(DEV), x0=x0.to(DEV), **kw)
    assert torch.equal(h["x"], g["x"].cpu())
    assert torch.equal(h["iters_used"], g["iters_used"].cpu())
    for b in (0, 6, 7, 4999):
        z, *_ = oracle.em_admm(pts[b].numpy().astype(np.float64), w[b].numpy().astype(np.float64), 0.0, 255.0, 1.0,
                               25, z0=x0[b].numpy().astype(np.float64))
        assert np.max(np.abs(h["x"][b].numpy() - z) / np.maximum(np.abs(z), 1.0)) <= 1e-4


def test_host_batch_arguments(nl):
    pts, w = _inputs(4300, 4, 5, 3, pinned=False)
    r = nl.em_solve_batch_host(pts[:0], w[:0], iters=3)          # B = 0: nothing to do
    assert r["x"].shape == (0, 3)
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch_host(pts, w, chunk=-1)
    assert e.value.code == -1
    with pytest.raises(ValueError):
        nl.em_solve_batch_host(pts.to(DEV), w.to(DEV))        # device tensors belong to em_solve_batch
    with pytest.raises(nl.NlemError) as e:
        nl.em_solve_batch_host(pts, w, rho=0.0)
    assert e.value.code == -1
