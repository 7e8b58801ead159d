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
