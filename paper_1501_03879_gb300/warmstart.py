"""Training of the learned warm start from solves the method itself produces.

For each training image, a seeded sample of pixels gets its features (nlem_features) and its
labels (nlem_ws_labels): every pixel is solved (tolerance 1e-4) from the weighted-mean start with
every penalty of a grid; the label penalty is the one that reaches the tolerance in the fewest
iterations, and the label start point is the solution patch of a tight solve (tolerance 1e-6)
with that penalty.  Targets for the network output y: y[0:d] = (z* - m) / 16 and y[d] = ln rho*.
Training runs the library's forward, backward and Adam kernels on shuffled minibatches
(nlem_ws_train).  All of it runs in the library; torch only holds device arrays and this module
only picks the pixels.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B

RHO_GRID = (1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1, 3e-1, 1.0)
DELTA_SCALE = 16.0


def make_training_set(images, hs, patch=7, window=21, per_image=4096, seed=0, tol=1e-4, check_every=5, cap=300,
                      tight_tol=1e-6, tight_cap=2000, rho_grid=RHO_GRID, ctx=None):
    """images: float32 CUDA tensors [H, W]; hs: their weight scales h; per_image: pixels sampled
    per image (one count, or one per image).  Returns (feats [N,2d+2], targets [N,d+1], info) on
    the device."""
    import torch
    d = patch * patch
    feats_all, tgt_all = [], []
    rng = np.random.default_rng(seed)
    best_counts = np.zeros(len(rho_grid), dtype=np.int64)
    counts = list(per_image) if isinstance(per_image, (list, tuple)) else [per_image] * len(images)
    for img, h, kk in zip(images, hs, counts):
        H, W = img.shape
        dev = img.device
        k = min(kk, H * W)
        pix_np = np.sort(rng.choice(H * W, k, replace=False)).astype(np.int32)
        pix = torch.from_numpy(pix_np).to(dev)
        feats = B.nlem_features(img, patch, window, h, pixels=pix, ctx=ctx)
        tgt, won = B.nlem_ws_labels(img, pix, feats, rho_grid, patch=patch, window=window, h=h, tol=tol,
                                       check_every=check_every, cap=cap, tight_tol=tight_tol, tight_cap=tight_cap,
                                       ctx=ctx)
        best_counts += np.asarray(won, dtype=np.int64)
        feats_all.append(feats)
        tgt_all.append(tgt)
    info = {"rho_grid": list(rho_grid), "best_rho_counts": best_counts.tolist()}
    return torch.cat(feats_all), torch.cat(tgt_all), info


def train(ws: B.WarmStart, feats, targets, epochs=10, batch=4096, lr=1e-3, seed=0):
    """Adam on shuffled minibatches of the training set, entirely in the library
    (nlem_ws_train); returns the mean minibatch loss of each epoch."""
    return ws.train(feats.contiguous(), targets.contiguous(), epochs, batch, lr, seed)


def evaluate(ws: B.WarmStart, image, h, patch=7, window=21, cap=300, tol=1e-4, check_every=10, rho_plain=1.0,
             ctx=None):
    """Warm-started vs plain EM-ADMM on one image: mean iterations to the tolerance and the
    number of pixels that fell back."""
    import torch
    warm = B.nlem_denoise_warm(ws, image, patch, window, h, rho_fallback=rho_plain, iters=cap, tol=tol,
                               check_every=check_every, ctx=ctx)
    plain = B.nlem_denoise(image, patch, window, h, rho=rho_plain, iters=cap, tol=tol, check_every=check_every,
                           ctx=ctx)
    torch.cuda.synchronize()
    return dict(warm_iters=float(warm["iters_used"].float().mean().item()),
                plain_iters=float(plain["iters_used"].float().mean().item()),
                fallback=warm["fallback"], warm=warm, plain=plain)
