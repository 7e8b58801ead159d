"""Seeded synthetic inputs shared by the CUDA path, the FP64 oracle, the tests and the bench.

This module holds no arithmetic of the denoising method: it only draws random numbers and
paints test images.  Every draw comes from one counter-based generator, SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), used
in counter mode: output ``i`` of a stream whose state starts at ``key`` is
``mix64(key + (i + 1) * GOLDEN)``.  Any element of any stream can therefore be regenerated on
its own, which lets the oracle recompute a sampled subset of a device-sized batch.

The one device-side generator (``gen_points.cu`` beside this file, built into
``libsynth.so``) implements the same published definition and uses only integer operations
and correctly rounded FP32 multiplies, so both sides produce identical bits.

Workloads follow the denoising experiments of the paper (Sec. 3: grayscale images, additive
i.i.d. Gaussian noise g = f + sigma*xi, patch k, search window S, h = 10*sigma).  The test
images themselves are not available, so a procedural image stands in for them: a linear
gradient with 8 axis-aligned rectangles and 4 disks of random intensity.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (one independent SplitMix64 stream per purpose)
STREAM_SHAPES = 1
STREAM_NOISE_A = 2
STREAM_NOISE_B = 3
STREAM_SP_SELECT = 4
STREAM_SP_VALUE = 5
STREAM_PTS_VALUE = 11
STREAM_PTS_OUTLIER = 12
STREAM_PTS_BERNOULLI = 13
STREAM_WEIGHTS = 14
STREAM_BATCH_META = 21

OUTLIER_THRESHOLD_24 = 1677721  # floor(0.1 * 2**24): a point is an outlier iff its 24-bit draw is below this


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output mixing function (the published finaliser), on uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Initial SplitMix64 state of stream ``stream`` under ``seed``."""
    s = np.array([((seed & 0xFFFFFFFF) << 32) | (stream & 0xFFFFFFFF)], dtype=np.uint64)
    return mix64(s)[0]


def draw_u64(key: np.uint64, idx) -> np.ndarray:
    """Output number ``idx`` (0-based) of the stream whose state starts at ``key``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(key) + (idx + np.uint64(1)) * GOLDEN
    return mix64(x)


def draw_u24(key, idx) -> np.ndarray:
    """Top 24 bits of a draw, as uint32 in [0, 2**24)."""
    return (draw_u64(key, idx) >> np.uint64(40)).astype(np.uint32)


def uniform53(key, idx) -> np.ndarray:
    """Uniform float64 in [0, 1) from the top 53 bits of a draw."""
    return (draw_u64(key, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_open53(key, idx) -> np.ndarray:
    """Uniform float64 in (0, 1]."""
    return ((draw_u64(key, idx) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


# ----------------------------------------------------------------------------------------
# images
# ----------------------------------------------------------------------------------------

def clean_image(seed: int, H: int, W: int) -> np.ndarray:
    """Procedural clean image in [0, 255] (float64, H x W).

    Draw order: a linear gradient ramping from 32 to 224 along a random direction across the
    image, then 8 axis-aligned rectangles (top-left corner uniform in the image, sides
    uniform on [side/8, side/2], clipped at the border) and 4 disks (centre uniform, radius
    uniform on [m/16, m/4], m = min(H, W)); each shape has an intensity uniform on [0, 255]
    and later shapes overwrite earlier ones.
    """
    key = stream_key(seed, STREAM_SHAPES)
    u = uniform53(key, np.arange(64))
    it = iter(u)
    theta = 2.0 * math.pi * next(it)
    rr, cc = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    proj = cc * math.cos(theta) + rr * math.sin(theta)
    corners = [0.0, (W - 1) * math.cos(theta), (H - 1) * math.sin(theta),
               (W - 1) * math.cos(theta) + (H - 1) * math.sin(theta)]
    pmin, pmax = min(corners), max(corners)
    span = pmax - pmin if pmax > pmin else 1.0
    img = 32.0 + 192.0 * (proj - pmin) / span
    for _ in range(8):
        hr = H / 8.0 + next(it) * (H / 2.0 - H / 8.0)
        wr = W / 8.0 + next(it) * (W / 2.0 - W / 8.0)
        r0 = int(next(it) * H)
        c0 = int(next(it) * W)
        val = 255.0 * next(it)
        img[r0:min(H, r0 + int(round(hr))), c0:min(W, c0 + int(round(wr)))] = val
    m = float(min(H, W))
    for _ in range(4):
        cr = next(it) * H
        ccen = next(it) * W
        rad = m / 16.0 + next(it) * (m / 4.0 - m / 16.0)
        val = 255.0 * next(it)
        img[(rr - cr) ** 2 + (cc - ccen) ** 2 <= rad * rad] = val
    return img


def gaussian(seed: int, count: int) -> np.ndarray:
    """count i.i.d. N(0,1) draws (Box-Muller on two independent uniform streams)."""
    idx = np.arange(count)
    u1 = uniform_open53(stream_key(seed, STREAM_NOISE_A), idx)
    u2 = uniform53(stream_key(seed, STREAM_NOISE_B), idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def noisy_image(seed: int, H: int, W: int, sigma: float, salt_pepper: float = 0.0):
    """Return (noisy float32 image, clean float64 image).

    Noise model of Sec. 3: g = f + sigma * xi, xi i.i.d. N(0,1), not clipped.  With
    ``salt_pepper`` > 0 that fraction of pixels is then replaced by 0 or 255 with
    probability 1/2 each (impulse noise on top of the Gaussian noise).
    """
    f = clean_image(seed, H, W)
    g = f + sigma * gaussian(seed, H * W).reshape(H, W)
    if salt_pepper > 0.0:
        idx = np.arange(H * W)
        sel = uniform53(stream_key(seed, STREAM_SP_SELECT), idx) < salt_pepper
        hi = uniform53(stream_key(seed, STREAM_SP_VALUE), idx) < 0.5
        flat = g.reshape(-1)
        flat[sel & hi] = 255.0
        flat[sel & ~hi] = 0.0
    return np.ascontiguousarray(g.astype(np.float32)), f


def psnr(x: np.ndarray, ref: np.ndarray, peak: float = 255.0) -> float:
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * math.log10(peak * peak / mse)


# ----------------------------------------------------------------------------------------
# standalone Euclidean-median batches: points uniform on [0,255], 10% whole-point outliers
# at 255*Bernoulli(1/2) per coordinate, weights Exp(1)
# ----------------------------------------------------------------------------------------

def em_points(seed: int, problems, n: int, d: int) -> np.ndarray:
    """Points of the listed problems, float32 array [len(problems), n, d].

    Element (b, k, q) has linear index L = (b*n + k)*d + q.  Non-outlier values are
    round_f32(255 * k24) * 2**-24 with k24 the top 24 bits of draw L of the value stream; a
    point is an outlier iff draw (b*n + k) of the outlier stream has k24 < 1677721, and then
    coordinate q is 255 if draw L of the Bernoulli stream has its top bit set, else 0.
    """
    problems = np.asarray(problems, dtype=np.int64).reshape(-1)
    kv = stream_key(seed, STREAM_PTS_VALUE)
    ko = stream_key(seed, STREAM_PTS_OUTLIER)
    kb = stream_key(seed, STREAM_PTS_BERNOULLI)
    pt = (problems[:, None] * n + np.arange(n)[None, :])            # [P, n] point index
    L = pt[:, :, None] * d + np.arange(d)[None, None, :]            # [P, n, d]
    k24 = draw_u24(kv, L.reshape(-1)).reshape(L.shape)
    val = k24.astype(np.float32) * np.float32(255.0)
    val = val * np.float32(2.0 ** -24)
    out_flag = draw_u24(ko, pt.reshape(-1)).reshape(pt.shape) < OUTLIER_THRESHOLD_24
    bern = (draw_u64(kb, L.reshape(-1)) >> np.uint64(63)).reshape(L.shape).astype(bool)
    ov = np.where(bern, np.float32(255.0), np.float32(0.0))
    return np.ascontiguousarray(np.where(out_flag[:, :, None], ov, val).astype(np.float32))


def em_weights(seed: int, problems, n: int) -> np.ndarray:
    """Weights Exp(1) of the listed problems, float32 [len(problems), n] (host only)."""
    problems = np.asarray(problems, dtype=np.int64).reshape(-1)
    idx = problems[:, None] * n + np.arange(n)[None, :]
    u = uniform_open53(stream_key(seed, STREAM_WEIGHTS), idx.reshape(-1))
    return np.ascontiguousarray((-np.log(u)).astype(np.float32).reshape(idx.shape))


# ----------------------------------------------------------------------------------------
# workload descriptions
# ----------------------------------------------------------------------------------------

@dataclass
class ImageSpec:
    seed: int
    H: int
    W: int
    sigma: float
    patch: int
    window: int
    salt_pepper: float = 0.0

    @property
    def h(self) -> float:
        return 10.0 * self.sigma          # h = 10*sigma (Sec. 3, NLM parameters)

    def make(self):
        return noisy_image(self.seed, self.H, self.W, self.sigma, self.salt_pepper)


def batch_specs(seed: int, count: int = 64, side_lo: int = 128, side_hi: int = 1024):
    """Uneven image batch: sides uniform on [side_lo, side_hi] drawn independently for H and
    W, sigma in {10,20,30,40}, search radius uniform on {5..10}, patch 5x5 or 7x7."""
    key = stream_key(seed, STREAM_BATCH_META)
    u = uniform53(key, np.arange(count * 8)).reshape(count, 8)
    specs = []
    for i in range(count):
        H = side_lo + int(u[i, 0] * (side_hi - side_lo + 1))
        W = side_lo + int(u[i, 1] * (side_hi - side_lo + 1))
        sigma = float((10, 20, 30, 40)[int(u[i, 2] * 4)])
        radius = 5 + int(u[i, 3] * 6)
        patch = 5 if u[i, 4] < 0.5 else 7
        specs.append(ImageSpec(seed * 1000 + i, H, W, sigma, patch, 2 * radius + 1))
    return specs


# ----------------------------------------------------------------------------------------
# device generator (same published definition; integer ops and correctly rounded multiplies)
# ----------------------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
SYNTH_LIB = os.path.join(_HERE, "libsynth.so")


def build_device_generator(verbose: bool = False) -> str:
    import subprocess
    src = os.path.join(_HERE, "gen_points.cu")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
           "-Xcompiler", "-fPIC", "-shared", "-o", SYNTH_LIB, src]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return SYNTH_LIB


def device_em_points(seed: int, B: int, n: int, d: int, out_ptr: int, stream_ptr: int = 0) -> None:
    """Fill a device float32 buffer [B, n, d] with em_points(seed, range(B), n, d)."""
    import ctypes
    lib = ctypes.CDLL(SYNTH_LIB)
    lib.synth_em_points.restype = ctypes.c_int
    lib.synth_em_points.argtypes = [ctypes.c_uint64] * 3 + [ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                                             ctypes.c_void_p, ctypes.c_void_p]
    rc = lib.synth_em_points(int(stream_key(seed, STREAM_PTS_VALUE)), int(stream_key(seed, STREAM_PTS_OUTLIER)),
                             int(stream_key(seed, STREAM_PTS_BERNOULLI)), B, n, d,
                             ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"synth_em_points failed with CUDA error {rc}")
