"""FP64 CPU oracle (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the CPU-baseline and
reference legs of bench.py.  It shares no code with the CUDA library (`paper_1501_03879_gb300`)
and never imports it.

Functions mirror the passages of Chaudhury & Ramakrishnan (arXiv 1501.03879) cited in
oracle.c: the closed-form prox (Sec. 2, Eq. closed-form), the conjugate prox (Eq. proxfstar),
the box projection (Sec. 3), Algorithm 1 (EM-ADMM) and the NLEM driver (Sec. 3,
Eq. L1regression).  Parity status of each function is listed in PINS below.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
SRC = os.path.join(_HERE, "oracle.c")

# every public function and what pins it (tests/test_oracle_*.py)
PINS = {
    "prox": "argmin of Eq. defprox by brute force (d=1,2), limits lam=0 / lam=inf, Moreau identity",
    "prox_conj": "ball projection: norm <= lam, Moreau identity",
    "project_box": "coordinate clamp, idempotent, nonexpansive",
    "em_admm": "n=1, n=2, d=1 weighted median, planar Fermat point, brute-force grid, KKT, "
               "Weiszfeld agreement, one step against numeric argmins of the augmented Lagrangian, "
               "invariances",
    "residuals": "r_pri / r_dual against their definitions on stored iterates (step-by-step replay)",
    "nlem": "patch/weight assembly against numpy.pad reflect; constant image; S=1; k=1 weighted median",
    "irls": "surrogate stationarity; converges to the EM within sqrt(eps)-scale",
    "em_admm_fast": "first two iterations equal Algorithm 1's; converges to em_admm's optimum (random "
                    "problems, d=1 weighted median, planar Fermat point); fewer iterations than Algorithm 1 "
                    "to the stopping rule at mu = 1 on NLEM problems",
    "project_set": "per-coordinate boxes: coordinate clamp; ball: brute-force argmin on a 2-D grid, "
                   "idempotent, interior points fixed",
    "em_admm_set": "equal bounds reproduce em_admm's box run; d=1 boxes give the clamped weighted median; "
                   "large ball gives the unconstrained median, radius 0 the centre; 2-D brute-force minimum "
                   "over the ball and over a box",
    "nlem_color": "identical channels equal grayscale NLEM at h/sqrt(C), mu*sqrt(C); one varying channel "
                  "beside constant ones equals grayscale NLEM; channel permutation; constant image",
    "nlem_irls": "k=1 windows: the weighted median of the window's pixels after many steps; constant "
                 "image; one pixel equals irls on nlem_problem; zero steps give the start point",
    "weiszfeld": "objective non-increasing; agrees with ADMM at convergence",
    "features": "weighted median: dominant weight, equal weights (ordinary median), d=1 problem (1) "
                "solution; entropy of uniform weights = log n; weighted mean = 1-point mean",
    "mlp": "loss gradient against central finite differences of the loss",
}

_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", LIB_PATH, SRC, "-lm", "-lpthread"]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
    return LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(LIB_PATH)
    D = ctypes.POINTER(ctypes.c_double)
    F = ctypes.POINTER(ctypes.c_float)
    I = ctypes.POINTER(ctypes.c_int)
    LL = ctypes.POINTER(ctypes.c_longlong)
    c_int, c_double, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.orc_prox.argtypes = [D, D, c_double, c_int, D]
    lib.orc_prox_conj.argtypes = [D, D, c_double, c_int, D]
    lib.orc_project_box.argtypes = [D, c_int, c_double, c_double, D]
    lib.orc_project_set.argtypes = [D, c_int, c_int, D, D, c_double, D]
    lib.orc_em_admm_fast.argtypes = [D, D, c_int, c_int, c_double, c_double, c_double, c_int, D, c_double, c_int,
                                     c_double, c_int, c_int, D, ctypes.POINTER(c_int), D, D, ctypes.POINTER(c_int), D]
    lib.orc_em_admm_fast.restype = c_int
    lib.orc_em_admm_set.argtypes = [D, D, c_int, c_int, c_int, D, D, c_double, c_double, c_int, D, c_double, c_int,
                                    D, ctypes.POINTER(c_int), D, D]
    lib.orc_em_admm_set.restype = c_int
    lib.orc_objective.argtypes = [D, D, D, c_int, c_int]
    lib.orc_objective.restype = c_double
    lib.orc_kkt_residual.argtypes = [D, D, D, c_int, c_int, c_double, c_double, c_double]
    lib.orc_kkt_residual.restype = c_double
    lib.orc_weighted_mean_start.argtypes = [D, D, c_int, c_int, c_double, c_double, D]
    lib.orc_em_admm.argtypes = [D, D, c_int, c_int, c_double, c_double, c_double, c_int, D,
                                c_double, c_int, D, I, D, D]
    lib.orc_em_admm.restype = c_int
    lib.orc_weiszfeld.argtypes = [D, D, c_int, c_int, D, c_int, D, D]
    lib.orc_irls.argtypes = [D, D, c_int, c_int, c_double, c_double, D, c_double, c_int, D, D]
    lib.orc_em_admm_batch.argtypes = [F, F, c_ll, c_int, c_int, c_double, c_double, c_double, c_int,
                                      F, c_double, c_int, D, I, D, D, c_int, c_int, I, D, c_int]
    lib.orc_em_admm_batch.restype = c_int
    lib.orc_nlem.argtypes = [F, c_int, c_int, c_int, c_int, c_double, c_double, c_int, c_double,
                             c_double, c_double, c_int, c_int, c_int, LL, c_ll, D, I, D, D, I, D, c_int, c_int, I,
                             D, c_int]
    lib.orc_nlem.restype = c_int
    lib.orc_em_admm_wpen.argtypes = [D, D, c_int, c_int, c_double, c_double, c_double, c_int, D, c_double, c_int,
                                     D, I, D, D]
    lib.orc_em_admm_wpen.restype = c_int
    lib.orc_nlem_problem.argtypes = [F, c_int, c_int, c_int, c_int, c_double, c_ll, c_int, D, D, D]
    lib.orc_nlem_problem.restype = c_int
    lib.orc_num_cores.restype = c_int
    lib.orc_features.argtypes = [D, D, c_int, c_int, D]
    lib.orc_mlp_forward.argtypes = [D, c_int, c_int, c_double, D, c_ll, D]
    lib.orc_mlp_loss_grad.argtypes = [D, c_int, c_int, c_double, D, D, c_ll, D]
    lib.orc_mlp_loss_grad.restype = c_double
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_cores() -> int:
    return int(_load().orc_num_cores())


def prox(v, u, lam):
    """Eq. (closed-form): Psi_lam(v, u)."""
    v, u = _f64(v), _f64(u)
    out = np.empty_like(v)
    _load().orc_prox(_dp(v), _dp(u), float(lam), v.size, _dp(out))
    return out


def prox_conj(v, u, lam):
    """Eq. (proxfstar): projection of v - u onto the ball of radius lam."""
    v, u = _f64(v), _f64(u)
    out = np.empty_like(v)
    _load().orc_prox_conj(_dp(v), _dp(u), float(lam), v.size, _dp(out))
    return out


def project_box(x, lo, hi):
    x = _f64(x)
    out = np.empty_like(x)
    _load().orc_project_box(_dp(x), x.size, float(lo), float(hi), _dp(out))
    return out


SET_COORD_BOXES = 1
SET_BALL = 2


def project_set(x, kind, a, b=None, r=0.0):
    """Projection onto per-coordinate boxes prod_q [a_q, b_q] (kind 1) or the ball ||x - a|| <= r
    (kind 2): the constraint sets beyond the box that problem (1) admits (Sec. 2)."""
    x, a = _f64(x), _f64(a)
    b = _f64(b) if b is not None else np.zeros_like(a)
    out = np.empty_like(x)
    _load().orc_project_set(_dp(x), x.size, int(kind), _dp(a), _dp(b), float(r), _dp(out))
    return out


def em_admm_fast(pts, w, lo, hi, mu, iters, z0=None, tol=0.0, check_every=1, eta=0.999, with_margin=False,
                 restart_every=0, combined=False):
    """Accelerated Algorithm 1 (fast ADMM with restart, Goldstein et al. 2014; accelerated ADMM is
    the future work Sec. 4 names).  The restart test compares the z-part mu n ||z - z_hat||^2 of
    Goldstein's combined residual (combined=True: the whole combined residual); restart_every = k > 0
    restarts after every k-th iteration instead.  Returns (z, iters_used, r_pri, r_dual, restarts),
    plus the decision margin min |c / (eta c_prev) - 1| with with_margin."""
    pts, w = _f64(pts), _f64(w)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, d = pts.shape
    z = np.empty(d)
    used = np.zeros(1, dtype=np.int32)
    rest = np.zeros(1, dtype=np.int32)
    rp = np.zeros(1)
    rd = np.zeros(1)
    z0a = _f64(z0) if z0 is not None else None
    marg = np.zeros(1)
    rc = _load().orc_em_admm_fast(_dp(pts), _dp(w), n, d, float(lo), float(hi), float(mu), int(iters), _dp(z0a),
                                  float(tol), int(check_every), float(eta), int(restart_every), int(bool(combined)),
                                  _dp(z), _ip(used), _dp(rp), _dp(rd), _ip(rest), _dp(marg))
    if rc != 0:
        raise MemoryError("oracle em_admm_fast out of memory")
    res = (z, int(used[0]), float(rp[0]), float(rd[0]), int(rest[0]))
    return res + (float(marg[0]),) if with_margin else res


def em_admm_wpen(pts, w, lo, hi, mu, iters, z0=None, tol=0.0, check_every=1):
    """Algorithm 1 with per-point penalties mu_k = mu w_k: prox radius 1/mu for every point, z the
    projected w-weighted mean, residuals in the w-weighted norm.  Returns (z, iters_used, r_pri, r_dual)."""
    pts, w = _f64(pts), _f64(w)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, d = pts.shape
    z = np.empty(d)
    used = np.zeros(1, dtype=np.int32)
    rp = np.zeros(1)
    rd = np.zeros(1)
    z0a = _f64(z0) if z0 is not None else None
    rc = _load().orc_em_admm_wpen(_dp(pts), _dp(w), n, d, float(lo), float(hi), float(mu), int(iters), _dp(z0a),
                                  float(tol), int(check_every), _dp(z), _ip(used), _dp(rp), _dp(rd))
    if rc != 0:
        raise MemoryError("oracle em_admm_wpen out of memory")
    return z, int(used[0]), float(rp[0]), float(rd[0])


def em_admm_set(pts, w, kind, a, b=None, r=0.0, mu=1.0, iters=100, z0=None, tol=0.0, check_every=1):
    """Algorithm 1 with the z-update projecting onto project_set's set (kind 1 or 2); the start is
    z0 as given, else the projected weighted mean.  Returns (z, iters_used, r_pri, r_dual)."""
    pts, w, a = _f64(pts), _f64(w), _f64(a)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, d = pts.shape
    b = _f64(b) if b is not None else np.zeros_like(a)
    z = np.empty(d)
    used = np.zeros(1, dtype=np.int32)
    rp = np.zeros(1)
    rd = np.zeros(1)
    z0a = _f64(z0) if z0 is not None else None
    rc = _load().orc_em_admm_set(_dp(pts), _dp(w), n, d, int(kind), _dp(a), _dp(b), float(r), float(mu), int(iters),
                                 _dp(z0a), float(tol), int(check_every), _dp(z), _ip(used), _dp(rp), _dp(rd))
    if rc != 0:
        raise MemoryError("oracle em_admm_set out of memory")
    return z, int(used[0]), float(rp[0]), float(rd[0])


def objective(z, pts, w):
    """Eq. (1) objective sum_k w_k ||z - a_k||."""
    z, pts, w = _f64(z), _f64(pts), _f64(w)
    n, d = pts.shape
    return float(_load().orc_objective(_dp(z), _dp(pts), _dp(w), n, d))


def kkt_residual(z, pts, w, lo, hi, tau=None):
    z, pts, w = _f64(z), _f64(pts), _f64(w)
    n, d = pts.shape
    if tau is None:
        tau = 1e-9 * max(1.0, abs(hi - lo))
    return float(_load().orc_kkt_residual(_dp(z), _dp(pts), _dp(w), n, d, float(lo), float(hi), float(tau)))


def weighted_mean_start(pts, w, lo, hi):
    pts, w = _f64(pts), _f64(w)
    n, d = pts.shape
    z = np.empty(d)
    _load().orc_weighted_mean_start(_dp(pts), _dp(w), n, d, float(lo), float(hi), _dp(z))
    return z


def em_admm(pts, w, lo, hi, mu, iters, z0=None, tol=0.0, check_every=1):
    """Algorithm 1 on one problem.  Returns (z, iters_used, r_pri, r_dual)."""
    pts, w = _f64(pts), _f64(w)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, d = pts.shape
    z = np.empty(d)
    used = np.zeros(1, dtype=np.int32)
    rp = np.zeros(1)
    rd = np.zeros(1)
    z0a = _f64(z0) if z0 is not None else None
    rc = _load().orc_em_admm(_dp(pts), _dp(w), n, d, float(lo), float(hi), float(mu), int(iters),
                             _dp(z0a), float(tol), int(check_every), _dp(z), _ip(used), _dp(rp), _dp(rd))
    if rc != 0:
        raise MemoryError("oracle em_admm out of memory")
    return z, int(used[0]), float(rp[0]), float(rd[0])


def weiszfeld(pts, w, x0, iters):
    pts, w, x0 = _f64(pts), _f64(w), _f64(x0)
    n, d = pts.shape
    x = np.empty(d)
    F = np.empty(max(iters, 1))
    _load().orc_weiszfeld(_dp(pts), _dp(w), n, d, _dp(x0), int(iters), _dp(x), _dp(F))
    return x, F[:iters]


def irls(pts, w, lo, hi, x0, eps, iters):
    pts, w, x0 = _f64(pts), _f64(w), _f64(x0)
    n, d = pts.shape
    x = np.empty(d)
    F = np.empty(max(iters, 1))
    _load().orc_irls(_dp(pts), _dp(w), n, d, float(lo), float(hi), _dp(x0), float(eps), int(iters), _dp(x), _dp(F))
    return x, F[:iters]


def em_admm_batch(pts, w, lo, hi, mu, iters, z0=None, tol=0.0, check_every=1, nthreads=0, penalty=0,
                  fast=False, extra=False, restart_every=0):
    """Algorithm 1 on a float32 batch [B, n, d] (threads over problems); penalty 1 solves each
    problem with em_admm_wpen instead, fast=True with em_admm_fast (eta = 0.999, restart_every as
    there).  Returns
    (z [B,d] float64, iters_used [B], r_pri [B], r_dual [B]); with extra also the restarts [B]
    and decision margins [B] of em_admm_fast."""
    pts = np.ascontiguousarray(pts, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    B, n, d = pts.shape
    z = np.empty((B, d))
    used = np.zeros(B, dtype=np.int32)
    rp = np.zeros(B)
    rd = np.zeros(B)
    z0a = np.ascontiguousarray(z0, dtype=np.float32) if z0 is not None else None
    rest = np.zeros(B, dtype=np.int32)
    marg = np.full(B, np.inf)
    method = 2 if fast else int(penalty)
    rc = _load().orc_em_admm_batch(_fp(pts), _fp(w), B, n, d, float(lo), float(hi), float(mu), int(iters),
                                   _fp(z0a), float(tol), int(check_every), _dp(z), _ip(used), _dp(rp), _dp(rd),
                                   int(nthreads), method, _ip(rest), _dp(marg), int(restart_every))
    if rc != 0:
        raise MemoryError("oracle em_admm_batch failed")
    return (z, used, rp, rd, rest, marg) if extra else (z, used, rp, rd)


def nlem(img, k, S, h, mu, iters, lo=0.0, hi=255.0, tol=0.0, check_every=1, init_mode=0,
         weight_mode=0, pixels=None, nthreads=0, penalty=0, fast=False, restart_every=0):
    """NLEM (Sec. 3) on a float32 image; penalty 1 solves each pixel's problem with em_admm_wpen
    (per-point penalties mu_k = mu w_k), fast=True with em_admm_fast (eta = 0.999, restart_every as
    there).  Returns a
    dict with out (float64), iters_used, r_pri, r_dual, n (points per problem), wsum (sum of
    weights), restarts and margin (em_admm_fast's; 0 and inf otherwise), one entry per processed
    pixel (all pixels row-major, or the listed linear indices)."""
    img = np.ascontiguousarray(img, dtype=np.float32)
    H, W = img.shape
    if pixels is None:
        npix = H * W
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64).reshape(-1))
        npix = pix.size
    out = np.empty(npix)
    used = np.zeros(npix, dtype=np.int32)
    rp = np.zeros(npix)
    rd = np.zeros(npix)
    nn = np.zeros(npix, dtype=np.int32)
    ws = np.zeros(npix)
    rest = np.zeros(npix, dtype=np.int32)
    marg = np.full(npix, np.inf)
    pixp = pix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if pix is not None else None
    method = 2 if fast else int(penalty)
    rc = _load().orc_nlem(_fp(img), H, W, int(k), int(S), float(h), float(mu), int(iters), float(lo), float(hi),
                          float(tol), int(check_every), int(init_mode), int(weight_mode), pixp, npix,
                          _dp(out), _ip(used), _dp(rp), _dp(rd), _ip(nn), _dp(ws), int(nthreads), method,
                          _ip(rest), _dp(marg), int(restart_every))
    if rc != 0:
        raise MemoryError("oracle nlem failed")
    res = dict(out=out, iters_used=used, r_pri=rp, r_dual=rd, n=nn, wsum=ws, restarts=rest, margin=marg)
    if pixels is None:
        for key in ("out", "iters_used", "r_pri", "r_dual", "n", "wsum", "restarts", "margin"):
            res[key] = res[key].reshape(H, W)
    return res


def nlem_problem(img, k, S, h, lin, weight_mode=0):
    """(points [n, k*k], weights [n], centre patch) that NLEM builds for pixel `lin`."""
    img = np.ascontiguousarray(img, dtype=np.float32)
    H, W = img.shape
    d = k * k
    pts = np.zeros((S * S, d))
    w = np.zeros(S * S)
    pc = np.zeros(d)
    n = _load().orc_nlem_problem(_fp(img), H, W, int(k), int(S), float(h), int(lin), int(weight_mode),
                                 _dp(pts), _dp(w), _dp(pc))
    return pts[:n].copy(), w[:n].copy(), pc


def nlem_irls(img, k, S, h, eps, iters, lo=0.0, hi=255.0, init_mode=0, pixels=None):
    """NLEM-IRLS, the comparison method of Sec. 3 (Table 1, Figs. 1-2): every listed pixel's
    problem (nlem_problem: patches, window, weights exp(-||P_i - P_j||^2 / h^2)) solved by IRLS on
    the surrogate of Eq. 2 (irls, projected onto [lo, hi]^d after every step) for exactly `iters`
    steps, from P_C(weighted mean) (init_mode 0) or the projected noisy patch (init_mode 1).
    Pure composition of nlem_problem, weighted_mean_start, project_box, irls and objective.
    Returns dict(out, step, obj, wsum) of float64 arrays: the centre coordinate of x(T),
    ||x(T) - x(T-1)|| / ||x(T)|| (0 when iters == 0), the objective of problem (1) at x(T) and the
    sum of the weights."""
    img = np.ascontiguousarray(img, dtype=np.float32)
    H, W = img.shape
    lins = np.arange(H * W) if pixels is None else np.asarray(pixels, dtype=np.int64).reshape(-1)
    out = np.empty(lins.size)
    step = np.zeros(lins.size)
    obj = np.empty(lins.size)
    wsum = np.empty(lins.size)
    c = (k * k - 1) // 2
    for i, lin in enumerate(lins):
        pts, w, pc = nlem_problem(img, k, S, h, int(lin))
        x = weighted_mean_start(pts, w, lo, hi) if init_mode == 0 else project_box(pc, lo, hi)
        if iters > 0:
            xp, _ = irls(pts, w, lo, hi, x, eps, iters - 1) if iters > 1 else (x, None)
            x, _ = irls(pts, w, lo, hi, xp, eps, 1)
            step[i] = np.linalg.norm(x - xp) / max(np.linalg.norm(x), 1e-300)
        out[i] = x[c]
        obj[i] = objective(x, pts, w)
        wsum[i] = float(np.sum(w))
    if pixels is None:
        out, step, obj, wsum = (a.reshape(H, W) for a in (out, step, obj, wsum))
    return dict(out=out, step=step, obj=obj, wsum=wsum)


def nlem_color(img, k, S, h, mu, iters, lo=0.0, hi=255.0, tol=0.0, check_every=1, init_mode=0, pixels=None):
    """NLEM (Sec. 3) on a planar multichannel image [C, H, W]: the patch of a pixel stacks the
    channels' k x k patches (coordinate c*k*k + r*k + s), so ||P_i - P_j||^2 sums over the channels
    and w_ij = exp(-sum_c D_c / h^2) is the product of the channels' weights.  Each pixel's problem
    is solved by Algorithm 1 (em_admm) from P_C(weighted mean) (init_mode 0) or the projected noisy
    patch (1).  Pure composition of nlem_problem, project_box and em_admm.
    Returns dict(out [C, ...], iters_used, r_pri, r_dual) per listed pixel."""
    img = np.ascontiguousarray(img, dtype=np.float32)
    C, H, W = img.shape
    lins = np.arange(H * W) if pixels is None else np.asarray(pixels, dtype=np.int64).reshape(-1)
    out = np.empty((C, lins.size))
    used = np.zeros(lins.size, dtype=np.int64)
    rp = np.zeros(lins.size)
    rd = np.zeros(lins.size)
    kk = k * k
    for i, lin in enumerate(lins):
        parts = [nlem_problem(img[c], k, S, h, int(lin)) for c in range(C)]
        pts = np.hstack([p[0] for p in parts])
        w = np.prod(np.stack([p[1] for p in parts]), axis=0)
        pc = np.concatenate([p[2] for p in parts])
        z0 = None if init_mode == 0 else project_box(pc, lo, hi)
        z, used[i], rp[i], rd[i] = em_admm(pts, w, lo, hi, mu, iters, z0=z0, tol=tol, check_every=check_every)
        out[:, i] = z[np.arange(C) * kk + (kk - 1) // 2]
    if pixels is None:
        out = out.reshape(C, H, W)
        used, rp, rd = used.reshape(H, W), rp.reshape(H, W), rd.reshape(H, W)
    return dict(out=out, iters_used=used, r_pri=rp, r_dual=rd)


def features(pts, w):
    """[m (d), q (d), H, pmax] of one problem (weighted mean, coordinate-wise lower weighted
    median, weight entropy, largest normalised weight)."""
    pts, w = _f64(pts), _f64(w)
    if pts.ndim == 1:
        pts = pts[:, None]
    n, d = pts.shape
    f = np.empty(2 * d + 2)
    _load().orc_features(_dp(pts), _dp(w), n, d, _dp(f))
    return f


def mlp_num_params(d, hidden=128):
    F, O = 2 * d + 2, d + 1
    return hidden * F + hidden + hidden * hidden + hidden + O * hidden + O


def mlp_forward(params, d, feats, hidden=128, nref=441.0):
    params, feats = _f64(params), _f64(feats)
    B = feats.shape[0]
    y = np.empty((B, d + 1))
    _load().orc_mlp_forward(_dp(params), d, hidden, float(nref), _dp(feats), B, _dp(y))
    return y


def mlp_loss_grad(params, d, feats, targets, hidden=128, nref=441.0):
    params, feats, targets = _f64(params), _f64(feats), _f64(targets)
    B = feats.shape[0]
    g = np.empty_like(params)
    L = _load().orc_mlp_loss_grad(_dp(params), d, hidden, float(nref), _dp(feats), _dp(targets), B, _dp(g))
    return float(L), g
