"""GB300-native constrained Euclidean medians (EM-ADMM) and NLEM denoising.

Thin Python binding over libnlem.so (C ABI in include/nlem.h).  Every step of the
computation runs in the library's CUDA kernels; this module only marshals arguments
(torch CUDA tensors -> device pointers, the current CUDA stream) and raises on errors.
There is no CPU fallback: importing the binding fails loudly if the library is missing.

Method: Chaudhury & Ramakrishnan, "A new ADMM algorithm for the Euclidean median and its
application to robust patch regression" (arXiv 1501.03879): problem (1), Algorithm 1
(EM-ADMM) and NLEM (Sec. 3).
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    INIT_NOISY_PATCH,
    INIT_WEIGHTED_MEAN,
    LAYOUT_AUTO,
    LAYOUT_PAIR,
    LAYOUT_PIXEL,
    PENALTY_UNIFORM,
    PENALTY_WEIGHTED,
    PREC_BF16,
    PREC_FP32,
    SOLVER_ADMM,
    SOLVER_FAST,
    SOLVER_IRLS,
    Context,
    WarmStart,
    NlemError,
    em_solve,
    em_solve_batch,
    em_solve_batch_host,
    em_solve_batch_set,
    lib_path,
    load_library,
    nlem_batch_config,
    nlem_batch_force_config,
    nlem_bf16_weights,
    nlem_denoise,
    nlem_denoise_batch,
    nlem_denoise_batch_noalloc,
    nlem_denoise_color,
    nlem_denoise_ex,
    nlem_denoise_host,
    nlem_debug_status,
    nlem_device_status,
    nlem_selftest_timeout,
    nlem_denoise_warm,
    nlem_features,
    nlem_fp32_peak,
    nlem_ws_labels,
)
