"""GB300 conditional-entropy (P, Pdot) period search (arXiv:2006.06866, gce).

The computation lives in the CUDA library ``_lib/libgce.so`` (C ABI in
``include/gce.h``); ``binding`` exposes it to Python with the same names.
Build with ``python -m paper_2006_06866_gb300.build``.
"""
from .binding import (GCE_ERR_CUDA, GCE_ERR_INVALID, GCE_ERR_NOMEM, GCE_ERR_UNSUPPORTED,
                      GCE_FLAG_NO_GRAPH, GCE_FLAG_OVERLAP, GCE_FLAG_TIME_KERNEL, GCE_MAX_BANDS,
                      GCE_MAX_CURVE_POINTS, GCE_MAX_MAG_BINS, GCE_MAX_PHASE_BINS, GCE_MAX_TOPK,
                      GCE_OK, GCE_PHASE_FIXED32, GCE_PHASE_FP64, GCE_PHASE_SPLIT32, MODES, Config,
                      GceError, Handle, gce_autotune, gce_autotune_job, gce_ce_counts,
                      gce_ce_detect, gce_ce_detect_bands, gce_ce_grid, gce_ce_grid_bands,
                      gce_ce_grid_single, gce_ce_topk, gce_ce_topk_host, gce_ce_topk_static,
                      gce_check_job, gce_get_tuning, gce_kernel_time, gce_last_launches,
                      gce_set_tuning, gce_stream_status, lib)

__all__ = [
    "GCE_ERR_CUDA", "GCE_ERR_INVALID", "GCE_ERR_NOMEM", "GCE_ERR_UNSUPPORTED", "GCE_FLAG_NO_GRAPH",
    "GCE_FLAG_OVERLAP", "GCE_FLAG_TIME_KERNEL", "GCE_MAX_BANDS", "GCE_MAX_CURVE_POINTS",
    "GCE_MAX_MAG_BINS", "GCE_MAX_PHASE_BINS", "GCE_MAX_TOPK", "GCE_OK", "GCE_PHASE_FIXED32",
    "GCE_PHASE_FP64", "GCE_PHASE_SPLIT32", "MODES", "Config", "GceError", "Handle", "gce_autotune",
    "gce_autotune_job", "gce_ce_counts", "gce_ce_detect", "gce_ce_detect_bands", "gce_ce_grid",
    "gce_ce_grid_bands", "gce_ce_grid_single", "gce_ce_topk", "gce_ce_topk_host",
    "gce_ce_topk_static", "gce_check_job", "gce_get_tuning", "gce_kernel_time",
    "gce_last_launches", "gce_set_tuning", "gce_stream_status", "lib",
]
