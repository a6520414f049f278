"""GB300 (sm_103a) shooting-and-bouncing-rays trace-integrate path for monostatic RCS.

The compute path lives in ``lib/libsbr.so`` (CUDA, C ABI in ``include/sbr.h``);
``sbr`` is its ctypes binding. Build with ``paper_2604_09243_gb300.build.build()``.
"""
from .sbr import (  # noqa: F401
    Context, SbrError, Surrogate, gemm_bf16_tn, gemm_bf16_tn_async, lib, ray_grid, spacing_for, version, POL_ORDER,
    EXPORTS, po_integrate_noalloc, probe_l2_bandwidth, probe_fp32_fma,
    TRACE_PHASE_LITERAL_2R, TRACE_REQUIRE_ESCAPE, TRACE_RECORD_HITS, TRACE_COUNT_VISITS, TRACE_TIME_PASSES,
    TRACE_NO_GRAPH,
)
