"""GB300-native exact exponential field solver for cylindrical PIC (azimuthal modes).

Thin Python binding over the C-ABI library ``lib/libfdetd.so`` (declared in
``include/fdetd.h``): argument marshalling only; every step of the solver runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.

    from paper_2605_12132_gb300 import fdetd_plan, fdetd_step
    plan = fdetd_plan(Nz, Nr, M, order, dz, dr, dt, precision="bf16x3")
    fdetd_step(plan, fields, J, nsteps)      # fields: cuda complex64 [M+1][6][Nz][Nr]

The library is loaded lazily on first use; importing this package does not need a GPU.
"""
from ._native import (  # noqa: F401
    J_ON_PRIMARY,
    SPECTRAL_COLUMNS,
    fdetd_host_split_parts,
    fdetd_plan_cache_set_limit,
    fdetd_plan_cache_stats,
    fdetd_plan_cache_warm,
    pipeline_report,
    PRECISIONS,
    EnvelopePlan,
    FdetdBatch,
    FdetdError,
    FdetdPlan,
    envelope_plan,
    envelope_step,
    envelope_step_absorbing,
    envelope_step_static,
    envelope_step_fused,
    fdetd_current_correct,
    fdetd_current_host_bands,
    fdetd_destagger,
    fdetd_host_coeffs,
    fdetd_host_spectral_order,
    fdetd_host_spectral_radices,
    fdetd_host_tables,
    fdetd_plan,
    fdetd_plan_modes,
    fdetd_probe_mma_rounding,
    TaylorPlan,
    fdetd_taylor_host_bands,
    fdetd_taylor_plan,
    fdetd_taylor_step,
    fdetd_step,
    fdetd_step_host,
    lib,
    lib_path,
)
