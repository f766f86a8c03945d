"""GB300 (sm_103a) implementation of the data-parallel hot path of the periodic QM/MM-Multipole
electrostatic embedding (arXiv 2408.03273): the region-I one-electron matrix over
Gaussian-smeared MM charges (Eq. 9), the multipolar Ewald coupling between QM multipoles and MM
charges (Eq. 6 QM-MM lines, Eq. 10) and their adjoint (Eq. 15 and the region-I integral
derivatives).

The compute lives in the C-ABI library ``_build/libqmmm_gb300.so`` (include/qmmm.h).  This
package is its thin binding: ``_lib`` exposes the C entry points under the same names,
``Handle`` bundles a handle with a workload, and ``QMMMEnergy`` is the torch.autograd.Function
whose backward is the hand-written adjoint kernel.
"""
from __future__ import annotations

from . import build  # noqa: F401
from ._lib import (  # noqa: F401
    EXPORTS,
    QMMM_FP64,
    QMMM_MIXED,
    QMMM_TUNE_BOTH_PRECISIONS,
    QMMM_TUNE_FORCES,
    QMMM_TUNE_V,
    SWEEP_KINDS,
    QMMMError,
    load,
    qmmm_batch_captures,
    qmmm_batch_counts,
    qmmm_batch_create,
    qmmm_batch_destroy,
    qmmm_batch_run,
    qmmm_batch_timing,
    qmmm_aspc_predict,
    qmmm_autotune,
    qmmm_get_tuning,
    qmmm_set_tuning,
    library_path,
    qmmm_create,
    qmmm_destroy,
    qmmm_energy,
    qmmm_density_gradient,
    qmmm_ewald,
    qmmm_forces,
    qmmm_get_info,
    qmmm_get_potential,
    qmmm_last_error,
    qmmm_last_timing,
    qmmm_nao,
    qmmm_nuclear_mm_energy_static,
    qmmm_octupole_error,
    qmmm_qm_images,
    qmmm_rcut_search,
    qmmm_set_positions,
    qmmm_selftest_bounded_wait,
    qmmm_set_precision,
    qmmm_set_recip_method,
    QMMM_RECIP_CUDA_CORES,
    QMMM_RECIP_TENSOR,
    QMMM_RECIP_AUTO,
    qmmm_set_stream,
    qmmm_strerror,
    qmmm_vpot,
)
from .handle import Batch, Handle, QMMMEnergy  # noqa: F401
