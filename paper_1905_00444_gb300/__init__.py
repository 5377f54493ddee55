"""GB300-native tensor-network amplitudes of random quantum circuits (arXiv:1905.00444).

The compute path is libqfx (CUDA for sm_103a, C ABI in include/qfx.h); this package is
its Python binding.  Importing it builds the library in-tree if it is missing or out of
date (nvcc is required) and raises if that fails: there is no CPU fallback.
"""
from .build import build as _build

_build()

from .qfx import (  # noqa: E402,F401
    Batch, Circuit, Plan, QfxError, amplitudes, amplitudes_backward, amplitudes_static, contract_step, header_symbols, launch_count, lib,
    autotune, frugal_sample, frugal_select, permute, profile_collect, profile_enable, sync,
    tensor_peak, version, debug_permute_withhold,
)
from .sharding import item_costs, partition_items, partition_slices, reduce_partials  # noqa: E402,F401
from .autograd import CircuitAmplitudes, circuit_amplitudes  # noqa: E402,F401
