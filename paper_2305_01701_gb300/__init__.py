"""GB300-native pseudo-transient solver for strain localization in a
(visco-)hypoelastic, perfectly plastic Drucker-Prager medium
(Alkhimenkov, Khakimova, Utkin, Podladchikov, arXiv:2305.01701).

The compute path is the CUDA library ``lib/libep.so`` (C ABI in
``include/ep.h``); this package only marshals arguments to it.
"""
from ._native import (measure_fp64_peak, PENDING, warm_in, warm_out, Batch, Net, FP32_MIXED, FP64, KERNEL_AUTO, KERNEL_FUSED, KERNEL_FUSED_TMA, KERNEL_FUSED_REG, KERNEL_STAGED, LOAD_XY, LOAD_XZ, EPError, Grid,
                      field_shape, lib, workspace_bytes)

__all__ = ["measure_fp64_peak", "PENDING", "warm_in", "warm_out", "Grid", "Batch", "Net", "EPError", "FP64", "FP32_MIXED", "LOAD_XY", "LOAD_XZ", "KERNEL_AUTO", "KERNEL_STAGED", "KERNEL_FUSED_REG",
           "KERNEL_FUSED", "KERNEL_FUSED_TMA", "field_shape", "lib", "workspace_bytes"]
