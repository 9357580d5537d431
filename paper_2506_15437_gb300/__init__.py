"""gb300fft: 2D complex-to-complex Cooley-Tukey FFT for the NVIDIA GB300.

The transforms run in hand-written sm_103a CUDA kernels behind the C ABI of
``_build/libgb300fft.so`` (include/gb300fft.h); this package only marshals
torch tensors into that ABI.
"""
from .fft import (ColumnPlan, FFT1Function, FFT2Function, Plan, RaggedPlan, WeightedPowerLoss, fft1, fft2, get_plan,
                  radices, reorder_map, slab_pack, slab_unpack, weighted_power_loss)
from ._native import FFTError, load as load_library

__all__ = ["ColumnPlan", "FFT1Function", "FFT2Function", "Plan", "RaggedPlan", "WeightedPowerLoss", "fft1", "fft2",
           "get_plan", "radices", "reorder_map", "slab_pack", "slab_unpack", "weighted_power_loss", "FFTError",
           "load_library"]
