"""GB300 (sm_103a) lattice Boltzmann library for capillary filling.

The D2Q9 free-energy MRT scheme of Pooley, Kusumaatmaja & Yeomans (liquid-gas
and binary models) runs in hand-written CUDA kernels behind the C ABI of
include/lb.h; this package holds the kernels (csrc/), their build (build.py) and
a thin ctypes binding (lb.py).
"""
from .lb import (Batch, Lattice, LbError, MODEL_BINARY, MODEL_LIQUID_GAS, STORAGE_F16_BLOCKED, STORAGE_F16DEV,
                 STORAGE_F32, STORAGE_F32_BLOCKED, STORAGE_F32_GELIM, STORAGE_F64, STORAGE_MOMENTS, STORAGE_MOMENTS_F16, library)

__all__ = ["Batch", "Lattice", "LbError", "MODEL_BINARY", "MODEL_LIQUID_GAS", "STORAGE_F16_BLOCKED", "STORAGE_F16DEV",
           "STORAGE_F32", "STORAGE_F32_BLOCKED", "STORAGE_F32_GELIM", "STORAGE_F64", "STORAGE_MOMENTS", "STORAGE_MOMENTS_F16", "library"]
