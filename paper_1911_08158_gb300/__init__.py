"""GB300-native alternating-direction isogeometric (ADS/IGA) implicit wave solver.

The compute path is the CUDA library ``_build/libads_gb300.so`` (sm_103a)
behind the C ABI of ``include/ads.h``; :mod:`.ads` is its thin ctypes binding
(argument marshalling only).  PyTorch supplies device memory (caching
allocator) and streams.  There is no CPU fallback: without the built library
and a CUDA device every call fails loudly.
"""
from .ads import (ADS_DEVICE, ADS_ELASTIC, ADS_FP32, ADS_FP64, ADS_HOST, ADS_OP_MASS, ADS_OP_MASS_SOLVE,
                  ADS_OP_SPLIT_SOLVE, ADS_OP_STIFF, ADS_SCALAR_WAVE, AdsError, Simulation, batch_step,
                  estimate_bytes, launch_count, library)

__all__ = ["Simulation", "AdsError", "batch_step", "estimate_bytes", "library", "launch_count", "ADS_FP32", "ADS_FP64",
           "ADS_SCALAR_WAVE", "ADS_ELASTIC", "ADS_HOST", "ADS_DEVICE", "ADS_OP_MASS", "ADS_OP_STIFF",
           "ADS_OP_MASS_SOLVE", "ADS_OP_SPLIT_SOLVE"]
