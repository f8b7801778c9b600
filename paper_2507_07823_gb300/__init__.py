"""GB300-native windowed Fourier projection (WFP) for 1D wave scattering by point springs.

The package holds the seeded workload generators (`workloads`) and the thin ctypes
binding (`wave1d`) over the CUDA C-ABI library built from `csrc/`.  Importing the
package does not load the CUDA library; `wave1d.lib()` does, and raises if it is
missing (there is no CPU fallback).
"""
__all__ = ["workloads", "wave1d"]
