"""GB300-native parallel multi-scale reduction of persistent-homology filtrations.

Implements the data-parallel hot path of Mendoza-Smith & Tanner, "Parallel multi-scale
reduction of persistent homology filtrations" (arXiv:1708.04710): Vietoris-Rips filtrations
built on the device, Algorithm 2 (Phase 0 / I / II with clearing and Corollary 10) reduced in
hand-written sm_103a CUDA kernels, pairs and essential simplices extracted on the device.

The C ABI is declared in ``include/ph_gb300.h``; ``native.Context`` is its thin binding.
"""
from .native import PS_FIELDS, Context, PHError, load_library  # noqa: F401

__all__ = ["Context", "PHError", "load_library", "PS_FIELDS"]
