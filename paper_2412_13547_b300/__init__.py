"""B300-native (sm_103a) hot path of Turbo-GS fitting: a differentiable,
tile-based 3D Gaussian splatting rasterizer with dilated rendering, the
densification statistics it feeds, and a fused Adam step.

All arithmetic runs in hand-written CUDA kernels in ``libturbogs.so`` behind
the C ABI declared in ``include/turbogs.h``; this package only marshals
arguments (see ``raster.py``). The library is loaded on first use and a
missing or stale build raises an error: there is no CPU fallback.
"""
__all__ = ["scenes"]
