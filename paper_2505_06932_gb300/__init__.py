"""GB300 (sm_103a) implementation of the front/fluid coupling hot path of sharp
front tracking (arXiv 2505.06932): binning, volume fraction, PPIC curvature,
CSF force and divergence-preserving velocity interpolation.

The compute lives in ``libfront.so`` (CUDA, C ABI in ``include/front.h``);
``paper_2505_06932_gb300._front`` is its ctypes binding.  ``inputs`` holds the
seeded synthetic workloads.  Nothing here falls back to the CPU.
"""

__all__ = ["inputs", "build"]
