"""GB300-native (sm_103a) NBGS hard-contact granular time step.

The compute path lives in ``libnbgs.so`` (CUDA C++ behind a C ABI declared in
``include/nbgs.h``); :mod:`paper_1501_05810_gb300.nbgs` is the thin ctypes
binding with the same entry-point names.  :mod:`paper_1501_05810_gb300.scenes`
holds the seeded input generators.  Submodules are imported lazily so that
the generators can be used on machines without a GPU.
"""

__all__ = ["nbgs", "scenes", "build"]
