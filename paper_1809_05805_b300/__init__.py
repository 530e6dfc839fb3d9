"""B300-native one-reduce (lagged-normalization, compact-WY) MGS-GMRES.

The solver runs in hand-written sm_103a CUDA kernels behind a C ABI
(``include/lsgmres.h``); :mod:`paper_1809_05805_b300.lsgmres` is the thin ctypes
binding. :mod:`paper_1809_05805_b300.problems` builds the seeded synthetic inputs.
Nothing is imported eagerly, so the input generators load without the CUDA library.
"""
__all__ = ["lsgmres", "problems"]
