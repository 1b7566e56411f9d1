"""GB300-native matrix-free high-order finite elements in persistent cell-wise storage.

The compute path lives in ``libfe.so`` (hand-written CUDA for sm_103a behind a C ABI, declared in
``include/fe.h``); :mod:`paper_2607_02335_gb300.fe` is the thin ctypes binding with the same call
names.  :mod:`paper_2607_02335_gb300.slab` holds the communicators of the slab decomposition (one
mesh over several processes or devices) and :mod:`paper_2607_02335_gb300.synth` the seeded input
generators.  Importing this package does not load the CUDA library; importing ``.fe`` does, and
fails loudly when the library has not been built.
"""
__all__ = ["fe", "slab", "synth"]
