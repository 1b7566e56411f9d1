"""GB300-native matrix-free high-order finite elements in persistent cell-wise storage.

The compute path lives in ``libfe.so`` (hand-written CUDA for sm_103a behind a C ABI, declared in
``include/fe.h``); :mod:`paper_2607_02335_gb300.fe` is the thin ctypes binding with the same call
names.  Importing this package does not load the CUDA library; importing ``.fe`` does, and fails
loudly when the library has not been built.
"""
__all__ = ["fe", "synth"]
