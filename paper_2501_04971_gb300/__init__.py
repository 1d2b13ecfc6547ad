"""GB300-native hot path of the Self-Adaptive Ising Machine (arXiv 2501.04971).

The compute path lives in ``libsais.so`` (hand-written CUDA for sm_103a behind the C-ABI
declared in ``include/sais.h``); :mod:`.sais` is its thin ctypes binding.  Importing this
package loads nothing: the library is opened on first use of :mod:`.sais`.
"""
__all__ = ["sais", "workloads", "build"]
