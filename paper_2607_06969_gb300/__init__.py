"""GB300-native (sm_103a) NEP per-atom evaluation and training backward.

The compute path lives in the CUDA library built from csrc/ (libnep.so);
`binding` exposes its C-ABI to Python.  Importing this package does not load
the library; `paper_2607_06969_gb300.binding.lib()` does, and raises if it
is missing.
"""
__all__ = ["inputs", "binding"]
