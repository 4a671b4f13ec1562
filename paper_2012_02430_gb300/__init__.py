"""GB300-native sliced bucket-elimination simulator for QAOA MaxCut amplitudes.

The compute path is the C-ABI library libqtensor.so (include/qtensor.h) with
hand-written sm_103a CUDA kernels; `qtensor` is its ctypes binding and
`inputs` the seeded instance generators. Importing the package itself loads
nothing native; `from paper_2012_02430_gb300 import qtensor` does.
"""

__all__ = ["inputs", "qtensor", "build"]
