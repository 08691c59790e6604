"""GB300-native linear-scaling response-density-matrix solve (TC2 + first-order
recursion) behind the C ABI of include/rdm.h.

The compute path is ``librdm.so`` (hand-written sm_103a CUDA kernels);
``paper_2009_03551_gb300.rdm`` is a ctypes binding with the C names.
Importing it raises ImportError if the library has not been built; there is
no CPU fallback.
"""
