"""Hercules exact k-NN query answering on one GB300 (sm_103a).

The compute path is a C-ABI CUDA library (include/hercules_gb300.h) built from
csrc/; `binding` marshals arguments to it.  There is no CPU fallback: without
the built library every call raises.
"""
