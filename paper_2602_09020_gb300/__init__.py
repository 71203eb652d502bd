"""Pauli-rotation statevector engine for GB300 (sm_103a).

The compute path lives in the C-ABI library ``libpaulirot.so`` (CUDA kernels
plus host C++); :mod:`paper_2602_09020_gb300.capi` marshals arguments into it.
Importing the package does not load the library: ``synth`` (seeded inputs) is
usable on machines without a GPU.
"""
__all__ = ["synth"]
