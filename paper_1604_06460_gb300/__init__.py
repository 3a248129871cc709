"""GB300-native state-vector emulator (Haener, Steiger, Smelyanskiy, Troyer,
"High Performance Emulation of Quantum Circuits", 2016).

``qe``      - Python binding of the C ABI in ``include/qe.h``;
``build``   - in-tree nvcc build of ``libqe.so`` for sm_103a;
``inputs``  - seeded synthetic inputs (gates, circuits, Hamiltonians).

Importing the package loads nothing; the CUDA library is loaded on first use.
"""
__all__ = ["qe", "build", "inputs"]
