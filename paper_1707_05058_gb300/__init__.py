"""GB300-native chordally decomposed ADMM for sparse SDPs.

The solver lives in the CUDA library `libcdsdp.so` (C ABI, include/cdsdp.h);
`cdsdp` is its ctypes binding.  Importing this package does not load the
library; `paper_1707_05058_gb300.cdsdp` does, and fails loudly when the
library has not been built.
"""
