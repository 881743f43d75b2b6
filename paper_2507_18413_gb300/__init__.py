"""GB300-native Compact-Table propagation: CUDA kernels behind a C ABI (libct.so)."""
