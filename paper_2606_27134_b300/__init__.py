"""B300-native periodized DMK: C-ABI CUDA library and its thin Python binding."""
