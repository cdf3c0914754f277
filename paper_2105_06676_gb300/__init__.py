"""GB300-native FFT stencil solver (package placeholder, filled by the CUDA binding)."""
