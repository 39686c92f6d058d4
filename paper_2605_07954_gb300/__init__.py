"""GB300-native iterated explicit 2D stencil sweeps (sm_103a CUDA behind a C-ABI)."""
