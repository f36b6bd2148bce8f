"""GB300-native RecSplit construction and lookup (sm_103a CUDA behind a C ABI)."""
