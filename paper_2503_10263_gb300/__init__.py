"""GB300-native KARL transport hot path (sm_103a CUDA behind a C ABI)."""
