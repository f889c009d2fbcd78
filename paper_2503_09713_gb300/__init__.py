"""GB300-native (sm_103a) SPH hot path of arXiv 2503.09713 behind a C-ABI library."""
