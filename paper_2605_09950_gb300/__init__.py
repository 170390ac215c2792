"""GB300-native GPU Boruta: the per-iteration forest fit, importance, hit and
decision steps as hand-written sm_103a CUDA kernels behind a C ABI."""
