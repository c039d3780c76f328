"""ASE-DF residual library for GB300 (sm_103a, FP64)."""
