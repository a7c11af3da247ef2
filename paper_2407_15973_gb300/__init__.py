"""Mixed-precision block-Jacobi PCG for one GB300 (sm_103a)."""
