"""CPU FP64 oracle of the CHNS residual / Jacobian-vector product (test infrastructure only)."""
