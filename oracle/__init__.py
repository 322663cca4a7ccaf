"""FP64 CPU oracle of the differentiable MLS-MPM step (test infrastructure only)."""
