"""CPU FP64 oracle of the PFC scheme and its FAS solver (test infrastructure only)."""
