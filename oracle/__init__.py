"""CPU FP64 oracle (test infrastructure only; see sfac_oracle)."""
