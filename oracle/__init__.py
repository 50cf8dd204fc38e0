"""CPU FP64 oracle (test infrastructure only; see df_oracle)."""
