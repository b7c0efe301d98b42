"""FP64 CPU oracle: test infrastructure only (see amg_oracle)."""
