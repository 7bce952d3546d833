"""FP64 CPU oracle (test infrastructure; see marfa_oracle)."""
