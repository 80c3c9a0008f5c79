"""FP64 CPU oracle (test infrastructure only; see octaoctree_oracle)."""
