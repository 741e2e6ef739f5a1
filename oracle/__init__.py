"""FP64 CPU oracle (test infrastructure only; see yk_oracle)."""
