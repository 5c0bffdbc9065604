"""FP64 CPU oracle (test infrastructure only; see psatd_oracle)."""
