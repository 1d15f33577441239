"""FP64 CPU oracle for ICNNM: test infrastructure only (see icnnm_oracle)."""
