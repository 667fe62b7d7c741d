"""FP64 CPU oracle (test infrastructure only; see sparc_oracle.py)."""
