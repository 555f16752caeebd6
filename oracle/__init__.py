"""FP64 CPU oracle (test infrastructure only; see psvd_oracle.py)."""
