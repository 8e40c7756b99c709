"""FP64 CPU oracle (test infrastructure only; see sgpic_oracle.py)."""
