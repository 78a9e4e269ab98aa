"""FP64 CPU oracle (test infrastructure only; see ilves_oracle.py)."""
