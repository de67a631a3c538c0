"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle (see oracle.py and sylv_oracle.c)."""
