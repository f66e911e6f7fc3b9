"""Plain FP64 CPU reference of SuperSCS (test infrastructure only; see oracle.py)."""
