"""FP64 CPU oracle for G-CVO (test infrastructure only; see oracle.py)."""
