"""CPU oracle of STZ (test infrastructure only; see oracle.py)."""
