"""FP64 CPU oracle for the LMA hot path (test infrastructure; never used by the product path)."""
