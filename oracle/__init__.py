"""FP64 CPU oracle of the synthesis hot path (test infrastructure only)."""
