"""FP64 CPU oracle for the NEP path (test infrastructure only)."""
