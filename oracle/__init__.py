"""CPU oracle for the reuse hot path (test infrastructure only)."""
