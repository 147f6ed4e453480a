"""FP64 CPU oracle of the staggered leap-frog Dirac scheme (test infrastructure only)."""
