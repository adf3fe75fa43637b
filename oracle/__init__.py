"""FP64 CPU oracle of the indexing path.  TEST INFRASTRUCTURE ONLY: imported by the
tests, the package smoke check and the benchmark's CPU-baseline leg, never by the
product path (which has no CPU fallback)."""
