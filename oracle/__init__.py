"""FP64 CPU oracle for the batched MPM path.  Test infrastructure only: imported by
tests/, the package smoke check and the benchmark's CPU-baseline leg, never by the
product library."""
