"""FP64 CPU oracle for speed-limited PIC (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library.
"""
