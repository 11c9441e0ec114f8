"""FP64 CPU oracle of the robust reference governor (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline and
reference legs may import this package.
"""
