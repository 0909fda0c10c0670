"""FP64 CPU oracle for the DISC hot path.

Test infrastructure only: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the library.
"""
