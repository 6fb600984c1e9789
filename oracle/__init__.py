"""FP64 CPU oracle for the Mosaic Flow sweep -- test infrastructure only.

Imported only by the tests, the smoke check and the benchmark's CPU-baseline leg.
"""
