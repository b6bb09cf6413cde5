"""FP64 CPU oracle of the SU(2) heat-bath method -- test infrastructure only.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package; the library path never does.
"""
