"""CPU oracle of the ph-AFQMC walker step: test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package; the product path never does.
"""
