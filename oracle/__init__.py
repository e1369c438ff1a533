"""CPU oracle of the HeatACO decoder -- test infrastructure only.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  The library under ``paper_2601_19041_gb300`` never does.
"""
