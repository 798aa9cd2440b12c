"""CPU float64 oracle of the P1-P1 IPCS step and of the learned pressure guess.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code, tables or
helpers with the CUDA path; the two meet only through the seeded inputs of
the ``workloads`` package.
"""
