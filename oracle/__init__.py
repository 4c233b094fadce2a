"""CPU oracle for the checkpoint/restart data pass.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the product library never does.
"""
