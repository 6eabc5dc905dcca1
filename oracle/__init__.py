"""CPU oracle for CD / CD-WAC core-level G0W0 (plain FP64 numpy).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py,
never by the CUDA library or its binding.
"""
