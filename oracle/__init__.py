"""FP64 CPU oracle for radiomic spatial mapping.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  The product package never imports
it.
"""
