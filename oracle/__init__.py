"""FP64 CPU oracle of the pseudopotential MRT-LB step and its analytic companions.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  It shares no
code with paper_2604_13407_gb300 (the CUDA library and its binding), and neither
imports the other.
"""
