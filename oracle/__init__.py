"""CPU oracle of the FHE-DiCSNN hot path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import
anything from this package.
"""
