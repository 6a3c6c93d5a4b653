"""FP64 CPU oracle for the IEWPF hot path: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this package.  The product path never calls it.
"""
