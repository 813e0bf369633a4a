"""FP64 CPU oracle of the periodic G0W0 hot path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline leg may
import this package. The product path (paper_2011_01400_gb300) never does.
"""
