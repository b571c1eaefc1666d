"""CPU oracle for the randomized ID (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  It shares no code with paper_1205_3830_gb300.
"""
from .rid_oracle import *  # noqa: F401,F403
from .rid_oracle import __all__  # noqa: F401
