"""CPU oracle for the Combined Sieve -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  The product path (paper_2012_03771_gb300)
never imports it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
