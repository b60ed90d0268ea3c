"""CPU oracle of the collective multigrid method (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this package.  The product package never imports it.
"""
from .cmg_oracle import *  # noqa: F401,F403
