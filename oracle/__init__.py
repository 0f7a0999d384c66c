"""FP64 CPU oracle (test infrastructure only; never imported by the product path).

See oracle/nmf_oracle.py for what it computes and which passages it follows.
"""
from .nmf_oracle import *  # noqa: F401,F403
from .nmf_oracle import __all__  # noqa: F401
