"""CPU FP64 oracle (test infrastructure only; never imported by the product path).

See ``oracle.qbvm_oracle`` for what each function follows in the paper.
"""
from .qbvm_oracle import *  # noqa: F401,F403
