"""CPU oracle for the LABFM hot path: test infrastructure, not product code.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It is independent of the CUDA library (no shared
code, no shared constants) and follows the paper's definitions in plain FP64.
``labfm_oracle`` (as ``core``) covers the interior method; ``boundary_oracle`` the
boundary operators of Section 7.1 and Appendix A.
"""
from .labfm_oracle import *  # noqa: F401,F403
from . import labfm_oracle as core  # noqa: F401
