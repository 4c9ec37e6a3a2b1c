"""FP64 CPU oracle for the randomized Tucker methods (arXiv 2211.13028).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (``paper_2211_13028_gb300``) never imports it and shares no code
with it.

Parity status: every function in ``tucker_ref`` is pinned by a ``-m "not gpu"``
test against brute force, a closed form, a printed value of the paper, or a
mathematical invariant (see the module docstring of ``tucker_ref``).
"""
from .tucker_ref import *  # noqa: F401,F403
