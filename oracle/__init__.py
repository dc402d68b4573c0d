"""CPU oracle for the sparse truncated state-vector method.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the product path never does.
"""
from .oracle import C64, C128, Oracle, build, fx, fx_to_double, prob  # noqa: F401
