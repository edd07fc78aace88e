"""Plain FP64 CPU oracle of the per-patch update (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.
"""
from .oracle import Oracle, build, lib  # noqa: F401
