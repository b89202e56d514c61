"""Plain FP64 CPU oracle for the forest-of-quadtrees patch method.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library package
never does, and nothing here imports the library package.
"""
from .fco import Oracle, OracleParams, build_oracle, oracle_lib  # noqa: F401
