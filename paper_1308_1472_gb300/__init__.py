"""GB300-native forest-of-quadtrees patch solver (wave propagation on every leaf
patch), behind the C ABI declared in include/fc.h.

The compute path is libfc.so (hand-written sm_103a CUDA); this package only
builds/loads it and marshals arguments (see ``fc``).  There is no CPU path.
"""
from . import fc  # noqa: F401
from .fc import Context, FCError  # noqa: F401
