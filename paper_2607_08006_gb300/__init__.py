"""shmemg: a GPU-aware OpenSHMEM symmetric heap on one GB300 (sm_103a).

npes virtual PEs are equal partitions of one HBM allocation; thread blocks or
thread-block clusters act as PEs.  The C ABI (include/shmemg.h) and every kernel live
in libshmemg.so; this package is its ctypes binding (argument marshalling only).
"""
from .builder import build  # noqa: F401
from .shmemg import *  # noqa: F401,F403
from .shmemg import Heap, Sym, ShmemgError, lib  # noqa: F401
