"""Binding of libcrac_testkit.so: workload mutators used by tests and the bench.

These kernels stand in for the application rewriting part of its memory
between checkpoints.  They are not part of the checkpoint/restart path.
"""
from __future__ import annotations

import ctypes
import os

from . import TESTKIT_PATH, _stream

if not os.path.exists(TESTKIT_PATH):
    raise ImportError(f"libcrac_testkit.so is not built ({TESTKIT_PATH})")

_tk = ctypes.CDLL(TESTKIT_PATH)
_tk.crac_testkit_mutate_xor.restype = ctypes.c_int
_tk.crac_testkit_mutate_xor.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
_tk.crac_testkit_rewrite.restype = ctypes.c_int
_tk.crac_testkit_rewrite.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
_tk.crac_testkit_delay.restype = ctypes.c_int
_tk.crac_testkit_delay.argtypes = [ctypes.c_uint64, ctypes.c_void_p]


def delay(ns: int, stream=None) -> None:
    """Keep `stream` busy for ns nanoseconds (at most 10 s) of device time."""
    e = _tk.crac_testkit_delay(ns, _stream(stream))
    if e:
        raise RuntimeError(f"delay launch failed: cudaError {e}")


def mutate_xor(entries_dev_ptr: int, n: int, stream=None) -> None:
    """entries: device array of n x {u64 ptr, u64 len, u32 mask, u32 0} (24 bytes)."""
    e = _tk.crac_testkit_mutate_xor(entries_dev_ptr, n, _stream(stream))
    if e:
        raise RuntimeError(f"mutate_xor launch failed: cudaError {e}")


def rewrite(entries_dev_ptr: int, n: int, stream=None) -> None:
    """entries: device array of n x {u64 dst, u64 src, u64 len}."""
    e = _tk.crac_testkit_rewrite(entries_dev_ptr, n, _stream(stream))
    if e:
        raise RuntimeError(f"rewrite launch failed: cudaError {e}")
