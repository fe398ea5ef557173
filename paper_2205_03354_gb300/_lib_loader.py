"""Loads the compiled C-ABI library; raises if it has not been built."""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libstencilcomp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libstencilcomp.so not found at {LIB_PATH}: build it first with "
        "`python paper_2205_03354_gb300/build.py` (needs nvcc); there is no CPU fallback")

lib = ctypes.CDLL(LIB_PATH)
lib.sc_last_error.restype = ctypes.c_char_p
lib.sc_version.restype = ctypes.c_int32

STATUS = {0: "SC_OK", 1: "SC_EINVAL", 2: "SC_ENOMEM", 3: "SC_ENOTCONV", 4: "SC_EBREAKDOWN",
          5: "SC_ETIMEOUT", 6: "SC_EBUSY", 7: "SC_ECUDA", 8: "SC_EOVERFLOW", 9: "SC_EPENDING"}


class ScError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check(rc: int) -> int:
    if rc != 0:
        raise ScError(rc, lib.sc_last_error().decode(errors="replace"))
    return rc
