"""Shared helper: make sure libdgnn.so exists and is newer than its sources."""
import os

from paper_2207_11571_gb300 import build as _build


def ensure_built():
    lib = _build.LIB
    srcs = [os.path.join(_build.CSRC, f) for f in os.listdir(_build.CSRC)]
    srcs.append(os.path.join(os.path.dirname(_build.PKG), "include", "dgnn.h"))
    if not os.path.exists(lib) or max(os.path.getmtime(s) for s in srcs) > os.path.getmtime(lib):
        _build.build()
    return lib
