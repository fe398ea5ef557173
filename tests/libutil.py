"""Helpers for tests that use the compiled library."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    """Builds libstencilcomp.so (nvcc, in-tree) if it is missing or stale."""
    spec = importlib.util.spec_from_file_location(
        "_sc_build", os.path.join(ROOT, "paper_2205_03354_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def header_functions():
    import re
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(sc_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))
