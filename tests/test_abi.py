"""The C ABI builds for sm_103a and exports every entry point include/pa.h
declares; the Python binding mirrors the same names.  No GPU needed: the
library is only loaded and inspected, never asked to compute."""
import ctypes
import os
import re

import pytest

from paper_1006_0252_gb300 import build, pa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pa.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pa_\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_core_boundary():
    names = declared_functions()
    for core in ("pa_create", "pa_step", "pa_observables", "pa_free_energy", "pa_weighted_average",
                 "pa_destroy", "pa_last_error", "pa_overlap", "pa_batch_run"):
        assert core in names


def test_library_exports_every_declared_symbol():
    lib_path = build.build_library()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_the_c_names():
    lib = pa.load()
    for n in declared_functions():
        assert hasattr(lib, n)
    for n in ("pa_create", "pa_step", "pa_step_target", "pa_sync", "pa_observables",
              "pa_free_energy", "pa_trajectory", "pa_overlap", "pa_weighted_average",
              "pa_bootstrap", "pa_copy_spins", "pa_copy_energies", "pa_copy_copies", "pa_destroy"):
        assert callable(getattr(pa, n)), n
    assert pa.pa_version() >= 10000


def test_library_is_built_for_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    # bit-exact parity needs every multiply and add rounded as written
    assert "-fmad=false" in build.NVCC_FLAGS
    assert not any("fast" in f or f.startswith("-fmad=t") for f in build.NVCC_FLAGS)
    assert os.path.exists(build.LIB)


def declared_parameter_counts():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pa_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every entry point of include/pa.h has its ctypes signature in the
    binding, with as many parameters as the C declaration."""
    lib = pa.load()
    counts = declared_parameter_counts()
    assert set(counts) == set(declared_functions())
    wrong = {n: (k, None if getattr(lib, n).argtypes is None else len(getattr(lib, n).argtypes))
             for n, k in counts.items()
             if getattr(lib, n).argtypes is None or len(getattr(lib, n).argtypes) != k}
    assert not wrong, wrong
