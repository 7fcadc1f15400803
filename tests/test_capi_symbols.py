"""The C-ABI library builds, loads on the host (no compute) and exports every
entry point that include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1610_05141_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["rs_create", "rs_destroy", "rs_sample", "rs_sample_with_replacement", "rs_bernoulli", "rs_sync",
              "rs_strerror", "rs_split_tree"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib_path):
    import paper_1610_05141_gb300 as rs
    rs.load(lib_path)
    assert rs.strerror(rs.RS_EINVAL) == "invalid argument"
    assert rs.strerror(99) == "unknown error code"
    assert rs.rs_plan(10**6, 10**9, 4096) == 8
    assert rs.rs_plan(10**9, 2**50, 4096) == 18
    assert rs.rs_plan(10, 4, 1) == 2
    with pytest.raises(rs.RSError):
        rs.rs_plan(1, 1, 0)


def test_plan_matches_oracle(lib_path, oracle):
    import paper_1610_05141_gb300 as rs
    rs.load(lib_path)
    for n, N, n0 in [(0, 0, 1), (1, 1, 1), (4097, 10**9, 4096), (10**9, 2**40, 4096), (999, 1000, 3),
                     (2**62, 2**62, 1), (12345, 10**7, 100)]:
        assert rs.rs_plan(n, N, n0) == oracle.depth(n, N, n0)


def test_binding_covers_every_declared_symbol():
    """The Python binding gives every entry point of include/*.h its C
    signature (argument marshalling only)."""
    src = open(os.path.join(ROOT, "paper_1610_05141_gb300", "__init__.py")).read()
    bound = set(re.findall(r'"(rs_\w+)":', src))
    missing = [n for n in _declared() if n not in bound]
    assert not missing, missing
