"""The C-ABI library builds, loads and exports every entry point that
include/hoph.h declares; argument validation answers without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1805_11254_gb300 import build_lib
from paper_1805_11254_gb300 import hoph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hoph.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return hoph.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("oph_build_sketches", "minwise_build_sketches", "hoph_query_batch",
                 "hoph_plan_create", "hoph_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(hoph._EXPORTS)


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(hoph.hoph_pair) == 16
    assert hoph.PAIR_DTYPE.itemsize == 16
    assert ctypes.sizeof(hoph.hoph_stats) == 8 * (3 * 16 + 4)
    assert ctypes.sizeof(hoph.hoph_params) == 64
    assert ctypes.sizeof(hoph.hoph_exec) == 32


def _header_fields(struct_name):
    """Member names of `typedef struct {...} struct_name;` in include/hoph.h."""
    text = open(os.path.join(ROOT, "include", "hoph.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*%s\s*;" % struct_name, text)
    assert m, struct_name
    names = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if decl:  # "type name[, name...]" with optional array suffixes
            _, declarators = decl.split(" ", 1)
            names += [re.sub(r"\[.*\]", "", d).strip(" *") for d in declarators.split(",")]
    return names


@pytest.mark.parametrize("name", ["hoph_params", "hoph_exec", "hoph_stats", "hoph_plan_info"])
def test_binding_structs_follow_the_header(name):
    """The ctypes mirrors of the ABI structs name the same members in the
    same order as include/hoph.h."""
    assert [f[0] for f in getattr(hoph, name)._fields_] == _header_fields(name)


@pytest.mark.parametrize("kw", [dict(k=100, k_group=32), dict(k=128, k_group=0),
                                dict(thr=(8, 7)), dict(thr=(0, 7)), dict(a=1, b=0),
                                dict(epsilon=-1.0), dict(empty_rule=7), dict(k=32 * 17, k_group=32),
                                dict(D=1 << 33), dict(perm_kind=1), dict(weighting=2),
                                # Algorithm 2's recursion over 8 groups of a 1:1000 split
                                # outgrows the 120-bit integers it is decided in
                                dict(D=1 << 30, k=128, k_group=16, a=1, b=1000, weighting=1)])
def test_invalid_parameters_rejected_before_any_cuda_call(lib, kw):
    base = dict(D=1 << 16, k=128, k_group=32)
    base.update(kw)
    p = hoph.make_params(**base)
    with pytest.raises(hoph.HophError) as e:
        hoph.hoph_plan_create(p)
    assert e.value.code == hoph.HOPH_ERR_PARAM


def test_status_strings(lib):
    assert hoph.hoph_status_string(0) == "ok"
    assert "capacity" in hoph.hoph_status_string(hoph.HOPH_ERR_CAPACITY)
    assert "captured" in hoph.hoph_status_string(hoph.HOPH_ERR_CAPTURE)
    assert hoph.hoph_status_string(12345) == "unknown status"


def test_null_plan_is_a_parameter_error(lib):
    assert lib.oph_build_sketches(None, None, None, 0, None, None) == hoph.HOPH_ERR_PARAM
    assert lib.hoph_query_batch(None, 0, None, 0, None, 0, None, 0, None, None, None) == \
        hoph.HOPH_ERR_PARAM


def test_binding_constants_follow_the_header():
    """Every HOPH_* integer #define of include/hoph.h has the same value in
    the Python binding."""
    text = open(os.path.join(ROOT, "include", "hoph.h")).read()
    found = re.findall(r"#define (HOPH_\w+) \(?(-?\d+)\)?\s", text)
    assert len(found) >= 9
    for name, val in found:
        if hasattr(hoph, name):
            assert getattr(hoph, name) == int(val), name
    for name, _ in found:
        if name.startswith("HOPH_ERR_"):
            assert hasattr(hoph, name), name
