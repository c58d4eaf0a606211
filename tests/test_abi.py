"""The C ABI library loads and exports every entry point that include/sunb.h
declares; argument validation that needs no GPU (CPU-only checks)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sunb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sunb_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_01713_b300 import build
    build.build()
    import paper_2405_01713_b300 as sb
    return sb.lib()


def test_header_declares_the_boundary():
    """The calls of the boundary: create / set_tolerances / set_params /
    integrate / stats / adjoint / destroy / last_error, plus the single steps."""
    names = _declared()
    for n in ("sunb_create", "sunb_set_tolerances", "sunb_set_params", "sunb_integrate",
              "sunb_stats", "sunb_adjoint", "sunb_destroy", "sunb_last_error", "sunb_rhs", "sunb_jac",
              "sunb_lu_solve_batched", "sunb_get_tapes"):
        assert n in names


def _signature(name):
    txt = open(os.path.join(ROOT, "include", "sunb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    m = re.search(r"\b" + name + r"\s*\(([^)]*)\)", txt)
    return [a.strip() for a in m.group(1).split(",")]


def test_boundary_signatures():
    """set_params carries the byte count of the parameter array, stats the
    host totals and the optional per-cell device counters."""
    assert _signature("sunb_set_params") == ["sunb_ctx *ctx", "const double *dev_params", "size_t bytes"]
    assert _signature("sunb_stats") == ["sunb_ctx *ctx", "sunb_stats_t *host_totals", "int32_t *dev_per_cell"]
    assert _signature("sunb_adjoint")[:3] == ["sunb_ctx *ctx", "const double *dev_dLdy", "double *dev_grad"]


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    import paper_2405_01713_b300 as sb
    assert set(_declared()) <= set(sb.SIGNATURES)


def test_version_and_null_arguments_without_gpu(lib):
    import paper_2405_01713_b300 as sb
    assert b"sm_103a" in lib.sunb_version()
    out = ctypes.c_void_p()
    assert lib.sunb_create(None, None, ctypes.byref(out)) == sb.ILL_INPUT
    assert out.value is None
    assert b"NULL" in lib.sunb_last_error(None)
    assert lib.sunb_lu_solve_batched(0, 1, None, None, None, None, None) == sb.ILL_INPUT
    assert lib.sunb_lu_solve_batched(65, 1, None, None, None, None, None) == sb.ILL_INPUT
    assert lib.sunb_destroy(None) == 0
    assert lib.sunb_set_params(None, None, 0) == sb.ILL_INPUT
    assert lib.sunb_stats(None, None, None) == sb.ILL_INPUT
    assert lib.sunb_get_tapes(None, 0, 0, None) == sb.ILL_INPUT
    assert lib.sunb_tape_stride(None) == 0


def test_library_is_built_for_sm_103a():
    from paper_2405_01713_b300 import build
    assert "arch=compute_103a,code=sm_103a" in build.FLAGS


def test_binding_constants_equal_the_header():
    """Every SUNB_* value the header defines (enumerators and #defines)
    has the same value in the binding, under its name without the prefix
    (status codes also in the binding's STATUS table)."""
    import paper_2405_01713_b300 as sb
    txt = open(os.path.join(ROOT, "include", "sunb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    vals = {k: int(v) for k, v in re.findall(r"\bSUNB_([A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    vals.update({k: int(v) for k, v in re.findall(r"#define\s+SUNB_([A-Z0-9_]+)\s+(-?\d+)", txt)})
    assert len(vals) >= 20
    statuses = {k for k in vals if vals[k] <= 0 and k in sb.STATUS.values()}
    for name, v in vals.items():
        if name in statuses:
            assert sb.STATUS[v] == name
        if hasattr(sb, name):
            assert getattr(sb, name) == v, name
    for name in ("ROBERTSON", "MECHANISM", "COSMOLOGY", "MIXED", "FP64", "MIXED32",
                 "SCHED_QUEUE", "SCHED_STATIC", "LS_DIRECT", "LS_GMRES", "METHOD_BDF", "METHOD_ERK"):
        assert getattr(sb, name) == vals[name], name
