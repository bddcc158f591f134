"""CPU checks of the C ABI library: it builds, loads, exports every symbol
include/fmm2d.h declares, and its planner rules agree with the oracle's."""
import os
import re

import pytest

from conftest import ROOT

from oracle import params as op


@pytest.fixture(scope="module")
def fm():
    from paper_1204_3105_gb300 import build, fmm2d
    build.build()
    fmm2d.lib()
    return fmm2d


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(fmm2d_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(fm):
    names = _declared()
    assert "fmm2d_build" in names and "fmm2d_evaluate" in names
    L = fm.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(fm.SYMBOLS) <= names


@pytest.mark.parametrize("tiling", ["quad", "sept", "tri"])
def test_planner_rules_match_oracle(fm, tiling):
    for n in (1000, 8192, 100000, 2 ** 20, 4 * 10 ** 6):
        L, p, r = fm.fmm2d_default_params(tiling, n, 64, 1e-6)
        assert L == op.auto_levels(tiling, n)
        assert p == op.p_from_eps(tiling, 1e-6)
        if tiling == "sept":
            assert r == op.sept_leaf_circumradius(L)          # bit-exact
        elif tiling == "tri":
            assert r == op.tri_root_inradius()
    for eps in (1e-3, 1e-4, 1e-8, 1e-10):
        assert fm.fmm2d_default_params(tiling, 1000, 64, eps)[1] == op.p_from_eps(tiling, eps)
    # leaf target 0: the S_opt level of Table 2 / App. A-C
    for n in (1000, 5120, 100000, 2 ** 20, 4 * 10 ** 6):
        for eps in (1e-4, 1e-6, 1e-10):
            L, p, _ = fm.fmm2d_default_params(tiling, n, 0, eps)
            assert L == op.sopt_levels(tiling, n, n, p), (n, eps)


def test_bad_arguments_rejected_without_gpu(fm):
    with pytest.raises(fm.FMM2DError) as e:
        fm.Plan("quad", levels=40)
    assert e.value.status == fm.EINVAL
    with pytest.raises(fm.FMM2DError):
        fm.Plan(7)
    with pytest.raises(fm.FMM2DError):
        fm.Plan("quad", p=0, eps=2.0)
    with pytest.raises(fm.FMM2DError):
        fm.fmm2d_default_params("quad", 100, 64, 0.0)


def _header():
    txt = open(os.path.join(ROOT, "include", "fmm2d.h")).read()
    return re.sub(r"/\*.*?\*/", "", txt, flags=re.S)


def _struct_fields(txt, name):
    """Field names, in order, of `typedef struct { ... } name;`."""
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", txt, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            part = re.sub(r"\[.*?\]", "", part).strip()   # arrays: keep the name
            fields.append(re.findall(r"\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*$", part)[0])
    return fields


def test_binding_matches_header(fm):
    """The ctypes binding's flag values and struct layouts are the header's:
    every flag macro, and the field order of the request, result, info and
    server-statistics structs."""
    txt = _header()
    macros = dict(re.findall(r"#define\s+(FMM2D_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+)u", txt))
    for name in ("PREC_FP64", "PREC_MIXED", "PREC_MIXED_TC", "PREC_HYBRID", "PREC_SPLIT",
                 "IN_F32", "ADAPTIVE", "SERVE_PREC_AS_GIVEN", "FIELD"):
        assert getattr(fm, name) == int(macros["FMM2D_" + name], 16), name
    for cname, py in (("fmm2d_request", fm.Request), ("fmm2d_result", fm.Result),
                      ("fmm2d_info", fm.Info), ("fmm2d_serve_info", fm.ServeInfo)):
        assert _struct_fields(txt, cname) == [f for f, _ in py._fields_], cname


def test_unknown_precision_form_rejected(fm):
    """Precision values past FMM2D_PREC_SPLIT are refused at plan creation."""
    for bad in (0x5, 0x6, 0x7, 0x8):
        with pytest.raises(fm.FMM2DError) as e:
            fm.Plan("quad", levels=4, p=8, flags=bad)
        assert e.value.status == fm.EINVAL
