"""The ctypes binding against include/uf.h, parsed as text: every enum
constant the binding mirrors has the header's value, and every struct the
binding mirrors has the header's fields in the header's order with
matching C types, so a change on one side cannot go unnoticed (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2204_01117_gb300 import uf

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "uf.h")


def header_text():
    text = open(HEADER).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def enum_values():
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", header_text(), flags=re.S):
        for name, value in re.findall(r"(UF_\w+)\s*=\s*(\d+)", body):
            vals[name] = int(value)
    return vals


def struct_fields(name):
    """[(C type, field)] of `typedef struct { ... } name;`, arrays as type[n]."""
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", header_text())
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        dm = re.match(r"(const\s+)?(long long|unsigned int|double|int|float|size_t|char)\s*(.*)$", decl)
        assert dm, decl
        base = (dm.group(1) or "") + dm.group(2)
        for var in dm.group(3).split(","):
            var = var.strip()
            stars = len(var) - len(var.lstrip("*"))
            var = var.lstrip("*").strip()
            arr = re.match(r"(\w+)\s*\[(\w+)\]$", var)
            if arr:
                out.append((f"{base}{'*' * stars}[{arr.group(2)}]", arr.group(1)))
            else:
                out.append((base + "*" * stars, var))
    return out


CT = {"int": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float, "long long": ctypes.c_longlong,
      "size_t": ctypes.c_size_t, "char": ctypes.c_char, "unsigned int": ctypes.c_uint}


def same_ctype(ctype, field_type, defines):
    arr = re.match(r"(.+)\[(\w+)\]$", ctype)
    if arr:
        n = arr.group(2)
        n = defines.get(n, None) if not n.isdigit() else int(n)
        return issubclass(field_type, ctypes.Array) and field_type._length_ == n and \
            same_ctype(arr.group(1), field_type._type_, defines)
    if ctype.endswith("*"):
        return field_type is ctypes.c_void_p or issubclass(field_type, ctypes._Pointer)
    return field_type is CT[ctype.replace("const ", "").strip()]


def test_enums_match_the_header():
    v = enum_values()
    assert v["UF_F32"] == uf.F32 and v["UF_F64"] == uf.F64
    for name, val in uf.PRECOND.items():
        assert v["UF_PRECOND_" + name.upper()] == val, name
    assert v["UF_STOP_RESIDUAL"] == uf.STOP_RULE["residual"] and v["UF_STOP_PAPER"] == uf.STOP_RULE["paper"]
    for name, val in uf.SMOOTHER.items():
        assert v["UF_SMOOTH_" + name.upper()] == val, name
    for name, val in uf.TRANSFER.items():
        assert v["UF_TRANSFER_" + name.upper()] == val, name
    for name, val in uf.FIELDS.items():
        assert v["UF_FIELD_" + name.upper()] == val, name
    for i, name in enumerate(uf.STATUS_NAMES):
        assert v[name] == i, name
    subs = {"eddy": "EDDY", "advect": "ADVECT", "diffuse": "DIFFUSE", "drag_bc": "DRAG_BC", "project": "PROJECT",
            "turb": "TURB"}
    for name, (which, _, _) in uf.SUBSTEPS.items():
        assert v["UF_SUB_" + subs[name]] == which, name
    assert v["UF_OBJ_COMFORT"] == 0 and v["UF_OBJ_REGIONS"] == 1


def defines():
    return {k: int(x) for k, x in re.findall(r"#define\s+(UF_\w+)\s+(\d+)\b", header_text())}


@pytest.mark.parametrize("cname, pyname", [("uf_grid_desc", "GridDesc"), ("uf_step_stats", "StepStats"),
                                           ("uf_objective_desc", "ObjectiveDesc"), ("uf_tuning", "Tuning"),
                                           ("uf_kernel_time", "KernelTime")])
def test_structs_match_the_header(cname, pyname):
    fields = struct_fields(cname)
    py = getattr(uf, pyname)._fields_
    assert [f for _, f in fields] == [f for f, _ in py], (cname, fields, py)
    d = defines()
    for (ctype, f), (_, ftype) in zip(fields, py):
        assert same_ctype(ctype, ftype, d), (cname, f, ctype, ftype)
