"""The Python binding marshals every call of include/ms.h with the header's
argument widths, and its structs have the header's fields in the header's
order (no GPU, no library needed): a mismatch would pass garbage through
ctypes without an error."""
import ctypes
import os
import re

import paper_2007_14283_gb300 as ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = open(os.path.join(ROOT, "include", "ms.h")).read()
CODE = re.sub(r"/\*.*?\*/", "", HEADER, flags=re.S)

C_SCALARS = {"int32_t": "i32", "ms_status": "i32", "int64_t": "i64", "uint64_t": "u64", "double": "f64",
             "float": "f32", "void": "void"}


def c_kind(decl):
    """'i32', 'i64', 'u64', 'f64', 'ptr' or 'void' for a C type (with or without a name)."""
    if "*" in decl:
        return "ptr"
    words = [w for w in re.findall(r"\w+", decl) if w not in ("const", "struct")]
    return C_SCALARS[words[0]]


def ctypes_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or isinstance(t, type(ctypes.POINTER(ctypes.c_int))):
        return "ptr"
    return {ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_uint64: "u64", ctypes.c_double: "f64",
            ctypes.c_float: "f32"}[t]


def header_functions():
    out = {}
    for m in re.finditer(r"MS_API\s+([\w\s\*]+?)\b(ms_\w+)\s*\((.*?)\)\s*;", CODE, re.S):
        ret, name, params = m.group(1), m.group(2), m.group(3).strip()
        args = [] if params in ("", "void") else [c_kind(p) for p in params.split(",")]
        out[name] = (c_kind(ret), args)
    return out


def header_struct(name):
    m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), CODE, re.S)
    fields = []
    for line in m.group(1).split(";"):
        line = line.strip()
        if not line:
            continue
        mm = re.match(r"(\w+)\s+(\w+)(?:\[(\d+)\])?$", line)
        fields.append((mm.group(2), C_SCALARS[mm.group(1)], int(mm.group(3) or 0)))
    return fields


def test_every_declaration_has_a_binding_with_the_same_widths():
    decl = header_functions()
    assert len(decl) >= 40
    assert set(decl) == set(ms._SIGNATURES), set(decl) ^ set(ms._SIGNATURES)
    for name, (ret, args) in decl.items():
        bret, bargs = ms._SIGNATURES[name]
        assert ctypes_kind(bret) == ret, (name, "return")
        assert [ctypes_kind(a) for a in bargs] == args, name


def test_structs_match_the_header_field_by_field():
    for cname, py in (("ms_config", ms.ms_config), ("ms_stats", ms.ms_stats),
                      ("ms_tune_result", ms.ms_tune_result)):
        want = header_struct(cname)
        got = []
        for fname, ftype in py._fields_:
            if issubclass(ftype, ctypes.Array):
                got.append((fname, ctypes_kind(ftype._type_), ftype._length_))
            else:
                got.append((fname, ctypes_kind(ftype), 0))
        assert got == want, cname


def test_the_checker_sees_a_planted_mismatch():
    """The parser itself: a width changed in a copy of the table is caught."""
    decl = header_functions()
    ret, args = decl["ms_set_state"]
    assert args == ["ptr", "i64"]
    bargs = [ctypes.c_void_p, ctypes.c_int32]
    assert [ctypes_kind(a) for a in bargs] != args
