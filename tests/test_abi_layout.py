"""The ctypes binding agrees with include/mfwh.h: struct layouts, constants and
function signatures.

A binding that disagrees with the header does not fail loudly: a field at the
wrong offset, an int passed where the library reads an int64_t, or a float where
it reads a double hands the library garbage.  The layouts and constants are
read from the header by a small C program compiled with the host compiler; the
signatures are read from the header's prototypes.  No GPU is needed.
"""

import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2507_23613_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADER = os.path.join(INCLUDE, "mfwh.h")

STRUCTS = {"mfwh_problem": _lib.Problem, "mfwh_setup": _lib.Setup,
           "mfwh_solve_info": _lib.SolveInfo}

# Status codes and modes: header name -> binding name (the header's MFWH_ prefix dropped).
CONSTANTS = ["MFWH_MAX_NF", "MFWH_OK", "MFWH_ERR_INVALID_ARG", "MFWH_ERR_SINGULAR",
             "MFWH_ERR_CUDA", "MFWH_ERR_NOMEM", "MFWH_ERR_NOT_CONVERGED", "MFWH_ERR_SPURIOUS",
             "MFWH_ERR_NONFINITE", "MFWH_ERR_TIMEOUT", "MFWH_FILTER_OPTIMIZED",
             "MFWH_FILTER_TRADITIONAL", "MFWH_FILTER_USER", "MFWH_PREC_FP64",
             "MFWH_PREC_FP32_KAHAN", "MFWH_PREC_FP32_BLOCKSUM", "MFWH_UPDATE_IMPLICIT",
             "MFWH_UPDATE_EXPLICIT", "MFWH_C_CONST", "MFWH_C_TWO_LAYER", "MFWH_C_FIELD",
             "MFWH_TIME_EXPLICIT", "MFWH_TIME_IMPLICIT"]


def _header_text():
    with open(HEADER) as fh:
        return fh.read()


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """sizeof / offsetof of every binding field and the constants, as the C compiler sees the
    header."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mfwh.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("field {cname}.{field} %zu %zu\\n", '
                         f"offsetof({cname}, {field}), sizeof((({cname}*)0)->{field}));")
    for name in CONSTANTS:
        lines.append(f'  printf("const {name} %lld\\n", (long long)({name}));')
    lines.append('  printf("const MFWH_NOALLOC_SCRATCH_DOUBLES %lld\\n", '
                 "(long long)MFWH_NOALLOC_SCRATCH_DOUBLES);")
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", INCLUDE, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, fields, consts = {}, {}, {}
    for line in out.splitlines():
        kind, name, *vals = line.split()
        if kind == "size":
            sizes[name] = int(vals[0])
        elif kind == "field":
            fields[name] = (int(vals[0]), int(vals[1]))
        else:
            consts[name] = int(vals[0])
    return sizes, fields, consts


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    sizes, fields, _ = c_layout
    py = STRUCTS[cname]
    assert C.sizeof(py) == sizes[cname], cname
    for field, _ in py._fields_:
        desc = getattr(py, field)
        assert (desc.offset, desc.size) == fields[f"{cname}.{field}"], f"{cname}.{field}"


def test_struct_fields_in_header_order():
    """Every field the header declares is in the binding, in the header's order (an extra field
    at the end of a C struct would not move any offset)."""
    text = re.sub(r"/\*.*?\*/", "", _header_text(), flags=re.S)
    for cname, py in STRUCTS.items():
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r"\s*;", text)
        assert body, cname
        names = []
        for decl in body.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "double c_lo, c_hi" declares two fields; array bounds and pointer stars are dropped
            head, *rest = decl.split(",")
            names.append(re.sub(r"\[.*", "", head.split()[-1]).lstrip("*"))
            names += [re.sub(r"\[.*", "", r.strip()).lstrip("*") for r in rest]
        assert names == [f for f, _ in py._fields_], cname


def test_constants_match_header(c_layout):
    _, _, consts = c_layout
    for name in CONSTANTS:
        assert getattr(_lib, name[len("MFWH_"):]) == consts[name], name
    assert consts["MFWH_NOALLOC_SCRATCH_DOUBLES"] == 32768


# C parameter type (const dropped, spaces normalised) -> the ctypes types that pass it intact.
_PTR_OK = (C.c_void_p, C.c_char_p)


def _scalar(ctype):
    return {"int": C.c_int, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double,
            "float": C.c_float, "mfwh_status": C.c_int}.get(ctype)


def _is_pointer(t):
    return t in _PTR_OK or (isinstance(t, type) and issubclass(t, C._Pointer))


def _prototypes():
    text = re.sub(r"/\*.*?\*/", "", _header_text(), flags=re.S)
    text = re.sub(r"#[^\n]*", "", text)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(mfwh_\w+)\s*\(([^;{]*?)\)\s*;", text):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3)
        ret = ret.split("\n")[-1].strip()
        plist = [] if params.strip() in ("", "void") else [p.strip() for p in params.split(",")]
        protos[name] = (ret, plist)
    return protos


def _param_type(decl):
    """'const double* v' -> ('double', 1, []); 'int64_t cells[16][3]' -> ('int64_t', 1, [3]):
    an array parameter decays to a pointer to its element, here an array of 3."""
    dims = [int(d) for d in re.findall(r"\[(\d+)\]", decl)]
    decl = " ".join(re.sub(r"\[.*", "", decl).replace("const", " ").split())
    stars = decl.count("*") + (1 if dims else 0)
    base = decl.replace("*", " ").split()[0]
    return base, stars, dims[1:]


def test_signatures_match_header():
    protos = _prototypes()
    assert sorted(protos) == sorted(_lib.declared_symbols())
    for name, (ret, params) in protos.items():
        res, args = _lib._SIGNATURES[name]
        assert len(args) == len(params), name
        # return type
        if ret == "void":
            assert res is None, name
        elif ret.endswith("*"):
            assert res is C.c_char_p, name
        else:
            assert res is _scalar(ret), (name, ret, res)
        for i, (decl, t) in enumerate(zip(params, args)):
            base, stars, inner = _param_type(decl)
            if base in ("mfwh_handle_t", "mfwh_cnn_t") and stars == 0:
                assert t is C.c_void_p, (name, i, decl)
            elif stars or base in ("mfwh_handle_t", "mfwh_cnn_t"):
                assert _is_pointer(t), (name, i, decl, t)
                if stars == 1 and base in ("double", "int", "int64_t") and t is not C.c_void_p:
                    want = _scalar(base)
                    for n in reversed(inner):
                        want = want * n
                    assert t._type_ is want or (
                        inner and t._type_._type_ is _scalar(base)
                        and t._type_._length_ == inner[-1]), (name, i, decl, t)
                if base in ("mfwh_problem", "mfwh_setup", "mfwh_solve_info") and t is not C.c_void_p:
                    assert t._type_ is STRUCTS[base], (name, i, decl, t)
            else:
                assert t is _scalar(base), (name, i, decl, t)
