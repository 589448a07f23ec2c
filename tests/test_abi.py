"""The C-ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dd_wilson.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2407_00041_gb300 import binding
    lib = binding.load()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same set
    assert set(binding.SIGNATURES) == set(names)


def test_host_side_argument_checks_without_gpu():
    from paper_2407_00041_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    for bad in ((3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 4, 5)):
        arr = (ctypes.c_int * 4)(*bad)
        assert lib.dd_lattice_create(arr, -1, ctypes.byref(h)) == binding.DD_ERR_ARG
        assert b"even" in lib.dd_last_error_detail()
    arr = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.dd_lattice_create(arr, 0, ctypes.byref(h)) == binding.DD_ERR_ARG
    assert lib.dd_lattice_create(arr, -1, ctypes.byref(h)) == 0
    assert lib.dd_lattice_volume(h) == 256
    lib.dd_lattice_destroy(h)
    assert lib.dd_error_string(-5) == b"DD_ERR_NOT_CONVERGED"
    p = binding.SolveParams()
    lib.dd_solve_params_default(ctypes.byref(p))
    assert p.tol == 1e-10 and p.restart == 30 and p.even_odd == 1
    assert p.refine_prec == binding.DD_PREC_F64 and p.amg is None


def test_no_cpu_fallback_in_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2407_00041_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, flags=re.M), f


def _ctype_of(decl):
    """Kind of ctypes type the binding must use for one C parameter
    declaration ("type name", "type* name", "type name[4]")."""
    decl = decl.strip()
    if "*" in decl or "[" in decl:
        return "char_p" if re.match(r"const\s+char\s*\*", decl) else "pointer"
    words = decl.replace("const", " ").split()
    base = " ".join(words[:-1])  # the last word is the parameter name
    return {"int": "int", "double": "double", "int64_t": "int64", "uint64_t": "size_t", "unsigned": "uint",
            "size_t": "size_t", "void": None}[base]


def test_binding_argument_and_return_types_match_the_header():
    """Every ctypes signature in the binding has the parameter count, the
    parameter kinds and the return type of its C declaration."""
    from paper_2407_00041_gb300 import binding
    kinds = {ctypes.c_void_p: "pointer", ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_int64: "int64",
             ctypes.c_uint: "uint", ctypes.c_size_t: "size_t", ctypes.c_char_p: "char_p", None: None}
    src = open(os.path.join(ROOT, "include", "dd_wilson.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    decls = re.findall(r"^([A-Za-z_][\w \*]*?)\b(dd_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S | re.M)
    assert len(decls) == len(binding.SIGNATURES)
    for ret, name, params in decls:
        res, args = binding.SIGNATURES[name]
        params = params.strip()
        plist = [] if params in ("", "void") else [p for p in params.split(",")]
        assert len(plist) == len(args), name
        assert kinds[res] == _ctype_of(ret.strip() + " x"), (name, ret)
        for i, (p, a) in enumerate(zip(plist, args)):
            assert kinds[a] == _ctype_of(p), (name, i, p)


def test_binding_structs_match_the_header():
    """The ctypes mirrors of dd_solve_params, dd_stats and dd_amg_params have
    the C structs' fields in the same order, with the same types and array
    lengths, so that their layouts agree."""
    from paper_2407_00041_gb300 import binding
    src = open(os.path.join(ROOT, "include", "dd_wilson.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double, "dd_amg*": ctypes.c_void_p}
    for cname, pyclass in (("dd_solve_params", binding.SolveParams), ("dd_stats", binding.Stats),
                           ("dd_amg_params", binding.AmgParams)):
        body = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + cname + r"\s*;", src, flags=re.S)
        assert body, cname
        fields = []
        for decl in body.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"^([A-Za-z_]\w*\s*\*?)\s*([A-Za-z_]\w*)\s*(?:\[(\d+)\])?$", decl)
            assert m, (cname, decl)
            typ = m.group(1).replace(" ", "")
            t = ctype[typ]
            fields.append((m.group(2), t * int(m.group(3)) if m.group(3) else t))
        py = [(n, t) for n, t in pyclass._fields_]
        assert [n for n, _ in py] == [n for n, _ in fields], cname
        for (n, t), (_, u) in zip(py, fields):
            assert ctypes.sizeof(t) == ctypes.sizeof(u) and getattr(t, "_type_", t) == getattr(u, "_type_", u), (cname, n)
