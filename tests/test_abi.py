"""The C-ABI library loads and exports every entry point its header declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mbinv_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    import paper_1612_00001_gb300 as mb
    return mb.build()


def test_header_declares_entry_points():
    names = declared()
    for must in ("mbinv_create", "mbinv_block", "mbinv_all_blocks", "mbinv_backward", "mbinv_batched_blocks",
                 "mbinv_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    import paper_1612_00001_gb300 as mb
    L = mb.lib()
    for n in declared():
        assert hasattr(L, n)
        assert n in mb.SIGNATURES, f"binding lacks {n}"
    assert L.mbinv_version().decode().startswith("mbinv")
    assert L.mbinv_status_string(mb.ESINGULAR).decode()
    o = mb.Options()
    L.mbinv_default_options(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(mb.Options) and o.precision == 0 and o.bf16_slices == 3


def test_invalid_arguments_rejected_without_gpu(libpath):
    import paper_1612_00001_gb300 as mb
    L = mb.lib()
    h = ctypes.c_void_p()
    # null matrix, bad k, bad dtype: rejected before any CUDA call
    assert L.mbinv_create(ctypes.byref(h), 16, 4, 0, None, 16, None) == mb.EINVAL
    buf = (ctypes.c_double * 256)()
    assert L.mbinv_create(ctypes.byref(h), 16, 0, 0, buf, 16, None) == mb.EINVAL
    assert L.mbinv_create(ctypes.byref(h), 16, 4, 7, buf, 16, None) == mb.EINVAL
    assert L.mbinv_create(ctypes.byref(h), 16, 4, 0, buf, 8, None) == mb.EINVAL
    assert L.mbinv_block(None, 0, 0, buf, 4, None) == mb.EINVAL
    assert L.mbinv_batched_blocks(-1, None, 0, None, None) == mb.EINVAL


# C type of a header field -> the ctypes type its mirror must use
_CTYPES = {"double": ctypes.c_double, "size_t": ctypes.c_size_t, "int64_t": ctypes.c_int64, "int": ctypes.c_int,
           "uint64_t": ctypes.c_uint64, "mbinv_precision": ctypes.c_int}


def header_struct(name):
    """Fields (name, C type, array length) of `typedef struct {...} name;` in include/mbinv.h."""
    text = open(os.path.join(ROOT, "include", "mbinv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        dm = re.match(r"(const\s+)?(\w+)\s*(\*?)\s*(.*)", decl)
        ctype, ptr, names = dm.group(2), dm.group(3), dm.group(4)
        for nm in names.split(","):
            nm = nm.strip()
            star = ptr or nm.startswith("*")
            nm = nm.lstrip("*").strip()
            am = re.match(r"(\w+)\[(\d+)\]", nm)
            fields.append((am.group(1) if am else nm, "void*" if star else ctype, int(am.group(2)) if am else 1))
    return fields


@pytest.mark.parametrize("cname,pyname", [("mbinv_report", "Report"), ("mbinv_options", "Options"),
                                          ("mbinv_problem", "Problem"), ("mbinv_rbf", "Rbf")])
def test_binding_structs_match_header(cname, pyname):
    """The ctypes mirrors declare the header's fields in the header's order
    with the same types (a drifted struct would shift every later field)."""
    import paper_1612_00001_gb300 as mb
    py = getattr(mb, pyname)._fields_
    hdr = header_struct(cname)
    assert [f[0] for f in py] == [h[0] for h in hdr], (cname, [f[0] for f in py], [h[0] for h in hdr])
    for (fname, ftype), (hname, htype, count) in zip(py, hdr):
        want = ctypes.c_void_p if htype == "void*" else _CTYPES[htype]
        if count > 1:
            want = want * count
        assert ctypes.sizeof(ftype) == ctypes.sizeof(want) and getattr(ftype, "_type_", None) == getattr(
            want, "_type_", None), (cname, fname, ftype, htype)


def test_product_library_exports_no_test_hooks(libpath):
    """The C-ABI symbols of libmbinv.so are the header's entry points; the
    test hooks live in libmbinv_test.so beside it."""
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.split() and l.split()[-1].startswith("mbinv_")}
    assert exported == set(declared()), sorted(exported ^ set(declared()))
    test_lib = os.path.join(os.path.dirname(libpath), "libmbinv_test.so")
    hooks = subprocess.run(["nm", "-D", "--defined-only", test_lib], capture_output=True, text=True,
                           check=True).stdout
    assert "mbinv_debug_oz_gemm" in hooks
