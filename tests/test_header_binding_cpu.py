"""The C header and the Python binding describe the same ABI: every
prototype in include/l1line.h has a ctypes signature in l1line.SIGNATURES
with the same arity, and each parameter and return type maps to the ctypes
type of the same size and kind (pointers to c_void_p, const char * results
to c_char_p).  ctypes converts by the declared types alone, so a drifted
signature would pass wrong bits without an error."""
import ctypes
import os
import re

import pytest

from paper_2402_16712_gb300 import l1line

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCALARS = {
    "int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
    "uint32_t": ctypes.c_uint32, "size_t": ctypes.c_size_t, "double": ctypes.c_double,
    "float": ctypes.c_float,
}


def _prototypes():
    src = open(os.path.join(ROOT, "include", "l1line.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = re.sub(r"#[^\n]*", " ", src)
    out = {}
    for ret, name, args in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(l1line_\w+)\s*\(([^;{]*?)\)\s*;",
                                      src):
        params = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        out[name] = (ret.strip(), params)
    return out


def _ctype_of(decl: str, is_return: bool = False):
    """ctypes type for a C parameter declaration or return type."""
    if "*" in decl:
        base = decl.replace("const", "").replace("*", " ").split()
        if is_return and base[:1] == ["char"]:
            return ctypes.c_char_p
        return ctypes.c_void_p
    words = decl.replace("const", "").split()
    # a parameter has a name after its type; a return type does not
    tname = words[0] if is_return or len(words) == 1 else " ".join(words[:-1])
    return SCALARS[tname]


def _same(a, b) -> bool:
    """Same size and kind (c_int64 and c_long are one type on LP64)."""
    if a is b:
        return True
    if ctypes.c_void_p in (a, b) or ctypes.c_char_p in (a, b):
        return False
    kind = lambda t: t._type_ in "fd" and "float" or (t._type_.isupper() and "u" or "s")  # noqa: E731
    return ctypes.sizeof(a) == ctypes.sizeof(b) and kind(a) == kind(b)


def test_every_prototype_has_a_binding_and_back():
    protos = _prototypes()
    assert len(protos) >= 40
    assert set(protos) == set(l1line.SIGNATURES)


@pytest.mark.parametrize("name", sorted(_prototypes()))
def test_prototype_types_match_the_binding(name):
    ret, params = _prototypes()[name]
    res, argtypes = l1line.SIGNATURES[name]
    assert len(params) == len(argtypes), (name, params, argtypes)
    want_ret = _ctype_of(ret, is_return=True)
    assert _same(want_ret, res), (name, ret, res)
    for p, a in zip(params, argtypes):
        assert _same(_ctype_of(p), a), (name, p, a)


def test_header_compiles_as_plain_c(tmp_path):
    """C callers include the header directly: it must be C99 (no C++-only
    constructs) and warning-free under -pedantic."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "l1line.h"\n'
                   "int main(void) {\n"
                   "    l1line_tuning t = {1, 2, 3, 4, 0, 1};\n"
                   "    int (*fit)(const float *, int64_t, int64_t, const double *, int64_t,\n"
                   "               float *, double *, int32_t *, void *, size_t, void *) =\n"
                   "        l1line_fit_f32;\n"
                   "    return (fit != 0 && t.warps == 1) ? 0 : 1;\n"
                   "}\n")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                    str(tmp_path / "use_header.o")], check=True)
