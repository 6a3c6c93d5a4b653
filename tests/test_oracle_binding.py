"""The oracle's ctypes binding against its C source, on the CPU: the
parameter structs' field offsets and sizes (a C program compiled with the
host compiler includes the oracle's source and prints them) and every
function's argument and return types (pointer or scalar, width,
signedness), so that a binding slip cannot feed the oracle wrong numbers."""
import ctypes
import json
import os
import re
import shutil
import subprocess

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "iewpf_oracle.c")

_C_SCALARS = {"int": (4, "i"), "long": (8, "i"), "int64_t": (8, "i"), "uint64_t": (8, "u"),
              "uint32_t": (4, "u"), "double": (8, "f"), "float": (4, "f")}


def _c_kind(param):
    p = " ".join(param.replace("const ", " ").split())
    if "*" in p or "[" in p:
        return ("ptr",)
    return _C_SCALARS[p.rsplit(" ", 1)[0]]


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return ("ptr",)
    if t in (ctypes.c_double, ctypes.c_float):
        return (ctypes.sizeof(t), "f")
    return (ctypes.sizeof(t), "i" if t(-1).value < 0 else "u")


def test_struct_layouts_match_the_source(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"orc_swe_t": O.SWE, "orc_err_t": O.ERR}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "%s"' % SRC, "int main(void) {",
             '    printf("{");']
    for cname, cls in structs.items():
        lines.append('    printf("\\"%s\\": %%zu, ", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('    printf("\\"%s.%s\\": [%%zu, %%zu], ", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (cname, fname, cname, fname, cname, fname))
    lines += ['    printf("\\"end\\": 0}\\n");', "    return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=gnu11", str(tmp_path / "layout.c"), "-o", str(exe), "-lm"], check=True)
    got = json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)
    for cname, cls in structs.items():
        assert got[cname] == ctypes.sizeof(cls), cname
        for fname, ftype in cls._fields_:
            off, size = got["%s.%s" % (cname, fname)]
            assert getattr(cls, fname).offset == off and ctypes.sizeof(ftype) == size, (cname, fname)


def test_function_types_match_the_source():
    src = re.sub(r"/\*.*?\*/", " ", open(SRC).read(), flags=re.S)
    defs = re.findall(r"^(void|int|double)\s+(orc_[a-z_0-9]+)\(([^)]*)\)\s*\{", src, flags=re.M)
    L = O.lib()
    bound = [n for n in dir(L) if n.startswith("orc_")]
    names = {name for _, name, _ in defs}
    declared = [name for name in names if getattr(L, name).argtypes is not None]
    assert declared, "no oracle function declared"
    for ret, name, args in defs:
        fn = getattr(L, name)
        if fn.argtypes is None:
            continue                      # not called through the binding
        params = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        assert len(fn.argtypes) == len(params), name
        for k, (p, t) in enumerate(zip(params, fn.argtypes)):
            assert _c_kind(p) == _ctypes_kind(t), "%s argument %d (%s)" % (name, k, p)
        if ret == "double":
            assert fn.restype is ctypes.c_double, name
        elif ret == "int":
            assert fn.restype is ctypes.c_int, name
    assert set(bound) <= names
