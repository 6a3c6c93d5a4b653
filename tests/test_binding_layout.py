"""The binding's ABI against include/iewpf.h, on the CPU: a C program
compiled with the host compiler prints every field's offset and size and
each struct's size, which must equal the ctypes layout; every exported
function's ctypes argument and return types match its prototype (pointer or
scalar, width, signedness); and the configuration -> parameter mapping puts
every value in its named field."""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

from paper_1910_01031_gb300 import iewpf, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"iewpf_params_t": iewpf.Params, "iewpf_obs_t": iewpf.Obs, "iewpf_diag_t": iewpf.Diag}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "iewpf.h"', "int main(void) {",
             '    printf("{");']
    for cname, cls in STRUCTS.items():
        lines.append('    printf("\\"%s\\": %%zu, ", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('    printf("\\"%s.%s\\": [%%zu, %%zu], ", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (cname, fname, cname, fname, cname, fname))
    lines += ['    printf("\\"end\\": 0}\\n");', "    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return json.loads(subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_ctypes_structure_matches_the_c_struct(c_layout, cname):
    cls = STRUCTS[cname]
    assert c_layout[cname] == ctypes.sizeof(cls)
    for fname, ftype in cls._fields_:
        off, size = c_layout["%s.%s" % (cname, fname)]
        assert getattr(cls, fname).offset == off, fname
        assert ctypes.sizeof(ftype) == size, fname


def test_params_from_config_fills_every_named_field():
    cfg = synth.config4()
    p = iewpf.params_from_config(cfg, n_drifters_max=7, scheme=iewpf.ONE_STAGE)
    expect = {"nx": cfg.nx, "ny": cfg.ny, "dx": cfg.dx, "dy": cfg.dy, "g": cfg.g, "f": cfg.f, "H_eq": cfg.H,
              "theta": cfg.theta, "courant": cfg.courant, "dt_model": cfg.dt_model, "c_omega": cfg.c_omega,
              "q0": cfg.q0, "L0": cfg.L0, "seed": cfg.seed, "n_particles": cfg.n_particles,
              "obs_kind": cfg.obs_kind, "n_obs_max": cfg.n_obs, "obs_sigma": cfg.obs_sigma,
              "dense_S": cfg.dense_S, "instance_id": 0, "n_drifters_max": 7, "scheme": iewpf.ONE_STAGE}
    assert set(expect) == {f for f, _ in iewpf.Params._fields_}
    for k, v in expect.items():
        assert getattr(p, k) == v, k
    assert iewpf.params_from_config(cfg, n_obs_max=3).n_obs_max == 3


_C_SCALARS = {"int": (4, "i"), "int64_t": (8, "i"), "uint64_t": (8, "u"), "uint32_t": (4, "u"),
              "double": (8, "f"), "float": (4, "f"), "size_t": (8, "u")}


def _c_kind(param):
    """('ptr',) for a pointer parameter, else (size, signedness) of its type."""
    p = " ".join(param.replace("const ", " ").split())
    if "*" in p:
        return ("ptr",)
    base = p.rsplit(" ", 1)[0] if " " in p else p
    return _C_SCALARS[base]


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return ("ptr",)
    size = ctypes.sizeof(t)
    if t in (ctypes.c_double, ctypes.c_float):
        return (size, "f")
    signed = t(-1).value < 0
    return (size, "i" if signed else "u")


def test_every_export_has_the_headers_argument_types():
    import re
    src = open(os.path.join(ROOT, "include", "iewpf.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    protos = re.findall(r"IEWPF_API\s+(int|const char\*)\s+([a-z_]+)\((.*?)\);", src, flags=re.S)
    assert len(protos) == len(iewpf.EXPORTS)
    L = iewpf.load()
    for ret, name, args in protos:
        fn = getattr(L, name)
        params = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        assert len(fn.argtypes) == len(params), name
        for k, (p, t) in enumerate(zip(params, fn.argtypes)):
            assert _c_kind(p) == _ctypes_kind(t), "%s argument %d (%s)" % (name, k, p)
        assert fn.restype is (ctypes.c_int if ret == "int" else ctypes.c_char_p), name


class _FakeTensor:
    """Stands in for a CUDA torch tensor: only what the binding inspects."""

    def __init__(self, shape, dtype="torch.float32", contiguous=True, cuda=True):
        self.shape, self.dtype, self._c, self.is_cuda = tuple(shape), dtype, contiguous, cuda

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("the library must not be reached")


def test_device_tensors_of_the_wrong_layout_are_refused_before_the_library():
    e = iewpf.Ensemble.__new__(iewpf.Ensemble)
    e.ne, e.nx, e.ny, e.L, e.h = 2, 16, 8, None, None
    good = (2, 3, 8, 16)
    for bad in (_FakeTensor((2, 3, 8, 15)), _FakeTensor((1, 3, 8, 16)), _FakeTensor(good, "torch.float64"),
                _FakeTensor(good, contiguous=False)):
        with pytest.raises(ValueError):
            e.set_state(bad)
        with pytest.raises(ValueError):
            e.get_state(bad)
    s = iewpf.Surrogate.__new__(iewpf.Surrogate)
    s.nx, s.ny, s.L, s.h = 16, 8, None, None
    for U, out in ((_FakeTensor((4, 3, 8, 15)), None), (_FakeTensor((4, 3, 8, 16), cuda=False), None),
                   (_FakeTensor((4, 3, 8, 16)), _FakeTensor((3, 3, 8, 16))),
                   (_FakeTensor((4, 3, 8, 16)), _FakeTensor((4, 3, 8, 16), "torch.bfloat16"))):
        with pytest.raises(ValueError):
            s.apply_device(U, out=out)
