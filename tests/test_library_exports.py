"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every entry point declared in include/iewpf.h, and its calls
fail with an error code (not a crash) when no GPU is present."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "iewpf.h")).read()
    return sorted(set(re.findall(r"IEWPF_API\s+(?:int|const char\*)\s+([a-z_]+)\(", src)))


def test_header_declares_the_binding_exports():
    from paper_1910_01031_gb300 import iewpf
    assert _declared() == sorted(iewpf.EXPORTS)


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1910_01031_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in _declared():
        assert name in exported, name
    # nothing but the C ABI is exported
    assert exported == set(_declared())


def test_library_loads_and_reports_errors_without_crashing():
    from paper_1910_01031_gb300 import iewpf
    L = iewpf.load()
    for name in iewpf.EXPORTS:
        assert hasattr(L, name)
    assert L.iewpf_last_error(None) == b"null context"
    assert L.iewpf_forecast(None, 1, 1) == -1
    assert L.iewpf_destroy(None) == 0
    bad = iewpf.Params()
    h = __import__("ctypes").c_void_p()
    assert L.iewpf_create(__import__("ctypes").byref(bad), None, __import__("ctypes").byref(h)) == -1
    # an unknown analysis scheme is refused before any device work
    from paper_1910_01031_gb300 import synth
    p = iewpf.params_from_config(synth.config1())
    p.scheme = 2
    assert L.iewpf_create(__import__("ctypes").byref(p), None, __import__("ctypes").byref(h)) == -1


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1910_01031_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("the oracle", ""), f


def test_every_export_has_its_argument_types_declared():
    # a C function called through ctypes without argtypes would have its
    # arguments converted by guesswork (doubles and 64-bit ints lost)
    from paper_1910_01031_gb300 import iewpf
    L = iewpf.load()
    assert [n for n in iewpf.EXPORTS if getattr(L, n).argtypes is None] == []


def test_building_blocks_refuse_bad_arguments_before_device_work():
    # these checks run on the host, so they hold without a GPU
    import ctypes
    import numpy as np
    from paper_1910_01031_gb300 import iewpf
    L = iewpf.load()
    dp = ctypes.POINTER(ctypes.c_double)
    one = np.ones(3)
    p = one.ctypes.data_as(dp)
    out = np.zeros(3)
    q = out.ctypes.data_as(dp)
    assert L.iewpf_weights(0, 10.0, p, p, p, q, q, q, q) == -1                 # no particles
    assert L.iewpf_weights(3, 0.0, p, p, p, q, q, q, q) == -1                  # N_psi not positive
    assert L.iewpf_weights(3, 10.0, None, p, p, q, q, q, q) == -1
    assert L.iewpf_weights_one_stage(3, -1.0, p, p, q, q, q, q) == -1
    neg = np.array([1.0, -0.5, 2.0])
    assert L.iewpf_alpha_gamma(3, 10.0, p, neg.ctypes.data_as(dp), q) == -1   # c* < 0
    assert L.iewpf_alpha_gamma(3, 10.0, neg.ctypes.data_as(dp), p, q) == -1   # gamma <= 0
    assert L.iewpf_normals(0, 0, 0, 0, 4, None, None) == -1                   # no output
