"""The ctypes structures of the binding against the C structs of
include/iewpf.h, on the CPU: a C program compiled with the host compiler
prints every field's offset and size and each struct's size, which must
equal the ctypes layout; and the configuration -> parameter mapping puts
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
