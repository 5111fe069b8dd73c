"""CPU checks of the C-ABI boundary: the library builds, loads and exports every entry point
declared in include/pic.h, and the ctypes structs match the C layout (offsets from gcc)."""

import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")


@pytest.fixture(scope="module")
def built_lib():
    from paper_2606_15035_gb300 import build
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pic_init", "pic_step", "pic_energy", "pic_diagnostics", "pic_get_state", "pic_set_state",
                     "pic_destroy", "pic_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = C.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pic_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_loads_and_defaults(built_lib):
    from paper_2606_15035_gb300 import sim
    cfg = sim.pic_config_default()
    assert tuple(cfg.n) == (8, 8, 8) and cfg.split_orbit_at_knots == 1 and cfg.precision == 0


def test_ctypes_layout_matches_c():
    from paper_2606_15035_gb300 import _lib
    structs = {
        "pic_config": _lib.PicConfig, "pic_particles": _lib.PicParticles, "pic_allocator": _lib.PicAllocator,
        "pic_step_info": _lib.PicStepInfo, "pic_energy_t": _lib.PicEnergy, "pic_diag_t": _lib.PicDiag,
        "pic_state_view": _lib.PicStateView, "pic_iterate_out": _lib.PicIterateOut, "pic_profile_t": _lib.PicProfile,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            fname = f[0]
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        cname, field, val = line.split()
        py = structs[cname]
        if field == "size":
            assert C.sizeof(py) == int(val), (cname, C.sizeof(py), val)
        else:
            assert getattr(py, field).offset == int(val), (cname, field)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2606_15035_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()
