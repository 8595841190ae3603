"""The C ABI without a GPU: exported symbols, struct layouts, status strings and the
argument checks md_create makes before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1107_2619_gb300 import build, inputs as I, md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md.h")


def header_functions():
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libmd():
    build.build()
    return md.lib()


def test_library_exports_every_declared_function(libmd):
    names = header_functions()
    assert len(names) >= 13
    raw = C.CDLL(md.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name
    assert set(names) == set(md.EXPORTS)


def test_struct_layouts_match_header(tmp_path, libmd):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "md.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(md_potential), sizeof(md_config), sizeof(md_energies),
         sizeof(md_profile), sizeof(md_surrogate), sizeof(md_passes));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(md_potential, tables), offsetof(md_config, stream),
         offsetof(md_energies, range_violations), offsetof(md_profile, ms_force), offsetof(md_surrogate, rd),
         offsetof(md_config, passes), offsetof(md_passes, active));
  printf("%zu\\n", offsetof(md_config, integrator));
  return 0;
}""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [C.sizeof(md.md_potential), C.sizeof(md.md_config), C.sizeof(md.md_energies),
            C.sizeof(md.md_profile), C.sizeof(md.md_surrogate), C.sizeof(md.md_passes), md.md_potential.tables.offset,
            md.md_config.stream.offset, md.md_energies.range_violations.offset, md.md_profile.ms_force.offset,
            md.md_surrogate.rd.offset, md.md_config.passes.offset, md.md_passes.active.offset,
            md.md_config.integrator.offset]
    assert got == want


def test_status_strings(libmd):
    assert libmd.md_abi_version() == 6
    assert md.status_string(md.MD_ERR_NBR_OVERFLOW) == "neighbour list overflow"
    assert md.status_string(md.MD_ERR_SPECIES) == "unsupported species"


def _create(w, **kw):
    cfg = md.make_config(w.n_atoms, kw.pop("box", w.box), w.skin, kw.pop("k_max", w.k_max), w.dt_fs)
    for k, v in kw.items():
        setattr(cfg, k, v)
    pot, keep = md.make_potential(w.potential)
    return cfg, pot, keep


@pytest.mark.parametrize("case,status", [("shear", md.MD_ERR_BOX), ("small", md.MD_ERR_BOX),
                                         ("species", md.MD_ERR_SPECIES), ("kmax", md.MD_ERR_ARG),
                                         ("nan", md.MD_ERR_NONFINITE), ("prec", md.MD_ERR_ARG)])
def test_create_rejects_bad_input_before_the_device(libmd, case, status):
    w = I.bcc_fe(4 if case == "small" else 8, seed=3)
    cfg, pot, keep = _create(w)
    pos, spc = w.pos.copy(), w.species.copy()
    if case == "shear":
        cfg.h[1] = 0.5
    if case == "species":
        spc[5] = 3
    if case == "kmax":
        cfg.k_max = 0
    if case == "nan":
        pos[7, 1] = np.nan
    if case == "prec":
        cfg.precision = 7
    out = C.c_void_p()
    st = libmd.md_create(C.byref(cfg), C.byref(pot), C.c_void_p(pos.ctypes.data), C.c_void_p(w.vel.ctypes.data),
                         C.c_void_p(spc.ctypes.data), 0, C.byref(out))
    assert st == status
    assert not out.value
