"""The C ABI library loads and exports every function include/mithra.h declares, and the
Python struct layouts agree with the C compiler's (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "mithra.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(mithra_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_exports_every_declared_symbol():
    import paper_2009_13645_gb300 as m
    L = m.load()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", m._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mithra_\w+)", out))
    assert set(names) <= exported, set(names) - exported


def test_struct_layouts_match_c(tmp_path):
    import paper_2009_13645_gb300 as m
    c = tmp_path / "sz.c"
    c.write_text('#include "mithra.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                 'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mithra_grid),'
                 ' sizeof(mithra_undulator), sizeof(mithra_bunch), offsetof(mithra_grid, sort_every),'
                 ' offsetof(mithra_undulator, dist_to_bunch_head), offsetof(mithra_bunch, lab_particles),'
                 ' offsetof(mithra_grid, nf_points), offsetof(mithra_grid, bunch_every),'
                 ' offsetof(mithra_undulator, n_modules), offsetof(mithra_undulator, taper));'
                 'printf("%zu %zu\\n", offsetof(mithra_grid, optimize_position), offsetof(mithra_bunch, seed));'
                 'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    py = [ctypes.sizeof(m.Grid), ctypes.sizeof(m.Undulator), ctypes.sizeof(m.Bunch),
          m.Grid.sort_every.offset, m.Undulator.dist_to_bunch_head.offset, m.Bunch.lab_particles.offset,
          m.Grid.nf_points.offset, m.Grid.bunch_every.offset, m.Undulator.n_modules.offset,
          m.Undulator.taper.offset, m.Grid.optimize_position.offset, m.Bunch.seed.offset]
    assert vals == py


def test_last_error_and_kernel_names_without_gpu():
    import paper_2009_13645_gb300 as m
    L = m.load()
    assert L.mithra_version() == 1
    assert [L.mithra_kernel_name(k).decode() for k in range(len(m.KERNELS))] == list(m.KERNELS)
    # create rejects bad sizes before touching the device
    g = m.Grid(nx=3, ny=8, nz=8, dx=1e-3, dy=1e-3, dz=1e-3, solver=0, courant=1.0, mur_order=2,
               space_charge=1, precision=0, substeps=1, power_plane_dist=0.0, norm_freq=1.0)
    u = m.Undulator(kind=-1, K=0.0, lambda_=1e-3)
    b = m.Bunch(n=0, charge_e=0.0, gamma=1.0, sig_z=0.0)
    h = ctypes.c_void_p()
    rc = L.mithra_create(ctypes.byref(g), 0.0, ctypes.byref(u), ctypes.byref(b), ctypes.byref(h))
    assert rc == m.EINVAL and b">= 6 nodes" in L.mithra_last_error()
