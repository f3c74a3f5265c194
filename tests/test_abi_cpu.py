"""CPU-only checks of the C-ABI library: it loads, exports every declared
symbol, and its host-side logic (reference element, transfer operators,
argument and mesh validation) agrees with the oracle. No GPU call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

from dg_inputs import jittered_grid
from oracle import refops

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    build.build()
    return P


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(P):
    L = P.lib()
    names = _declared()
    assert "dg_poisson_apply" in names and "dg_pcg_solve" in names
    for n in sorted(names):
        assert hasattr(L, n), n


@pytest.mark.parametrize("N", range(1, 11))
def test_library_reference_element_matches_oracle(P, N):
    a = P.reference_operators(N)
    o = refops.reference_operators(N)
    assert np.abs(a["r"] - o["r"]).max() < 1e-14 and np.abs(a["s"] - o["s"]).max() < 1e-14
    for k in ("M", "Dr", "Ds", "Mf"):
        assert np.abs(a[k] - o[k]).max() < 1e-12 * max(1.0, np.abs(o[k]).max()), k
    assert (a["fmask"] == np.array(o["faces"])).all()


@pytest.mark.parametrize("Nf,Nc", [(8, 4), (4, 2), (2, 1), (6, 3), (3, 1), (8, 1), (10, 5), (9, 4)])
def test_library_interpolation_matches_oracle(P, Nf, Nc):
    assert np.abs(P.interpolation_matrix(Nf, Nc) - refops.interpolation(Nf, Nc)).max() < 1e-12


def test_status_strings_and_argument_errors(P):
    L = P.lib()
    assert L.dg_status_string(0) == b"ok"
    assert L.dg_status_string(4) == b"not converged"
    m = jittered_grid(2, 2)
    with pytest.raises(P.DgError) as ei:
        P.Mesh(0, m.VX, m.VY, m.EToV, m.bc)
    assert ei.value.name == "DG_ERR_ARG"
    with pytest.raises(P.DgError) as ei:
        P.Mesh(11, m.VX, m.VY, m.EToV, m.bc)
    assert ei.value.name == "DG_ERR_ARG"


def test_mesh_validation_rejects_bad_meshes_before_any_device_work(P):
    m = jittered_grid(2, 2)
    cw = m.EToV[:, ::-1].copy()          # clockwise elements
    with pytest.raises(P.DgError) as ei:
        P.Mesh(2, m.VX, m.VY, cw, m.bc)
    assert ei.value.name == "DG_ERR_MESH"
    bad = m.bc.copy()
    bad[m.bc == 0] = 1                    # interior face tagged Dirichlet
    with pytest.raises(P.DgError) as ei:
        P.Mesh(2, m.VX, m.VY, m.EToV, bad)
    assert ei.value.name == "DG_ERR_MESH"
    bad = m.bc.copy()
    bad[m.bc != 0] = 0                    # boundary face without a tag
    with pytest.raises(P.DgError) as ei:
        P.Mesh(2, m.VX, m.VY, m.EToV, bad)
    assert ei.value.name == "DG_ERR_MESH"
    e = m.EToV.copy()
    e[0, 0] = 999                          # vertex index out of range
    with pytest.raises(P.DgError) as ei:
        P.Mesh(2, m.VX, m.VY, e, m.bc)
    assert ei.value.name == "DG_ERR_ARG"


def test_tet_mesh_validation_rejects_before_any_device_work(P):
    from dg_inputs.tetmesh import jittered_tet_grid
    m = jittered_tet_grid(1)
    for N in (0, 6):                       # tetrahedral degrees are 1..5
        with pytest.raises(P.DgError) as ei:
            P.TetMesh.from_inputs(m, N)
        assert ei.value.name == "DG_ERR_ARG"
    e = m.EToV.copy()
    e[0, 0] = 999
    with pytest.raises(P.DgError) as ei:
        P.TetMesh(2, m.VX, m.VY, m.VZ, e, m.bc)
    assert ei.value.name == "DG_ERR_MESH"
    e = m.EToV.copy()
    e[0, [1, 2]] = e[0, [2, 1]]            # negative Jacobian
    with pytest.raises(P.DgError) as ei:
        P.TetMesh(2, m.VX, m.VY, m.VZ, e, m.bc)
    assert ei.value.name == "DG_ERR_MESH"
    bad = m.bc.copy()
    bad[m.bc != 0] = 0                     # boundary face without a tag
    with pytest.raises(P.DgError) as ei:
        P.TetMesh(2, m.VX, m.VY, m.VZ, m.EToV, bad)
    assert ei.value.name == "DG_ERR_MESH"


C_CONSUMER = r"""
#include <stdio.h>
#include "dg.h"
int main(void) {
  double r[45], s[45];
  int32_t fmask[27];
  dg_solver_opts o;
  dg_status st = dg_reference_operators(8, r, s, NULL, NULL, NULL, NULL, fmask);
  dg_solver_opts_default(&o);
  printf("%d %.17g %.17g %g %d %s\n", (int)st, r[0], s[44], o.tol, o.max_iter,
         dg_status_string(DG_ERR_BREAKDOWN));
  return st != DG_OK;
}
"""


def test_header_is_c_and_a_c_program_links_and_runs(P, tmp_path):
    """include/dg.h is plain C (C99, -pedantic, no warnings) and a C program
    links against the library and calls its host-side entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "consumer.c"
    src.write_text(C_CONSUMER)
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(P.lib_path())
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L" + libdir, "-ldg_gb300", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    st, r0, s_last, tol, max_iter, name = out.stdout.split(None, 5)
    assert st == "0" and float(r0) == -1.0 and float(s_last) == 1.0   # vertices v0 and v2 of the reference triangle
    assert float(tol) == 1e-10 and int(max_iter) == 1000 and name.strip()


def test_new_entry_points_reject_bad_arguments_before_device_work(P):
    """dg_apply_host and the tetrahedral calls check their arguments on the host:
    a NULL mesh or pointer is DG_ERR_ARG with no device call."""
    import ctypes
    L = P.lib()
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert L.dg_apply_host(None, 0, P.DG_F64, 1, 0.0, p, p, None) == 1
    assert L.dg_tet_apply(None, P.DG_F64, 1, 0.0, p, p, None) == 1
    assert L.dg_tet_rhs(None, 1, p, p, p, None) == 1
    assert L.dg_tet_pcg_jacobi_solve(None, 1, 0.0, 1e-10, 10, p, p, None, None) == 1
    assert L.dg_tet_mesh_info(None, None, None, None) == 1
    assert L.dg_tet_mesh_destroy(None) == 0
    out = ctypes.c_void_p()
    VX = (ctypes.c_double * 4)(0, 1, 0, 0)
    VY = (ctypes.c_double * 4)(0, 0, 1, 0)
    VZ = (ctypes.c_double * 4)(0, 0, 0, 1)
    E = (ctypes.c_int32 * 4)(0, 1, 2, 3)
    bc = (ctypes.c_int8 * 4)(1, 1, 1, 1)
    assert L.dg_tet_mesh_setup(6, 4, VX, VY, VZ, 1, E, bc, None, ctypes.byref(out)) == 1   # degree 6
    assert L.dg_tet_mesh_setup(2, 4, VX, VY, VZ, 1, E, None, None, ctypes.byref(out)) == 1  # NULL tags
    assert not out.value
