"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and rejects invalid input on the host before touching a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2609_00535_b300 import inputs, semlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header="sem_lbm.h", prefix="sem_lbm_"):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"\b(%s\w+)\s*\(" % prefix, txt))


def test_every_header_is_covered():
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == \
        ["sem_lbm.h", "semlbm_peak.h"]


def test_peak_library_exports_its_symbol():
    lib = ctypes.CDLL(semlbm.PEAK_PATH)
    names = declared_symbols("semlbm_peak.h", "semlbm_")
    assert names == {"semlbm_fp64_peak"}
    for n in names:
        assert hasattr(lib, n)


def test_library_exports_every_declared_symbol():
    lib = semlbm.load()
    names = declared_symbols()
    assert {"sem_lbm_create", "sem_lbm_step", "sem_lbm_diagnostics"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(semlbm.EXPORTED) <= names


def _create(mesh, N, lattice, theta_tag=(), beta=1e-3, kappa=1e-6, tau=0.5):
    lib = semlbm.load()
    m, keep = semlbm.mesh_struct(mesh)
    tags = np.asarray(theta_tag, dtype=np.float64)
    p = semlbm.ParamsC(1.0, 0.1, 0.01, 0.0, 0.0, len(tags), tags.ctypes.data if len(tags) else None,
                       None, None, 0)
    h = ctypes.c_void_p()
    rc = lib.sem_lbm_create(ctypes.byref(m), N, lattice, beta, kappa, tau, math.pi / 3,
                            ctypes.byref(p), ctypes.byref(h))
    return rc, lib.sem_lbm_last_error().decode()


def test_host_validation_errors():
    m2 = inputs.box((2, 2), (0, 0), (1, 1), 4, face_tags={2: 0})
    m3 = inputs.box((1, 1, 1), (0, 0, 0), (1, 1, 1), 3)
    rc, msg = _create(m2, 4, semlbm.D3Q13)
    assert rc == -1 and "lattice" in msg
    rc, msg = _create(m2, 17, semlbm.D2Q9)
    assert rc == -6
    rc, msg = _create(m3, 9, semlbm.D3Q13)
    assert rc == -6
    rc, msg = _create(m2, 4, semlbm.D2Q9, beta=-1.0)
    assert rc == -1
    bad = inputs.box((2, 2), (0, 0), (1, 1), 4, face_tags={2: 3})   # tag 3 has no angle
    rc, msg = _create(bad, 4, semlbm.D2Q9, theta_tag=(1.0,))
    assert rc == -1 and "tag 3" in msg
    fk = inputs.box((2, 2), (0, 0), (1, 1), 4)
    fk.face_kind[0, 0] = 7
    rc, msg = _create(fk, 4, semlbm.D2Q9)
    assert rc == -1 and "face_kind" in msg


def test_null_arguments_are_rejected_on_the_host():
    """Entry points given a NULL solver or buffer return SEMLBM_EINVAL (-1) and a
    message before touching a device."""
    import ctypes
    L = semlbm.load()
    buf = (ctypes.c_double * 4)()
    step = ctypes.c_int64()
    ids = (ctypes.c_int64 * 4)()
    assert L.sem_lbm_get_state_global(None, buf, 0, ctypes.byref(step)) == -1
    assert L.sem_lbm_set_state_global(None, buf, 0, 0) == -1
    assert L.sem_lbm_get_global_nodes(None, ids) == -1
    assert L.sem_lbm_get_state(None, buf, 0, ctypes.byref(step)) == -1
    assert L.sem_lbm_set_state(None, buf, 0, 0) == -1
    assert L.sem_lbm_step(None, 1) == -1
    assert b"NULL" in L.sem_lbm_last_error()


def test_workspace_bytes_is_host_only_and_scales():
    b1 = semlbm.workspace_bytes(inputs.box((2, 2), (0, 0), (1, 1), 4), 4, "D2Q9")
    b2 = semlbm.workspace_bytes(inputs.box((4, 4), (0, 0), (1, 1), 4), 4, "D2Q9")
    assert 0 < b1 < b2
    # 4 state copies of Q*V doubles dominate
    V = 16 * 25
    assert b2 > 4 * 9 * V * 8
    assert semlbm.workspace_bytes(inputs.box((2, 2), (0, 0), (1, 1), 4), 4, "D3Q13") == 0


STRUCTS = [("sem_lbm_mesh", semlbm.MeshC), ("sem_lbm_params", semlbm.ParamsC),
           ("sem_lbm_diag", semlbm.DiagC), ("sem_lbm_profile_t", semlbm.ProfileC),
           ("sem_lbm_info_t", semlbm.InfoC), ("sem_lbm_batch_group_info", semlbm.GroupInfoC),
           ("sem_lbm_wetting", semlbm.WettingC)]


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler gives
    the header's struct (guards the binding when the ABI grows)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sem_lbm.h"', 'int main(void) {']
    for cname, py in STRUCTS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, py in STRUCTS:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
