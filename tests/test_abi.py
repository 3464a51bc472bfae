"""The C-ABI library builds, loads and exports every function include/bem.h
declares; argument errors come back as status codes (no GPU needed)."""
import ctypes

import pytest

from paper_2003_12663_gb300 import bem, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return bem.lib()


def test_every_header_symbol_is_exported(L):
    names = bem.header_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(bem._SIGS), set(names) ^ set(bem._SIGS)


def test_default_params(L):
    p = bem.default_params()
    assert p.eta == 4.0 and p.far_order == 3 and p.gmres_restart == 100


def test_argument_errors_without_device(L):
    h = ctypes.c_void_p()
    assert L.bem_create(None, None, None, None) == -1
    assert L.bem_create(ctypes.byref(h), None, None, None) == -1
    assert b"NULL" in L.bem_last_error(None)
    m = bem.bem_mesh()
    m.nv, m.np = 3, 1
    assert L.bem_create(ctypes.byref(h), ctypes.byref(m), None, None) == -1
    assert not h.value
    # calls on a NULL context are argument errors
    assert L.bem_matvec(None, 0, 1, None, None) == -1
    assert L.bem_solve(None, 0, 1, None, None, 1e-8, None, None) == -1
    assert L.bem_eval_field(None, 0, None, 0, None, None, None) == -1
    assert L.bem_destroy(None) == 0


def test_bad_mesh_rejected_before_device(L):
    import numpy as np
    X = np.zeros((3, 3))
    tri = np.array([[0, 1, 5]], np.int32)
    reg = np.zeros(1, np.int32)
    regs = (bem.bem_region * 1)()
    m = bem.bem_mesh(3, 1, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     reg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1, regs)
    h = ctypes.c_void_p()
    assert L.bem_create(ctypes.byref(h), ctypes.byref(m), None, None) == -1
    assert b"out of range" in L.bem_last_error(None)
    p = bem.default_params(eta=0.5)
    tri[0, 2] = 2
    assert L.bem_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(p), None) == -1
    assert b"eta" in L.bem_last_error(None)


def test_region_kinds_match_header():
    """The binding's region kinds are the header's enum values."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(build.__file__), "..", "include", "bem.h")).read()
    vals = dict((k, int(v)) for k, v in re.findall(r"BEM_(CONDUCTOR|FLOATING|DIELECTRIC|SHEET) = (\d+)", hdr))
    assert vals == {"CONDUCTOR": bem.CONDUCTOR, "FLOATING": bem.FLOATING,
                    "DIELECTRIC": bem.DIELECTRIC, "SHEET": bem.SHEET}
    assert bem._KIND["sheet"] == bem.SHEET


def test_bad_regions_rejected_before_device(L):
    """Region descriptors are checked before any device work: an unknown kind, a
    sheet with eps- < 0 or a floating id out of range, and a floating id that no
    triangle carries."""
    import numpy as np
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    tri = np.array([[0, 1, 2], [0, 1, 3]], np.int32)
    reg = np.array([0, 1], np.int32)

    def create(r1, r0=None):
        regs = (bem.bem_region * 2)()
        regs[0].kind, regs[0].V0 = bem.CONDUCTOR, 1.0
        if r0:
            for k, v in r0.items():
                setattr(regs[0], k, v)
        for k, v in r1.items():
            setattr(regs[1], k, v)
        m = bem.bem_mesh(4, 2, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         reg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 2, regs)
        h = ctypes.c_void_p()
        rc = L.bem_create(ctypes.byref(h), ctypes.byref(m), None, None)
        assert not h.value
        return rc, L.bem_last_error(None)

    rc, msg = create({"kind": 4})
    assert rc == -1 and b"unknown kind" in msg
    rc, msg = create({"kind": bem.SHEET, "floating_id": 0, "eps_plus": 1.0, "eps_minus": -1.0})
    assert rc == -1 and b"eps_minus" in msg
    rc, msg = create({"kind": bem.SHEET, "floating_id": 7, "eps_plus": 1.0, "eps_minus": 1.0})
    assert rc == -1 and b"floating_id" in msg
    rc, msg = create({"kind": bem.SHEET, "floating_id": 0, "eps_plus": 0.0, "eps_minus": 1.0})
    assert rc == -1 and b"eps_plus" in msg
    # floating id 1 is used by a region that no triangle carries, id 0 by none at all
    rc, msg = create({"kind": bem.CONDUCTOR, "V0": 0.0},
                     {"kind": bem.SHEET, "floating_id": 1, "eps_plus": 1.0, "eps_minus": 1.0})
    assert rc == -1 and b"no triangles" in msg


STRUCTS = ["bem_region", "bem_mesh", "bem_params", "bem_trace_params", "bem_counters", "bem_tuning",
           "bem_p1_params", "bem_batch_counters"]


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and field
    offsets (a stale mirror would pass arguments at the wrong offsets)."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bem.h"', 'int main(void) {']
    for name in STRUCTS:
        cls = getattr(bem, name)
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in STRUCTS:
        cls = getattr(bem, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_new_defaults(L):
    p = bem.default_params()
    assert p.residual == bem.RESIDUAL_DF_UPDATE      # one double-FP32 residual per solve
    assert p.trace_cluster == 0 and p.far32_variant == 0
    assert p.adjoint_checkpoint == 128 and p.adjoint_lines == 256
