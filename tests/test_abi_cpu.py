"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/ewh.h; argument validation works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_12344_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ewh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ewh_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ewh_create", "ewh_apply_S", "ewh_apply_Pi0", "ewh_solve", "ewh_destroy", "ewh_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2205_12344_gb300 import _lib
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, "binding lacks %s" % name


def test_exports_have_c_linkage(lib):
    path = lib._name
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in declared_symbols():
        assert name in exported, name


def _desc(**kw):
    from paper_2205_12344_gb300 import api
    args = dict(dim=2, n=[10, 10, 1], h=0.1, order=2, bc=[0] * 6)
    args.update(kw)
    return api.make_desc(**args)


def _call_create(lib, desc, rho, lam, mu, omega=3.0, nrhs=1):
    from paper_2205_12344_gb300 import _lib
    out = ctypes.c_void_p()
    s = lib.ewh_create(ctypes.byref(desc), _lib._ptr(rho), _lib._ptr(lam), _lib._ptr(mu), omega, None, nrhs,
                       None, ctypes.byref(out))
    return s, out


@pytest.mark.parametrize("kw,msg", [({"dim": 4}, "dim"), ({"order": 3}, "order"), ({"n": [3, 10, 1]}, "n[0]"),
                                    ({"order": 4, "n": [7, 10, 1]}, "n[0]"), ({"h": -1.0}, "h must"),
                                    ({"cfl": 1.5}, "cfl"), ({"periods": 0}, "periods"),
                                    ({"bc": [0, 0, 2, 0, 0, 0]}, "bc")])
def test_invalid_descriptor_rejected(lib, kw, msg):
    from paper_2205_12344_gb300 import _lib
    m = np.ones((10, 10))
    s, out = _call_create(lib, _desc(**kw), m, m, m)
    assert s == _lib.EWH_EINVAL
    assert not out.value
    assert msg in lib.ewh_last_error(None).decode()


@pytest.mark.parametrize("field,val", [("mu", -1.0), ("rho", 0.0), ("lam", np.nan), ("lam", -5.0)])
def test_invalid_medium_rejected(lib, field, val):
    from paper_2205_12344_gb300 import _lib
    arrs = {k: np.ones((10, 10)) for k in ("rho", "lam", "mu")}
    arrs[field][3, 4] = val
    s, out = _call_create(lib, _desc(), arrs["rho"], arrs["lam"], arrs["mu"])
    assert s == _lib.EWH_EINVAL
    assert "invalid medium" in lib.ewh_last_error(None).decode()


def test_invalid_omega_rejected(lib):
    from paper_2205_12344_gb300 import _lib
    m = np.ones((10, 10))
    for om in (0.0, -2.0, float("inf")):
        s, _ = _call_create(lib, _desc(), m, m, m, omega=om)
        assert s == _lib.EWH_EINVAL


def test_status_strings(lib):
    assert lib.ewh_status_string(0) == b"EWH_OK"
    assert lib.ewh_status_string(5) == b"EWH_EBREAKDOWN"


def _call_create_mapped(lib, desc, X, Y, m):
    from paper_2205_12344_gb300 import _lib
    out = ctypes.c_void_p()
    s = lib.ewh_create_mapped(ctypes.byref(desc), _lib._ptr(X), _lib._ptr(Y), _lib._ptr(m), _lib._ptr(m),
                              _lib._ptr(m), 3.0, None, 1, None, ctypes.byref(out))
    return s, out


@pytest.mark.parametrize("case,msg", [("no_x", "x and y"), ("order2", "dim 2 and order 4"),
                                      ("dim3", "dim 2 and order 4"), ("nan", "finite"), ("bad_desc", "h must")])
def test_mapped_create_validates_on_the_host(lib, case, msg):
    """ewh_create_mapped rejects missing or non-finite coordinates and grids
    other than 2D order 4 before touching the device."""
    from paper_2205_12344_gb300 import _lib
    n = [10, 12, 1]
    m = np.ones((12, 10))
    Q, R = np.meshgrid(np.arange(10) * 0.1, np.arange(12) * 0.1)
    kw = {"order": 4, "n": n}
    if case == "order2":
        kw["order"] = 2
    if case == "dim3":
        kw.update(dim=3, n=[10, 12, 9])
        m = np.ones((9, 12, 10))
        Q, R = np.ones((9, 12, 10)), np.ones((9, 12, 10))
    if case == "bad_desc":
        kw["h"] = -1.0
    if case == "nan":
        Q = Q.copy()
        Q[3, 4] = np.nan
    s, out = _call_create_mapped(lib, _desc(**kw), None if case == "no_x" else Q, R, m)
    assert s == _lib.EWH_EINVAL
    assert not out.value
    assert msg in lib.ewh_last_error(None).decode()


def test_mapped_create_without_device_reports_ecuda(lib):
    """Valid arguments on a machine without a CUDA device: the metric terms
    are computed on the device, so creation fails with EWH_ECUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2205_12344_gb300 import _lib
    m = np.ones((12, 10))
    Q, R = np.meshgrid(np.arange(10) * 0.1, np.arange(12) * 0.1)
    s, out = _call_create_mapped(lib, _desc(order=4, n=[10, 12, 1]), Q, R, m)
    assert s == _lib.EWH_ECUDA
    assert not out.value


def test_ctypes_structures_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of
    the header's C struct (compiled with the host compiler): a field added on
    one side only would shift the others silently."""
    import shutil
    import subprocess
    from paper_2205_12344_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"ewh_grid_desc": _lib.ewh_grid_desc, "ewh_problem_info": _lib.ewh_problem_info,
               "ewh_solve_info": _lib.ewh_solve_info, "ewh_stats": _lib.ewh_stats, "ewh_problem": _lib.ewh_problem}
    c_name = {"lambda_": "lambda"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ewh.h"', "int main(void) {"]
    for s, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in cls._fields_:
            cf = c_name.get(f, f)
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, cf))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for s, cls in structs.items():
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)
