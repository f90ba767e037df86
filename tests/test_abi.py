"""The C-ABI library builds, loads and exports every entry point that
include/wf.h declares; argument errors are reported before any CUDA work
(these calls need no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(wf_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def wflib():
    from paper_1702_08852_gb300 import build
    build.build()
    from paper_1702_08852_gb300 import wf
    return wf


def test_header_lists_the_entry_points():
    names = declared_functions()
    for n in ("wf_plan", "wf_solve", "wf_residual", "wf_alm2map", "wf_map2alm",
              "wf_destroy", "wf_solve_host"):
        assert n in names


def test_every_declared_symbol_is_exported(wflib):
    L = ctypes.CDLL(wflib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing


def test_defaults_and_strings(wflib):
    o = wflib.wf_opts_default()
    assert o.beta == 0.75 and o.eps_final == 1e-6 and o.band_limit == 1
    assert wflib.wf_status_str(0) == "ok"
    assert "argument" in wflib.wf_status_str(1)
    L = wflib.lib()
    assert L.wf_npix(1024) == 12 * 1024 * 1024
    assert L.wf_nalm(2048) == 2049 * 2050 // 2


@pytest.mark.parametrize("nside,lmax,cl_bad", [(0, 4, False), (4, 12, False),
                                               (4, 0, False), (4, 8, True)])
def test_plan_rejects_bad_arguments_before_cuda(wflib, nside, lmax, cl_bad):
    L = wflib.lib()
    cl = np.ones(max(lmax, 1) + 1)
    if cl_bad:
        cl[3] = -1.0
    h = ctypes.c_void_p()
    o = wflib.wf_opts_default()
    st = L.wf_plan(ctypes.byref(h), nside, lmax, cl.ctypes.data_as(ctypes.c_void_p),
                   None, None, ctypes.byref(o), None)
    assert st == wflib.WF_ERR_ARG
    assert h.value is None
    assert wflib.wf_last_error()


def test_bad_options_rejected(wflib):
    L = wflib.lib()
    cl = np.ones(9)
    for field, val in (("beta", 1.0), ("beta", 0.0), ("eps_final", 0.0),
                       ("max_iter", 0), ("precision", 7), ("stop_rule", 3)):
        o = wflib.wf_opts_default(**{field: val})
        h = ctypes.c_void_p()
        st = L.wf_plan(ctypes.byref(h), 4, 8, cl.ctypes.data_as(ctypes.c_void_p),
                       None, None, ctypes.byref(o), None)
        assert st == wflib.WF_ERR_ARG, field


def test_null_plan_calls(wflib):
    L = wflib.lib()
    assert L.wf_solve(None, None, None, None, None, None, None) == wflib.WF_ERR_ARG
    assert L.wf_alm2map(None, None, None) == wflib.WF_ERR_ARG
    L.wf_destroy(None)


def _c_layout(tmp_path, structs):
    """sizeof and field offsets of the header's structs, from a C program
    compiled against include/wf.h (gcc, the host ABI the library uses)."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "wf.h"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    return got


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field
    offsets (a field added to one side only would shift every later field)."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1702_08852_gb300 import wf
    pairs = {"wf_opts": wf.wf_opts, "wf_stats": wf.wf_stats, "wf_tuning": wf._Tuning}
    structs = {c: [f for f, _ in py._fields_] for c, py in pairs.items()}
    got = _c_layout(tmp_path, structs)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_binding_checks_host_array_lengths():
    """Host arrays handed to the library by pointer are checked against the
    lengths it reads before any call (no plan, no GPU needed)."""
    from paper_1702_08852_gb300 import wf
    p = wf.Plan.__new__(wf.Plan)
    p.nside, p.lmax, p.npix, p.nalm, p.handle = 4, 8, wf.wf_npix(4), wf.wf_nalm(8), None
    with pytest.raises(ValueError):
        p.set_cl(np.ones(8))
    with pytest.raises(ValueError):
        p.solve_host(np.zeros(p.npix - 1))
    with pytest.raises(ValueError):
        wf.Plan(4, 8, np.ones(5))


def test_alu_peak_rejects_bad_arguments_before_cuda(wflib):
    import ctypes as C
    L = wflib.lib()
    t = C.c_double()
    assert L.wf_alu_peak(3, 1, C.byref(t), None, None) == wflib.WF_ERR_ARG
    assert L.wf_alu_peak(1, 0, C.byref(t), None, None) == wflib.WF_ERR_ARG
    assert L.wf_alu_peak(1, 1, None, None, None) == wflib.WF_ERR_ARG


def test_flat_plan_rejects_bad_sizes_before_cuda(wflib):
    import ctypes as C
    L = wflib.lib()
    h = C.c_void_p()
    ck = np.ones(100)
    dummy = C.c_void_p(8)  # never dereferenced: the size check comes first
    assert L.wf_flat_plan(C.byref(h), 10, 1e-6, ck.ctypes.data_as(C.c_void_p), dummy,
                          None, None) == wflib.WF_ERR_ARG
    assert L.wf_flat_plan(C.byref(h), 4096, 1e-6, ck.ctypes.data_as(C.c_void_p), dummy,
                          None, None) == wflib.WF_ERR_ARG
    assert L.wf_flat_plan(C.byref(h), 8, 0.0, ck.ctypes.data_as(C.c_void_p), dummy,
                          None, None) == wflib.WF_ERR_ARG
