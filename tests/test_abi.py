"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/reg.h declares (no compute call is made here)."""
import ctypes
import os
import re

from paper_1408_6299_gb300 import build, lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^REG_API\s+[\w\s\*]+?\b(reg_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_api():
    names = declared_symbols()
    for must in ("reg_create", "reg_objective", "reg_gradient", "reg_hessvec", "reg_solve", "reg_precond"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    L = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert set(lib.EXPORTED) <= declared_symbols()


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    with_err = None
    try:
        lib.Registration((16, 16), 4)
    except lib.RegError as e:
        with_err = e
    assert with_err is not None and with_err.status in (lib.REG_ECUDA, lib.REG_ENOMEM)


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of the header's structs: same size and field offsets
    import subprocess
    structs = {"reg_solve_opts": lib.SolveOpts, "reg_solve_report": lib.SolveReport, "reg_problem": lib.ProblemC,
               "reg_cont_opts": lib.ContOpts, "reg_cont_report": lib.ContReport}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "reg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, f, val = line.split()
            got[(cname, f)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_solve_option_defaults_and_unknown_names():
    L = lib.load()
    o = lib.SolveOpts.make(L, {"grad_rtol": 1e-3, "method": lib.REG_METHOD_PICARD})
    assert o.grad_rtol == 1e-3 and o.method == lib.REG_METHOD_PICARD
    assert o.max_outer == 50 and o.step_memory == 1 and o.stop_rule == lib.REG_STOP_GRAD_REL and o.tau_J == 1e-3
    import pytest
    with pytest.raises(TypeError):
        lib.SolveOpts.make(L, {"grad_rtoll": 1e-3})
    c = lib.ContOpts()
    L.reg_cont_opts_default(ctypes.byref(c))
    assert (c.beta0, c.beta_min, c.eps_F, c.beta_rtol, c.dist_rtol, c.max_solves) == (1.0, 1e-6, 0.1, 0.05, 1e-2, 50)
