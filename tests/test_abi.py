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
