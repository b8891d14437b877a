"""The C-ABI library builds, loads without a GPU, and exports every entry point
include/simnet.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2105_05821_b300 import build as B
from paper_2105_05821_b300 import simnet as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(simnet_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_exports_every_declared_symbol(libpath):
    decl = declared_functions()
    assert "simnet_simulate" in decl and "simnet_init" in decl
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (simnet_\w+)", out))
    missing = [d for d in decl if d not in exported]
    assert not missing, missing
    assert set(S.EXPORTS) <= exported


def test_loads_and_reports_version(libpath):
    L = ctypes.CDLL(libpath)
    assert L.simnet_abi_version() == 4


def test_sm103a_only(libpath):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath],
                         capture_output=True, text=True).stdout
    arches = set(re.findall(r"sm_(\d+a?)", out))
    assert arches == {"103a"}, arches


def test_init_without_device_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    L = S.lib()
    cfg = S._Config(32, 2, 64, 256, 8, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    assert L.simnet_init(ctypes.byref(cfg), ctypes.byref(h)) == 3      # ECUDA
    bad = S._Config(33, 2, 64, 256, 8, 0, 0, 0, 0)                       # W not divisible by 4
    assert L.simnet_init(ctypes.byref(bad), ctypes.byref(h)) == 1       # EINVAL
    L.simnet_destroy(None)
