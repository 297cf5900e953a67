"""The C ABI library loads and exports every entry point include/pf.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1407_8071_gb300 import pf, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^PF_API[^(;]*?\b(pf_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = declared()
    for core in ("pf_create", "pf_step", "pf_estimate", "pf_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    path = pf.lib()._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared() - exported
    assert not missing, missing
    # and nothing else leaks out of the library under a pf_ name
    assert {e for e in exported if e.startswith("pf_")} == declared()


def test_binding_covers_every_symbol():
    assert set(pf.declared_symbols()) == declared()
    L = pf.lib()
    for name in declared():
        assert isinstance(getattr(L, name), ctypes._CFuncPtr)


def test_build_targets_sm_103a_only():
    from paper_1407_8071_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_validates_before_touching_the_device():
    spec = W.lorenz63()
    s = pf._Structs(spec, seed=1)
    h = ctypes.c_void_p()
    N = (ctypes.c_int32 * 1)(0)
    st = pf.lib().pf_create(ctypes.byref(s.model), 1, N, spec.dt, ctypes.byref(s.obs), ctypes.byref(s.noise),
                            ctypes.byref(h))
    assert st == pf.PF_EINVAL and not h.value
    assert b"N[m]" in pf.lib().pf_last_error(None)
    bad = pf._Structs(W.lorenz63(), seed=1)
    bad.model.dx = 4
    N = (ctypes.c_int32 * 1)(16)
    st = pf.lib().pf_create(ctypes.byref(bad.model), 1, N, spec.dt, ctypes.byref(bad.obs), ctypes.byref(bad.noise),
                            ctypes.byref(h))
    assert st == pf.PF_EINVAL
    fhn = pf._Structs(W.fhn_lattice(J=7), seed=1)
    st = pf.lib().pf_create(ctypes.byref(fhn.model), 1, N, 0.05, ctypes.byref(fhn.obs), ctypes.byref(fhn.noise),
                            ctypes.byref(h))
    assert st == pf.PF_EINVAL  # odd lattice side
    assert pf.lib().pf_systematic_scratch_bytes(0, 10) == 0
    assert pf.lib().pf_systematic_scratch_bytes(3, 5000) > 5000 * 12
    pf.lib().pf_destroy(None)  # NULL-safe
