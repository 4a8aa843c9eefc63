"""The C ABI: the library builds for sm_103a, loads without a GPU, and exports every function include/mc.h
declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mc_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared("mc.h")
    for must in ["mc_create", "mc_create_batch", "mc_sweep", "mc_energy", "mc_gr_histogram", "mc_get_positions",
                 "mc_get_state", "mc_set_state", "mc_stats", "mc_destroy", "mc_last_error"]:
        assert must in names, must


def test_library_exports_every_declared_symbol():
    import paper_1602_05716_gb300 as pkg
    path = pkg.build()
    L = ctypes.CDLL(path)
    for header in sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")):
        for name in _declared(header):
            assert hasattr(L, name), f"{name} declared in {header} but not exported"


def test_option_constants_match_the_header():
    """Every MC_OPT_* value of include/mc.h is the binding's OPT_* constant of the same name."""
    import paper_1602_05716_gb300 as pkg
    src = open(os.path.join(ROOT, "include", "mc.h")).read()
    defs = dict(re.findall(r"^#define MC_(OPT_[A-Z0-9_]+)\s+(\d+)", src, flags=re.M))
    assert "OPT_SHARED_GUARD" in defs and len(defs) >= 13
    for name, value in defs.items():
        assert getattr(pkg, name) == int(value), name


def test_binding_loads_without_gpu():
    import paper_1602_05716_gb300 as pkg
    pkg.build()
    L = pkg.lib()
    assert L.mc_last_error() is not None


def test_record_capacity_is_kept_per_chain(monkeypatch):
    """The binding reads each chain's records and timeline with the capacity enabled for that chain (a fake
    library stands in for the C calls: nothing runs on a device)."""
    from paper_1602_05716_gb300 import api

    class _Fake:
        def __init__(self):
            self.read = []

        def mc_record_enable(self, h, chain, cap):
            return 0

        mc_trace_enable = mc_record_enable

        def mc_record_read(self, h, chain, out, cap):
            self.read.append((chain, cap))
            return 0

        mc_trace_read = mc_record_read

    fake = _Fake()
    monkeypatch.setattr(api, "lib", lambda: fake)
    s = api.System.__new__(api.System)
    s._h, s._rec_caps, s._trace_caps = None, {}, {}
    s.record_enable(4500, chain=0)
    s.record_enable(1920, chain=3)
    s.trace_enable(70, chain=1)
    s.records(0), s.records(3), s.records(2), s.trace(1)
    assert fake.read == [(0, 4500), (3, 1920), (2, 0), (1, 70)]


def test_reduction_run_refuses_an_unknown_scheme():
    """The scheme is checked with the description, before any device call."""
    import numpy as np
    from paper_1602_05716_gb300 import api
    api.build()
    p = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]], np.float32)
    q = np.array([1.0, -1.0], np.float32)
    d = api._Desc(p.ctypes.data, q.ctypes.data, 2, 1.0, 0.7, 5.0, 0.3, 1, 0)
    out = np.zeros_like(p)
    rc = api.lib().mc_reduction_run(ctypes.byref(d), 1, 2, out.ctypes.data, None, None, None)
    assert rc == api.ERR_INVALID


def test_binding_declares_every_abi_function():
    """The Python binding gives every function of include/mc.h a ctypes signature under the same name."""
    from paper_1602_05716_gb300 import api
    api.build()
    L = api.lib()
    for name in _declared("mc.h"):
        f = getattr(L, name)
        assert f.argtypes is not None, name
