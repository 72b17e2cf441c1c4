"""The C-ABI library loads on a CPU-only machine and exports every function
that include/pdhcg.h declares (no compute calls)."""
import ctypes
import os

import pytest


def test_library_exports_declared_symbols():
    import __graft_entry__ as g
    g.build()
    from paper_2506_06258_gb300 import capi
    lib = ctypes.CDLL(capi.LIB_PATH)
    names = capi.declared_symbols()
    assert len(names) >= 11
    missing = [s for s in names if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_and_defaults():
    from paper_2506_06258_gb300 import capi
    capi.load()
    assert capi.status_string(0) == "ok"
    p = capi.default_params()
    assert p.tol == 1e-6 and p.kkt_check_every == 64
    assert (p.beta_suff, p.beta_nec, p.beta_art, p.theta) == (0.2, 0.8, 0.2, 0.2)
    assert (p.eta_lo, p.eta_hi) == (0.01, 3.0) and p.omega_reset_every == 3
