"""The C-ABI library without a GPU: it builds, loads, exports every symbol the
header declares, and rejects malformed problems in host validation (which
runs before any device call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2301_05726_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_05726_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ucc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ucc_[a-z_]+)\s*\(", src)))


def test_header_and_exports(lib):
    from paper_2301_05726_gb300 import _lib
    names = declared_functions()
    assert names == sorted(_lib.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def _create(lib, prob, exc=None, theta=None):
    from paper_2301_05726_gb300._lib import Ansatz, Hamiltonian
    h = np.ascontiguousarray(prob.h)
    g = np.ascontiguousarray(prob.g)
    e = np.ascontiguousarray(prob.exc if exc is None else exc, dtype=np.int32).reshape(-1)
    t = np.ascontiguousarray(prob.theta if theta is None else theta)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ham = Hamiltonian(prob.n_spatial, prob.n_alpha, prob.n_beta, 0.0, dp(h), dp(g))
    an = Ansatz(len(e) // 4, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), dp(t))
    out = ctypes.c_void_p()
    st = lib.ucc_create(ctypes.byref(ham), ctypes.byref(an), None, ctypes.byref(out))
    return st, out, lib.ucc_last_error().decode()


@pytest.mark.parametrize("row,why", [
    ((0, 1, 4, 4), "repeated"),
    ((0, 2, 5, 7), "spin"),          # alpha alpha -> beta beta
    ((0, -1, 5, -1), "spin"),        # alpha -> beta single
    ((0, 1, 40, 41), "range"),
    ((0, -1, 4, 6), "malformed"),
])
def test_validation_rejects(lib, row, why):
    from paper_2301_05726_gb300._lib import UCC_EINVAL
    prob = synth.config_problem(1)
    exc = np.array([row], dtype=np.int32)
    st, out, msg = _create(lib, prob, exc=exc, theta=np.array([0.1]))
    assert st == UCC_EINVAL, msg
    assert why in msg or (why == "range" and "out of range" in msg)


def test_validation_rejects_nan_theta(lib):
    from paper_2301_05726_gb300._lib import UCC_EINVAL
    prob = synth.config_problem(1)
    th = prob.theta.copy()
    th[3] = np.nan
    st, _, msg = _create(lib, prob, theta=th)
    assert st == UCC_EINVAL and "theta" in msg


def test_validation_rejects_too_many_orbitals(lib):
    from paper_2301_05726_gb300._lib import UCC_EINVAL
    prob = synth.config_problem(1)
    import dataclasses
    # up to 64 spatial orbitals (two-word keys); 65 is refused before any device call
    big = dataclasses.replace(prob, n_spatial=65, h=np.zeros((65, 65)), g=np.zeros((65,) * 4))
    st, _, msg = _create(lib, big)
    assert st == UCC_EINVAL and "n_spatial" in msg


def test_static_energy_rejects_on_the_host(lib):
    """ucc_energy_static checks its sizes, counts and pointers before any
    device call: oversized and empty inputs and null outputs are refused with
    UCC_EINVAL and a message (the header's UCC_STATIC_MAX_DETS is the limit)."""
    from paper_2301_05726_gb300._lib import UCC_EINVAL
    src = open(os.path.join(ROOT, "include", "ucc.h")).read()
    cap = int(re.search(r"#define UCC_STATIC_MAX_DETS (\d+)", src).group(1))
    buf = np.zeros(8)
    p = ctypes.c_void_p(buf.ctypes.data)
    E, n2 = ctypes.c_double(), ctypes.c_double()

    def call(n_spatial=6, n_det=16, sigma=p, e_nuc=0.0):
        st = lib.ucc_energy_static(n_spatial, 2, 2, e_nuc, p, p, n_det, p, p, sigma, ctypes.byref(E),
                                   ctypes.byref(n2), None)
        return st, lib.ucc_last_error().decode()

    st, msg = call(n_det=cap + 1)
    assert st == UCC_EINVAL and str(cap) in msg
    st, msg = call(n_det=0)
    assert st == UCC_EINVAL and "n_det" in msg
    st, msg = call(n_spatial=33)
    assert st == UCC_EINVAL and "out of range" in msg
    st, msg = call(sigma=None)
    assert st == UCC_EINVAL and "null" in msg
    st, msg = call(e_nuc=float("nan"))
    assert st == UCC_EINVAL and "e_nuc" in msg


def test_no_cpu_fallback_in_binding():
    # The binding has no path that computes without the library.
    src = open(os.path.join(ROOT, "paper_2301_05726_gb300", "api.py")).read()
    assert "oracle" not in src
    assert "import oracle" not in open(os.path.join(ROOT, "paper_2301_05726_gb300", "_lib.py")).read()
