"""CPU oracle for the sparse UCC path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library in
``paper_2301_05726_gb300``; the two meet only through the seeded inputs of
``paper_2301_05726_gb300.synth`` (which holds none of the method's
arithmetic).

``ucc_oracle.cpp`` is the sparse reference (Eq. 3 factor by factor on a
``std::unordered_map``, Slater-Condon energy, checkpointed adjoint), built
with 64-bit and with 128-bit determinant keys;
``dense.py`` is an independent state-vector brute force used to pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucc_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libucc_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no fused multiply-add contraction): the same
    source twice, with 64-bit keys (entry points orc_*) and with 128-bit keys
    (orc128_*), linked into one library."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        objs = []
        for bits in (64, 128):
            obj = f"{tmp}.{bits}.o"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-c",
                                   f"-DORC_KEY_BITS={bits}", "-o", obj, _SRC])
            objs.append(obj)
        subprocess.check_call(["g++", "-shared", "-o", tmp] + objs)
        for obj in objs:
            os.remove(obj)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Counts(ctypes.Structure):
    _fields_ = [("rotations", ctypes.c_longlong), ("created", ctypes.c_longlong),
                ("dropped_new", ctypes.c_longlong), ("dropped_old", ctypes.c_longlong),
                ("cut", ctypes.c_longlong)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, dp, ip, u64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), \
            ctypes.POINTER(ctypes.c_uint64)
        lib.orc_problem_new.restype = vp
        lib.orc_problem_new.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ip]
        lib.orc_problem_free.argtypes = [vp]
        lib.orc_apply.restype = vp
        lib.orc_apply.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong,
                                  ctypes.POINTER(_Counts), dp]
        lib.orc_wf_from_arrays.restype = vp
        lib.orc_wf_from_arrays.argtypes = [ctypes.c_longlong, u64p, dp]
        lib.orc_wf_size.restype = ctypes.c_longlong
        lib.orc_wf_size.argtypes = [vp]
        lib.orc_wf_export.argtypes = [vp, u64p, dp]
        lib.orc_wf_free.argtypes = [vp]
        lib.orc_sigma.argtypes = [vp, vp, ctypes.c_int, dp]
        lib.orc_energy.argtypes = [vp, vp, ctypes.c_int, dp, dp]
        lib.orc_sigma_at.argtypes = [vp, vp, ctypes.c_longlong, u64p, dp]
        lib.orc_hmat.restype = ctypes.c_double
        lib.orc_hmat.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_tau.restype = ctypes.c_int
        lib.orc_tau.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, u64p]
        lib.orc_gradient.argtypes = [vp, dp, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int,
                                     dp, dp]
        # the 128-bit build: the same calls, keys as (low, high) pairs of words
        for name in ("problem_new", "problem_free", "apply", "wf_from_arrays", "wf_size", "wf_export", "wf_free",
                     "sigma", "energy", "sigma_at", "gradient"):
            f64, f128 = getattr(lib, "orc_" + name), getattr(lib, "orc128_" + name)
            f128.restype, f128.argtypes = f64.restype, f64.argtypes
        lib.orc128_hmat.restype = ctypes.c_double
        lib.orc128_hmat.argtypes = [vp, u64p, u64p]
        lib.orc128_tau.restype = ctypes.c_int
        lib.orc128_tau.argtypes = [vp, ctypes.c_int, ctypes.c_int, u64p, u64p]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One problem loaded into the oracle (integrals + factor list).

    key_bits: 64 (keys are uint64 arrays) or 128 (keys are (n, 2) uint64
    arrays of (low, high) words; needed above 64 spin-orbitals).  By default
    the smallest that holds the problem's spin-orbitals."""

    def __init__(self, prob, key_bits=None):
        self.lib = _load()
        self.prob = prob
        n_so = 2 * int(prob.n_spatial)
        if key_bits is None:
            key_bits = 64 if n_so <= 64 else 128
        if key_bits not in (64, 128) or n_so > key_bits:
            raise ValueError(f"{n_so} spin-orbitals do not fit {key_bits}-bit keys")
        self.key_bits = key_bits
        self._p = "orc_" if key_bits == 64 else "orc128_"
        self._h = np.ascontiguousarray(prob.h, dtype=np.float64)
        self._g = np.ascontiguousarray(prob.g, dtype=np.float64)
        self._exc = np.ascontiguousarray(prob.exc, dtype=np.int32)
        self.handle = self._f("problem_new")(
            prob.n_spatial, prob.n_alpha, prob.n_beta, _dp(self._h), _dp(self._g), int(self._exc.shape[0]),
            self._exc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))

    def _f(self, name):
        return getattr(self.lib, self._p + name)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self._f("problem_free")(h)
            self.handle = None

    def _theta(self, theta):
        t = self.prob.theta if theta is None else theta
        return np.ascontiguousarray(t, dtype=np.float64)

    def _cut(self, n_max, n_cut):
        if n_max is None:
            return int(getattr(self.prob, "n_max", 0)), int(getattr(self.prob, "n_cut", 0))
        return int(n_max), int(n_cut or 0)

    def apply(self, theta=None, eps=None, n_factors=None, n_max=None, n_cut=None):
        """Eq. 3 on the reference with the eps rule (and the problem's N_MAX/N_CUT
        cut unless given).  Returns (keys, amps, counts) sorted by key; counts has
        rotations/created/dropped_new/dropped_old/cut."""
        th = self._theta(theta)
        eps = self.prob.eps if eps is None else eps
        n_max, n_cut = self._cut(n_max, n_cut)
        nf = len(th) if n_factors is None else int(n_factors)
        cnt = _Counts()
        wf = self._f("apply")(self.handle, _dp(th), nf, float(eps), int(n_max), int(n_cut), ctypes.byref(cnt),
                                None)
        keys, amps = self._export(wf)
        self._f("wf_free")(wf)
        counts = {f: getattr(cnt, f) for f, _ in _Counts._fields_}
        return keys, amps, counts

    def entropy_per_factor(self, theta=None, eps=None, n_factors=None, n_max=None, n_cut=None):
        """Eq. 6 after each factor (array of n_factors)."""
        th = self._theta(theta)
        eps = self.prob.eps if eps is None else eps
        n_max, n_cut = self._cut(n_max, n_cut)
        nf = len(th) if n_factors is None else int(n_factors)
        out = np.zeros(nf)
        cnt = _Counts()
        wf = self._f("apply")(self.handle, _dp(th), nf, float(eps), int(n_max), int(n_cut), ctypes.byref(cnt),
                                _dp(out))
        self._f("wf_free")(wf)
        return out

    def _keys(self, keys):
        k = np.ascontiguousarray(keys, dtype=np.uint64)
        if self.key_bits == 128 and (k.ndim != 2 or k.shape[1] != 2):
            raise ValueError("128-bit keys are (n, 2) arrays of (low, high) words")
        return k

    def _export(self, wf):
        n = self._f("wf_size")(wf)
        keys = np.zeros((n,) if self.key_bits == 64 else (n, 2), dtype=np.uint64)
        amps = np.zeros(n, dtype=np.float64)
        if n:
            self._f("wf_export")(wf, keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(amps))
        return keys, amps

    def _wf(self, keys, amps):
        keys = self._keys(keys)
        amps = np.ascontiguousarray(amps, dtype=np.float64)
        return self._f("wf_from_arrays")(len(keys), keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                         _dp(amps))

    def energy(self, keys, amps, route="lookup"):
        """(E, <psi|psi>) of the map keys -> amps; route 'lookup' or 'pairwise'."""
        wf = self._wf(keys, amps)
        E, n2 = ctypes.c_double(), ctypes.c_double()
        self._f("energy")(self.handle, wf, 1 if route == "pairwise" else 0, ctypes.byref(E), ctypes.byref(n2))
        self._f("wf_free")(wf)
        return E.value, n2.value

    def sigma(self, keys, amps, route="lookup"):
        """sigma_I = sum_J <I|H|J> c_J over the map, in sorted-key order."""
        wf = self._wf(keys, amps)
        n = self._f("wf_size")(wf)
        sk, _ = self._export(wf)
        out = np.zeros(n)
        self._f("sigma")(self.handle, wf, 1 if route == "pairwise" else 0, _dp(out))
        self._f("wf_free")(wf)
        return sk, out

    def sigma_at(self, keys, amps, query):
        """sigma at the given determinants only (one by one)."""
        wf = self._wf(keys, amps)
        q = self._keys(query)
        out = np.zeros(len(q))
        self._f("sigma_at")(self.handle, wf, len(q), q.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(out))
        self._f("wf_free")(wf)
        return out

    def hmat(self, I, J):
        """<J|H|I> for determinants given as Python integers."""
        if self.key_bits == 64:
            return self.lib.orc_hmat(self.handle, int(I), int(J))
        a, b = words(int(I)), words(int(J))
        return self.lib.orc128_hmat(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                    b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))

    def tau(self, k, det, dagger=False):
        """(sign, tau_k |det>) or (0, None), determinants as Python integers."""
        if self.key_bits == 64:
            out = ctypes.c_uint64()
            s = self.lib.orc_tau(self.handle, int(k), 1 if dagger else 0, int(det), ctypes.byref(out))
            return (s, out.value) if s else (0, None)
        d, out = words(int(det)), np.zeros(2, dtype=np.uint64)
        s = self.lib.orc128_tau(self.handle, int(k), 1 if dagger else 0,
                                d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        return (s, int(out[0]) | (int(out[1]) << 64)) if s else (0, None)

    def run_energy(self, theta=None, eps=None, n_factors=None, n_max=None, n_cut=None):
        keys, amps, _ = self.apply(theta, eps, n_factors, n_max, n_cut)
        return self.energy(keys, amps)[0]

    def gradient(self, theta=None, eps=None, stride=0, n_max=None, n_cut=None):
        """(E, dE/dtheta) by the checkpointed adjoint sweep (stride 0 = ceil(sqrt K))."""
        th = self._theta(theta)
        eps = self.prob.eps if eps is None else eps
        n_max, n_cut = self._cut(n_max, n_cut)
        g = np.zeros(len(th))
        E = ctypes.c_double()
        self._f("gradient")(self.handle, _dp(th), float(eps), int(n_max), int(n_cut), int(stride),
                              ctypes.byref(E), _dp(g))
        return E.value, g


def words(key: int) -> np.ndarray:
    """A determinant key as its (low, high) 64-bit words."""
    return np.array([key & 0xFFFFFFFFFFFFFFFF, key >> 64], dtype=np.uint64)


def key_ints(keys) -> list:
    """Keys (a uint64 array, or an (n, 2) array of (low, high) words) as Python integers."""
    k = np.asarray(keys, dtype=np.uint64)
    if k.ndim == 1:
        return [int(x) for x in k]
    return [int(lo) | (int(hi) << 64) for lo, hi in k]
