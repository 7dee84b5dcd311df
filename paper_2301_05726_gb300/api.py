"""Python face of libucc.so: one context per problem, plus a torch autograd op.

Every step of the path (apply, energy, adjoint) runs in the library's CUDA
kernels; this module only marshals arguments.  PyTorch supplies the CUDA
stream (``torch.cuda.current_stream()``) and, for device-side results, the
output tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import Ansatz, Hamiltonian, Options, Stats, check


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _current_stream():
    try:
        import torch
    except ImportError:  # pragma: no cover
        return None
    if not torch.cuda.is_available():
        raise RuntimeError("libucc needs a CUDA device")
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class UCCContext:
    """A problem (integrals + factor list + theta) resident on the GPU.

    ``prob`` is a ``synth.Problem`` or anything with the same attributes
    (n_spatial, n_alpha, n_beta, h, g, exc, theta, e_nuc).
    """

    def __init__(self, prob, stream=None, probe_width: int = 0, max_entries: int = 0):
        self.lib = _lib.load()
        self.prob = prob
        self.K = int(prob.exc.shape[0])
        self.key_words = 2 if 2 * int(prob.n_spatial) > 64 else 1  # uint64 words per determinant key
        self._h = np.ascontiguousarray(prob.h, dtype=np.float64)
        self._g = np.ascontiguousarray(prob.g, dtype=np.float64)
        self._exc = np.ascontiguousarray(prob.exc, dtype=np.int32).reshape(-1)
        self._theta = np.ascontiguousarray(prob.theta, dtype=np.float64)
        ham = Hamiltonian(prob.n_spatial, prob.n_alpha, prob.n_beta, float(getattr(prob, "e_nuc", 0.0)),
                          _dp(self._h), _dp(self._g))
        an = Ansatz(self.K, self._exc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(self._theta))
        self.stream = stream if stream is not None else _current_stream()
        handle = ctypes.c_void_p()
        check(self.lib.ucc_create(ctypes.byref(ham), ctypes.byref(an), self.stream, ctypes.byref(handle)))
        self.handle = handle
        self._opt = dict(n_max=int(getattr(prob, "n_max", 0)), n_cut=int(getattr(prob, "n_cut", 0)),
                         max_entries=int(max_entries), probe_width=int(probe_width), checkpoint_stride=0,
                         tape_budget_mb=0, record_entropy=0, batch_wait_ms=0, batch_test_skip_block=0,
                         batch_tiles=0, energy_route=0, energy_test_partitions=0, energy_test_buffer_records=0,
                         rebuild_test_regions=0)
        self.set_options()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ucc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def set_options(self, **changes):
        """Update run options (the rest keep their values): n_max, n_cut,
        max_entries, probe_width, checkpoint_stride, tape_budget_mb,
        record_entropy, batch_wait_ms, batch_test_skip_block, batch_tiles, energy_route,
        energy_test_partitions, energy_test_buffer_records, rebuild_test_regions.  The problem's
        own cut is the starting point."""
        unknown = set(changes) - set(self._opt)
        if unknown:
            raise TypeError(f"unknown options {sorted(unknown)}")
        self._opt.update({k: int(v) for k, v in changes.items()})
        o = self._opt
        o = Options(o["n_max"], o["n_cut"], o["max_entries"], o["probe_width"], o["checkpoint_stride"],
                    o["tape_budget_mb"], o["record_entropy"], o["batch_wait_ms"], o["batch_test_skip_block"],
                    o["batch_tiles"], o["energy_route"], o["energy_test_partitions"],
                    o["energy_test_buffer_records"], o["rebuild_test_regions"], 0)
        check(self.lib.ucc_set_options(self.handle, ctypes.byref(o)))

    def set_theta(self, theta):
        """theta: numpy array (host) or a CUDA torch tensor (device)."""
        if hasattr(theta, "is_cuda") and theta.is_cuda:
            t = theta.detach().to(dtype=__import__("torch").float64).contiguous()
            assert t.numel() == self.K
            check(self.lib.ucc_set_theta(self.handle, ctypes.c_void_p(t.data_ptr()), 1))
        else:
            t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
            assert t.shape == (self.K,)
            check(self.lib.ucc_set_theta(self.handle, t.ctypes.data_as(ctypes.c_void_p), 0))

    def apply(self, eps=None):
        eps = float(self.prob.eps if eps is None else eps)
        check(self.lib.ucc_apply(self.handle, eps))

    def energy(self):
        E, n2 = ctypes.c_double(), ctypes.c_double()
        check(self.lib.ucc_energy(self.handle, ctypes.byref(E), ctypes.byref(n2)))
        return E.value, n2.value

    def gradient(self, eps=None, out=None):
        """(E, dE/dtheta).  ``out`` may be a CUDA float64 tensor of K entries
        (result stays on the device) or None (host numpy array)."""
        eps = float(self.prob.eps if eps is None else eps)
        E = ctypes.c_double()
        if out is not None:
            assert out.is_cuda and out.numel() == self.K
            check(self.lib.ucc_gradient(self.handle, eps, ctypes.byref(E), ctypes.c_void_p(out.data_ptr()), 1))
            return E.value, out
        g = np.zeros(self.K)
        check(self.lib.ucc_gradient(self.handle, eps, ctypes.byref(E), g.ctypes.data_as(ctypes.c_void_p), 0))
        return E.value, g

    def wavefunction(self, with_sigma=False):
        """(keys, amps[, sigma]) of the held state, sorted by key (host).  Above
        64 spin-orbitals keys is an (n, 2) array of (low, high) words."""
        n = ctypes.c_size_t()
        st = self.lib.ucc_get_wavefunction(self.handle, 0, ctypes.byref(n), None, None, None, 0)
        if st not in (_lib.UCC_OK, _lib.UCC_ECAPACITY):
            check(st)
        cap = n.value
        keys = np.zeros(cap * self.key_words, dtype=np.uint64)
        amps = np.zeros(cap, dtype=np.float64)
        sig = np.zeros(cap, dtype=np.float64) if with_sigma else None
        check(self.lib.ucc_get_wavefunction(self.handle, cap, ctypes.byref(n), keys.ctypes.data_as(ctypes.c_void_p),
                                            amps.ctypes.data_as(ctypes.c_void_p),
                                            sig.ctypes.data_as(ctypes.c_void_p) if with_sigma else None, 0))
        if self.key_words == 2:
            keys = keys.reshape(cap, 2)
            order = np.lexsort((keys[:, 0], keys[:, 1]))
        else:
            order = np.argsort(keys, kind="stable")
        if with_sigma:
            return keys[order], amps[order], sig[order]
        return keys[order], amps[order]

    def entropy(self):
        """Eq. 6 entropy after each factor of the last apply (needs record_entropy)."""
        S = np.zeros(self.K)
        check(self.lib.ucc_get_entropy(self.handle, _dp(S), self.K))
        return S

    def stats(self):
        s = Stats()
        check(self.lib.ucc_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()


def batch_run(contexts, eps, with_grad=True):
    """Energies (and gradients) of many contexts through ucc_batch_run."""
    lib = _lib.load()
    n = len(contexts)
    handles = (ctypes.c_void_p * n)(*[c.handle for c in contexts])
    E = np.zeros(n)
    grads = [np.zeros(c.K) for c in contexts] if with_grad else None
    gp = (ctypes.c_void_p * n)(*[g.ctypes.data_as(ctypes.c_void_p) for g in grads]) if with_grad else None
    check(lib.ucc_batch_run(n, handles, float(eps), _dp(E), gp))
    return E, grads


def _autograd():
    import torch

    class UCCEnergy(torch.autograd.Function):
        """E(theta) with dE/dtheta from the library's one-sweep adjoint.

        forward(ctx, context, theta, eps) -> scalar energy tensor on theta's
        device; backward returns grad_out * dE/dtheta (a CUDA float64 tensor).
        """

        @staticmethod
        def forward(fctx, context, theta, eps):
            context.set_theta(theta)
            grad = torch.empty(context.K, dtype=torch.float64, device=theta.device)
            E, _ = context.gradient(eps=eps, out=grad)
            fctx.save_for_backward(grad)
            return torch.tensor(E, dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(fctx, grad_out):
            (grad,) = fctx.saved_tensors
            return None, grad_out * grad, None

    return UCCEnergy


def ucc_energy(context, theta, eps=None):
    """Differentiable E(theta) (torch autograd; CUDA float64 theta)."""
    eps = float(context.prob.eps if eps is None else eps)
    return _autograd().apply(context, theta, eps)
