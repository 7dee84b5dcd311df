"""ucc_energy_static: the energy pass for callers that cannot allocate device
memory when they call it (cudaMalloc/cudaFree may synchronise the device, the
memory may all belong to another allocator, or the device may be out of
memory).  Its scratch is a fixed device array inside the library.

The test holds the wavefunction of the 24-spin-orbital workload (245,025
determinants) in caller-owned device buffers, calls the entry point through
the C ABI twice in a row, and checks each result against the context path
(ucc_apply + ucc_energy) and against the CPU oracle (its stored energy of that
state, and sigma at sampled determinants) within the energy tolerance of the
other GPU tests.  This file is collected last so that a failure here comes
after every other test has run.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_2301_05726_gb300 import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-10
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_energy(name):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    return float(rows[0][0])


def test_energy_static_matches_context_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05726_gb300 import build, _lib
    from paper_2301_05726_gb300.api import UCCContext
    build.build()
    lib = _lib.load()
    prob = synth.config_problem(2)
    ctx = UCCContext(prob)
    ctx.apply()
    E_ref, n2_ref = ctx.energy()
    keys, amps, sig_ref = ctx.wavefunction(with_sigma=True)
    assert len(keys) <= 262144

    dev = torch.device("cuda")
    d_keys = torch.from_numpy(keys.view(np.int64)).to(dev)
    d_amps = torch.from_numpy(amps).to(dev)
    d_h = torch.from_numpy(np.ascontiguousarray(prob.h)).to(dev)
    d_g = torch.from_numpy(np.ascontiguousarray(prob.g)).to(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    # The oracle's side: its energy of this state (written by
    # tests/golden/make_golden.py from the oracle alone; the GPU state is
    # bit-identical to the oracle's, which the parity tests check) and sigma
    # at a sample of determinants.
    import oracle
    E_oracle = golden_energy("cfg2_energy_gradient.txt")
    sample = np.random.default_rng(3).choice(len(keys), 200, replace=False)
    sig_oracle = oracle.Oracle(prob).sigma_at(keys, amps, keys[sample])
    for call in range(2):
        d_sig = torch.full((len(keys),), float("nan"), dtype=torch.float64, device=dev)
        E = ctypes.c_double()
        n2 = ctypes.c_double()
        st = lib.ucc_energy_static(prob.n_spatial, prob.n_alpha, prob.n_beta, 0.0, vp(d_h), vp(d_g), len(keys),
                                   vp(d_keys), vp(d_amps), vp(d_sig), ctypes.byref(E), ctypes.byref(n2), stream)
        assert st == 0, lib.ucc_last_error().decode()
        assert abs(E.value - E_ref) <= E_TOL, (call, E.value, E_ref)
        assert abs(E.value - E_oracle) <= E_TOL, (call, E.value, E_oracle)
        assert abs(n2.value - n2_ref) <= 1e-12
        sig = d_sig.cpu().numpy()
        assert np.max(np.abs(sig - sig_ref)) <= E_TOL, call
        assert np.max(np.abs(sig[sample] - sig_oracle)) <= E_TOL, call

    # Sizes past the stated maximum are rejected before any device work.
    E = ctypes.c_double()
    st = lib.ucc_energy_static(prob.n_spatial, prob.n_alpha, prob.n_beta, 0.0, vp(d_h), vp(d_g), 262145,
                               vp(d_keys), vp(d_amps), vp(d_amps), ctypes.byref(E), None, stream)
    assert st == _lib.UCC_EINVAL and "n_det" in lib.ucc_last_error().decode()

    # A determinant with the right electron count but the wrong alpha/beta
    # split (one alpha electron moved to a beta orbital) is rejected by the
    # kernel's key check.
    bad = keys.copy()
    k0 = int(bad[0])
    a_bits = [p for p in range(0, prob.n_so, 2) if (k0 >> p) & 1]
    b_free = [p for p in range(1, prob.n_so, 2) if not (k0 >> p) & 1]
    bad[0] = np.uint64(k0 & ~(1 << a_bits[0]) | (1 << b_free[0]))
    d_bad = torch.from_numpy(bad.view(np.int64)).to(dev)
    d_sig = torch.empty(len(keys), dtype=torch.float64, device=dev)
    st = lib.ucc_energy_static(prob.n_spatial, prob.n_alpha, prob.n_beta, 0.0, vp(d_h), vp(d_g), len(keys),
                               vp(d_bad), vp(d_amps), vp(d_sig), ctypes.byref(E), None, stream)
    assert st == _lib.UCC_EINVAL and "alpha" in lib.ucc_last_error().decode()
