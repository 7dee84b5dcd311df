"""ucc_energy_static: the energy pass for callers that cannot allocate device
memory when they call it (cudaMalloc/cudaFree may synchronise the device, the
memory may all belong to another allocator, or the device may be out of
memory).  Its scratch is a fixed device array inside the library.

The test holds the wavefunction of the 24-spin-orbital workload (245,025
determinants) in caller-owned device buffers, calls the entry point through
the C ABI twice in a row, and checks each result against the context path
(ucc_apply + ucc_energy) within the energy tolerance of the other GPU tests.
This file is collected last so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2301_05726_gb300 import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-10


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
    for call in range(2):
        d_sig = torch.full((len(keys),), float("nan"), dtype=torch.float64, device=dev)
        E = ctypes.c_double()
        n2 = ctypes.c_double()
        st = lib.ucc_energy_static(prob.n_spatial, prob.n_alpha, prob.n_beta, 0.0, vp(d_h), vp(d_g), len(keys),
                                   vp(d_keys), vp(d_amps), vp(d_sig), ctypes.byref(E), ctypes.byref(n2), stream)
        assert st == 0, lib.ucc_last_error().decode()
        assert abs(E.value - E_ref) <= E_TOL, (call, E.value, E_ref)
        assert abs(n2.value - n2_ref) <= 1e-12
        sig = d_sig.cpu().numpy()
        assert np.max(np.abs(sig - sig_ref)) <= E_TOL, call

    # Sizes past the stated maximum are rejected before any device work.
    E = ctypes.c_double()
    st = lib.ucc_energy_static(prob.n_spatial, prob.n_alpha, prob.n_beta, 0.0, vp(d_h), vp(d_g), 262145,
                               vp(d_keys), vp(d_amps), vp(d_amps), ctypes.byref(E), None, stream)
    assert st == _lib.UCC_EINVAL and "n_det" in lib.ucc_last_error().decode()
