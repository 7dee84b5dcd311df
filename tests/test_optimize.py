"""The optimiser driver (SLSQP, as in the Methods section) on the CPU with the
oracle's adjoint gradient, and on the GPU context.  Pins: the variational
bound E >= E_FCI (dense diagonalisation of the sector Hamiltonian), energy
decrease from the start, and a vanishing gradient at the optimum."""
import numpy as np
import pytest

from paper_2301_05726_gb300 import synth
from paper_2301_05726_gb300.optimize import minimize_energy


def fci_energy(prob):
    # Lowest eigenvalue of H in the (n_alpha, n_beta) sector, with the
    # Slater-Condon elements that tests/test_oracle_pins.py pins to the dense
    # RDM contraction.
    from oracle import Oracle
    o = Oracle(prob)
    na = prob.n_alpha
    dets = [x for x in range(1 << prob.n_so)
            if bin(x).count("1") == prob.n_elec and bin(x & 0x5555555555555555).count("1") == na]
    H = np.array([[o.hmat(I, J) for J in dets] for I in dets])
    return float(np.linalg.eigvalsh(H)[0])


@pytest.fixture(scope="module")
def small():
    # 10 spin-orbitals, 4 electrons: 100 determinants, 48 factors
    return synth.make_problem(41, 5, 2, 2, 0.05)


def test_slsqp_with_oracle_gradient(small):
    from oracle import Oracle
    o = Oracle(small)
    E0, _ = o.gradient()
    res = minimize_energy(lambda th: o.gradient(th), small.theta, method="SLSQP", maxiter=300)
    e_fci = fci_energy(small)
    assert res.energy < E0
    assert res.energy >= e_fci - 1e-10          # variational bound
    assert res.energy - e_fci < 5e-3             # UCCSD recovers most of the correlation
    assert res.grad_norm < 1e-5


@pytest.mark.gpu
def test_slsqp_on_gpu_matches_oracle(small):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import Oracle
    from paper_2301_05726_gb300 import build
    from paper_2301_05726_gb300.api import UCCContext
    from paper_2301_05726_gb300.optimize import minimize_context
    build.build()
    ctx = UCCContext(small)
    res = minimize_context(ctx, method="SLSQP", maxiter=300)
    o = Oracle(small)
    ref = minimize_energy(lambda th: o.gradient(th), small.theta, method="SLSQP", maxiter=300)
    assert abs(res.energy - ref.energy) < 1e-9
    assert res.grad_norm < 1e-5
