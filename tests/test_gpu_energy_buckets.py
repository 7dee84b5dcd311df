"""The energy by buckets of shared cores against the per-connection energy
and the oracle, through the C ABI.

Both routes compute sigma_I = sum_{J in S} <I|H|J> c_J over the stored set
(Slater-Condon rules; the energy of the Results section is <psi|sigma> /
<psi|psi>).  They differ only in how the connected pairs are found, so sigma
agrees to rounding (its sums run in other orders), E within 1e-12 of each
other and within 1e-10 of the oracle, and the number of connected stored
pairs found is the same integer.
"""
import os

import numpy as np
import pytest

from paper_2301_05726_gb300 import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05726_gb300 import build
    build.build()
    return torch


def ctx_for(prob):
    from paper_2301_05726_gb300.api import UCCContext
    return UCCContext(prob)


def energy_by(ctx, route, **test):
    ctx.set_options(energy_route=route, energy_test_partitions=test.get("partitions", 0),
                    energy_test_buffer_records=test.get("buffer_records", 0))
    E, n2 = ctx.energy()
    st = ctx.stats()
    assert st["energy_route"] == route
    k, a, s = ctx.wavefunction(with_sigma=True)
    return E, n2, s, st


def assert_routes_agree(ctx, **test):
    E1, n1, s1, st1 = energy_by(ctx, 1)
    E2, n2, s2, st2 = energy_by(ctx, 2, **test)
    scale = max(1.0, float(np.max(np.abs(s1))))
    assert np.max(np.abs(s1 - s2)) <= 1e-12 * scale
    assert abs(E1 - E2) <= 1e-12 and abs(n1 - n2) <= 1e-14
    assert st1["sigma_hits"] == st2["sigma_hits"] > 0
    return E2


def fourteen():
    # 14 spin-orbitals, 6 electrons: the whole 1,225-determinant sector is
    # reached (21 records per determinant).
    return synth.make_problem(21, 7, 3, 3, 0.1)


def golden_energy(name):
    # written by tests/golden/make_golden.py from the oracle alone: E on the
    # first line that is not a comment
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden", name))
            if ln.strip() and not ln.startswith("#")]
    return float(rows[0][0])


@pytest.mark.parametrize("case", ["cfg1", "cfg2", "cfg4_prefix300_cut", "pruned_cut"])
def test_routes_agree_and_match_the_oracle(torch_cuda, case):
    import oracle
    if case == "cfg1":
        prob = synth.config_problem(1)
    elif case == "cfg2":
        prob = synth.config_problem(2)
    elif case == "cfg4_prefix300_cut":
        prob = synth.config_problem(4).prefix(300)
        prob.n_max, prob.n_cut = 8000, 5000
    else:
        import dataclasses
        prob = dataclasses.replace(synth.config_problem(2).prefix(150), eps=1e-7, n_max=1500, n_cut=1000)
    ctx = ctx_for(prob)
    ctx.apply()
    E = assert_routes_agree(ctx)
    if case == "cfg2":
        # the oracle's own energy of the whole 245,025-determinant sector takes minutes
        E_o = golden_energy("cfg2_energy_gradient.txt")
    else:
        o = oracle.Oracle(prob)
        k, a, _ = o.apply()
        E_o, _ = o.energy(k, a)
    assert abs(E - E_o) <= E_TOL


def test_default_route_is_buckets(torch_cuda):
    ctx = ctx_for(synth.config_problem(2))
    ctx.apply()
    ctx.energy()
    assert ctx.stats()["energy_route"] == 2


def test_oversized_partitions_take_the_global_walk(torch_cuda):
    # Four partitions for ~25,700 records: ~6,400 each, over the 3,072 a block
    # holds in shared memory.
    ctx = ctx_for(fourteen())
    ctx.apply()
    assert ctx.stats()["n_det"] == 1225
    assert_routes_agree(ctx, partitions=4)


def test_records_in_many_rounds(torch_cuda):
    # A 4,000-record buffer: the partitions are processed in several rounds.
    ctx = ctx_for(fourteen())
    ctx.apply()
    assert_routes_agree(ctx, buffer_records=4000)


def test_gradient_through_either_route(torch_cuda):
    # The adjoint starts from sigma (lambda_K = (sigma - E psi) / <psi|psi>).
    prob = synth.config_problem(2)
    ctx = ctx_for(prob)
    ctx.set_options(energy_route=1)
    E1, g1 = ctx.gradient()
    ctx.set_options(energy_route=2)
    E2, g2 = ctx.gradient()
    assert abs(E1 - E2) <= 1e-12 and np.max(np.abs(g1 - g2)) <= 1e-10


def test_two_word_keys(torch_cuda):
    import oracle
    from test_gpu_wide_keys import ch2o_like
    prob = ch2o_like().prefix(300)
    ctx = ctx_for(prob)
    ctx.apply()
    E = assert_routes_agree(ctx)
    o = oracle.Oracle(prob, key_bits=128)
    k, a, _ = o.apply()
    E_o, _ = o.energy(k, a)
    assert abs(E - E_o) <= E_TOL


def test_invalid_route_options_are_rejected(torch_cuda):
    from paper_2301_05726_gb300._lib import UCCError
    ctx = ctx_for(synth.config_problem(1))
    for bad in (dict(energy_route=3), dict(energy_test_partitions=3), dict(energy_test_buffer_records=-1)):
        with pytest.raises(UCCError):
            ctx.set_options(**bad)
