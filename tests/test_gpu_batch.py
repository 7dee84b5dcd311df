"""Batched form: many independent jobs of uneven size advanced together by
one persistent launch per pass, through ucc_batch_run.

Each job of the batch must give what it gives alone: the same determinants
and bit-identical amplitudes (energy-only batches keep the state), energies
within 1e-10 Ha and gradients within 1e-8 of the single-job path and of the
CPU oracle.  Jobs are drawn from the 256-job workload (16-36 spin-orbitals,
4-12 electrons, theta ~ N(0, 0.02), eps = 1e-8), restricted to those whose
Hilbert space the oracle covers in seconds.
"""
import numpy as np
import pytest

from paper_2301_05726_gb300 import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-10
G_TOL = 1e-8


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_05726_gb300 import build
    build.build()
    return torch


def small_jobs(limit, max_hilbert):
    out = []
    for j in range(256):
        n_sp, na, nb = synth.batch_job_shape(j)
        if synth.hilbert_size(n_sp, na, nb) <= max_hilbert:
            out.append(j)
    return out[:limit]


def test_batch_gradients_match_single_path(torch_cuda):
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    jobs = small_jobs(24, 60000)
    assert len(jobs) == 24
    probs = [synth.batch_job_problem(j) for j in jobs]
    ctxs = [UCCContext(p) for p in probs]
    E, grads = batch_run(ctxs, eps=1e-8, with_grad=True)
    sizes = set()
    for p, e, g in zip(probs, E, grads):
        ref = UCCContext(p)
        Er, gr = ref.gradient(eps=1e-8)
        assert abs(e - Er) <= E_TOL, p.name
        assert np.max(np.abs(g - gr)) <= G_TOL, p.name
        sizes.add(p.n_exc)
    assert len(sizes) > 5  # uneven jobs


def test_batch_energy_state_vs_oracle(torch_cuda):
    import oracle
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    jobs = small_jobs(8, 20000)
    probs = [synth.batch_job_problem(j) for j in jobs]
    ctxs = [UCCContext(p) for p in probs]
    E, _ = batch_run(ctxs, eps=1e-8, with_grad=False)
    for p, c, e in zip(probs, ctxs, E):
        o = oracle.Oracle(p)
        ok, oa, oc = o.apply(eps=1e-8)
        gk, ga = c.wavefunction()
        assert np.array_equal(gk, ok), p.name
        assert not np.any(ga != oa), p.name
        assert c.stats()["rotations"] == oc["rotations"]
        E_ref, _ = o.energy(ok, oa)
        assert abs(e - E_ref) <= E_TOL, p.name


def test_batch_gradient_vs_oracle(torch_cuda):
    import oracle
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    jobs = small_jobs(6, 8000)
    probs = [synth.batch_job_problem(j) for j in jobs]
    ctxs = [UCCContext(p) for p in probs]
    E, grads = batch_run(ctxs, eps=1e-8, with_grad=True)
    for p, e, g in zip(probs, E, grads):
        Er, gr = oracle.Oracle(p).gradient(eps=1e-8)
        assert abs(e - Er) <= E_TOL, p.name
        assert np.max(np.abs(g - gr)) <= G_TOL, p.name


def test_batch_with_a_cut_job_and_a_large_job(torch_cuda):
    # A job with the N_MAX/N_CUT cut (cut on the device inside the persistent
    # launch) and a job whose table holds its whole 245,025-determinant sector
    # share the batch with a small one.
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    big = synth.config_problem(2)
    cut = synth.config_problem(3).prefix(120)
    cut.n_max, cut.n_cut = 100000, 62500
    small = synth.batch_job_problem(small_jobs(1, 5000)[0])
    probs = [small, big, cut]
    ctxs = [UCCContext(p) for p in probs]
    E, grads = batch_run(ctxs, eps=0.0, with_grad=True)
    for p, e, g in zip(probs, E, grads):
        Er, gr = UCCContext(p).gradient(eps=0.0)
        assert abs(e - Er) <= E_TOL, p.name
        assert np.max(np.abs(g - gr)) <= G_TOL, p.name


def paper_cut(prob):
    # The paper's production truncation (Methods section: N_MAX = 8,000,
    # N_CUT = 5,000), carried by every job of the 256-job workload.
    prob.n_max, prob.n_cut = 8000, 5000
    return prob


def test_batch_256_workload_jobs_vs_single_path(torch_cuda):
    # Jobs of the 256-job workload, large ones included (their sectors hold up
    # to 3.4e8 determinants; the cut keeps 5,000-8,000), against the one-job
    # path with the same cut (host-driven cuts, one launch per factor).
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    picks = [0, 3, 21, 54, 65, 98, 120, 131, 186, 197, 230, 251]
    probs = [paper_cut(synth.batch_job_problem(j)) for j in picks]
    ctxs = [UCCContext(p) for p in probs]
    E, grads = batch_run(ctxs, eps=1e-8, with_grad=True)
    st = ctxs[0].stats()
    assert st["batch_tiles"] in (1, 2, 4, 8) and st["probe_width"] in (1, 2, 4)
    cut_jobs = 0
    for p, c, e, g in zip(probs, ctxs, E, grads):
        ref = UCCContext(p)
        Er, gr = ref.gradient(eps=1e-8)
        assert abs(e - Er) <= E_TOL, p.name
        assert np.max(np.abs(g - gr)) <= G_TOL, p.name
        assert c.stats()["cut"] == ref.stats()["cut"], p.name
        cut_jobs += ref.stats()["cut"] > 0
    assert cut_jobs >= 4


def test_batch_cut_job_state_vs_oracle(torch_cuda):
    # Energy-only batch: a cut job's determinants and amplitudes after the
    # device-side cuts are the oracle's, bit for bit.
    import oracle
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    probs = [paper_cut(synth.batch_job_problem(j).prefix(300)) for j in (54, 120)]
    probs.append(synth.batch_job_problem(0))
    ctxs = [UCCContext(p) for p in probs]
    E, _ = batch_run(ctxs, eps=1e-8, with_grad=False)
    for p, c, e in zip(probs, ctxs, E):
        o = oracle.Oracle(p)
        ok, oa, oc = o.apply(eps=1e-8)
        gk, ga = c.wavefunction()
        assert np.array_equal(gk, ok), p.name
        assert not np.any(ga != oa), p.name
        assert c.stats()["cut"] == oc["cut"] and c.stats()["rotations"] == oc["rotations"], p.name
        assert abs(e - o.energy(ok, oa)[0]) <= E_TOL, p.name
    assert sum(c.stats()["cut"] > 0 for c in ctxs) == 2


def test_batch_barrier_timeout_returns_an_error(torch_cuda):
    # One block of the persistent forward launch leaves before its first grid
    # barrier (a test hook), so the other blocks' waits run out after 50 ms:
    # the call returns UCC_ETIMEOUT, and the same contexts then run normally.
    from paper_2301_05726_gb300 import _lib
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    probs = [synth.batch_job_problem(j) for j in small_jobs(4, 8000)]
    ctxs = [UCCContext(p) for p in probs]
    ctxs[0].set_options(batch_wait_ms=50, batch_test_skip_block=1)
    with pytest.raises(_lib.UCCError) as err:
        batch_run(ctxs, eps=1e-8, with_grad=True)
    assert err.value.status == _lib.UCC_ETIMEOUT
    ctxs[0].set_options(batch_wait_ms=0, batch_test_skip_block=0)
    E, grads = batch_run(ctxs, eps=1e-8, with_grad=True)
    for p, e, g in zip(probs, E, grads):
        Er, gr = UCCContext(p).gradient(eps=1e-8)
        assert abs(e - Er) <= E_TOL and np.max(np.abs(g - gr)) <= G_TOL, p.name
