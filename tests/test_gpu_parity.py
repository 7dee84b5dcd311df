"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bars: determinant keys and amplitudes bit-identical (the rotation is two
rounded products and one rounded sum on both sides, cos/sin from the same
libm); integer counters identical; energies within 1e-10 Ha; gradients within
1e-8.
"""
import os

import numpy as np
import pytest

from paper_2301_05726_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
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


def ctx_for(prob, **kw):
    from paper_2301_05726_gb300.api import UCCContext
    return UCCContext(prob, **kw)


def oracle_for(prob):
    import oracle
    return oracle.Oracle(prob)


def load_golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    E = float(rows[0][0])
    g = np.array([float(r[1]) for r in rows[1:]])
    return E, g


def assert_same_state(gk, ga, ok, oa):
    assert len(gk) == len(ok), f"{len(gk)} determinants on the GPU vs {len(ok)} in the oracle"
    assert np.array_equal(gk, ok)
    assert not np.any(np.isnan(ga))
    # bit-identical up to the sign of zero
    diff = ga != oa
    assert not diff.any(), f"{diff.sum()} amplitudes differ; max |d| = {np.max(np.abs(ga - oa))}"


def small_pruned():
    return synth.make_problem(31, 9, 3, 3, 0.08, eps=1e-5)


@pytest.mark.parametrize("case", ["cfg1", "cfg2", "cfg3_prefix150", "cfg4_prefix300", "pruned_small"])
def test_state_bit_exact(torch_cuda, case):
    if case == "cfg1":
        prob = synth.config_problem(1)
    elif case == "cfg2":
        prob = synth.config_problem(2)
    elif case == "cfg3_prefix150":
        prob = synth.config_problem(3).prefix(150)
    elif case == "cfg4_prefix300":
        prob = synth.config_problem(4).prefix(300)
    else:
        prob = small_pruned()
    ok, oa, oc = oracle_for(prob).apply()
    ctx = ctx_for(prob)
    ctx.apply()
    gk, ga = ctx.wavefunction()
    st = ctx.stats()
    assert_same_state(gk, ga, ok, oa)
    assert st["rotations"] == oc["rotations"]
    assert st["created"] == oc["created"]
    assert st["dropped_new"] == oc["dropped_new"]
    assert st["dropped_old"] == oc["dropped_old"]
    assert st["n_det"] == len(ok)
    assert st["probe_width"] in (1, 2, 4, 8)  # autotuned once the table passes 2^16 entries


@pytest.mark.parametrize("pw", [1, 2, 4, 8])
def test_probe_widths_agree(torch_cuda, pw):
    prob = synth.config_problem(3).prefix(100)
    ok, oa, _ = oracle_for(prob).apply()
    ctx = ctx_for(prob, probe_width=pw)
    ctx.apply()
    gk, ga = ctx.wavefunction()
    assert_same_state(gk, ga, ok, oa)


def test_energy_cfg1_and_sigma(torch_cuda):
    prob = synth.config_problem(1)
    o = oracle_for(prob)
    ok, oa, _ = o.apply()
    E_ref, n2_ref = o.energy(ok, oa)
    ctx = ctx_for(prob)
    ctx.apply()
    E, n2 = ctx.energy()
    assert abs(E - E_ref) <= E_TOL
    assert abs(n2 - n2_ref) <= 1e-13
    gk, ga, gs = ctx.wavefunction(with_sigma=True)
    sk, ss = o.sigma(ok, oa)
    assert np.array_equal(gk, sk)
    assert np.max(np.abs(gs - ss)) <= E_TOL


def test_energy_cfg2(torch_cuda):
    prob = synth.config_problem(2)
    E_ref, _ = load_golden("cfg2_energy_gradient.txt")
    ctx = ctx_for(prob)
    ctx.apply()
    E, n2 = ctx.energy()
    assert abs(E - E_ref) <= E_TOL
    assert abs(n2 - 1.0) <= 1e-12
    # sigma at sampled determinants, one by one in the oracle
    gk, ga, gs = ctx.wavefunction(with_sigma=True)
    rng = np.random.default_rng(0)
    pick = rng.choice(len(gk), 200, replace=False)
    o = oracle_for(prob)
    ref = o.sigma_at(gk, ga, gk[pick])
    assert np.max(np.abs(gs[pick] - ref)) <= E_TOL


@pytest.mark.parametrize("prefix", [80, 300])
def test_energy_cfg4_prefix_sampled_sigma(torch_cuda, prefix):
    prob = synth.config_problem(4).prefix(prefix)
    ctx = ctx_for(prob)
    ctx.apply()
    E, n2 = ctx.energy()
    gk, ga, gs = ctx.wavefunction(with_sigma=True)
    o = oracle_for(prob)
    rng = np.random.default_rng(1)
    pick = rng.choice(len(gk), min(64, len(gk)), replace=False)
    ref = o.sigma_at(gk, ga, gk[pick])
    assert np.max(np.abs(gs[pick] - ref)) <= E_TOL
    # the energy is the Rayleigh quotient of the exported sigma
    assert abs(E - float(ga @ gs) / float(ga @ ga)) <= 1e-12
    if prefix == 80:
        E_ref, _ = o.energy(gk, ga)
        assert abs(E - E_ref) <= E_TOL


@pytest.mark.parametrize("case", ["cfg1", "cfg3_prefix60", "pruned_small"])
def test_gradient_vs_oracle(torch_cuda, case):
    if case == "pruned_small":
        prob = small_pruned()
        E_ref, g_ref = oracle_for(prob).gradient()
    else:
        cfg, pre = (1, None) if case == "cfg1" else (3, 60)
        prob = synth.config_problem(cfg)
        if pre:
            prob = prob.prefix(pre)
        E_ref, g_ref = load_golden(f"{case}_energy_gradient.txt")
    ctx = ctx_for(prob)
    E, g = ctx.gradient()
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL
    st = ctx.stats()
    if case == "pruned_small":
        assert st["tape_entries"] > 0  # the irreversible path was exercised


def test_reverse_sweep_compacts(torch_cuda):
    """The reverse sweep removes the entries each factor created; on this
    prefix (39k determinants) a third of the table is dropped well before the
    sweep ends, so it compacts the table (keeping the adjoint) at least once,
    and the gradient still matches the oracle's."""
    prob = synth.config_problem(3).prefix(60)
    E_ref, g_ref = load_golden("cfg3_prefix60_energy_gradient.txt")
    ctx = ctx_for(prob)
    E, g = ctx.gradient()
    st = ctx.stats()
    assert st["reverse_compactions"] >= 1
    assert st["reverse_scanned"] > 0
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL


def test_gradient_cfg2(torch_cuda):
    prob = synth.config_problem(2)
    E_ref, g_ref = load_golden("cfg2_energy_gradient.txt")
    ctx = ctx_for(prob)
    E, g = ctx.gradient()
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL


def test_gradient_vs_central_fd_on_gpu(torch_cuda):
    # Independent of the oracle: central differences of the GPU energy.
    prob = synth.config_problem(1)
    ctx = ctx_for(prob)
    E0, g = ctx.gradient()
    th = prob.theta.copy()
    h = 1e-6
    for k in (0, 10, 45, 91):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        ctx.set_theta(tp)
        ctx.apply()
        Ep, _ = ctx.energy()
        ctx.set_theta(tm)
        ctx.apply()
        Em, _ = ctx.energy()
        assert abs(g[k] - (Ep - Em) / (2 * h)) <= max(G_TOL, 5e-9 * abs(E0))


def test_edge_cases(torch_cuda):
    base = synth.config_problem(1)
    o_hf = oracle_for(base)
    # empty ansatz: psi = HF, E = E_HF, empty gradient
    empty = synth.Problem(base.n_spatial, base.n_alpha, base.n_beta, base.h, base.g,
                          np.zeros((0, 4), np.int32), np.zeros(0))
    ctx = ctx_for(empty)
    ctx.apply()
    k, a = ctx.wavefunction()
    assert list(k) == [base.hf_key] and list(a) == [1.0]
    E, _ = ctx.energy()
    assert abs(E - o_hf.hmat(base.hf_key, base.hf_key)) <= E_TOL
    E2, g = ctx.gradient()
    assert g.shape == (0,) and abs(E2 - E) <= E_TOL
    # theta = 0 with pruning: only the reference survives
    zero = base.with_theta(np.zeros(base.n_exc))
    ctx = ctx_for(zero)
    ctx.apply(eps=1e-12)
    k, a = ctx.wavefunction()
    assert list(k) == [base.hf_key] and list(a) == [1.0]
    # energy before apply is a state error
    from paper_2301_05726_gb300._lib import UCCError, UCC_ESTATE, UCC_EINVAL
    ctx = ctx_for(base)
    with pytest.raises(UCCError) as ei:
        ctx.energy()
    assert ei.value.status == UCC_ESTATE
    with pytest.raises(UCCError) as ei:
        ctx.apply(eps=float("nan"))
    assert ei.value.status == UCC_EINVAL
    # run twice: identical state (deterministic per key)
    ctx.apply()
    k1, a1 = ctx.wavefunction()
    ctx.apply()
    k2, a2 = ctx.wavefunction()
    assert np.array_equal(k1, k2) and np.array_equal(a1, a2)


def test_theta_on_device_and_autograd(torch_cuda):
    torch = torch_cuda
    from paper_2301_05726_gb300.api import ucc_energy
    prob = synth.config_problem(1)
    ctx = ctx_for(prob)
    E_ref, g_ref = load_golden("cfg1_energy_gradient.txt")
    theta = torch.tensor(prob.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    E = ucc_energy(ctx, theta)
    E.backward()
    assert abs(E.item() - E_ref) <= E_TOL
    assert torch.max(torch.abs(theta.grad.cpu() - torch.tensor(g_ref))).item() <= G_TOL


# ---------------------------------------------------------------------------
# Methods-section truncation (N_MAX / N_CUT) on the device
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case,n_max,n_cut", [
    ("cfg3_prefix150", 200000, 125000),
    ("cfg4_prefix300", 50000, 31250),
    ("pruned_small", 3000, 1875),
])
def test_truncation_bit_exact(torch_cuda, case, n_max, n_cut):
    if case == "cfg3_prefix150":
        prob = synth.config_problem(3).prefix(150)
    elif case == "cfg4_prefix300":
        prob = synth.config_problem(4).prefix(300)
    else:
        prob = small_pruned()
    ok, oa, oc = oracle_for(prob).apply(n_max=n_max, n_cut=n_cut)
    assert oc["cut"] > 0
    ctx = ctx_for(prob)
    ctx.set_options(n_max=n_max, n_cut=n_cut)
    ctx.apply()
    gk, ga = ctx.wavefunction()
    st = ctx.stats()
    assert_same_state(gk, ga, ok, oa)
    assert st["cut"] == oc["cut"]
    assert st["rotations"] == oc["rotations"]


def test_truncation_gradient(torch_cuda):
    prob = small_pruned()
    E_ref, g_ref = oracle_for(prob).gradient(n_max=3000, n_cut=1875)
    ctx = ctx_for(prob)
    ctx.set_options(n_max=3000, n_cut=1875)
    E, g = ctx.gradient()
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL
    assert ctx.stats()["cut"] > 0


@pytest.mark.parametrize("case,stride", [("pruned_small", 7), ("pruned_small", 1), ("cfg2", 38)])
def test_gradient_segment_checkpoints(torch_cuda, case, stride):
    # Snapshots every `stride` factors, each segment recomputed and swept
    # backward: the same gradient as the oracle's checkpointed adjoint.
    if case == "cfg2":
        prob = synth.config_problem(2)
        E_ref, g_ref = load_golden("cfg2_energy_gradient.txt")
    else:
        prob = small_pruned()
        E_ref, g_ref = oracle_for(prob).gradient()
    ctx = ctx_for(prob)
    ctx.set_options(checkpoint_stride=stride)
    E, g = ctx.gradient()
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL


def test_gradient_tape_budget_falls_back_to_segments(torch_cuda):
    # A 1 MiB tape budget cannot hold even one 24 MB tape page: the gradient
    # falls back to segment checkpoints (with recomputation) and still matches
    # the oracle's adjoint.
    prob = small_pruned()
    E_ref, g_ref = oracle_for(prob).gradient(n_max=3000, n_cut=1875)
    ctx = ctx_for(prob)
    ctx.set_options(n_max=3000, n_cut=1875, tape_budget_mb=1)
    E, g = ctx.gradient()
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL
    assert ctx.stats()["recompute_rotations"] > 0
    # With room for the tape, one segment and no recomputation.
    ctx.set_options(n_max=3000, n_cut=1875, tape_budget_mb=0)
    E2, g2 = ctx.gradient()
    assert ctx.stats()["recompute_rotations"] == 0
    assert np.max(np.abs(g2 - g_ref)) <= G_TOL


@pytest.mark.parametrize("case", ["cfg2", "cfg3_prefix150", "pruned_cut"])
def test_entropy_per_factor(torch_cuda, case):
    # Eq. 6 after every factor, accumulated on the device from the changes of
    # the touched pairs (and the cut), vs the oracle's direct sum.
    if case == "cfg2":
        prob = synth.config_problem(2)
        cut = {}
    elif case == "cfg3_prefix150":
        prob = synth.config_problem(3).prefix(150)
        cut = {}
    else:
        prob = small_pruned()
        cut = dict(n_max=3000, n_cut=1875)
    S_ref = oracle_for(prob).entropy_per_factor(**cut)
    ctx = ctx_for(prob)
    ctx.set_options(record_entropy=True, **cut)
    ctx.apply()
    S = ctx.entropy()
    assert np.max(np.abs(S - S_ref)) <= 1e-10
    assert S_ref[-1] > 0.0


# ---------------------------------------------------------------------------
# The benchmarked configuration: 64 spin-orbitals, eps = 1e-6, with the cut
# ---------------------------------------------------------------------------
def test_gradient_64so_with_cut_vs_oracle(torch_cuda):
    # The first 400 factors of the 64-spin-orbital workload with the paper's own
    # production cut (N_MAX = 8,000, N_CUT = 5,000; Methods section): the cut
    # fires after most factors, so this runs the bench's path -- one tape over
    # the whole run with the cut's records, in-place inverse rotations, lone
    # members divided by cos(theta), bulk re-insertion of cut records.
    prob = synth.config_problem(4).prefix(400)
    n_max, n_cut = 8000, 5000
    o = oracle_for(prob)
    ok, oa, oc = o.apply(n_max=n_max, n_cut=n_cut)
    E_ref, g_ref = o.gradient(n_max=n_max, n_cut=n_cut)
    assert oc["cut"] > 100 * n_cut
    ctx = ctx_for(prob)
    ctx.set_options(n_max=n_max, n_cut=n_cut)
    ctx.apply()
    gk, ga = ctx.wavefunction()
    assert_same_state(gk, ga, ok, oa)
    assert ctx.stats()["cut"] == oc["cut"]
    E, g = ctx.gradient()
    assert abs(E - E_ref) <= E_TOL
    assert np.max(np.abs(g - g_ref)) <= G_TOL
    st = ctx.stats()
    assert st["recompute_rotations"] == 0 and st["tape_entries"] >= oc["cut"]


def test_one_tape_vs_sqrt_k_checkpoints_64so(torch_cuda):
    # 1,500 factors of the 64-spin-orbital workload with a cut that fires every
    # few factors (N_MAX = 1e6, N_CUT = 6.25e5): the one-tape sweep undoes
    # every factor in place (inverse rotations, 1/cos(theta) on lone members),
    # the checkpointed sweep recomputes each sqrt(K)-long segment forward from
    # a snapshot.  The two gradients differ only by the round-off the in-place
    # inversion accumulates.
    prob = synth.config_problem(4).prefix(1500)
    ctx = ctx_for(prob)
    ctx.set_options(n_max=1_000_000, n_cut=625_000)
    E1, g1 = ctx.gradient()
    st1 = ctx.stats()
    assert st1["cut"] > 0 and st1["recompute_rotations"] == 0
    stride = int(np.ceil(np.sqrt(prob.n_exc)))
    ctx.set_options(checkpoint_stride=stride)
    E2, g2 = ctx.gradient()
    st2 = ctx.stats()
    assert st2["recompute_rotations"] > 0
    assert abs(E1 - E2) <= 1e-12  # the same state; sigma sums in a different order
    drift = np.max(np.abs(g1 - g2))
    print(f"one tape vs sqrt(K) checkpoints: max |dg| = {drift:.3e} (|g|max = {np.max(np.abs(g1)):.3e})")
    assert drift <= 1e-10


def test_truncation_with_many_exact_ties(torch_cuda):
    # Zero angles after the first eight factors: every partner they create has
    # amplitude exactly 0 (eps = 0 keeps it), so each cut's threshold is 0 with
    # about 1e5 exactly tied entries, more than the selection's candidate buffer
    # holds: the tie-break by smaller key runs on the table itself.
    prob = synth.config_problem(2).prefix(300)
    th = prob.theta.copy()
    th[8:] = 0.0
    prob = prob.with_theta(th)
    n_max, n_cut = 100_000, 70_000
    ok, oa, oc = oracle_for(prob).apply(n_max=n_max, n_cut=n_cut)
    assert oc["cut"] > 4 * n_cut and np.sum(oa == 0.0) > 0.9 * len(oa)
    ctx = ctx_for(prob)
    ctx.set_options(n_max=n_max, n_cut=n_cut)
    ctx.apply()
    gk, ga = ctx.wavefunction()
    assert_same_state(gk, ga, ok, oa)
    st = ctx.stats()
    assert st["cut"] == oc["cut"] and st["rotations"] == oc["rotations"]


def test_reevaluate_fixed_theta_at_larger_cuts(torch_cuda):
    # Results, discussion of Fig. 3c: with the parameters held fixed, the
    # energy is computed again while the wavefunction may grow past the N_CUT
    # used in the optimisation.  One context, its cut changed between
    # evaluations: every evaluation matches the oracle at that cut (state
    # bit-identical, E within 1e-10), and returning to the first cut gives
    # the first state bit for bit (nothing of the larger runs is kept; the
    # energy's summation order follows the table's layout, which the larger
    # runs resized, so E agrees to rounding).
    prob = synth.fig3_problem().prefix(400)
    o = oracle_for(prob)
    ctx = ctx_for(prob)
    energies, states = [], []
    for n_cut in (300, 600, 1200, 2400, 300):
        n_max = 8 * n_cut // 5
        ctx.set_options(n_max=n_max, n_cut=n_cut)
        ctx.apply()
        E, n2 = ctx.energy()
        ok, oa, oc = o.apply(n_max=n_max, n_cut=n_cut)
        gk, ga = ctx.wavefunction()
        assert np.array_equal(gk, ok) and not np.any(ga != oa), n_cut
        assert ctx.stats()["cut"] == oc["cut"] > 0
        E_o, n2_o = o.energy(ok, oa)
        assert abs(E - E_o) <= E_TOL and abs(n2 - n2_o) <= 1e-12
        energies.append(E)
        states.append((gk, ga))
    assert np.array_equal(states[-1][0], states[0][0]) and np.array_equal(states[-1][1], states[0][1])
    assert abs(energies[-1] - energies[0]) <= 1e-12
    assert len(set(energies[:4])) == 4
