"""Pins for the CPU oracle: each test ties it to something other than itself.

* sizes the paper prints (tests/golden/paper_counts.txt);
* the dense state-vector brute force (oracle/dense.py: Taylor-series matrix
  exponentials and RDM contractions, no 2x2 closed form, no Slater-Condon);
* closed forms (Hartree-Fock energy from spatial integrals; one factor on the
  reference);
* invariants (norm, Hermiticity, reachable set, checkpoint-stride
  independence);
* the exact four-term parameter-shift rule and central finite differences.
"""
import math
import os

import numpy as np
import pytest

from paper_2301_05726_gb300 import synth
from oracle import Oracle
from oracle.dense import Dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(seed=7, n_spatial=6, na=2, nb=2, sigma=0.05, eps=0.0, m_doubles=None):
    return synth.make_problem(seed, n_spatial, na, nb, sigma, eps=eps, m_doubles=m_doubles)


@pytest.fixture(scope="module")
def cfg1():
    return synth.config_problem(1)


@pytest.fixture(scope="module")
def nh3_shape():
    # 16 spin-orbitals, 10 electrons: the size of the NH3/STO-3G entropy study
    # (315 factors, Results discussion of Fig. 4).
    return small_problem(seed=11, n_spatial=8, na=5, nb=5, sigma=0.05)


# ---------------------------------------------------------------------------
# Paper-printed sizes
# ---------------------------------------------------------------------------
def test_paper_counts():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_counts.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 4
    for n_sp, na, nb, nexc, hil, _cite in rows:
        n_sp, na, nb = int(n_sp), int(na), int(nb)
        s, d = synth.enumerate_excitations(n_sp, na, nb)
        if nexc != "-":
            assert len(s) + len(d) == int(nexc)
        if hil != "-":
            h = synth.hilbert_size(n_sp, na, nb)
            if "e" in hil:  # printed to two significant figures
                assert abs(h - float(hil)) / float(hil) < 0.02
            else:
                assert h == int(hil)


def test_config_factor_counts():
    # Spin-conserving UCCSD counts of the four single-job workloads; the
    # 64-spin-orbital one keeps all singles and the 29,616 largest doubles.
    assert synth.config_problem(1).n_exc == 92
    assert synth.config_problem(2).n_exc == 1424
    s, d = synth.enumerate_excitations(20, 6, 6)
    assert (len(s), len(d)) == (168, 9786)
    s, d = synth.enumerate_excitations(32, 8, 8)
    assert (len(s), len(d)) == (384, 52320)


def test_factor_order(cfg1):
    exc, th = cfg1.exc, cfg1.theta
    is_double = exc[:, 1] >= 0
    nd = int(is_double.sum())
    assert is_double[:nd].all() and not is_double[nd:].any()  # doubles first, singles applied last
    assert np.all(np.diff(np.abs(th[:nd])) <= 0)  # largest |theta| applied first


# ---------------------------------------------------------------------------
# Operators and matrix elements vs the dense brute force
# ---------------------------------------------------------------------------
def test_tau_signs_vs_dense(cfg1):
    o, d = Oracle(cfg1), Dense(cfg1)
    rng = np.random.default_rng(3)
    ne = cfg1.n_elec
    dets = [k for k in range(d.dim) if bin(k).count("1") == ne]
    for k in range(cfg1.n_exc):
        for det in rng.choice(dets, 12, replace=False):
            v = np.zeros(d.dim)
            v[det] = 1.0
            for dagger in (False, True):
                w = d.tau_dagger(cfg1.exc[k], v) if dagger else d.tau(cfg1.exc[k], v)
                s, out = o.tau(k, det, dagger)
                nz = np.nonzero(w)[0]
                if s == 0:
                    assert len(nz) == 0
                else:
                    assert list(nz) == [out] and w[out] == s
            # tau|E> = s|D>  implies  tau^+|D> = s|E>
            s, D = o.tau(k, det)
            if s:
                s2, back = o.tau(k, D, dagger=True)
                assert back == det and s2 == s


def test_slater_condon_vs_dense(cfg1):
    o, d = Oracle(cfg1), Dense(cfg1)
    rng = np.random.default_rng(5)
    ne = cfg1.n_elec
    dets = np.array([k for k in range(d.dim) if bin(k).count("1") == ne])
    seen = set()
    for _ in range(60):
        I, J = (int(x) for x in rng.choice(dets, 2))
        level = bin(I & ~J).count("1")
        seen.add(level)
        ref = d.hmat(I, J)
        assert o.hmat(I, J) == pytest.approx(ref, abs=1e-12)
        assert o.hmat(J, I) == pytest.approx(o.hmat(I, J), abs=1e-14)  # Hermitian
    for I in dets[:10]:
        assert o.hmat(int(I), int(I)) == pytest.approx(d.hmat(int(I), int(I)), abs=1e-12)
    assert {1, 2}.issubset(seen)


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------
def hf_energy_spatial(prob):
    """E_HF of the closed-shell reference from spatial integrals:
    2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)], i, j over doubly occupied orbitals."""
    assert prob.n_alpha == prob.n_beta
    occ = range(prob.n_alpha)
    h, g = prob.h, prob.g
    e = 2.0 * sum(h[i, i] for i in occ)
    e += sum(2.0 * g[i, i, j, j] - g[i, j, j, i] for i in occ for j in occ)
    return e


@pytest.mark.parametrize("cfg", [1, 2, 4])
def test_theta_zero_gives_hf_energy(cfg):
    prob = synth.config_problem(cfg)
    if cfg == 2:
        prob = prob.prefix(40)
    o = Oracle(prob)
    zero = np.zeros(prob.n_exc)
    eps = 1e-12 if cfg == 4 else 0.0  # drops the zero-amplitude partners of the 64-qubit case
    keys, amps, _ = o.apply(zero, eps=eps)
    assert amps[np.searchsorted(keys, prob.hf_key)] == 1.0
    assert np.all(amps[keys != prob.hf_key] == 0.0)
    E, n2 = o.energy(keys, amps)
    assert n2 == 1.0
    assert E == pytest.approx(hf_energy_spatial(prob), abs=1e-12)


def test_single_factor_closed_form(cfg1):
    # One double on the reference: psi = cos t |HF> + s sin t |D>, so
    # E(t) = cos^2 t H_00 + sin^2 t H_DD + 2 s sin t cos t H_0D.
    d = Dense(cfg1)
    hf = cfg1.hf_key
    for k in (0, 3, 40):
        prob = synth.Problem(cfg1.n_spatial, cfg1.n_alpha, cfg1.n_beta, cfg1.h, cfg1.g,
                             cfg1.exc[k:k + 1].copy(), np.array([0.0]))
        o = Oracle(prob)
        s, D = o.tau(0, hf)
        assert s != 0
        H00, HDD, H0D = d.hmat(hf, hf), d.hmat(D, D), d.hmat(hf, D)
        for t in (0.3, -1.1, 2.0):
            keys, amps, cnt = o.apply(np.array([t]))
            assert list(keys) == sorted([hf, D])
            got = dict(zip(keys.tolist(), amps.tolist()))
            assert got[hf] == pytest.approx(math.cos(t), abs=1e-15)
            assert got[D] == pytest.approx(s * math.sin(t), abs=1e-15)
            E, _ = o.energy(keys, amps)
            ref = math.cos(t) ** 2 * H00 + math.sin(t) ** 2 * HDD + 2 * s * math.sin(t) * math.cos(t) * H0D
            assert E == pytest.approx(ref, abs=1e-12)
            assert cnt["rotations"] == 1 and cnt["created"] == 1


# ---------------------------------------------------------------------------
# Whole ansatz vs the dense brute force (eps = 0)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["cfg1", "nh3_shape"])
def test_state_and_energy_vs_dense(which, request):
    prob = request.getfixturevalue(which)
    o, d = Oracle(prob), Dense(prob)
    keys, amps, cnt = o.apply()
    v = d.state()
    idx = keys.astype(np.int64)
    assert np.max(np.abs(v[idx] - amps)) < 1e-13
    outside = np.ones(d.dim, bool)
    outside[idx] = False
    assert np.max(np.abs(v[outside])) == 0.0  # every nonzero dense amplitude is a key
    E, n2 = o.energy(keys, amps)
    assert E == pytest.approx(d.energy(v), abs=1e-11)
    assert n2 == pytest.approx(1.0, abs=prob.n_exc * 1e-15)


def test_reachable_set_is_structural(cfg1):
    o = Oracle(cfg1)
    k0, a0, _ = o.apply(np.zeros(cfg1.n_exc))
    k1, a1, _ = o.apply()
    assert np.array_equal(k0, k1)  # eps = 0: the key set does not depend on theta
    assert len(k1) == synth.hilbert_size(6, 2, 2)  # and the 92 factors reach the whole sector


def test_norm_with_and_without_pruning():
    prob = synth.config_problem(3).prefix(60)
    o = Oracle(prob)
    _, a, cnt = o.apply(eps=0.0)
    assert float(a @ a) == pytest.approx(1.0, abs=1e-13)
    prev = 1.0
    for nf in (15, 30, 45, 60):
        _, a, cnt = o.apply(eps=1e-6, n_factors=nf)
        n2 = float(a @ a)
        assert n2 <= prev + 1e-15 and n2 <= 1.0 + 1e-15
        prev = n2
    assert cnt["dropped_new"] > 0


def test_sigma_routes_agree():
    prob = synth.config_problem(3).prefix(40)
    o = Oracle(prob)
    keys, amps, _ = o.apply(eps=1e-5)
    assert 50 < len(keys) < 3000
    k1, s1 = o.sigma(keys, amps, "lookup")
    k2, s2 = o.sigma(keys, amps, "pairwise")
    assert np.array_equal(k1, k2)
    assert np.max(np.abs(s1 - s2)) < 1e-12
    sample = keys[::7]
    s3 = o.sigma_at(keys, amps, sample)
    assert np.max(np.abs(s3 - s1[::7])) == 0.0


def test_eps_rule_counts():
    prob = synth.config_problem(3).prefix(60)
    o = Oracle(prob)
    k0, a0, c0 = o.apply(eps=0.0)
    k1, a1, c1 = o.apply(eps=1e-6)
    assert c0["dropped_new"] == 0 and c0["dropped_old"] == 0
    assert set(k1.tolist()) <= set(k0.tolist())
    assert np.all(np.abs(a1) >= 1e-6)


# ---------------------------------------------------------------------------
# Gradient pins
# ---------------------------------------------------------------------------
def shift_rule(f, t):
    """Exact derivative of a trigonometric polynomial of degree 2:
    f'(t) = [f(t+pi/4) - f(t-pi/4)] / (8 sin^2(pi/8)) - [f(t+3pi/4) - f(t-3pi/4)] / (8 sin^2(3pi/8))."""
    a, b = math.pi / 4, 3 * math.pi / 4
    return (f(t + a) - f(t - a)) / (8 * math.sin(a / 2) ** 2) - (f(t + b) - f(t - b)) / (8 * math.sin(b / 2) ** 2)


def test_shift_rule_on_trig_polynomials():
    rng = np.random.default_rng(0)
    for _ in range(5):
        c = rng.normal(size=5)
        f = lambda t: c[0] + c[1] * math.cos(t) + c[2] * math.sin(t) + c[3] * math.cos(2 * t) + c[4] * math.sin(2 * t)
        df = lambda t: -c[1] * math.sin(t) + c[2] * math.cos(t) - 2 * c[3] * math.sin(2 * t) + 2 * c[4] * math.cos(2 * t)
        for t in (0.0, 0.7, -2.2):
            assert shift_rule(f, t) == pytest.approx(df(t), abs=1e-13)


def test_gradient_vs_dense_parameter_shift(cfg1):
    # Fully independent chain: dense energies + the exact shift rule.
    o, d = Oracle(cfg1), Dense(cfg1)
    E, g = o.gradient()
    th = cfg1.theta
    for k in (0, 17, 60, 91):
        def f(t, k=k):
            tt = th.copy()
            tt[k] = t
            return d.energy(d.state(tt))
        assert g[k] == pytest.approx(shift_rule(f, th[k]), abs=1e-10)


def test_gradient_vs_fd_and_shift():
    prob = small_problem(seed=21, n_spatial=7, na=3, nb=3, sigma=0.1)
    o = Oracle(prob)
    E, g = o.gradient()
    th = prob.theta
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in rng.choice(prob.n_exc, 12, replace=False):
        def f(t, k=k):
            tt = th.copy()
            tt[k] = t
            return o.run_energy(tt)
        fd = (f(th[k] + h) - f(th[k] - h)) / (2 * h)
        tol = max(1e-8, 5e-9 * abs(E))
        assert abs(g[k] - fd) < tol
        assert g[k] == pytest.approx(shift_rule(f, th[k]), abs=1e-11)


def test_gradient_checkpoint_stride_independent(cfg1):
    o = Oracle(cfg1)
    _, g0 = o.gradient(stride=0)
    for stride in (1, 5, 92):
        _, g1 = o.gradient(stride=stride)
        assert np.max(np.abs(g1 - g0)) == 0.0


def test_gradient_with_pruning_where_masks_are_stable():
    # With eps > 0 the gradient is that of the pruned map with the kept sets
    # held fixed; finite differences agree wherever a +-h change of theta_k
    # keeps every prune decision (same key set and the same numbers of
    # created / dropped entries at theta +- h).
    prob = small_problem(seed=31, n_spatial=9, na=3, nb=3, sigma=0.08)
    eps = 1e-5
    o = Oracle(prob)
    E, g = o.gradient(eps=eps)
    th = prob.theta
    k_ref, _, c_ref = o.apply(eps=eps)
    h = 1e-6
    checked = 0
    for k in range(0, prob.n_exc, max(1, prob.n_exc // 40)):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        kp, ap, cp = o.apply(tp, eps=eps)
        km, am, cm = o.apply(tm, eps=eps)
        if not (np.array_equal(kp, k_ref) and np.array_equal(km, k_ref) and cp == c_ref and cm == c_ref):
            continue
        fd = (o.energy(kp, ap)[0] - o.energy(km, am)[0]) / (2 * h)
        assert abs(g[k] - fd) < max(1e-8, 5e-9 * abs(E))
        checked += 1
    assert checked >= 20 and c_ref["dropped_old"] > 0 and c_ref["dropped_new"] > 0


def test_gradient_at_theta_zero(cfg1):
    # At theta = 0 every factor is the identity, so dE/dtheta_k = 2 <HF|H A_k|HF>
    # = 2 s_k <D_k|H|HF> when tau_k excites the reference and 0 otherwise.
    o, d = Oracle(cfg1), Dense(cfg1)
    E, g = o.gradient(np.zeros(cfg1.n_exc))
    hf = cfg1.hf_key
    nonzero = 0
    for k in range(cfg1.n_exc):
        s, D = o.tau(k, hf)
        ref = 2 * s * d.hmat(hf, D) if s else 0.0
        assert g[k] == pytest.approx(ref, abs=1e-12)
        nonzero += s != 0
    assert nonzero > 10
    assert E == pytest.approx(hf_energy_spatial(cfg1), abs=1e-12)


# ---------------------------------------------------------------------------
# Eq. 6 entropy after each factor
# ---------------------------------------------------------------------------
def test_entropy_per_factor_vs_dense_and_closed_form(cfg1):
    o, d = Oracle(cfg1), Dense(cfg1)
    S = o.entropy_per_factor()
    assert S.shape == (cfg1.n_exc,)
    for nf in (1, 10, 50, 92):
        v = d.state(n_factors=nf)
        p = v * v
        p = p[p > 0]
        assert S[nf - 1] == pytest.approx(float(-(p * np.log(p)).sum()), abs=1e-12)
    # one factor on the reference: S = -cos^2 ln cos^2 - sin^2 ln sin^2
    t = cfg1.theta[0]
    c2, s2 = math.cos(t) ** 2, math.sin(t) ** 2
    assert S[0] == pytest.approx(-c2 * math.log(c2) - s2 * math.log(s2), abs=1e-14)
    assert np.all(o.entropy_per_factor(np.zeros(cfg1.n_exc)) == 0.0)
