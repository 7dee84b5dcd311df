"""Host logic of bench.py that needs no GPU: sizing the oracle's prefix for
the CPU baseline and the reference arm."""
import types

import bench


def _fake_problem(n_exc):
    return types.SimpleNamespace(n_exc=n_exc)


def test_oracle_prefix_stays_within_budget(monkeypatch):
    # cost grows steeply with the prefix (the map grows), like the oracle's
    calls = []

    def fake_time(prob, n, with_grad=True):
        calls.append(n)
        return 1000 * n, 1e-4 * n ** 2.5

    monkeypatch.setattr(bench, "oracle_time", fake_time)
    nf, rot, dt = bench.oracle_prefix(_fake_problem(30000), seconds=15.0)
    assert dt <= 15.0 and rot == 1000 * nf
    # the next prefix (1.5x) would have passed the budget
    assert 1e-4 * int(nf * 1.5) ** 2.5 > 15.0 / 2
    # prefixes grew by 1.5x from 16 and were timed once each
    assert calls[0] == 16 and all(b == max(a + 1, int(a * 1.5)) for a, b in zip(calls, calls[1:]))


def test_oracle_prefix_caps_at_the_workload(monkeypatch):
    monkeypatch.setattr(bench, "oracle_time", lambda prob, n, with_grad=True: (n, 1e-6 * n))
    nf, _, _ = bench.oracle_prefix(_fake_problem(40), seconds=100.0)
    assert nf == 40


def test_oracle_sample_reuses_a_fixed_prefix(monkeypatch):
    seen = []

    def fake_time(prob, n, with_grad=True):
        seen.append(n)
        return 10 * n, 0.5

    monkeypatch.setattr(bench, "oracle_time", fake_time)
    rate, evals, nf, dt = bench.oracle_sample(_fake_problem(30000), 15.0, n_factors=54)
    assert seen == [54] and nf == 54 and rate == 10 * 54 / 0.5 and evals == 2.0


def test_traffic_is_scaled_by_the_entries_scanned(monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PER_SCANNED_ENTRY", {"k_reverse": 47.0})
    r = bench._roofline("k_reverse", 4e9, 10.0, 4, 6000.0, "measured", scanned=4e7)
    assert r["traffic"] == 47.0 * 1e7
    assert bench._roofline("energy", 1e9, 10.0, 1, 6000.0, "measured")["traffic"] is None
    assert bench._roofline("k_reverse", 4e9, 10.0, 4, 6000.0, "measured")["traffic"] is None


def test_member_model_charges_lone_rotations_one_member():
    tot = dict(scanned=1000, recompute_scanned=0, rotations=100, recompute_rotations=0, created=10,
               recompute_created=0, dropped_new=80, reverse_pairs=100, n_det=50, sigma_hits=7)
    m = bench.byte_models(tot)
    # 90 lone rotations (10 created + 80 dropped), 10 with both members stored
    assert m["pair"]["k_forward"] == 8 * 1000 + 48 * 100 + 32 * 10
    assert m["member"]["k_forward"] == 8 * 1000 + 16 * 90 + 48 * 10 + 32 * 10
    assert m["pair"]["k_reverse"] == 8 * 1000 + 80 * 100
    assert m["member"]["k_reverse"] == 8 * 1000 + 32 * 80 + 80 * 20
    assert m["member"]["energy"] == m["pair"]["energy"] == 24 * 50 + 16 * 7
    tot.update(energy_route_last=2, sigma_probes=900)
    assert bench.byte_models(tot)["member"]["energy"] == 64 * 900 + 40 * 50


def test_host_info_names_the_cpu():
    h = bench.host_info()
    assert h["nproc"] >= 1 and h["machine"]
