"""The plain profiler arithmetic against the summary the paper prints."""
import random

import pytest

from oracle import profile
from tests import golden_profile


def test_profile_oracle_reproduces_paper_summary():
    fx = golden_profile.load()
    evs = [profile.Event(*e) for e in golden_profile.synthetic_events(fx)]
    a = profile.analyse(evs, fx["elapsed"])
    # Printed absolute times carry 5 significant digits, relative shares 4
    # decimals: compare at the printed precision.
    for name, (rel, abs_s) in fx["agg"].items():
        assert a.aggregate[name] == pytest.approx(abs_s, rel=1e-9)
        assert a.relative[name] == pytest.approx(rel, abs=2e-3)
    assert a.total == pytest.approx(fx["agg_total"], abs=1e-4)
    assert a.overlaps == {("RNG_KERNEL", "READ_BUFFER"): pytest.approx(fx["overlap_total"], rel=1e-9)}
    assert a.effective == pytest.approx(fx["effective"], abs=5e-5)
    assert a.device_pct == pytest.approx(fx["device_pct"], abs=5e-3)
    assert a.host_pct == pytest.approx(fx["host_pct"], abs=5e-3)


def test_printed_summary_is_self_consistent():
    # The paper's own numbers obey effective = total - overlap and
    # device share = effective / elapsed; this pins the definitions.
    fx = golden_profile.load()
    assert fx["agg_total"] - fx["overlap_total"] == pytest.approx(fx["effective"], abs=5e-5)
    assert 100 * fx["effective"] / fx["elapsed"] == pytest.approx(fx["device_pct"], abs=5e-3)
    assert fx["device_pct"] + fx["host_pct"] == pytest.approx(100.0)
    total = sum(v[1] for v in fx["agg"].values())
    for rel, abs_s in fx["agg"].values():
        assert 100 * abs_s / total == pytest.approx(rel, abs=2e-3)


def test_effective_time_is_union_for_two_in_order_queues():
    # With two queues whose own events never overlap, total - pairwise
    # overlaps equals the measure of the union of all intervals.
    rng = random.Random(11)
    for _ in range(50):
        evs = []
        for q in ("Main", "Comms"):
            t = rng.random()
            for k in range(rng.randint(0, 8)):
                d = rng.random()
                evs.append(profile.Event(q, rng.choice("ABC"), t, t + d))
                t += d + rng.random() * 0.5
        a = profile.analyse(evs, 100.0)
        pts = sorted((e.start, e.end) for e in evs)
        union, cur_s, cur_e = 0.0, None, None
        for s, e in pts:
            if cur_e is None or s > cur_e:
                if cur_e is not None:
                    union += cur_e - cur_s
                cur_s, cur_e = s, e
            else:
                cur_e = max(cur_e, e)
        if cur_e is not None:
            union += cur_e - cur_s
        assert a.effective == pytest.approx(union, abs=1e-9)
