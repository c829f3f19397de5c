"""The run monitor's schedule and records (no GPU: the library calls are
replaced by a stand-in context that counts steps)."""
import json

import numpy as np
import pytest

from paper_2107_07315_gb300 import monitor
from paper_2107_07315_gb300 import sph


class _FakeCtx:
    def __init__(self):
        self.steps = 0
        self.calls = []


def _install(monkeypatch, ctx):
    def step(c, dt, k):
        c.calls.append(("step", dt, k))
        c.steps += k

    def stats(c):
        out = np.zeros(32, np.int64)
        out[9] = c.steps
        out[0] = 1000 + c.steps
        out[18] = c.steps // 4
        return out

    def totals(c):
        t = np.arange(16, dtype=np.float64)
        t[0] = 1.0
        t[6] = 2.0 + c.steps
        return t

    def per_star(c, ns):
        return np.tile(np.arange(16, dtype=np.float64), (ns, 1)) + c.steps

    monkeypatch.setattr(sph, "sph_step", step)
    monkeypatch.setattr(sph, "sph_sync", lambda c: None)
    monkeypatch.setattr(sph, "sph_stats", stats)
    monkeypatch.setattr(sph, "sph_totals", totals)
    monkeypatch.setattr(sph, "sph_totals_per_star", per_star)


def test_chunks_and_lines(tmp_path, monkeypatch):
    ctx = _FakeCtx()
    _install(monkeypatch, ctx)
    path = tmp_path / "run.jsonl"
    n = monitor.run_logged(ctx, 0.5, 10, 4, str(path), nstars=3, t0=1.0)
    assert n == 4  # the initial state and after steps 4, 8, 10
    assert [c[2] for c in ctx.calls] == [4, 4, 2]
    recs = [json.loads(l) for l in path.read_text().splitlines()]
    assert [r["step"] for r in recs] == [0, 4, 8, 10]
    assert [r["t"] for r in recs] == [1.0, 3.0, 5.0, 6.0]
    assert recs[-1]["totals"]["energy"] == 12.0 and recs[0]["totals"]["mass"] == 1.0
    assert len(recs[1]["stars"]) == 3 and recs[1]["stars"][2]["yielded"] == 14.0
    assert recs[2]["candidate_builds"] == 2 and recs[3]["pairs_last_rhs"] == 1010
    assert set(monitor.TOTAL_NAMES) == set(recs[0]["totals"])


def test_bad_schedule_rejected(tmp_path, monkeypatch):
    ctx = _FakeCtx()
    _install(monkeypatch, ctx)
    with pytest.raises(ValueError):
        monitor.run_logged(ctx, 0.1, 5, 0, str(tmp_path / "x.jsonl"))
