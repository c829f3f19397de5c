"""The run monitor on a real context: one JSON line per chunk with the
library's totals; mass is conserved exactly and the step counter advances."""
import json

import numpy as np
import pytest
import torch

from _parity import stream
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import monitor
from paper_2107_07315_gb300 import sph

pytestmark = pytest.mark.gpu


def test_monitor_lines_on_a_batch(tmp_path):
    st, eos, met, _ = I.ensemble_state(nstars=6, seed=2107, scale_n=0.02, nr=512)
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, dict(I.DEFAULT_MATERIAL), met, sph.SPH_MIXED,
                       dict(sort_every=4), stream=stream().cuda_stream)
    path = tmp_path / "run.jsonl"
    dt = 0.5 * I.cfl_dt(st, eos)
    assert monitor.run_logged(ctx, dt, 6, 2, str(path), nstars=6) == 4
    recs = [json.loads(l) for l in path.read_text().splitlines()]
    assert [r["step"] for r in recs] == [0, 2, 4, 6]
    m0 = recs[0]["totals"]["mass"]
    assert m0 == pytest.approx(float(np.sum(st["m"])), rel=1e-14)
    for r in recs:
        assert r["totals"]["mass"] == m0
        assert sum(s["mass"] for s in r["stars"]) == pytest.approx(m0, rel=1e-14)
    assert recs[-1]["pairs_last_rhs"] > 0
    sph.sph_free(ctx)
