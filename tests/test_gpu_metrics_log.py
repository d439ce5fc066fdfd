"""Per-solve metrics log: one JSON line per solve with cycles, the relative
residual after each cycle, time, algorithmic bytes and bandwidth.  The
logged residual history of an FMG solve is checked cycle by cycle against
the CPU oracle's FMG stopped after 1, 2, ... cycles."""
import json

import pytest

import oracle
from helpers import load_inputs, pair

pytestmark = pytest.mark.gpu
PEAK = 6796.5


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_metrics_log_lines(tmp_path):
    dom, st, o, g = pair("streamer_small")
    load_inputs(dom, st, o, g)
    path = tmp_path / "solves.jsonl"
    g.set_metrics_log(str(path), PEAK)
    rc1, rel1, c1 = g.fmg(1e-8, 30)
    g.set_graphs(False)
    rc2, rel2, c2 = g.solve(1e-10, 30)
    g.set_graphs(True)
    g.set_metrics_log(None)
    g.fmg(1e-8, 30)  # not logged
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2
    a, b = lines
    assert (a["seq"], a["call"], a["precision"], a["path"]) == (1, "fmg", "fp64", "graph")
    assert (b["seq"], b["call"], b["path"]) == (2, "solve", "host")
    for ln, rc, rel, c in ((a, rc1, rel1, c1), (b, rc2, rel2, c2)):
        assert ln["status"] == rc == 0 and ln["cycles"] == c and ln["rel"] == rel
        h = ln["residual_history"]
        assert len(h) == c and h[-1] == rel
        assert all(h[i + 1] < h[i] for i in range(c - 1))
        assert ln["leaf_cells"] == 512 * int((o.tables()["child"][:, 0] < 0).sum())
        assert ln["bytes"] == pytest.approx(ln["vcycle_bytes"] * c, rel=1e-12)
        assert ln["ms"] > 0 and ln["gbs"] == pytest.approx(ln["bytes"] / (ln["ms"] * 1e-3) / 1e9, rel=1e-9)
        assert ln["hbm_frac"] == pytest.approx(ln["gbs"] / PEAK, rel=1e-9)
    assert a["tol"] == 1e-8 and b["tol"] == 1e-10
    # the FMG history, cycle by cycle, against the oracle's FMG of k cycles
    for k, r in enumerate(a["residual_history"], start=1):
        _, rel_o, c_o = o.fmg(0.0, k)
        assert c_o == k
        assert r == pytest.approx(rel_o, rel=1e-6)


def test_metrics_log_bad_path_is_an_error(tmp_path):
    dom, st, o, g = pair("streamer_small")
    import paper_1708_08434_gb300 as pkg
    with pytest.raises(pkg.SmError):
        g.set_metrics_log(str(tmp_path / "no_such_dir" / "x.jsonl"))
