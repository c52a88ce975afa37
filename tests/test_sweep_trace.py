"""Host logic of the sweep's JSON-lines trace (no GPU: a stand-in context
records the calls)."""
import json


class FakeBatch:
    n = 2

    def __init__(self):
        self.steps = []
        self.t = 0

    def step(self, k):
        self.steps.append(k)
        self.t += k

    def status(self, i):
        return 0 if i == 0 else -4

    def stats(self, i):
        return {"mass": 1.0 + self.t, "mom_x": 0.0, "mom_y": 0.0, "ke": 0.5, "umax": 0.01}


def test_trace_records_every_interval_and_steps_exactly(tmp_path):
    from paper_1412_7228_gb300 import sweep as SW
    path = tmp_path / "trace.jsonl"
    tr = SW.Trace(str(path), 300)
    b = FakeBatch()
    done = SW._advance(b, 1000, 0, tr)
    done = SW._advance(b, 250, done, tr)
    tr.close()
    assert done == 1250 and b.t == 1250
    assert b.steps == [300, 300, 300, 100, 200, 50]   # stops at 300, 600, 900, 1200
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert [(r["step"], r["instance"]) for r in lines] == [(300, 0), (300, 1), (600, 0), (600, 1), (900, 0),
                                                          (900, 1), (1200, 0), (1200, 1)]
    assert lines[0]["mass"] == 301.0 and "mass" not in lines[1] and lines[1]["status"] == -4


def test_advance_without_a_trace_is_one_call():
    from paper_1412_7228_gb300 import sweep as SW
    b = FakeBatch()
    assert SW._advance(b, 777, 23, None) == 800 and b.steps == [777]
