"""Host logic of the trajectory tool (paper_2606_03140_gb300.md) without a GPU: the per-step
metric records and the chunking of the run around checkpoints, with the library calls replaced by
a recording stand-in."""
import io
import json

import numpy as np


class _FakeLib:
    def __init__(self):
        self.calls = []

    def sedacs_xlbomd_step(self, ctx, R, V, m, dt, e):
        start = sum(c[1] for c in self.calls if c[0] == "step")
        self.calls.append(("step", m))
        e[:, 0] = np.arange(start, start + m) + 1.0
        e[:, 1] = -2.0
        e[:, 2] = e[:, 0] + e[:, 1]
        return e

    def sedacs_density_info(self, ctx):
        return {"history": [(-0.25, 0.0, 0.0)], "dmu_linear": 0.01, "passes": 2, "count_err": 1e-6}

    def sedacs_checkpoint_save(self, ctx, path):
        done = sum(c[1] for c in self.calls if c[0] == "step")
        self.calls.append(("save", done))


def test_step_records_number_steps_and_carry_diagnostics_on_the_last():
    from paper_2606_03140_gb300 import md

    E = np.array([[1.0, -3.0, -2.0], [1.5, -3.2, -1.7]])
    recs = md.step_records(E, 10, 0.25, {"history": [(-0.2, 0, 0)], "dmu_linear": 0.05, "passes": 1,
                                         "count_err": 2e-7})
    assert [r["step"] for r in recs] == [11, 12] and recs[1]["t_fs"] == 3.0
    assert recs[0]["e_tot_ha"] == -2.0 and "mu_ha" not in recs[0]
    assert abs(recs[1]["mu_ha"] - (-0.15)) < 1e-15 and recs[1]["fermi_evaluations"] == 1


def test_run_chunks_land_on_checkpoints_and_write_one_record_per_step(monkeypatch):
    from paper_2606_03140_gb300 import md

    fake = _FakeLib()
    monkeypatch.setattr(md, "S", fake)
    buf = io.StringIO()
    R = np.zeros((3, 3))
    V = np.zeros((3, 3))
    E = md._md(None, R, V, 23, 0.25, chunk=10, first_step=5, jsonl=buf, ck_path="x.ck", ck_every=8)
    steps = [c[1] for c in fake.calls if c[0] == "step"]
    saves = [c[1] for c in fake.calls if c[0] == "save"]
    # global steps 6..28: chunks end at 8, 16, 24 (checkpoints) and 28
    assert steps == [3, 8, 8, 4] and saves == [3, 11, 19]
    assert np.array_equal(E[:, 0], np.arange(1, 24, dtype=float))
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [x["step"] for x in lines] == list(range(6, 29))
    assert sum("mu_ha" in x for x in lines) == 4
