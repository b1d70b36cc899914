"""Host logic of checkpoint / resume (paper_1112_6072_gb300/checkpoint.py,
no GPU): snapshot round trip, refusal of damaged snapshots and of another
job list, and the per-matrix sums (256-bit with carries, or modulo p)."""
import os

import numpy as np
import pytest

from paper_1112_6072_gb300 import checkpoint as C
from paper_1112_6072_gb300 import dist


def state(n=10, count=3):
    rng = np.random.default_rng(1)
    return {"fingerprint": C.fingerprint(rng.integers(1, 12, n), np.zeros(n), [97] * count),
            "queue": rng.permutation(n).astype(np.uint32), "done": (rng.random(n) < 0.5).astype(np.uint8),
            "sums": rng.integers(0, 2**63, size=(count, 4)).astype(np.uint64), "chunk": 2, "chunks": 5,
            "modulus": 0}


def test_round_trip(tmp_path):
    p = str(tmp_path / "snap")
    st = state()
    C.save(p, st)
    got = C.load(p)
    for k in st:
        assert np.array_equal(np.asarray(got[k]), np.asarray(st[k])), k
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]


def test_damaged_and_foreign_snapshots_are_refused(tmp_path):
    p = str(tmp_path / "snap")
    C.save(p, state())
    raw = bytearray(open(p, "rb").read())
    raw[-20] ^= 0x40
    open(p, "wb").write(bytes(raw))
    with pytest.raises(C.CheckpointError):
        C.load(p)
    open(p, "wb").write(b"short")
    with pytest.raises(C.CheckpointError):
        C.load(p)


def test_fingerprint_tracks_the_job_list():
    o = np.array([11, 11, 10, 9], np.int32)
    m = np.array([0, 0, 1, 1], np.int32)
    f = C.fingerprint(o, m, [97, 97])
    assert f == C.fingerprint(o.copy(), m.copy(), [97, 97])
    assert f != C.fingerprint(o[::-1], m, [97, 97])
    assert f != C.fingerprint(o, m[::-1], [97, 97])
    assert f != C.fingerprint(o, m, [97, 225])
    assert f != C.fingerprint(o, m, [97, 97], modulus=65537)


def test_sums_carry_and_residues():
    a, b = (1 << 200) - 5, -(1 << 130) + 7
    s = C.add_sums(np.array([dist.words_from_int(a)]), np.array([dist.words_from_int(b)]), 0)
    assert dist.int_from_words(s[0]) == a + b
    p = 2147483647
    s = C.add_sums(np.array([[p - 1, 0, 0, 0]], np.uint64), np.array([[5, 0, 0, 0]], np.uint64), p)
    assert s[0].tolist() == [4, 0, 0, 0]


# ---------------------------------------------------------------- chunk logic against a fake plan
class FakePlan:
    """The calls CheckpointedRun makes, over a fixed job list with known
    values; `fault` makes one evaluate_subset call drop a job, run a job
    outside its sub-queue, or report a failed status."""

    REC = np.dtype([("status", np.int32), ("queue_pos", np.int32)])

    def __init__(self, values, mats, counts, fault=None, fault_call=1):
        self.values = [int(v) for v in values]
        self.mats = np.asarray(mats, np.int32)
        self.njobs = len(self.values)
        self._count = counts
        self._desc = {"n": np.full(counts, 5)}
        self._opts = type("O", (), {"modulus": 0})()
        self.fault, self.fault_call, self.calls = fault, fault_call, 0
        self.words = None

    def expand(self):
        return self.njobs

    def job_orders(self):
        return np.full(self.njobs, 7, np.int32), self.mats

    def result_bits(self, i):
        return 200

    def order(self, kind):
        return np.arange(self.njobs, dtype=np.uint32)[::-1].copy()

    def evaluate_subset(self, queue, records=False):
        self.calls += 1
        rec = np.zeros(self.njobs, self.REC)
        rec["status"] = 0
        rec["queue_pos"] = -1
        q = [int(j) for j in queue]
        if self.fault and self.calls == self.fault_call:
            if self.fault == "drop":
                q = q[1:]
            elif self.fault == "extra":
                q = q + [j for j in range(self.njobs) if j not in q][:1]
            elif self.fault == "status":
                rec["status"][q[0]] = 2
        sums = [0] * self._count
        for k, j in enumerate(q):
            rec["queue_pos"][j] = k
            sums[self.mats[j]] += self.values[j]
        self.words = np.array([dist.words_from_int(v) for v in sums])
        return rec

    def result_words(self):
        return self.words


def fake_case():
    rng = np.random.default_rng(4)
    values = [int(v) * (1 << 120) + int(w) for v, w in zip(rng.integers(-9, 9, 23), rng.integers(0, 1 << 62, 23))]
    mats = rng.integers(0, 3, 23)
    want = [sum(v for v, m in zip(values, mats) if m == i) for i in range(3)]
    return values, mats, want


def test_chunks_stop_and_resume_on_a_fake_plan(tmp_path):
    values, mats, want = fake_case()
    path = str(tmp_path / "snap")
    assert C.CheckpointedRun(FakePlan(values, mats, 3), path, chunks=5).run(stop_after=3) is None
    run = C.CheckpointedRun(FakePlan(values, mats, 3), path)
    assert run.state["chunk"] == 3
    assert run.run() == want
    # a finished snapshot gives the same results again without evaluating
    fp = FakePlan(values, mats, 3)
    assert C.CheckpointedRun(fp, path).run() == want and fp.calls == 0


@pytest.mark.parametrize("fault", ["drop", "extra", "status"])
def test_dropped_extra_or_failed_jobs_fail_the_run(tmp_path, fault):
    values, mats, _ = fake_case()
    path = str(tmp_path / "snap")
    run = C.CheckpointedRun(FakePlan(values, mats, 3, fault=fault, fault_call=2), path, chunks=4)
    with pytest.raises(C.CheckpointError):
        run.run()
    # the snapshot holds the chunk before the fault, and a clean restart finishes
    st = C.load(path)
    assert st["chunk"] == 1
    assert C.CheckpointedRun(FakePlan(values, mats, 3), path).run() == fake_case()[2]


def test_another_job_list_is_refused(tmp_path):
    values, mats, _ = fake_case()
    path = str(tmp_path / "snap")
    C.CheckpointedRun(FakePlan(values, mats, 3), path, chunks=4).run(stop_after=1)
    other = np.array(mats)
    other[0] = (other[0] + 1) % 3
    with pytest.raises(C.CheckpointError):
        C.CheckpointedRun(FakePlan(values, other, 3), path)
