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
