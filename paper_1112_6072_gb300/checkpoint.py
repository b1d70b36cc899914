"""Checkpoint and resume of a long evaluation at job boundaries.

Algorithm PH evaluates independent jobs and sums them (Steps 3-4), so a run
can stop after any set of finished jobs and continue later: the queue is
evaluated in chunks (consecutive queue positions, each chunk one
``perm_eval_subset`` call), and after every chunk a snapshot is written
with

* the job list's fingerprint (job count, every job's order and source
  matrix, the matrices' exact widths and the modulus) -- the expansion is
  deterministic, so a new plan of the same matrices and options gives the
  same list, and a snapshot of another list is refused;
* the queue, the completion bitmap (one byte per job) and the number of
  chunks done;
* the partial sums per matrix: four 64-bit words each, the 256-bit sum of
  the finished jobs' coef * per (residues modulo p on the residue path);
* a SHA-256 of all of the above, so a damaged file is refused.

Each chunk's records are checked before they are counted: every job of the
chunk finished with status 0 and no job outside it ran (a dropped or
repeated job fails the run instead of corrupting the sum).  The snapshot is
written to a temporary file and renamed over the old one, so a crash while
writing leaves the previous snapshot intact.
"""
from __future__ import annotations

import hashlib
import io
import os

import numpy as np

from . import dist

VERSION = 1


class CheckpointError(RuntimeError):
    pass


def fingerprint(orders, mats, bits, modulus: int = 0) -> str:
    """SHA-256 of a job list's shape: job orders and source matrices (int32
    arrays), the per-matrix exact widths and the modulus."""
    h = hashlib.sha256()
    o = np.ascontiguousarray(orders, dtype=np.int32)
    m = np.ascontiguousarray(mats, dtype=np.int32)
    h.update(np.int64(o.size).tobytes())
    h.update(o.tobytes())
    h.update(m.tobytes())
    h.update(np.ascontiguousarray(bits, dtype=np.int32).tobytes())
    h.update(np.int64(modulus).tobytes())
    return h.hexdigest()


def _payload(state: dict) -> bytes:
    buf = io.BytesIO()
    np.savez(buf, version=np.int64(VERSION), fingerprint=np.frombuffer(state["fingerprint"].encode(), np.uint8),
             queue=state["queue"], done=state["done"], sums=state["sums"], chunk=np.int64(state["chunk"]),
             chunks=np.int64(state["chunks"]), modulus=np.int64(state["modulus"]))
    return buf.getvalue()


def save(path: str, state: dict) -> None:
    """Write a snapshot atomically (temporary file, then rename)."""
    body = _payload(state)
    digest = hashlib.sha256(body).digest()
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(digest)
        f.write(body)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path: str) -> dict:
    """Read a snapshot; CheckpointError if it is damaged or of another version."""
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) < 32 or hashlib.sha256(raw[32:]).digest() != raw[:32]:
        raise CheckpointError(f"{path}: checksum mismatch (damaged snapshot)")
    z = np.load(io.BytesIO(raw[32:]))
    if int(z["version"]) != VERSION:
        raise CheckpointError(f"{path}: snapshot version {int(z['version'])}, expected {VERSION}")
    return {"fingerprint": bytes(z["fingerprint"]).decode(), "queue": z["queue"], "done": z["done"].copy(),
            "sums": z["sums"].copy(), "chunk": int(z["chunk"]), "chunks": int(z["chunks"]),
            "modulus": int(z["modulus"])}


def add_sums(sums, words, modulus: int):
    """sums + words per matrix: 256-bit with carries, or modulo p."""
    out = np.array(sums, dtype=np.uint64, copy=True)
    for i in range(out.shape[0]):
        if modulus:
            out[i] = 0
            out[i, 0] = (int(sums[i, 0]) + int(words[i, 0])) % modulus
        else:
            out[i] = dist.combine_words([sums[i], words[i]])
    return out


class CheckpointedRun:
    """Evaluate a plan's queue in `chunks` consecutive sub-queues with a
    snapshot at `path` after each; `run()` resumes from the snapshot when
    one exists (same job list, same queue), else starts afresh."""

    def __init__(self, plan, path: str, chunks: int = 8, order: str = "natural"):
        self.plan = plan
        self.path = path
        self.modulus = int(plan._opts.modulus)
        if plan.njobs == 0:
            plan.expand()
        orders, mats = plan.job_orders()
        self.count = plan._count
        bits = [plan.result_bits(i) for i in range(self.count)]
        self.bits = bits
        self.fp = fingerprint(orders, mats, bits, self.modulus)
        if os.path.exists(path):
            st = load(path)
            if st["fingerprint"] != self.fp:
                raise CheckpointError(f"{path}: snapshot of another job list")
            if st["modulus"] != self.modulus or st["sums"].shape != (self.count, 4):
                raise CheckpointError(f"{path}: snapshot of another plan")
            self.state = st
        else:
            q = np.asarray(plan.order(order), dtype=np.uint32)
            self.state = {"fingerprint": self.fp, "queue": q, "done": np.zeros(plan.njobs, np.uint8),
                          "sums": np.zeros((self.count, 4), np.uint64), "chunk": 0, "chunks": int(chunks),
                          "modulus": self.modulus}

    def _bounds(self, c):
        n = len(self.state["queue"])
        k = self.state["chunks"]
        return (n * c) // k, (n * (c + 1)) // k

    def run(self, stop_after: int | None = None):
        """Evaluate the remaining chunks (at most stop_after of them); the
        final results (as Plan.results) once every chunk is done, else None."""
        st = self.state
        ran = 0
        while st["chunk"] < st["chunks"]:
            if stop_after is not None and ran >= stop_after:
                return None
            lo, hi = self._bounds(st["chunk"])
            sub = st["queue"][lo:hi]
            if sub.size:
                rec = self.plan.evaluate_subset(sub, records="array")
                inside = np.zeros(self.plan.njobs, bool)
                inside[sub] = True
                if (rec["status"][sub] != 0).any() or (rec["queue_pos"][sub] < 0).any():
                    raise CheckpointError(f"chunk {st['chunk']}: a job did not finish")
                if (rec["queue_pos"][~inside] >= 0).any():
                    raise CheckpointError(f"chunk {st['chunk']}: a job outside the chunk ran")
                if st["done"][sub].any():
                    raise CheckpointError(f"chunk {st['chunk']}: a job ran twice")
                st["sums"] = add_sums(st["sums"], self.plan.result_words(), self.modulus)
                st["done"][sub] = 1
            st["chunk"] += 1
            save(self.path, st)
            ran += 1
        if not st["done"].all():
            raise CheckpointError("finished with jobs not done")
        return self.results()

    def results(self):
        """Per-matrix results from the summed words (exact in result_bits
        bits; residues on the residue path).  A matrix without jobs has
        per = 1 (order 0) or 0 (a zero line)."""
        out = []
        for i in range(self.count):
            w = self.state["sums"][i]
            if self.modulus:
                out.append(int(w[0]) % self.modulus)
            else:
                out.append(dist.int_from_words(w, self.bits[i]))
        _, mats = self.plan.job_orders()
        has_jobs = np.zeros(self.count, bool)
        has_jobs[np.asarray(mats, dtype=np.int64)] = True
        orders = np.asarray(self.plan._desc["n"])
        for i in range(self.count):
            if not has_jobs[i]:
                out[i] = 1 if int(orders[i]) == 0 else 0
        return out
