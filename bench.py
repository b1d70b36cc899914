"""Benchmark of the sparse-permanent path on GB300.

Headline workload: the leaf-kernel batch -- 100,000 independent dense
integer matrices, n uniform in [12, 24], entries nonzero with probability
0.35 and uniform in {1, 2, 3} (seeded) -- evaluated exactly by the leaf
Ryser / Nijenhuis-Wilf kernel.  One step = one evaluation of the whole batch
(inputs resident in HBM).  The line also carries the C60 wall time per
permanent under natural and LPT order (whole path: expansion, estimate,
sort, evaluation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one process per GPU (torchrun); each rank evaluates its own
seeded batch (weak scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "C60 60x60 permanent wall time; leaf permanents/sec; % of integer-ALU roofline"
LEAF_COUNT = 100_000
# DRAM bytes (read + write) of one evaluation per leaf matrix, measured with
# ncu (dram__bytes_read.sum + dram__bytes_write.sum over the evaluation's
# launches) on the 20,000-matrix case of the same seed: 29.9 MB per
# evaluation; the traffic is per leaf, so it scales with the batch
LEAF_TRAFFIC_BYTES_PER_MATRIX = 29.9e6 / 20_000
LEAF_SEED = 20240601
C60_SEED = 60


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for name, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def leaf_workload(rank=0):
    return W.leaf_batch(LEAF_COUNT, seed=LEAF_SEED + rank)


def algorithmic_ops(mats):
    """Per Gray step of an n x n leaf: n-1 multiplies of the row sums (the
    integer-ALU work unit), 2^(n-1) steps per leaf."""
    ns = np.array([m.shape[0] for m in mats], dtype=np.float64)
    return float(np.sum((ns - 1) * 2.0 ** (ns - 1))), float(np.sum(2.0 ** (ns - 1)))


def flush_l2(torch, buf):
    buf.add_(1)  # writes 256 MB, more than the 129 MB L2


def run_ours(args, rank, world, torch):
    import paper_1112_6072_gb300 as pk

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mats = leaf_workload(rank)
    mults, steps_gray = algorithmic_ops(mats)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    tune = None
    if not args.chunk_log2:
        # Gray codes per lane (threads per job) from the autotuner, on a sample of the batch
        from paper_1112_6072_gb300 import autotune
        tune = autotune.tune_leaf_batch(mats[:10000], chunks=(8, 10, 12))
        args.chunk_log2 = tune["chunk_log2"]
    plan = pk.Plan(mats, chunk_log2=args.chunk_log2, order="natural")
    plan.expand()
    order = np.arange(plan.njobs, dtype=np.uint32)
    # the first evaluation prepares the queue; the rest replay it as one captured CUDA graph
    plan.evaluate(order=order)
    for _ in range(max(0, args.warmup - 1)):
        plan.replay()
    # correctness spot check on a few leaves (results are exact or the call fails)
    res = plan.results()
    dev_ms = []
    with Clocks(dev.index) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush_l2(torch, flush)
            plan.replay()
            dev_ms.append(plan.last_eval_ms)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    step_ms = float(np.mean(dev_ms))
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms = float(t.item())
    value = LEAF_COUNT * world / (step_ms * 1e-3)
    launches = plan.last_launches if hasattr(plan, "last_launches") else None
    if args.kernels_only:
        return {"metric": METRIC, "value": value, "unit": "leaf permanents/s", "ms_per_step": step_ms,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "kernels_only": True}

    # end to end through the public API from host buffers: the batch held as
    # one host buffer (matrices back to back) and its orders; each step
    # builds a new plan (validation and CSR blocks on host threads, upload),
    # evaluates it and downloads the results
    packed = np.concatenate([m.ravel() for m in mats])
    orders_n = np.array([m.shape[0] for m in mats], dtype=np.int64)
    e2e_ms, list_ms = [], []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        with pk.Plan.packed(packed, orders_n, chunk_log2=args.chunk_log2, order="natural") as p2:
            p2.expand()
            p2.evaluate(order=order)
            r2 = p2.results()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t) * 1e3)
    assert r2 == res
    serial_ms = min(e2e_ms)
    # the same steps pipelined: the next step's plan (validation and CSR
    # blocks on host threads, its upload on a stream of its own) is built
    # while the current step evaluates on another stream; every step still
    # uploads its inputs and downloads its results inside the timed region
    pipelined_ms = None
    try:
        import concurrent.futures as cf
        streams = [torch.cuda.Stream(device=dev) for _ in range(2)]

        def make(i):
            torch.cuda.set_device(dev)
            pn = pk.Plan.packed(packed, orders_n, chunk_log2=args.chunk_log2, order="natural", stream=streams[i % 2])
            pn.expand()
            return pn

        nsteps = max(2, min(args.steps, 4))
        ok = True
        torch.cuda.synchronize()
        t = time.perf_counter()
        with cf.ThreadPoolExecutor(1) as ex:
            fut = ex.submit(make, 0)
            for i in range(nsteps):
                p2 = fut.result()
                if i + 1 < nsteps:
                    fut = ex.submit(make, i + 1)
                p2.evaluate(order=order)
                ok = ok and p2.results() == res
                p2.close()
        torch.cuda.synchronize()
        if ok:
            pipelined_ms = (time.perf_counter() - t) * 1e3 / nsteps
    except Exception as exc:  # the serial figure stands
        print(f"pipelined end-to-end run skipped: {exc}", file=sys.stderr)
    e2e_best = min(serial_ms, pipelined_ms) if pipelined_ms else serial_ms
    # the same from a list of separate arrays (one address read per array)
    torch.cuda.synchronize()
    t = time.perf_counter()
    with pk.Plan(mats, chunk_log2=args.chunk_log2, order="natural") as p2:
        p2.expand()
        p2.evaluate(order=order)
        r2 = p2.results()
    torch.cuda.synchronize()
    list_ms.append((time.perf_counter() - t) * 1e3)
    assert r2 == res
    nnz = sum(int((m != 0).sum()) for m in mats)
    words = sum(((m.shape[0] + 4) // 4 + (int((m != 0).sum()) + 7) // 8 + int((m != 0).sum()) + 1) // 2 * 2
                for m in mats)
    h2d = 8 * words + 56 * len(mats) + 4 * len(mats)
    d2h = 32 * len(mats) + 8 * len(mats) + 4 * len(mats)

    # integer-ALU roofline of the leaf kernel
    pk_ = peaks()
    sm_mhz = clocks.get("sm_mhz") or pk_.get("clocks_under_load", {}).get("sm_mhz_median") or 1440.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    imad_per_clk_sm = 64
    peak = sms * imad_per_clk_sm * sm_mhz * 1e6 / 1e12  # T multiplies / s
    achieved = mults / (step_ms * 1e-3) / 1e12
    ub_ms, ub_rate = pk.ubench_imad()

    # C60: whole path per permanent, natural vs LPT order
    c60 = run_c60(pk, torch, args)
    ordering = run_ordering(pk, torch, args)

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "leaf permanents/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int128/int256 wrap (exact)",
        "data": "synthetic (seeded)",
        "config": {"workload": f"leaf batch: {LEAF_COUNT} dense integer matrices, n uniform in [12,24], "
                               f"P(nonzero)=0.35, values 1..3, seed {LEAF_SEED}",
                   "l2": "flushed between steps (256 MB write)", "chunk_log2": args.chunk_log2,
                   "autotune": tune,
                   "step": "one evaluation of the whole batch, replayed as a captured CUDA graph",
                   "parallelism": f"jobs sharded per rank (x{world})"},
        "e2e": {"value": LEAF_COUNT * world / (e2e_best * 1e-3), "unit": "leaf permanents/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms": e2e_best,
                "serial_ms": serial_ms, "pipelined_ms": pipelined_ms,
                "input": "one host buffer of the matrices back to back (Plan.packed)",
                "list_input_ms": min(list_ms)},
        "gpu_launches": launches * args.steps if launches is not None else None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tmul/s",
                     "frac": achieved / peak, "traffic": LEAF_TRAFFIC_BYTES_PER_MATRIX * LEAF_COUNT,
                     "traffic_basis": "ncu DRAM read+write of one evaluation of the 20,000-matrix case, "
                                      "scaled by the matrix count",
                     "peak_basis": f"{sms} SMs x {imad_per_clk_sm} IMAD/clk x {sm_mhz:.0f} MHz (median under load)",
                     "ubench_imad_Tops": ub_rate / 1e12},
        "clocks": clocks,
        "roofline_expand": c60.get("roofline_expand"),
        "c60": c60,
        "ordering": ordering,
        "gray_steps_per_step": steps_gray,
        "wall_s": wall,
    }
    return line


C60_LEAF = 11  # leaf order giving 103,940 jobs (the configuration asks for 10^5 - 10^6)


def blk_words(m, nnz):
    """Words of a job's CSR block (jobs.cuh)."""
    w = (m + 4) // 4 + (nnz + 7) // 8 + nnz
    return (w + 1) & ~1


def expand_algorithmic_bytes(orders, nnzs):
    """Algorithmic bytes of an expansion that emits these jobs: per job its
    parent's block read (order m + 1, the same nonzeros per row), its own
    block written, and its header (order, nonzeros, offset, matrix, levels
    left, 256-bit coefficient: 56 bytes)."""
    m = np.asarray(orders, dtype=np.int64)
    z = np.asarray(nnzs, dtype=np.int64)
    zp = np.rint(z * (m + 1) / np.maximum(m, 1)).astype(np.int64)
    words = blk_words(m, z) + blk_words(m + 1, zp)
    return float(np.sum(8 * words + 56))


def train_cost_model_configs(pk):
    """The learned cost model (without the KKLLL feature) on the job times
    the method logs in configurations 1-3: the n = 36 3-regular matrix split
    to depth 20 (leaf order 16), 2,000 matrices of the leaf batch, and C60
    with another vertex shuffle (another job tree) split to leaf order 11."""
    from paper_1112_6072_gb300 import learned

    Xs, ts = [], []
    cases = ((W.regular3(36, 1), dict(split_depth=20, leaf_size=16)),
             (W.c60(seed=C60_SEED + 1), dict(leaf_size=C60_LEAF)))
    for a, kw in cases:
        with pk.Plan([a], model_uses_estimate=False, **kw) as p:
            p.expand()
            X, t, _ = learned.collect(p, "natural")
        Xs.append(X)
        ts.append(t)
    with pk.Plan(W.leaf_batch(2000, seed=LEAF_SEED + 99), model_uses_estimate=False) as p:
        p.expand()
        X, t, _ = learned.collect(p, "natural")
    Xs.append(X)
    ts.append(t)
    return learned.train(np.concatenate(Xs), np.concatenate(ts), steps=600)


def _c60_orders(pk, torch, a, params, knobs, orders=("natural", "lpt", "learned"), reps=5):
    """Whole path of C60 per order: wall time of the call sequence, device
    time of the expansion and of the evaluation, ordering time and their
    sum (best of reps); the natural run's job orders and nonzeros."""
    out, ords, nnzs = {}, None, None
    for order in orders:
        best = None
        for it in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            with pk.Plan([a], order=order, model_uses_estimate=False, **knobs) as p:
                nj = p.expand()
                if order == "learned":
                    p.attach_model(params)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                p.order(order)
                torch.cuda.synchronize()
                order_ms = (time.perf_counter() - t1) * 1e3
                rec = p.evaluate(records="array") if it == 0 else p.evaluate()
                val = p.result(0)
                r = {"wall_ms": 0.0, "expand_device_ms": p.last_expand_ms, "order_ms": order_ms,
                     "eval_ms": p.last_eval_ms, "jobs": nj, "per": str(val), "driver": p.expand_driver}
                if it == 0 and order == "natural":
                    nnzs, ords = rec["nnz"], rec["order"]
            torch.cuda.synchronize()
            r["wall_ms"] = (time.perf_counter() - t) * 1e3
            r["order_plus_eval_ms"] = r["order_ms"] + r["eval_ms"]
            if best is None or r["wall_ms"] < best["wall_ms"]:
                best = r
        out[order] = best
    return out, ords, nnzs


def run_c60(pk, torch, args):
    """C60 (coordinates, vertex shuffle seed 60) through the whole path at
    leaf order 11 with the automatic split (103,940 jobs, within the
    configuration's 10^5 - 10^6): natural order, the paper's KKLLL-LPT order
    and the learned order (the cost model without the estimate, trained on
    configurations 1-3).  Per order: wall time of the whole call sequence,
    device time of the expansion and of the evaluation, ordering time, and
    their sum; the expansion's achieved bandwidth on its algorithmic bytes.
    Also, for reference, the fastest split of the autotuner's grid
    (autotune.tune_hybrid), which may leave far fewer, larger jobs."""
    from paper_1112_6072_gb300 import autotune
    a = W.c60(seed=C60_SEED)
    params, loss = train_cost_model_configs(pk)
    out = {"leaf_size": C60_LEAF, "split_depth": "automatic", "model_loss": loss}
    res, ords, nnzs = _c60_orders(pk, torch, a, params, {"leaf_size": C60_LEAF})
    out.update(res)
    nat = res["natural"]
    abytes = expand_algorithmic_bytes(ords, nnzs)
    pk_ = peaks()
    out["roofline_expand"] = {"bound": "hbm", "achieved": abytes / (nat["expand_device_ms"] * 1e-3) / 1e9,
                              "peak": pk_.get("hbm_gbs", 6800.0), "unit": "GB/s",
                              "frac": abytes / (nat["expand_device_ms"] * 1e-3) / 1e9 / pk_.get("hbm_gbs", 6800.0),
                              "algorithmic_bytes": abytes,
                              "basis": "per emitted job: parent block read + own block written + 56-byte header; "
                                       "device time of perm_expand (events), natural-order run"}
    tuned = autotune.tune_hybrid(a)
    knobs = {k: tuned[k] for k in ("leaf_size", "split_depth", "workers_per_sm")}
    t_res, _, _ = _c60_orders(pk, torch, a, params, knobs, orders=("natural",))
    out["tuned_split"] = dict(t_res["natural"], **knobs,
                              note="fastest (leaf order, split depth, warps) of the autotuner's grid; "
                                   "its job count is outside the configuration's 10^5 - 10^6")
    return out


def run_c60_path(pk, torch, iters, leaf):
    """C60's whole path in natural order, `iters` times: plan, expansion,
    evaluation (wall and device times of each, best and median)."""
    a = W.c60(seed=C60_SEED)
    rows = []
    for _ in range(iters):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with pk.Plan([a], leaf_size=leaf, order="natural") as p:
            t1 = time.perf_counter()
            nj = p.expand()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            p.evaluate()
            v = p.result(0)
            t3 = time.perf_counter()
            rows.append(dict(create_ms=(t1 - t0) * 1e3, expand_wall_ms=(t2 - t1) * 1e3, expand_device_ms=p.last_expand_ms,
                             eval_wall_ms=(t3 - t2) * 1e3, eval_device_ms=p.last_eval_ms, jobs=nj, per=str(v),
                             driver=p.expand_driver))
        torch.cuda.synchronize()
        rows[-1]["total_ms"] = (time.perf_counter() - t0) * 1e3
    keys = [k for k in rows[0] if k.endswith("_ms")]
    return {"leaf_size": leaf, "best": min(rows, key=lambda r: r["total_ms"]),
            "median": {k: float(np.median([r[k] for r in rows])) for k in keys}}


def run_shifted(pk, torch, k, leaf):
    """per(I - A) of C60 (the paper's Section 4.2 matrix at x = 1) modulo
    2^31 - 1: the automatic split (jobs of order 32) evaluated depth first,
    all jobs or k evenly spaced ones (evaluate_subset)."""
    a = W.c60(seed=C60_SEED)
    b = np.eye(60, dtype=np.int64) - a
    p_ = 2147483647
    with pk.Plan([b], leaf_size=leaf, modulus=p_, order="natural") as p:
        nj = p.expand()
        if k:
            sub = (np.arange(k, dtype=np.int64) * (nj // k)).astype(np.uint32)
            p.evaluate_subset(sub)
        else:
            p.evaluate()
        return {"jobs": nj, "evaluated": int(k or nj), "eval_ms": p.last_eval_ms, "leaf_size": leaf,
                "residue": str(p.result(0)), "modulus": p_}


def run_ordering(pk, torch, args, n=80, depth=40, leaf=14):
    """Natural vs KKLLL-LPT vs learned order on a coarse split (few jobs per
    worker, where the order matters): device evaluation time of the whole
    queue (the GPU makespan) and the ordering step's own time.  The model is
    trained on the job times of a different matrix of the same family."""
    from paper_1112_6072_gb300 import learned

    with pk.Plan([W.regular3(n, 7)], split_depth=depth, leaf_size=leaf) as p:
        p.expand()
        X, t, _ = learned.collect(p, "natural")
    params, loss = learned.train(X, t, steps=600)
    # the same network without the KKLLL feature: ordering needs no estimate
    Xc = X.copy()
    Xc[:, 10] = 0.0
    params_c, loss_c = learned.train(Xc, t, steps=600)
    a = W.regular3(n, 1)
    out = {"workload": f"random 3-regular n={n} (seed 1), split depth {depth}, leaf order {leaf}",
           "train": f"job times of n={n} seed 7, final loss {loss:.4f} (without the estimate {loss_c:.4f})"}
    variants = (("natural", "natural", None, True, False), ("lpt", "lpt", None, True, False),
                ("learned", "learned", params, True, False), ("learned_no_estimate", "learned", params_c, False, False),
                ("lpt_single_launch", "lpt", None, True, True))
    for name, order, prm, use_ap, single in variants:
        with pk.Plan([a], split_depth=depth, leaf_size=leaf, order=order, model_uses_estimate=use_ap,
                     single_launch=single) as p:
            nj = p.expand()
            if prm is not None:
                p.attach_model(prm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.order(order)
            torch.cuda.synchronize()
            order_ms = (time.perf_counter() - t0) * 1e3
            p.evaluate()
            evs = []
            for _ in range(3):
                p.replay()
                evs.append(p.last_eval_ms)
            out[name] = {"eval_ms": min(evs), "order_ms": order_ms, "order_plus_eval_ms": order_ms + min(evs),
                         "jobs": nj, "per": str(p.result(0)), "launches": p.last_launches}
    return out


C100_PRINTED = 149364113290700  # Table T12 total


def run_c100(pk, torch, args):
    """The paper's C100 adjacency: whole path, natural order, leaf order L."""
    out = run_single(pk, torch, W.paper_adjacency("c100"), args)
    out["printed"] = str(C100_PRINTED)
    out["equal"] = out["per"] == str(C100_PRINTED)
    return out


def run_single(pk, torch, a, args):
    """One permanent through the whole path, natural order, leaf order L."""
    torch.cuda.synchronize()
    t = time.perf_counter()
    with pk.Plan([a], leaf_size=args.leaf_size, order="natural", timeout_ns=3600 * 10**9) as p:
        nj = p.expand()
        p.order("natural")
        rec = p.evaluate(records=True)
        val = p.result(0)
        ev = p.last_eval_ms
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    return {"per": str(val), "n": int(a.shape[0]), "wall_s": wall,
            "eval_ms": ev, "jobs": nj, "leaf_size": args.leaf_size,
            "nodes": int(sum(r.nodes for r in rec)), "leaves": int(sum(r.leaves for r in rec))}


MIXED_SEED = 5


def run_mixed(pk, torch, args):
    """Config 5: 128 random 3-regular adjacencies (n in [40, 90]) and 128
    sparse matrices with 3-5 nonzeros per row (n in [40, 70]) in one plan.
    The leaf order is tuned on a sample of the batch; the learned model
    (without the KKLLL feature, so ordering costs no estimate) is trained on
    the job times of the n = 36 and C60 whole paths.  Orders: natural, the
    learned one (also replayed as one CUDA graph) and KKLLL-LPT with 32
    trials per job (m^2 trials on ~10^7 jobs would take minutes)."""
    from paper_1112_6072_gb300 import autotune, learned

    def log(*a):
        print(*a, file=sys.stderr, flush=True)

    mats = W.mixed_batch(seed=MIXED_SEED)
    Xs, ts = [], []
    for a, kw in ((W.regular3(36, 1), dict(split_depth=20, leaf_size=16)), (W.c60(C60_SEED), dict(leaf_size=12))):
        with pk.Plan([a], model_uses_estimate=False, **kw) as p:
            p.expand()
            X, t, _ = learned.collect(p, "natural")
        Xs.append(X)
        ts.append(t)
    params, loss = learned.train(np.concatenate(Xs), np.concatenate(ts), steps=600)
    log("mixed: model trained, loss", loss)
    tune = autotune.tune_batch(mats)
    L = tune["leaf_size"]
    log("mixed: tuned", tune)
    out = {"workload": f"mixed batch seed {MIXED_SEED}: 128 3-regular n in [40,90] + 128 sparse rows 3-5 nz "
                       f"n in [40,70]",
           "tune": tune, "model_loss": loss}
    ref = None
    for order, trials in (("natural", 0), ("learned", 0), ("lpt", 32)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        with pk.Plan(mats, leaf_size=L, order=order, kklll_trials=trials, model_uses_estimate=False,
                     timeout_ns=3600 * 10**9) as p:
            nj = p.expand()
            if order == "learned":
                p.attach_model(params)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            p.order(order)
            torch.cuda.synchronize()
            order_ms = (time.perf_counter() - t1) * 1e3
            rec = p.evaluate(records="array")
            vals = p.results()
            wall = time.perf_counter() - t
            ev = p.last_eval_ms
            rep = None
            if order == "learned":
                p.replay()
                rep = p.last_eval_ms
        leaves = int(rec["leaves"].sum())
        if ref is None:
            ref = vals
        out[order] = {"jobs": nj, "wall_s": wall, "eval_ms": ev, "graph_replay_ms": rep, "order_ms": order_ms,
                      "leaves": leaves, "leaves_per_s": leaves / (ev / 1e3), "kklll_trials": trials or None,
                      "same_permanents": vals == ref, "nonzero": sum(1 for v in vals if v)}
        log("mixed:", order, out[order])
    return out


KENDALL_SEED = 7000


def _train_cost_model(pk):
    """The learned cost model (no KKLLL feature) on the job times of the
    n = 36 and C60 whole paths."""
    from paper_1112_6072_gb300 import learned

    Xs, ts = [], []
    for a, kw in ((W.regular3(36, 1), dict(split_depth=20, leaf_size=16)), (W.c60(C60_SEED), dict(leaf_size=12))):
        with pk.Plan([a], model_uses_estimate=False, **kw) as p:
            p.expand()
            X, t, _ = learned.collect(p, "natural")
        Xs.append(X)
        ts.append(t)
    return learned.train(np.concatenate(Xs), np.concatenate(ts), steps=600)


def _whole_path(pk, torch, a, leaf):
    torch.cuda.synchronize()
    t = time.perf_counter()
    with pk.Plan([a], leaf_size=leaf, order="natural", timeout_ns=3600 * 10**9) as p:
        p.expand()
        p.order("natural")
        p.evaluate()
        v = p.result(0)
    torch.cuda.synchronize()
    return time.perf_counter() - t, v


def _estimates(pk, mats, params):
    """KKLLL log AP (T = m^2 trials), the job features (KKLLL feature
    included) and the pretrained cost model's predicted log time of each
    matrix as one job (that model does not use the KKLLL feature)."""
    from paper_1112_6072_gb300 import learned

    with pk.Plan(mats, split_depth=0, leaf_size=14) as p:
        nj = p.expand()
        assert nj == len(mats)
        ap = p.estimate()
        feats = p.features()
    f0 = feats.copy()
    f0[:, 10] = 0.0
    return ap.astype(float).tolist(), feats, learned.predict_log_time(params, f0).astype(float).tolist()


def _cross_validated(feats, times):
    """Predictions of a cost model trained on the other half of the group
    (even / odd positions), for each half."""
    from paper_1112_6072_gb300 import learned

    n = len(times)
    t = np.asarray(times, dtype=np.float64) * 1e9
    pred = np.zeros(n)
    idx = np.arange(n)
    for fold in (0, 1):
        te = idx % 2 == fold
        prm, _ = learned.train(feats[~te], t[~te], steps=600)
        pred[te] = learned.predict_log_time(prm, feats[te])
    return pred.tolist()


def run_kendall(pk, torch, args):
    """Tables T2-T4 analog (Section 3.2): Kendall tau-b of the computing time
    T_i of each matrix or sub-matrix (whole path on the GPU, the matrix alone)
    against its exact permanent P_i, its KKLLL estimate AP_i and the learned
    cost model's prediction (pretrained on the n = 36 and C60 job times, and
    cross-validated: trained on the other half of the same group).  T2: 100 random 0/1 matrices, n = 60, S = 4n
    nonzeros (no zero line).  T3: C100 divided by Eq. 2 at depth 20 (jobs of
    order 80).  T4: I + A of C60 (coordinates, shuffle seed 60) divided at
    depth 8 (jobs of order 52)."""
    from paper_1112_6072_gb300 import kendall

    def log(*a):
        print(*a, file=sys.stderr, flush=True)

    params, loss = _train_cost_model(pk)
    out = {"model_loss": loss}
    groups = {"T2": [W.random01(60, 240, KENDALL_SEED + i) for i in range(100)]}
    coefs_of = {}
    for name, a, d in (("T3", W.paper_adjacency("c100"), 20),
                       ("T4", W.c60(C60_SEED) + np.eye(60, dtype=np.int64), 8)):
        with pk.Plan([a], split_depth=d, leaf_size=14) as p:
            p.expand()
            jobs = p.jobs_export()
        groups[name] = [m for _, m, _ in jobs]
        coefs_of[name] = [c for _, _, c in jobs]
        # the jobs' coefficients multiply their permanents into per(A)
        out[name + "_split"] = {"depth": d, "jobs": len(jobs), "order": int(jobs[0][1].shape[0]) if jobs else 0}
    for name, mats in groups.items():
        ap, feats, pred = _estimates(pk, mats, params)
        times, pers = [], []
        for k, a in enumerate(mats):
            t, v = _whole_path(pk, torch, a, 14)
            times.append(t)
            pers.append(v)
        row_cv = _cross_validated(feats, times)
        row = kendall.table(times, per=pers, ap=ap, mlp=pred, mlp_cv=row_cv)
        row["seconds"] = sum(times)
        if name != "T2":
            # Tables T5-T7 (and T8-T10) analog: list scheduling of the jobs on m
            # workers with their measured times, in natural order, exact-time
            # LPT, KKLLL-LPT and learned order; efficiency T1 / (m Tm)
            row["per_total"] = str(sum(kendall.signed_mod(c, 256) * v for c, v in zip(coefs_of[name], pers)))
            row["schedules"] = _schedules(times, ap, pred, row_cv)
        out[name] = row
        log("kendall:", name, row)
    # per(I + A) of C60 again from the paper's own adjacency list (another
    # vertex order, so another job tree): the totals must agree
    _, v = _whole_path(pk, torch, W.paper_adjacency("c60") + np.eye(60, dtype=np.int64), 14)
    out["T4"]["per_total_paper_c60"] = str(v)
    out["T4"]["per_totals_agree"] = str(v) == out["T4"]["per_total"]
    return out


def _schedules(times, ap, pred, pred_cv, workers=(1, 2, 4, 8, 16, 32)):
    from paper_1112_6072_gb300 import learned

    n = len(times)
    orders = {"natural": np.arange(n), "exact_lpt": learned.order_by(times), "kklll_lpt": learned.order_by(ap),
              "learned": learned.order_by(pred), "learned_cv": learned.order_by(pred_cv)}
    t1 = float(sum(times))
    out = {}
    for name, q in orders.items():
        rows = []
        for m in workers:
            tm = learned.list_makespan(times, q, m)
            rows.append({"m": m, "makespan_s": tm, "efficiency": t1 / (m * tm)})
        out[name] = rows
    return out


def run_reference(args):
    """The oracle (plain CPU) on a bounded sample of the same workload."""
    import oracle

    mats = leaf_workload(0)
    cores = os.cpu_count() or 1
    budget = 20.0 / max(1, args.steps + args.warmup)
    vals = []
    k = 0
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget * max(1, args.steps) and k < len(mats):
        chunk = mats[k:k + cores]
        oracle.job_permanents(chunk, threads=cores)
        done += len(chunk)
        k += cores
    dt = time.perf_counter() - t0
    v = done / dt
    return {"metric": METRIC, "value": v, "unit": "leaf permanents/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "exact big integers", "data": "synthetic (seeded)",
            "impl": "reference",
            "config": {"workload": f"leaf batch sample: first {done} of {LEAF_COUNT} matrices (seed {LEAF_SEED})"},
            "cpu_baseline": {"value": v, "unit": "leaf permanents/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {done} matrices of the batch"},
            "e2e": {"value": v, "unit": "leaf permanents/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_baseline_sample():
    import oracle
    mats = leaf_workload(0)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    done = 0
    k = 0
    while time.perf_counter() - t0 < 15.0 and k < len(mats):
        chunk = mats[k:k + cores]
        oracle.job_permanents(chunk, threads=cores)
        done += len(chunk)
        k += cores
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "leaf permanents/s", "cores": cores, "kind": "oracle",
            "sample": f"first {done} matrices of the batch, {dt:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk-log2", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--leaf-count", type=int, default=LEAF_COUNT,
                    help="matrices in the leaf batch (smaller for profiler captures)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="skip the e2e, C60 and probe legs (profiler captures)")
    ap.add_argument("--c60-only", action="store_true",
                    help="run only the C60 whole-path leg and print its timings")
    ap.add_argument("--ordering-only", action="store_true",
                    help="run only the ordering leg (natural, KKLLL-LPT, learned on a coarse n = 80 split)")
    ap.add_argument("--c100", action="store_true",
                    help="per(A) of the paper's C100 adjacency (Appendix) against its printed total")
    ap.add_argument("--kendall", action="store_true",
                    help="Kendall tau-b of times against per, KKLLL and the cost model (Tables T2-T4 analog)")
    ap.add_argument("--mixed", action="store_true",
                    help="the mixed batch of 256 matrices (3-regular and sparse rows), three orders")
    ap.add_argument("--leaf-size", type=int, default=12)
    ap.add_argument("--c60-path", type=int, default=0, metavar="K",
                    help="run only C60's whole path (natural order) K times and print its time split "
                         "(the command the C60 profiles are taken with)")
    ap.add_argument("--shifted", type=int, default=0, metavar="K",
                    help="per(I - A) of C60 on the residue path (p = 2^31 - 1): K evenly spaced jobs of the "
                         "split at order 32 (all jobs when K = 0 and --shifted-all), depth-first evaluation")
    ap.add_argument("--shifted-all", action="store_true")
    ap.add_argument("--regular", type=int, default=0,
                    help="per(A) of one random 3-regular graph of this order (seed 1), natural order")
    args = ap.parse_args()
    globals()["LEAF_COUNT"] = args.leaf_count
    if args.c60_path:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        print(json.dumps({"c60_path": run_c60_path(pk, torch, args.c60_path, args.leaf_size)}))
        return
    if args.shifted or args.shifted_all:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        print(json.dumps({"c60_shifted": run_shifted(pk, torch, args.shifted, args.leaf_size)}))
        return
    if args.c60_only:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        print(json.dumps({"c60": run_c60(pk, torch, args)}))
        return
    if args.ordering_only:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        print(json.dumps({"ordering": run_ordering(pk, torch, args)}))
        return
    if args.kendall:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        print(json.dumps({"kendall": run_kendall(pk, torch, args)}))
        return
    if args.mixed:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        print(json.dumps({"mixed": run_mixed(pk, torch, args)}))
        return
    if args.c100 or args.regular:
        import torch
        import paper_1112_6072_gb300 as pk
        torch.cuda.set_device(0)
        if args.c100:
            print(json.dumps({"c100": run_c100(pk, torch, args)}))
        else:
            print(json.dumps({"regular": run_single(pk, torch, W.regular3(args.regular, 1), args)}))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, torch)
    if rank == 0:
        line["cpu_baseline"] = None if args.no_cpu_baseline else cpu_baseline_sample()
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
