"""Python binding of libperm.so (include/perm.h): exact permanents of sparse
integer matrices on one GB300 by the parallel hybrid method of Wang, Liang,
Bai and Huo (arXiv 1112.6072).

The binding only marshals arguments: every step of the computation runs in
the library's CUDA kernels.  PyTorch, when present, supplies the CUDA stream
and (optionally) the device memory through its caching allocator.  Importing
this package does not build anything; if the shared library is missing every
call raises ``PermError`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libperm.so")

MAX_N = 128
MAX_JOB_N = 64
MAX_LEAF = 32
MLP_FEATURES = 12
MLP_HIDDEN = 64
MLP_PARAMS = 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1

ORDER = {"natural": 0, "lpt": 1, "learned": 2}
STATUS = {0: "ok", 1: "invalid argument", 2: "overflow", 3: "timeout", 4: "cuda error",
          5: "short buffer", 6: "out of memory", 7: "out of sequence"}

EXPORTED = [
    "perm_opts_default", "perm_plan_create", "perm_plan_destroy", "perm_expand", "perm_estimate",
    "perm_order", "perm_eval_batch", "perm_last_eval_ms", "perm_last_eval_launches", "perm_result", "perm_result_bits",
    "perm_result_words", "perm_jobs_export", "perm_exact", "perm_job_features", "perm_mlp_grad",
    "perm_mlp_train", "perm_mlp_predict", "perm_mlp_attach", "perm_ubench_imad",
    "perm_status_string", "perm_last_error", "perm_leaf_batch_noalloc", "perm_eval_replay",
    "perm_eval_subset", "perm_jobs_select", "perm_expand_driver", "perm_last_expand_ms", "perm_crt",
]


class PermError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        try:
            extra = _lib().perm_last_error().decode()
            if extra and status == 4:
                msg += f" ({extra})"
        except Exception:
            pass
        super().__init__(msg)


alloc_fn_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
free_fn_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class perm_matrix(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("a", ctypes.POINTER(ctypes.c_int64)), ("ld", ctypes.c_int64)]


_MATRIX_DTYPE = np.dtype([("n", np.int32), ("a", np.uintp), ("ld", np.int64)], align=True)


class perm_opts(ctypes.Structure):
    _fields_ = [("split_depth", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("order", ctypes.c_int32),
                ("kklll_trials", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("workers_per_sm", ctypes.c_int32), ("chunk_log2", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("alloc", alloc_fn_t), ("free", free_fn_t),
                ("alloc_ctx", ctypes.c_void_p), ("timeout_ns", ctypes.c_int64),
                ("model_uses_estimate", ctypes.c_int32), ("fused_levels", ctypes.c_int32),
                ("dense_split", ctypes.c_int32), ("expand_walk", ctypes.c_int32),
                ("modulus", ctypes.c_uint32), ("single_launch", ctypes.c_int32)]


class perm_job_result(ctypes.Structure):
    _fields_ = [("matrix", ctypes.c_int32), ("order", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("status", ctypes.c_int32), ("value", ctypes.c_uint64 * 4), ("t_start_ns", ctypes.c_int64),
                ("t_end_ns", ctypes.c_int64), ("sm", ctypes.c_int32), ("queue_pos", ctypes.c_int32),
                ("leaves", ctypes.c_int64), ("nodes", ctypes.c_int64)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise PermError(4, "libperm.so is not built (call __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.perm_opts_default.argtypes = [P(perm_opts)]
        lib.perm_opts_default.restype = None
        lib.perm_plan_create.argtypes = [P(perm_matrix), ctypes.c_int32, P(perm_opts), P(vp)]
        lib.perm_plan_destroy.argtypes = [vp]
        lib.perm_plan_destroy.restype = None
        lib.perm_expand.argtypes = [vp, P(vp), P(ctypes.c_int64)]
        lib.perm_estimate.argtypes = [vp, P(ctypes.c_float)]
        lib.perm_expand_driver.argtypes = [vp, P(ctypes.c_int32)]
        lib.perm_last_expand_ms.argtypes = [vp, P(ctypes.c_float)]
        lib.perm_order.argtypes = [vp, ctypes.c_int32, P(ctypes.c_uint32)]
        lib.perm_eval_batch.argtypes = [vp, P(ctypes.c_uint32), P(perm_job_result)]
        lib.perm_eval_replay.argtypes = [vp, P(perm_job_result)]
        lib.perm_eval_subset.argtypes = [vp, P(ctypes.c_uint32), ctypes.c_int64, P(perm_job_result)]
        lib.perm_last_eval_ms.argtypes = [vp, P(ctypes.c_float)]
        lib.perm_last_eval_launches.argtypes = [vp, P(ctypes.c_int32)]
        lib.perm_result.argtypes = [vp, ctypes.c_int32, P(ctypes.c_uint32), ctypes.c_int32,
                                    P(ctypes.c_int32), P(ctypes.c_int32)]
        lib.perm_result_bits.argtypes = [vp, ctypes.c_int32, P(ctypes.c_int32)]
        lib.perm_result_words.argtypes = [vp, P(ctypes.c_uint64), ctypes.c_int32]
        lib.perm_jobs_export.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int64),
                                         P(ctypes.c_uint64), P(ctypes.c_int32)]
        lib.perm_exact.argtypes = [P(perm_matrix), P(perm_opts), P(ctypes.c_uint32), ctypes.c_int32,
                                   P(ctypes.c_int32), P(ctypes.c_int32)]
        lib.perm_jobs_select.argtypes = [vp, P(ctypes.c_int64), ctypes.c_int64, P(ctypes.c_int32),
                                         P(ctypes.c_int64), ctypes.c_int64, P(ctypes.c_uint64),
                                         P(ctypes.c_int32), P(ctypes.c_int64)]
        lib.perm_job_features.argtypes = [vp, P(ctypes.c_float)]
        f = P(ctypes.c_float)
        lib.perm_mlp_grad.argtypes = [f, f, f, ctypes.c_int32, vp, f, f]
        lib.perm_mlp_train.argtypes = [f, f, f, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, vp, f]
        lib.perm_mlp_predict.argtypes = [f, f, ctypes.c_int32, vp, f]
        lib.perm_mlp_attach.argtypes = [vp, f]
        lib.perm_ubench_imad.argtypes = [ctypes.c_int32, ctypes.c_int32, vp, f, P(ctypes.c_double)]
        lib.perm_leaf_batch_noalloc.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp]
        lib.perm_crt.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), ctypes.c_int32, ctypes.c_int32,
                                 P(ctypes.c_uint32), P(ctypes.c_int32), vp]
        lib.perm_status_string.argtypes = [ctypes.c_int]
        lib.perm_status_string.restype = ctypes.c_char_p
        lib.perm_last_error.argtypes = []
        lib.perm_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            fn = getattr(lib, name)
            if name not in ("perm_opts_default", "perm_plan_destroy", "perm_status_string", "perm_last_error"):
                fn.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _ck(st, where):
    if st != 0:
        raise PermError(st, where)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _stream_handle(stream):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self._a = alloc_fn_t(self._alloc)
        self._f = free_fn_t(self._free)

    def _alloc(self, nbytes, stream, ctx):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.dev, stream or 0))
        except Exception:
            return None

    def _free(self, ptr, stream, ctx):
        if ptr:
            self.torch.cuda.caching_allocator_delete(ptr)


def _limbs_to_int(limbs, n, sign):
    v = 0
    for k in range(n - 1, -1, -1):
        v = (v << 32) | int(limbs[k])
    return -v if sign < 0 else v


def _words_to_int(words):
    v = 0
    for k in range(3, -1, -1):
        v = (v << 64) | int(words[k])
    return v


@dataclass
class JobRecord:
    matrix: int
    order: int
    nnz: int
    status: int
    value_mod: int      # coef * per(job) modulo 2^256
    t_start_ns: int
    t_end_ns: int
    sm: int
    queue_pos: int
    leaves: int
    nodes: int


def packed_descriptors(data, orders):
    """(buffer, perm_matrix records) for matrices stored back to back in one
    int64 buffer: record i has n = orders[i], ld = max(n, 1) and the address
    of data[off_i], off_i the sum of the earlier orders squared.  The buffer
    returned is the contiguous int64 array the addresses point into (the
    input itself when it already is one)."""
    data = np.asarray(data)
    if data.dtype != np.int64 or not data.flags.c_contiguous:
        data = np.ascontiguousarray(data, dtype=np.int64)
    data = data.reshape(-1)
    orders = np.asarray(orders, dtype=np.int64).reshape(-1)
    if orders.size == 0 or (orders < 0).any():
        raise ValueError("orders must be non-negative, at least one matrix")
    sizes = orders * orders
    off = np.zeros(orders.size, dtype=np.int64)
    np.cumsum(sizes[:-1], out=off[1:])
    if int(off[-1] + sizes[-1]) != data.size:
        raise ValueError("data must hold exactly the matrices, back to back")
    desc = np.zeros(orders.size, dtype=_MATRIX_DTYPE)
    desc["n"] = orders
    desc["a"] = np.uint64(data.__array_interface__["data"][0]) + (8 * off).astype(np.uint64)
    desc["ld"] = np.maximum(orders, 1)
    return data, desc


class Plan:
    """A batch of matrices through the whole path: expand, order, evaluate.

    Options mirror ``perm_opts`` in include/perm.h.
    """

    def __init__(self, mats, **opts):
        mats = [np.ascontiguousarray(np.asarray(m, dtype=np.int64)) for m in mats]
        for m in mats:
            if m.ndim != 2 or m.shape[0] != m.shape[1]:
                raise ValueError("square matrices expected")
        # the perm_matrix descriptors, built as one numpy record array (a
        # ctypes loop costs about 4 us per matrix, reading each array's
        # address about 1 us: Plan.packed avoids both)
        desc = np.zeros(len(mats), dtype=_MATRIX_DTYPE)
        desc["n"] = [m.shape[0] for m in mats]
        desc["a"] = [m.__array_interface__["data"][0] for m in mats]
        desc["ld"] = np.maximum(desc["n"], 1)
        self._create(desc, mats, **opts)

    @classmethod
    def packed(cls, data, orders, **opts):
        """A plan over matrices stored back to back in one int64 buffer:
        matrix i, of order orders[i], is data[off_i : off_i + orders[i]**2]
        in row-major order, off_i the sum of the earlier orders squared.
        The descriptors come from one prefix sum.  Options as for Plan."""
        data, desc = packed_descriptors(data, orders)
        obj = cls.__new__(cls)
        obj._create(desc, data, **opts)
        return obj

    def _create(self, desc, keep, split_depth=-1, leaf_size=0, order="lpt", kklll_trials=0, seed=0x5EED,
                workers_per_sm=0, chunk_log2=0, stream=None, torch_allocator=False, timeout_ns=0,
                model_uses_estimate=True, fused_levels=True, dense_split=False, expand_walk=True, modulus=0,
                single_launch=False):
        lib = _lib()
        self._h = None
        self._keep = keep  # the host matrices the descriptors point into
        self._count = len(desc)
        self._desc = desc
        arr = (perm_matrix * len(desc)).from_buffer(desc)
        o = perm_opts()
        lib.perm_opts_default(ctypes.byref(o))
        o.split_depth = int(split_depth)
        o.leaf_size = int(leaf_size)
        o.order = ORDER[order] if isinstance(order, str) else int(order)
        o.kklll_trials = int(kklll_trials)
        o.seed = int(seed) & ((1 << 64) - 1)
        o.workers_per_sm = int(workers_per_sm)
        o.chunk_log2 = int(chunk_log2)
        o.stream = _stream_handle(stream)
        o.timeout_ns = int(timeout_ns)
        o.model_uses_estimate = 1 if model_uses_estimate else 0
        o.fused_levels = 1 if fused_levels else 0
        o.dense_split = 1 if dense_split else 0
        o.expand_walk = 1 if expand_walk else 0
        o.modulus = int(modulus)
        o.single_launch = 1 if single_launch else 0
        self._alloc = None
        if torch_allocator:
            self._alloc = _TorchAllocator()
            o.alloc = self._alloc._a
            o.free = self._alloc._f
        self._opts = o
        self._stream = o.stream
        h = ctypes.c_void_p()
        _ck(lib.perm_plan_create(arr, len(desc), ctypes.byref(o), ctypes.byref(h)), "perm_plan_create")
        self._h = h
        self._jobs = None
        self.njobs = 0

    # a2, a3
    def expand(self) -> int:
        j = ctypes.c_void_p()
        n = ctypes.c_int64()
        _ck(_lib().perm_expand(self._h, ctypes.byref(j), ctypes.byref(n)), "perm_expand")
        self._jobs = j
        self.njobs = n.value
        return self.njobs

    @property
    def expand_driver(self) -> str:
        """Driver of the last expansion: "levels", "fused" or "walk"."""
        v = ctypes.c_int32()
        _ck(_lib().perm_expand_driver(self._h, ctypes.byref(v)), "perm_expand_driver")
        return ("levels", "fused", "walk")[v.value]

    def _need_jobs(self):
        if self._jobs is None:
            self.expand()

    # a4
    def estimate(self) -> np.ndarray:
        self._need_jobs()
        out = np.zeros(max(self.njobs, 1), dtype=np.float32)
        _ck(_lib().perm_estimate(self._jobs, _fptr(out)), "perm_estimate")
        return out[:self.njobs]

    # a5, a6
    def order(self, kind="lpt") -> np.ndarray:
        self._need_jobs()
        out = np.zeros(max(self.njobs, 1), dtype=np.uint32)
        k = ORDER[kind] if isinstance(kind, str) else int(kind)
        _ck(_lib().perm_order(self._jobs, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
            "perm_order")
        return out[:self.njobs]

    def features(self) -> np.ndarray:
        self._need_jobs()
        out = np.zeros((max(self.njobs, 1), MLP_FEATURES), dtype=np.float32)
        _ck(_lib().perm_job_features(self._jobs, _fptr(out)), "perm_job_features")
        return out[:self.njobs]

    def attach_model(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_PARAMS:
            raise ValueError("parameter count")
        _ck(_lib().perm_mlp_attach(self._h, _fptr(p)), "perm_mlp_attach")

    # a7, a8
    def evaluate(self, order=None, records=False):
        self._need_jobs()
        lib = _lib()
        optr = None
        if order is not None:
            oa = np.ascontiguousarray(order, dtype=np.uint32)
            if oa.size != self.njobs:
                raise ValueError("order must be a permutation of the jobs")
            optr = oa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        res = (perm_job_result * max(self.njobs, 1))() if records else None
        _ck(lib.perm_eval_batch(self._jobs, optr, res), "perm_eval_batch")
        return self._records(res, records)

    def evaluate_subset(self, queue, records=False):
        """Evaluate only the jobs in ``queue`` (distinct job indices, in that
        order); ``results()`` then holds each matrix's sum over those jobs,
        modulo 2^K (see ``result_bits``).  Disjoint sub-queues covering every
        job sum to the permanents (one GPU each, Algorithm PH, Steps 3-4)."""
        self._need_jobs()
        qa = np.ascontiguousarray(queue, dtype=np.uint32).reshape(-1)
        res = (perm_job_result * max(self.njobs, 1))() if records else None
        _ck(_lib().perm_eval_subset(self._jobs, qa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), qa.size, res),
            "perm_eval_subset")
        return self._records(res, records)

    def result_words(self) -> np.ndarray:
        """Each matrix's result as four little-endian uint64 words (mod 2^256,
        exact in its low result_bits(i) bits)."""
        c = self._count
        w = np.zeros(4 * c, dtype=np.uint64)
        _ck(_lib().perm_result_words(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), c),
            "perm_result_words")
        return w.reshape(c, 4)

    def replay(self, records=False):
        """Repeat the last evaluation as a captured CUDA graph."""
        res = (perm_job_result * max(self.njobs, 1))() if records else None
        _ck(_lib().perm_eval_replay(self._jobs, res), "perm_eval_replay")
        return self._records(res, records)

    def _records(self, res, records):
        """records=True: a list of JobRecord; records="array": the raw
        perm_job_result array as a numpy structured array (fields as in
        include/perm.h; value holds the four little-endian words)."""
        if not records:
            return None
        if records == "array":
            return np.ctypeslib.as_array(res)[:self.njobs].copy()
        return [JobRecord(r.matrix, r.order, r.nnz, r.status, _words_to_int(r.value), r.t_start_ns,
                          r.t_end_ns, r.sm, r.queue_pos, r.leaves, r.nodes) for r in res[:self.njobs]]

    @property
    def last_eval_ms(self) -> float:
        v = ctypes.c_float()
        _ck(_lib().perm_last_eval_ms(self._h, ctypes.byref(v)), "perm_last_eval_ms")
        return v.value

    @property
    def last_expand_ms(self) -> float:
        """Device time of the last expansion (ms)."""
        v = ctypes.c_float()
        _ck(_lib().perm_last_expand_ms(self._h, ctypes.byref(v)), "perm_last_expand_ms")
        return v.value

    @property
    def last_launches(self) -> int:
        v = ctypes.c_int32()
        _ck(_lib().perm_last_eval_launches(self._h, ctypes.byref(v)), "perm_last_eval_launches")
        return v.value

    def result_bits(self, i) -> int:
        b = ctypes.c_int32()
        _ck(_lib().perm_result_bits(self._h, int(i), ctypes.byref(b)), "perm_result_bits")
        return b.value

    def result(self, i) -> int:
        limbs = (ctypes.c_uint32 * 16)()
        n, s = ctypes.c_int32(), ctypes.c_int32()
        _ck(_lib().perm_result(self._h, int(i), limbs, 16, ctypes.byref(n), ctypes.byref(s)), "perm_result")
        return _limbs_to_int(limbs, n.value, s.value)

    def results(self):
        c = self._count
        w = np.zeros(4 * c, dtype=np.uint64)
        _ck(_lib().perm_result_words(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), c),
            "perm_result_words")
        w = w.reshape(c, 4)
        # values that fit int64 (the upper words repeat the sign) convert in bulk
        lo = w[:, 0].view(np.int64)
        ext = np.where(lo < 0, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
        small = (w[:, 1] == ext) & (w[:, 2] == ext) & (w[:, 3] == ext)
        out = lo.tolist()
        for i in np.flatnonzero(~small).tolist():
            v = _words_to_int(w[i])
            out[i] = v - (1 << 256) if v >> 255 else v
        return out

    def job_coefs(self):
        """Orders, coefficients (Python ints, mod 2^256) and source matrices
        of the jobs, without the dense job matrices."""
        self._need_jobs()
        lib = _lib()
        tot = ctypes.c_int64()
        n = self.njobs
        sizes = np.zeros(max(n, 1), dtype=np.int32)
        coef = np.zeros(4 * max(n, 1), dtype=np.uint64)
        mid = np.zeros(max(n, 1), dtype=np.int32)
        _ck(lib.perm_jobs_export(self._jobs, ctypes.byref(tot),
                                 sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None,
                                 coef.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 mid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "perm_jobs_export")
        return sizes[:n].copy(), [_words_to_int(coef[4 * j:4 * j + 4]) for j in range(n)], mid[:n].copy()

    def job_orders(self):
        """(order, source matrix) of every job as two int32 arrays."""
        self._need_jobs()
        n = self.njobs
        tot = ctypes.c_int64()
        sizes = np.zeros(max(n, 1), dtype=np.int32)
        mid = np.zeros(max(n, 1), dtype=np.int32)
        _ck(_lib().perm_jobs_export(self._jobs, ctypes.byref(tot),
                                    sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, None,
                                    mid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "perm_jobs_export")
        return sizes[:n].copy(), mid[:n].copy()

    def jobs_select(self, idx):
        """Chosen jobs as (matrix index, dense job, coefficient mod 2^256)."""
        self._need_jobs()
        lib = _lib()
        ia = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1)
        k = ia.size
        sizes = np.zeros(max(k, 1), dtype=np.int32)
        coef = np.zeros(4 * max(k, 1), dtype=np.uint64)
        mid = np.zeros(max(k, 1), dtype=np.int32)
        ent = ctypes.c_int64()
        ip = ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        _ck(lib.perm_jobs_select(self._jobs, ip, k, sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, 0,
                                 None, None, ctypes.byref(ent)), "perm_jobs_select")
        mats = np.zeros(max(ent.value, 1), dtype=np.int64)
        _ck(lib.perm_jobs_select(self._jobs, ip, k, sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 mats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ent.value,
                                 coef.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 mid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(ent)),
            "perm_jobs_select")
        out, off = [], 0
        for j in range(k):
            m = int(sizes[j])
            out.append((int(mid[j]), mats[off:off + m * m].reshape(m, m).copy(), _words_to_int(coef[4 * j:4 * j + 4])))
            off += m * m
        return out

    def jobs_export(self):
        """The job list as (matrix index, dense job, coefficient mod 2^256)."""
        self._need_jobs()
        lib = _lib()
        tot = ctypes.c_int64()
        _ck(lib.perm_jobs_export(self._jobs, ctypes.byref(tot), None, None, None, None), "perm_jobs_export")
        n = self.njobs
        sizes = np.zeros(max(n, 1), dtype=np.int32)
        mats = np.zeros(max(tot.value, 1), dtype=np.int64)
        coef = np.zeros(4 * max(n, 1), dtype=np.uint64)
        mid = np.zeros(max(n, 1), dtype=np.int32)
        _ck(lib.perm_jobs_export(self._jobs, ctypes.byref(tot),
                                 sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 mats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 coef.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 mid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "perm_jobs_export")
        out, off = [], 0
        for j in range(n):
            m = int(sizes[j])
            out.append((int(mid[j]), mats[off:off + m * m].reshape(m, m).copy(),
                        _words_to_int(coef[4 * j:4 * j + 4])))
            off += m * m
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib().perm_plan_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def permanent(a, **opts) -> int:
    """per(A) of one integer matrix (perm_exact)."""
    lib = _lib()
    m = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    pm = perm_matrix(m.shape[0], m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), max(m.shape[0], 1))
    o = perm_opts()
    lib.perm_opts_default(ctypes.byref(o))
    for k, v in opts.items():
        if k == "order":
            v = ORDER[v] if isinstance(v, str) else int(v)
        setattr(o, k, v)
    if not opts.get("stream"):
        o.stream = _stream_handle(None)
    limbs = (ctypes.c_uint32 * 16)()
    n, s = ctypes.c_int32(), ctypes.c_int32()
    _ck(lib.perm_exact(ctypes.byref(pm), ctypes.byref(o), limbs, 16, ctypes.byref(n), ctypes.byref(s)),
        "perm_exact")
    return _limbs_to_int(limbs, n.value, s.value)


def mlp_grad(params, feats, target, stream=None):
    """Loss and gradient of the cost network on a batch (device kernels)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(feats, dtype=np.float32)
    y = np.ascontiguousarray(target, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _ck(_lib().perm_mlp_grad(_fptr(p), _fptr(x), _fptr(y), len(y), _stream_handle(stream), _fptr(loss),
                             _fptr(g)), "perm_mlp_grad")
    return float(loss[0]), g


def mlp_train(params, feats, target, steps=500, lr=3e-3, stream=None):
    p = np.array(params, dtype=np.float32, copy=True)
    x = np.ascontiguousarray(feats, dtype=np.float32)
    y = np.ascontiguousarray(target, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _ck(_lib().perm_mlp_train(_fptr(p), _fptr(x), _fptr(y), len(y), int(steps), float(lr),
                              _stream_handle(stream), _fptr(loss)), "perm_mlp_train")
    return p, float(loss[0])


def mlp_predict(params, feats, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(feats, dtype=np.float32)
    out = np.zeros(len(x), dtype=np.float32)
    _ck(_lib().perm_mlp_predict(_fptr(p), _fptr(x), len(x), _stream_handle(stream), _fptr(out)),
        "perm_mlp_predict")
    return out


def mlp_init(seed=0):
    """Seeded He-style initial parameters of the cost network (host data)."""
    rng = np.random.default_rng(seed)
    F, H = MLP_FEATURES, MLP_HIDDEN
    w1 = rng.normal(0, (2.0 / F) ** 0.5, size=(H, F))
    w2 = rng.normal(0, (2.0 / H) ** 0.5, size=(H, H))
    w3 = rng.normal(0, (1.0 / H) ** 0.5, size=H)
    return np.concatenate([w1.ravel(), np.zeros(H), w2.ravel(), np.zeros(H), w3, np.zeros(1)]).astype(np.float32)


def ubench_imad(blocks=152 * 8, iters=4096, stream=None):
    ms = ctypes.c_float()
    rate = ctypes.c_double()
    _ck(_lib().perm_ubench_imad(int(blocks), int(iters), _stream_handle(stream), ctypes.byref(ms),
                                ctypes.byref(rate)), "perm_ubench_imad")
    return ms.value, rate.value


def leaf_batch_noalloc(a_ptr, n, count, out_ptr, status_ptr, stream=None):
    """Allocation-free leaf batch (perm_leaf_batch_noalloc): for callers that
    cannot allocate device memory while they run -- a host framework whose
    allocator owns every device allocation, or a loop that may not allocate
    after start-up.  All pointers are device addresses the caller owns: ``count``
    row-major int64 n x n matrices, ``count * 4`` uint64 result words (256-bit
    two's complement) and ``count`` int32 statuses.  The work is only
    enqueued on the stream; calls whose work overlaps on the GPU race on the
    library's one scratch array, so issue them in order on one stream."""
    _ck(_lib().perm_leaf_batch_noalloc(ctypes.c_void_p(int(a_ptr)), int(n), int(count),
                                       ctypes.c_void_p(int(out_ptr)), ctypes.c_void_p(int(status_ptr)),
                                       ctypes.c_void_p(_stream_handle(stream))), "perm_leaf_batch_noalloc")


def crt(residues, primes, stream=None):
    """Integers from their residues (perm_crt): residues[v][i] is value v
    modulo primes[i] (distinct odd primes below 2^31); every value of
    absolute value below half the product of the primes comes back exactly
    (the balanced residue)."""
    pr = np.ascontiguousarray(primes, dtype=np.uint32).reshape(-1)
    k = pr.size
    r = np.ascontiguousarray(residues, dtype=np.uint32).reshape(-1, k)
    count = r.shape[0]
    limbs = np.zeros((count, k + 1), dtype=np.uint32)
    signs = np.zeros(count, dtype=np.int32)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    _ck(_lib().perm_crt(r.ctypes.data_as(u32), pr.ctypes.data_as(u32), k, count, limbs.ctypes.data_as(u32),
                        signs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream)), "perm_crt")
    return [_limbs_to_int(limbs[v], k + 1, int(signs[v])) for v in range(count)]
