"""Parity of the CUDA path with the oracle for the entry points that the
per-job tests do not reach: the job features (K5 input), training by Adam
(K5), perm_exact with its two-call buffer protocol, and the evaluator's
watchdog.  Every call goes through the C ABI."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import features as ofeat
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

pk = pytest.importorskip("paper_1112_6072_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _jobs_equal(got, want):
    assert len(got) == len(want)
    for (_, gm, gc), (wm, wc) in zip(got, want):
        assert gm.shape == wm.shape and (gm == wm).all() and gc == wc % (1 << 256)


# ---------------------------------------------------------------- features (a5)
@pytest.mark.parametrize("case", ["c60", "config1"])
def test_features_match_oracle(case):
    """Every job's twelve features against the oracle's fp64 statement of
    them (FP32 on the device: rtol 1e-6), without the estimate feature."""
    if case == "c60":
        a, d, L = W.c60(60), 48, 12
    else:
        a, d, L = W.regular3(36, 1), 20, 16
    want_jobs = oracle.jobs(a, d, L)
    with pk.Plan([a], split_depth=d, leaf_size=L, model_uses_estimate=False) as p:
        p.expand()
        _jobs_equal(p.jobs_export(), want_jobs)
        got = p.features()
    want = ofeat.features([m for m, _ in want_jobs])
    assert got.shape == want.shape
    assert np.allclose(got, want, rtol=1e-6, atol=1e-7), np.abs(got - want).max()
    assert (got[:, 10] == 0).all()


def test_estimate_feature_matches_oracle():
    """With the estimate, feature 10 is log AP / 64 within the estimator's
    1e-5 on log AP; the other eleven are unchanged."""
    a, d, L = W.regular3(36, 1), 20, 16
    want_jobs = oracle.jobs(a, d, L)
    with pk.Plan([a], split_depth=d, leaf_size=L, model_uses_estimate=True, seed=99) as p:
        p.expand()
        got = p.features()
    base = ofeat.features([m for m, _ in want_jobs])
    assert np.allclose(np.delete(got, 10, axis=1), np.delete(base, 10, axis=1), rtol=1e-6, atol=1e-7)
    rng = np.random.default_rng(1)
    for j in rng.choice(len(want_jobs), size=8, replace=False):
        la = oracle.kklll_log_ap(want_jobs[j][0], seed=99, job=int(j))
        f = ofeat.job_features(want_jobs[j][0], la)
        assert abs(float(got[j, 10]) - f[10]) < 1e-5 / 64, (j, got[j, 10], f[10])


# ---------------------------------------------------------------- Adam (a9)
@pytest.mark.parametrize("steps", [1, 2, 10])
def test_adam_training_matches_oracle(steps):
    """perm_mlp_train (device forward, backward and Adam) against the fp64
    oracle's full-batch Adam.  An Adam step moves a parameter by about lr
    times the sign of its (bias-corrected) gradient, so where the oracle's
    gradient is well away from zero at every step the parameters must agree
    to FP32 rounding; elsewhere (a sign the rounding can flip) they may
    differ by at most 2 lr per step."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=(400, pk.MLP_FEATURES)).astype(np.float32)
    y = (x[:, 0] - 0.5 * x[:, 7] + 0.1 * rng.normal(size=400)).astype(np.float32)
    p0 = pk.mlp_init(11)
    lr = 1e-3
    got, loss = pk.mlp_train(p0, x, y, steps=steps, lr=lr)
    want, wloss, grads = omlp.train(p0.astype(np.float64), x.astype(np.float64), y.astype(np.float64),
                                    steps, lr)
    gmax = np.abs(grads).max(axis=1, keepdims=True)
    firm = (np.abs(grads) > 1e-3 * gmax).all(axis=0)
    assert firm.mean() > 0.5
    diff = np.abs(got.astype(np.float64) - want)
    assert (diff[firm] <= 1e-6 + 1e-5 * np.abs(want[firm]) + 1e-3 * lr * steps).all(), diff[firm].max()
    assert (diff <= 2 * lr * steps + 1e-6).all()
    assert abs(loss - wloss) <= 1e-4 * max(1.0, wloss)


# ---------------------------------------------------------------- perm_exact (b)
@pytest.mark.parametrize("case", ["config1", "c60", "signed"])
def test_perm_exact_matches_oracle(case):
    if case == "config1":
        a, kw = W.regular3(36, 1), dict(leaf_size=16)
    elif case == "c60":
        a, kw = W.c60(60), dict(leaf_size=12, order=0)
    else:
        a = W.random_small(22, 31, lo=-3, hi=3, density=0.3)
        a[np.arange(22), np.arange(22)] = 2
        kw = dict(leaf_size=10)
    want = oracle.permanent(a)
    assert pk.permanent(a, **kw) == want


def _exact_raw(a, cap, limbs):
    lib = pk._lib()
    m = np.ascontiguousarray(a, dtype=np.int64)
    pm = pk.perm_matrix(m.shape[0], m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), max(m.shape[0], 1))
    o = pk.perm_opts()
    lib.perm_opts_default(ctypes.byref(o))
    o.order = 0
    o.stream = pk._stream_handle(None)
    n, s = ctypes.c_int32(-1), ctypes.c_int32(7)
    st = lib.perm_exact(ctypes.byref(pm), ctypes.byref(o), limbs, int(cap), ctypes.byref(n), ctypes.byref(s))
    return st, n.value, s.value


def test_perm_exact_short_buffer_protocol():
    """cap = 0 and no buffer: PERM_ESHORTBUF with the required limb count;
    a second call with that many limbs returns the value; a too-short buffer
    is left alone."""
    a = W.c60(60)
    want = oracle.permanent(a, d=12)
    st, n, s = _exact_raw(a, 0, None)
    assert st == 5 and n == (want.bit_length() + 31) // 32 and s == 1
    short = (ctypes.c_uint32 * 1)(0xABCD)
    st, n2, _ = _exact_raw(a, n - 1, short)
    assert st == 5 and n2 == n and short[0] == 0xABCD
    limbs = (ctypes.c_uint32 * n)()
    st, n3, s3 = _exact_raw(a, n, limbs)
    assert st == 0 and n3 == n and s3 == 1
    assert sum(int(limbs[k]) << (32 * k) for k in range(n)) == want


def test_perm_exact_sign_and_zero():
    a = -np.eye(5, dtype=np.int64)
    limbs = (ctypes.c_uint32 * 4)()
    st, n, s = _exact_raw(a, 4, limbs)
    assert st == 0 and n == 1 and s == -1 and limbs[0] == 1      # per(-I_5) = -1
    z = np.ones((4, 4), dtype=np.int64)
    z[:, 1] = 0
    st, n, s = _exact_raw(z, 4, limbs)
    assert st == 0 and n == 0 and s == 0


# ---------------------------------------------------------------- watchdog (failure detection)
def test_watchdog_returns_timeout_status():
    """A deadline of 1 ns on one job that visits far more than 4,096 nodes:
    the evaluator checks the deadline every 4,096 nodes, sets
    PERM_ETIMEOUT for the job and returns by itself; the call reports
    status 3 and the context stays usable."""
    a = W.regular3(60, 1)
    with pk.Plan([a], split_depth=0, leaf_size=8, timeout_ns=1, order="natural") as p:
        assert p.expand() == 1
        with pytest.raises(pk.PermError) as e:
            p.evaluate(records=False)
        assert e.value.status == 3
    # the same device context evaluates the next plan normally
    b = W.regular3(20, 2)
    assert pk.permanent(b, leaf_size=8) == oracle.permanent(b)
