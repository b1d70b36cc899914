"""The C-ABI library builds for sm_103a and exports every entry point that
include/perm.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "perm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(perm_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_boundary_calls():
    names = declared_functions()
    for required in ("perm_plan_create", "perm_expand", "perm_eval_batch", "perm_exact", "perm_estimate",
                     "perm_order", "perm_result"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_1112_6072_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    import paper_1112_6072_gb300 as pk
    assert sorted(pk.EXPORTED) == declared_functions()


def test_status_strings_without_gpu():
    import paper_1112_6072_gb300 as pk
    lib = pk._lib()
    assert lib.perm_status_string(0) == b"ok"
    assert lib.perm_status_string(2).startswith(b"value or bound")


def test_packed_plan_rejects_a_buffer_of_the_wrong_size():
    """Plan.packed checks the buffer against the orders before any library
    call (so this runs without a GPU)."""
    import numpy as np
    import paper_1112_6072_gb300 as pk
    with pytest.raises(ValueError):
        pk.Plan.packed(np.zeros(18, dtype=np.int64), [2, 3, 2])  # the matrices hold 4 + 9 + 4 = 17
    with pytest.raises(ValueError):
        pk.Plan.packed(np.zeros(4, dtype=np.int64), [2, -1])
    with pytest.raises(ValueError):
        pk.Plan.packed(np.zeros(0, dtype=np.int64), [])


def test_packed_descriptors_address_each_matrix():
    """Each record of a packed batch points at its matrix: the same address
    as a view of that matrix in the buffer, with its order and row stride."""
    import numpy as np
    import paper_1112_6072_gb300 as pk
    rng = np.random.default_rng(4)
    orders = [int(x) for x in rng.integers(0, 9, size=40)] + [1, 0, 24]
    mats = [rng.integers(-3, 4, size=(n, n)).astype(np.int64) for n in orders]
    data, desc = pk.packed_descriptors(np.concatenate([m.ravel() for m in mats]), orders)
    off = 0
    for i, m in enumerate(mats):
        n = m.shape[0]
        view = data[off:off + n * n]
        assert int(desc["n"][i]) == n and int(desc["ld"][i]) == max(n, 1)
        if n > 0:  # numpy gives an empty slice the buffer's base address; order 0 reads nothing
            assert int(desc["a"][i]) == view.__array_interface__["data"][0]
        assert np.array_equal(view.reshape(n, n), m)
        off += n * n
    # a contiguous int64 input is used in place, anything else converted once
    buf = np.arange(4 + 9, dtype=np.int64)
    same, _ = pk.packed_descriptors(buf, [2, 3])
    assert same.__array_interface__["data"][0] == buf.__array_interface__["data"][0]
    conv, d2 = pk.packed_descriptors(buf.astype(np.int32), [2, 3])
    assert conv.dtype == np.int64 and int(d2["a"][1]) - int(d2["a"][0]) == 8 * 4
