"""Caller-provided scratch (mt_workspace_query / mt_set_workspace): counts with
an attached torch buffer equal the library-allocated ones, a too-small buffer
is refused, and detaching restores the default.  GPU only."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from gpu_helpers import oracle_dense

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [3, 5, 6])
def test_attached_workspace_counts(lib, k):
    import torch
    lib.load_library()
    t = lib.table_build(k)
    g = syn.chung_lu_digraph(300, 1000, 2.2, None, 0.15, 20 + k) if k < 6 else \
        syn.chung_lu_digraph(160, 420, 2.2, None, 0.15, 16)
    dg = lib.graph_from(g)
    want = lib.to_numpy_u64(lib.count(dg, t))
    need = lib.workspace_query(dg, k)
    assert need > 0
    # exactly the queried size, then a larger one; two counts each
    for size in (need, need + 4096):
        buf = torch.empty(size, dtype=torch.uint8, device="cuda")
        lib.set_workspace(dg, buf)
        for _ in range(2):
            np.testing.assert_array_equal(lib.to_numpy_u64(lib.count(dg, t)), want)
            np.testing.assert_array_equal(lib.count_host(dg, t), want)
    ref, sets = oracle.count(g, k)
    assert int(want.sum()) == sets
    np.testing.assert_array_equal(want, oracle_dense(ref, t.class_masks()))
    # too small: refused, nothing allocated in its place
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    lib.set_workspace(dg, small)
    with pytest.raises(lib.MotifsError):
        lib.count(dg, t)
    # misaligned or host memory: refused
    with pytest.raises(lib.MotifsError):
        lib.set_workspace(dg, buf[1:])
    with pytest.raises(lib.MotifsError):
        lib.set_workspace(dg, torch.empty(need, dtype=torch.uint8))
    # detached: the library allocates again
    lib.set_workspace(dg, None)
    np.testing.assert_array_equal(lib.to_numpy_u64(lib.count(dg, t)), want)
    dg.free()
    t.free()
