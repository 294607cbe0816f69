"""mt_count_noalloc: the count for callers that must not allocate GPU memory
while running (a fixed device-memory budget reserved up front, or a loop that
cannot pay for cudaMalloc/cudaFree).  It must give exactly mt_count's histogram,
also on back-to-back calls that reuse its fixed scratch; its status word must
be readable afterwards (mt_count_noalloc_error); and the calls must leave the
device's free memory unchanged.  GPU only; this file is collected last."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["chunglu_k4", "nullmodel_k5", "nullmodel_k6"])
def test_noalloc_matches_count_twice(name):
    import torch

    import paper_1804_09741_gb300 as mt
    lib = mt.load_library()
    w = syn.WORKLOADS[name]
    g = syn.workload_graph(name)
    t = mt.table_build(w["k"])
    dg = mt.graph_from(g)
    want = mt.to_numpy_u64(mt.count(dg, t))
    assert want.sum() > 0
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full((t.num_classes,), -1, dtype=torch.int64, device="cuda")
        st = lib.mt_count_noalloc(dg.handle, t.handle, out.data_ptr(), stream)
        assert st == mt.MT_OK, lib.mt_last_error()
        assert mt.count_noalloc_error() == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(mt.to_numpy_u64(out), want)


def test_noalloc_allocates_no_device_memory():
    """After one warm-up call, further calls (and their status reads) leave the
    device's free memory exactly where it was."""
    import torch

    import paper_1804_09741_gb300 as mt
    mt.load_library()
    g = syn.workload_graph("chunglu_k4")
    t = mt.table_build(4)
    dg = mt.graph_from(g)
    out = torch.empty(t.num_classes, dtype=torch.int64, device="cuda")
    mt.count_noalloc(dg, t, out)
    assert mt.count_noalloc_error() == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        mt.count_noalloc(dg, t, out)
        assert mt.count_noalloc_error() == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_reports_an_expired_wait():
    """Fault injection from the host (no GPU fault, trap or hang): with an
    idle-wait limit of a few nanoseconds the count's warps give up, and the
    status read after the count says so; with the limit restored the next call
    is exact and reads a zero word."""
    import torch

    import paper_1804_09741_gb300 as mt
    mt.load_library()
    g = syn.workload_graph("nullmodel_k5")
    t = mt.table_build(5)
    dg = mt.graph_from(g)
    want = mt.to_numpy_u64(mt.count(dg, t))
    out = torch.empty(t.num_classes, dtype=torch.int64, device="cuda")
    try:
        mt.set_wait_limit(5)
        mt.count_noalloc(dg, t, out)
        with pytest.raises(mt.MotifsError) as err:
            mt.count_noalloc_error()
        assert err.value.status == mt.MT_ETIMEOUT
    finally:
        mt.set_wait_limit(0)
    mt.count_noalloc(dg, t, out)
    assert mt.count_noalloc_error() == 0
    np.testing.assert_array_equal(mt.to_numpy_u64(out), want)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    import torch

    import paper_1804_09741_gb300 as mt
    lib = mt.load_library()
    g = syn.chung_lu_digraph(20000, 120000, 2.5, 150, 0.1, 5)
    t = mt.table_build(4)
    dg = mt.graph_from(g)
    out = torch.zeros(t.num_classes, dtype=torch.int64, device="cuda")
    st = lib.mt_count_noalloc(dg.handle, t.handle, out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert st == mt.MT_EUNSUPPORTED
    assert b"fixed scratch" in lib.mt_last_error()
    host = np.zeros(t.num_classes, np.uint64)
    assert lib.mt_count_noalloc(dg.handle, t.handle, host.ctypes.data, None) == mt.MT_EINVAL
