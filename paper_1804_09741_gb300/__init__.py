"""Python binding of the GB300 Motifs-k library (``include/motifs.h``).

Argument marshalling only: every step of the counting path runs in the CUDA
kernels of ``_build/libmotifs.so``.  PyTorch supplies device buffers and the
current CUDA stream.  Importing this module does not need a GPU; calling it
does, and every call fails loudly (``MotifsError``) when the library is not
built or a status is not MT_OK.  There is no CPU fallback.

Names follow the C ABI with the ``mt_`` prefix dropped:

    g = graph_load_csr(n, row_ptr, col)        # host int32 CSR
    t = table_build(5)                         # isomorphism table for k = 5
    h = count(g, t)                            # torch uint64-as-int64, on the GPU
    hn = count_host(g, t)                      # numpy uint64, through a host buffer
    r = randomize(g, seed, swaps)              # null graph
    b = Batch(g, t, R, swaps); hs, z = b.run(seeds)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmotifs.so")

MT_OK, MT_EINVAL, MT_EUNSUPPORTED, MT_ENOMEM, MT_ECUDA, MT_ETIMEOUT, MT_EOVERFLOW, MT_EBUSY = range(8)
NUM_CLASSES = {3: 13, 4: 199, 5: 9364, 6: 1530843}

class Tuning(ctypes.Structure):
    """mt_tuning: root-split threshold (absolute or scale of the automatic one),
    block size in warps, candidate-stack entries per warp; 0 = automatic."""
    _fields_ = [("split_cost", ctypes.c_double), ("split_scale", ctypes.c_double),
                ("warps_per_block", ctypes.c_int), ("stack_cap", ctypes.c_int),
                ("method", ctypes.c_int)]


METHOD_ENUMERATE, METHOD_CELLS = 0, 1
NULL_ARC_SWAP, NULL_DYAD_SWAP = 0, 1


# Every entry point of include/motifs.h with its ctypes signature.
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i32, _u32, _u64, _f64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
SIGNATURES = {
    "mt_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "mt_last_error": (ctypes.c_char_p, []),
    "mt_graph_load_csr": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _P(_vp)]),
    "mt_graph_free": (ctypes.c_int, [_vp]),
    "mt_graph_info": (ctypes.c_int, [_vp, _P(_i32), _P(_i32), _P(_i32), _P(_i32)]),
    "mt_graph_copy_csr": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mt_table_build": (ctypes.c_int, [ctypes.c_int, _vp, _P(_vp)]),
    "mt_table_build_compact": (ctypes.c_int, [ctypes.c_int, _vp, _P(_vp)]),
    "mt_table_is_compact": (ctypes.c_int, [_vp, _P(ctypes.c_int)]),
    "mt_table_free": (ctypes.c_int, [_vp]),
    "mt_table_k": (ctypes.c_int, [_vp, _P(ctypes.c_int)]),
    "mt_table_num_classes": (ctypes.c_int, [_vp, _P(_u32)]),
    "mt_table_class_masks": (ctypes.c_int, [_vp, _vp]),
    "mt_table_entries": (ctypes.c_int, [_vp, _u64, _u64, _vp]),
    "mt_count": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mt_count_roots": (ctypes.c_int, [_vp, _vp, _i32, _i32, _vp, _vp]),
    "mt_count_tuned": (ctypes.c_int, [_vp, _vp, _vp, _P(Tuning), _vp]),
    "mt_count_stats": (ctypes.c_int, [_vp, _P(_u64), _P(_u32), _P(ctypes.c_float)]),
    "mt_count_launch_info": (ctypes.c_int, [_vp, ctypes.c_int, _P(_i32), _P(_i32), _P(_i32),
                                            _P(_u32)]),
    "mt_count_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mt_count_noalloc_error": (ctypes.c_int, [_P(_u32), _vp]),
    "mt_workspace_query": (ctypes.c_int, [_vp, ctypes.c_int, _P(ctypes.c_size_t)]),
    "mt_set_workspace": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "mt_set_wait_limit": (ctypes.c_int, [_u64]),
    "mt_randomize": (ctypes.c_int, [_vp, _u64, _u64, _vp, _P(_vp)]),
    "mt_randomize_dyads": (ctypes.c_int, [_vp, _u64, _u64, _vp, _P(_vp)]),
    "mt_batch_create": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _u64, _P(_vp)]),
    "mt_batch_create_tuned": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _u64, _P(Tuning), _P(_vp)]),
    "mt_batch_create_ex": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _u64, ctypes.c_int, _P(Tuning),
                                          _P(_vp)]),
    "mt_batch_free": (ctypes.c_int, [_vp]),
    "mt_batch_run": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "mt_batch_phase_ms": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "mt_batch_error": (ctypes.c_int, [_vp, _P(_u32)]),
    "mt_count_batch": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _u64, _vp, _vp, _vp]),
    "mt_probe_rates": (ctypes.c_int, [_u64, _u64, _P(_f64), _P(_f64)]),
    "mt_server_create": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_size_t, ctypes.c_int, _f64,
                                        _P(_vp)]),
    "mt_server_free": (ctypes.c_int, [_vp]),
    "mt_server_submit": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _vp, _vp, _P(_u64)]),
    "mt_server_step": (ctypes.c_int, [_vp, _P(_i32), _P(_i32), _P(_i32)]),
    "mt_server_result": (ctypes.c_int, [_vp, _u64, _P(_i32), _vp, _P(_f64)]),
    "mt_server_used_bytes": (ctypes.c_int, [_vp, _P(ctypes.c_size_t)]),
    "mt_server_set_method": (ctypes.c_int, [_vp, ctypes.c_int]),
}


class MotifsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({_status_text(status)}) {detail}".strip())


_lib = None


def _status_text(st: int) -> str:
    if _lib is None:
        return "?"
    return _lib.mt_status_str(st).decode()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the built library; raise if it is missing (build it with
    ``python -c "import __graft_entry__ as g; g.build()"``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} is missing")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != MT_OK:
        detail = _lib.mt_last_error().decode() if _lib is not None else ""
        raise MotifsError(st, where, detail)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise MotifsError(MT_ECUDA, "torch", "no CUDA device")
    return torch


def _stream(stream=None) -> int:
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------------ graphs


class Graph:
    """A graph loaded into device memory (mt_graph)."""

    def __init__(self, handle: int):
        self.handle = handle
        n, m, mu, dmax = _i32(), _i32(), _i32(), _i32()
        _check(_lib.mt_graph_info(handle, n, m, mu, dmax), "mt_graph_info")
        self.n, self.m, self.m_undirected, self.max_degree = n.value, m.value, mu.value, dmax.value

    def copy_csr(self, stream=None):
        rp = np.empty(self.n + 1, np.int32)
        col = np.empty(max(self.m, 1), np.int32)
        _check(_lib.mt_graph_copy_csr(self.handle, _ptr(rp), _ptr(col), _stream(stream)),
               "mt_graph_copy_csr")
        return rp, col[: self.m].copy()

    def free(self):
        if self.handle:
            _lib.mt_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def graph_load_csr(n: int, row_ptr, col, stream=None) -> Graph:
    load_library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    if c.size == 0:
        c = np.zeros(1, np.int32)
    h = _vp()
    m = int(rp[-1]) if rp.size else 0
    _check(_lib.mt_graph_load_csr(n, m, _ptr(rp), _ptr(c), _stream(stream), ctypes.byref(h)),
           "mt_graph_load_csr")
    return Graph(h.value)


def graph_from(g, stream=None) -> Graph:
    """Load a ``synthetic.Graph``-like object (n, row_ptr, col)."""
    return graph_load_csr(g.n, g.row_ptr, g.col, stream)


# ------------------------------------------------------------------ tables


class Table:
    """Device-resident isomorphism table (mt_table)."""

    def __init__(self, handle: int):
        self.handle = handle
        k, c = ctypes.c_int(), _u32()
        _check(_lib.mt_table_k(handle, ctypes.byref(k)), "mt_table_k")
        _check(_lib.mt_table_num_classes(handle, ctypes.byref(c)), "mt_table_num_classes")
        self.k, self.num_classes = k.value, c.value
        cp = ctypes.c_int()
        _check(_lib.mt_table_is_compact(handle, ctypes.byref(cp)), "mt_table_is_compact")
        self.compact = bool(cp.value)
        self._masks = None

    def class_masks(self) -> np.ndarray:
        if self._masks is None:
            out = np.empty(self.num_classes, np.uint32)
            _check(_lib.mt_table_class_masks(self.handle, _ptr(out)), "mt_table_class_masks")
            self._masks = out
        return self._masks

    def entries(self, first: int, count: int) -> np.ndarray:
        out = np.empty(max(count, 1), np.uint32)
        _check(_lib.mt_table_entries(self.handle, first, count, _ptr(out)), "mt_table_entries")
        return out[:count]

    def free(self):
        if self.handle:
            _lib.mt_table_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def table_build(k: int, stream=None, compact: bool = False) -> Table:
    """mt_table_build, or mt_table_build_compact (k = 6 only) with `compact`."""
    load_library()
    h = _vp()
    if compact:
        _check(_lib.mt_table_build_compact(k, _stream(stream), ctypes.byref(h)),
               "mt_table_build_compact")
    else:
        _check(_lib.mt_table_build(k, _stream(stream), ctypes.byref(h)), "mt_table_build")
    return Table(h.value)


# ------------------------------------------------------------------ counting


def _dev_hist(t: Table, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty(t.num_classes, dtype=torch.int64, device="cuda")
    return out


def count(g: Graph, t: Table, out=None, stream=None):
    """H_k(G) into a device tensor (int64 storage holding uint64 counts)."""
    out = _dev_hist(t, out)
    _check(_lib.mt_count(g.handle, t.handle, out.data_ptr(), _stream(stream)), "mt_count")
    return out


def count_host(g: Graph, t: Table, stream=None) -> np.ndarray:
    """H_k(G) through a host buffer (the call copies and synchronises)."""
    out = np.empty(t.num_classes, np.uint64)
    _check(_lib.mt_count(g.handle, t.handle, _ptr(out), _stream(stream)), "mt_count")
    return out


def count_roots(g: Graph, t: Table, root_begin: int, root_end: int, stream=None) -> np.ndarray:
    out = np.empty(t.num_classes, np.uint64)
    _check(_lib.mt_count_roots(g.handle, t.handle, root_begin, root_end, _ptr(out),
                               _stream(stream)), "mt_count_roots")
    return out


def make_tuning(split_cost: float = 0.0, warps_per_block: int = 0, split_scale: float = 0.0,
                stack_cap: int = 0, method: int = METHOD_ENUMERATE) -> Tuning:
    return Tuning(float(split_cost), float(split_scale), int(warps_per_block), int(stack_cap),
                  int(method))


def count_tuned(g: Graph, t: Table, split_cost: float = 0.0, warps_per_block: int = 0, out=None,
                stream=None, split_scale: float = 0.0, stack_cap: int = 0,
                method: int = METHOD_ENUMERATE):
    """mt_count_tuned: `method` METHOD_ENUMERATE classifies every k-set,
    METHOD_CELLS counts the last two vertices per cell pair (Algorithm 1)."""
    out = _dev_hist(t, out)
    tun = make_tuning(split_cost, warps_per_block, split_scale, stack_cap, method)
    _check(_lib.mt_count_tuned(g.handle, t.handle, out.data_ptr(), ctypes.byref(tun),
                               _stream(stream)), "mt_count_tuned")
    return out


def count_noalloc(g: Graph, t: Table, out=None, stream=None):
    """mt_count without any GPU allocation inside the call (fixed scratch in the
    library; calls must not overlap on the GPU).  ``out`` must be on the GPU."""
    out = _dev_hist(t, out)
    _check(_lib.mt_count_noalloc(g.handle, t.handle, out.data_ptr(), _stream(stream)),
           "mt_count_noalloc")
    return out


def count_noalloc_error(stream=None) -> int:
    """Status word of the last count_noalloc on this device (waits for the
    stream; 0 = exact).  Raises MotifsError (MT_ETIMEOUT / MT_EOVERFLOW) when
    the word is non-zero, i.e. the histogram is invalid."""
    err = _u32()
    st = _lib.mt_count_noalloc_error(ctypes.byref(err), _stream(stream))
    if st in (MT_ETIMEOUT, MT_EOVERFLOW):
        raise MotifsError(st, "mt_count_noalloc_error", f"status word {err.value:#x}")
    _check(st, "mt_count_noalloc_error")
    return int(err.value)


def launch_info(g: Graph, k: int) -> dict:
    """The automatic counting launch for `g` at k (mt_count_launch_info)."""
    w, b, cap, lay = _i32(), _i32(), _i32(), _u32()
    _check(_lib.mt_count_launch_info(g.handle, int(k), w, b, cap, lay), "mt_count_launch_info")
    return {"warps_per_block": w.value, "blocks": b.value, "stack_cap": cap.value,
            "graph_in_smem": bool(lay.value & 1), "words_in_smem": bool(lay.value & 2),
            "stacks_in_global": bool(lay.value & 4)}


def workspace_query(g: Graph, k: int) -> int:
    """Bytes of scratch a count of `g` at k needs (mt_workspace_query)."""
    out = ctypes.c_size_t()
    _check(_lib.mt_workspace_query(g.handle, int(k), ctypes.byref(out)), "mt_workspace_query")
    return int(out.value)


def set_workspace(g: Graph, buf=None):
    """Attach a device buffer (a CUDA tensor; it is kept alive with the handle)
    as the scratch of the counts of `g` (mt_set_workspace); None detaches."""
    if buf is None:
        _check(_lib.mt_set_workspace(g.handle, None, 0), "mt_set_workspace")
        g._workspace = None
        return
    nbytes = buf.numel() * buf.element_size()
    _check(_lib.mt_set_workspace(g.handle, buf.data_ptr(), nbytes), "mt_set_workspace")
    g._workspace = buf


def set_wait_limit(ns: int = 0):
    """mt_set_wait_limit: the idle-wait limit of later launches (0 = default)."""
    load_library()
    _check(_lib.mt_set_wait_limit(int(ns)), "mt_set_wait_limit")


def count_stats(g: Graph):
    items, err, ms = _u64(), _u32(), ctypes.c_float()
    _check(_lib.mt_count_stats(g.handle, items, err, ms), "mt_count_stats")
    return int(items.value), int(err.value), float(ms.value)


def probe_rates(table_words: int = 1 << 20, hist_words: int = 1 << 14):
    """(random table reads/s, random 64-bit atomic adds/s) measured on the GPU."""
    load_library()
    g, a = _f64(), _f64()
    _check(_lib.mt_probe_rates(table_words, hist_words, ctypes.byref(g), ctypes.byref(a)),
           "mt_probe_rates")
    return g.value, a.value


def to_numpy_u64(t) -> np.ndarray:
    """Device int64 tensor holding uint64 counts -> numpy uint64."""
    return t.cpu().numpy().view(np.uint64)


def hist_to_dict(hist: np.ndarray, table: Table) -> dict:
    """{canonical mask: count} for the non-zero classes."""
    masks = table.class_masks()
    nz = np.nonzero(hist)[0]
    return dict(zip(masks[nz].tolist(), hist[nz].astype(np.uint64).tolist()))


# ------------------------------------------------------------------ null model


def randomize(g: Graph, seed: int, swaps: int, stream=None) -> Graph:
    h = _vp()
    _check(_lib.mt_randomize(g.handle, seed, swaps, _stream(stream), ctypes.byref(h)),
           "mt_randomize")
    return Graph(h.value)


def randomize_dyads(g: Graph, seed: int, attempts: int, stream=None) -> Graph:
    """Null graph that keeps reciprocity (mt_randomize_dyads)."""
    h = _vp()
    _check(_lib.mt_randomize_dyads(g.handle, seed, attempts, _stream(stream), ctypes.byref(h)),
           "mt_randomize_dyads")
    return Graph(h.value)


class Batch:
    """The original graph plus R null graphs counted in one captured step."""

    def __init__(self, g: Graph, t: Table, R: int, swaps: int, tuning: Tuning | None = None,
                 null_model: int = 0):
        self.g, self.t, self.R, self.swaps = g, t, R, swaps
        h = _vp()
        if null_model:
            _check(_lib.mt_batch_create_ex(g.handle, t.handle, R, swaps, int(null_model),
                                           ctypes.byref(tuning) if tuning is not None else None,
                                           ctypes.byref(h)), "mt_batch_create_ex")
        elif tuning is None:
            _check(_lib.mt_batch_create(g.handle, t.handle, R, swaps, ctypes.byref(h)),
                   "mt_batch_create")
        else:
            _check(_lib.mt_batch_create_tuned(g.handle, t.handle, R, swaps, ctypes.byref(tuning),
                                              ctypes.byref(h)), "mt_batch_create_tuned")
        self.handle = h.value

    def run(self, seeds, hists=None, z=None, stream=None):
        """Run one step; returns (hists, z) as device tensors ((R+1) x C int64 and
        C float64) unless host numpy arrays are passed in."""
        torch = _torch()
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        assert seeds.size == self.R
        C = self.t.num_classes
        if hists is None:
            hists = torch.empty((self.R + 1, C), dtype=torch.int64, device="cuda")
        if z is None:
            z = torch.empty(C, dtype=torch.float64, device="cuda")
        hp = hists.data_ptr() if hasattr(hists, "data_ptr") else _ptr(hists)
        zp = z.data_ptr() if hasattr(z, "data_ptr") else _ptr(z)
        _check(_lib.mt_batch_run(self.handle, _ptr(seeds), hp, zp, _stream(stream)), "mt_batch_run")
        return hists, z

    def phase_ms(self):
        out = (ctypes.c_float * 3)()
        _check(_lib.mt_batch_phase_ms(self.handle, out), "mt_batch_phase_ms")
        return list(out)

    def error(self) -> int:
        e = _u32()
        _check(_lib.mt_batch_error(self.handle, ctypes.byref(e)), "mt_batch_error")
        return int(e.value)

    def free(self):
        if getattr(self, "handle", None):
            _lib.mt_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def count_batch(g: Graph, t: Table, seeds, swaps: int, stream=None):
    """One-shot batch through host buffers: (hists (R+1) x C uint64, z float64)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    R = seeds.size
    C = t.num_classes
    hists = np.empty((R + 1, C), np.uint64)
    z = np.empty(C, np.float64)
    _check(_lib.mt_count_batch(g.handle, t.handle, _ptr(seeds), R, swaps, _ptr(hists), _ptr(z),
                               _stream(stream)), "mt_count_batch")
    return hists, z
