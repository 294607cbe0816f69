"""Helpers for the GPU parity tests (test side only: no CUDA-path code here)."""
import numpy as np

import oracle


def ext_key_to_mask(k: int, keys: np.ndarray) -> np.ndarray:
    """Extension-order key (layout documented in include/motifs.h) -> the
    canonical-layout mask of the same labelled digraph."""
    keys = np.asarray(keys, dtype=np.uint64)
    out = np.zeros(keys.shape, dtype=np.uint64)
    for p in range(1, k):
        off = k * (k - 1) - p * (p + 1)
        for q in range(p):
            fwd = (keys >> np.uint64(off + 2 * q)) & np.uint64(1)      # q -> p
            back = (keys >> np.uint64(off + 2 * q + 1)) & np.uint64(1)  # p -> q
            out |= fwd << np.uint64(oracle.bit_index(k, q, p))
            out |= back << np.uint64(oracle.bit_index(k, p, q))
    return out.astype(np.uint32)


def expected_ids(k: int, keys: np.ndarray, class_masks: np.ndarray) -> np.ndarray:
    """Dense class id of each key by the oracle (brute-force canonical form,
    rank among the oracle's connected canonical masks), 0xFFFFFFFF if
    disconnected."""
    masks = ext_key_to_mask(k, keys)
    can = oracle.canon_many(k, masks)
    pos = np.searchsorted(class_masks, can)
    pos_c = np.minimum(pos, len(class_masks) - 1)
    found = class_masks[pos_c] == can
    return np.where(found, pos_c, 0xFFFFFFFF).astype(np.uint32)


def oracle_dense(hdict: dict, class_masks: np.ndarray) -> np.ndarray:
    """Oracle {canonical mask: count} -> dense uint64 histogram over class_masks."""
    out = np.zeros(len(class_masks), np.uint64)
    if hdict:
        m = np.array(list(hdict.keys()), dtype=np.uint32)
        c = np.array(list(hdict.values()), dtype=np.uint64)
        pos = np.searchsorted(class_masks, m)
        assert np.all(class_masks[np.minimum(pos, len(class_masks) - 1)] == m), \
            "oracle class not in the table's class list"
        out[pos] = c
    return out
