"""The oracle's tree and IDs in the library's plan-exchange format — oracle
(test infrastructure only).

Lets the GPU apply run on operators computed entirely by the oracle, so that
a parity test compares two implementations of Algorithm 2 on identical
inputs (the ID's pivot choice is otherwise free to differ between two correct
implementations near ties).
"""
from __future__ import annotations

import numpy as np

from .skeleton import Skeletons


def to_exchange(sk: Skeletons) -> dict:
    t = sk.tree
    nb = t.n_boxes
    idx_ptr = np.zeros(nb + 1, np.int64)
    T_ptr = np.zeros(nb + 1, np.int64)
    idx, piv, T = [], [], []
    k = np.zeros(nb, np.int32)
    for b in range(nb):
        if sk.idx[b] is None:          # the root of a tree with more than one box
            idx_ptr[b + 1] = idx_ptr[b]
            T_ptr[b + 1] = T_ptr[b]
            continue
        n = sk.idx[b].shape[0]
        idx.append(sk.idx[b])
        piv.append(np.asarray(sk.piv[b], dtype=np.int64))
        k[b] = int(sk.k[b])
        T.append(np.asarray(sk.T[b]).reshape(-1, order="F"))
        idx_ptr[b + 1] = idx_ptr[b] + n
        T_ptr[b + 1] = T_ptr[b] + sk.T[b].size
    cat = lambda v, dt: np.concatenate(v).astype(dt) if v else np.zeros(0, dt)
    tdt = np.complex128 if np.iscomplexobj(sk.T[1 if nb > 1 else 0]) else np.float64
    return {
        "level": t.level.astype(np.int32),
        "coord": np.array(t.coord, dtype=np.int32).reshape(nb, t.dim),
        "parent": t.parent.astype(np.int64),
        "is_leaf": t.is_leaf.astype(np.int8),
        "idx_ptr": idx_ptr, "idx": cat(idx, np.int64), "piv": cat(piv, np.int64), "k": k,
        "T_ptr": T_ptr, "T": cat(T, tdt),
        "center": np.asarray(t.center, dtype=np.float64), "side": float(t.side),
    }
