"""Algorithm 2 (FMM apply), step by step — oracle (test infrastructure only).

Notation follows Section 3.3 and the table of translation operators:
q_B, u_B live on the index set I_B of box B (slot order, see skeleton.py);
qhat_S, uhat_S on its skeleton S_B; T_B is the ID of box B.

Steps, in the paper's order:
 1. leaves: q_L = given charges on I_L.
 2. upward, l = L..1: a tree box gathers q_B = [qhat_{S_c}] of its
    children; every box sets qhat_S = q_S + T q_R.
 3. u_B = 0, uhat_S = 0 for every box.
 4. ifo, every box B on levels >= 2 and every colleague B_j (B included):
    u_B += A_{B,B_j} q_{B_j};  uhat_S -= A_{S,S_j} qhat_{S_j}.
 5. ifs, every box B with a coarse neighbor leaf L_j:
    u_B += A_{B,L_j} q_{L_j};  uhat_S -= A_{S,L_j} q_{L_j}.
 6. tfo, every leaf L with a fine neighbor B_j:
    u_L += A_{L,B_j} q_{B_j} - A_{L,S_j} qhat_{S_j}.
 7. level 1: u_B += sum over all level-1 boxes B_j of A_{B,B_j} q_{B_j}.
 8. downward, l = 2..L: uhat_S += (u_P restricted to the entries of S_B),
    then u_S += uhat_S and u_R += T^* uhat_S.
 9. leaves: the result u is read off u_L.

Readings (the paper is ambiguous here):
* Algorithm 2 lists the ifo loop "for all boxes" and a separate level-1
  sum; applying both at level 1 would count the level-1 interactions twice,
  so the ifo loop runs on levels >= 2 and level 1 gets only the direct sum.
* The downward step's "u_{S_p}" is read as the entries of the parent's u_P
  that correspond to the child's skeleton S_B (a slice of I_P), not the
  parent's own skeleton.
* If the root is a leaf (N <= b) the apply is the direct sum over the root.

``transpose=True`` applies A~^T instead of A~: the same steps with T
replaced by conj(T) (so the downward step uses T^T). For real kernels this is
the same operator (A~ is symmetric).
"""
from __future__ import annotations

import numpy as np

from . import kernels
from .skeleton import Skeletons


def skeleton_apply(sk: Skeletons, q: np.ndarray, transpose: bool = False) -> np.ndarray:
    tree = sk.tree
    x = tree.x
    kind, kappa = sk.kind, sk.kappa
    squeeze = q.ndim == 1
    q2 = q[:, None] if squeeze else q
    cplx = kernels.is_complex(kind) or np.iscomplexobj(q2)
    dtype = np.complex128 if cplx else np.float64
    q2 = q2.astype(dtype)
    nrhs = q2.shape[1]

    def A(ti, si):
        return kernels.kernel_matrix(kind, x[ti], x[si], kappa)

    def Tmat(b):
        t = sk.T[b]
        return np.conj(t) if transpose else t

    L = tree.n_levels
    if L == 0:
        u = A(sk.idx[0], sk.idx[0]) @ q2
        out = np.zeros((tree.n, nrhs), dtype=dtype)
        out[sk.idx[0]] = u
        return out[:, 0] if squeeze else out

    nb = tree.n_boxes
    S = [sk.piv[b][: sk.k[b]] if sk.idx[b] is not None else None for b in range(nb)]
    R = [sk.piv[b][sk.k[b]:] if sk.idx[b] is not None else None for b in range(nb)]
    lv = tree.level

    # 1-2. charges at the leaves, upward pass
    qv = [None] * nb
    qhat = [None] * nb
    for b in tree.leaves():
        qv[b] = q2[sk.idx[b]]
    for lvl in range(L, 0, -1):
        for b in tree.boxes_at[lvl]:
            if not tree.is_leaf[b]:
                qv[b] = np.concatenate([qhat[c] for c in tree.children[b]], axis=0)
            qhat[b] = qv[b][S[b]] + Tmat(b) @ qv[b][R[b]]

    # 3. zero incoming representations
    u = [None] * nb
    uhat = [None] * nb
    for b in range(1, nb):
        u[b] = np.zeros((sk.idx[b].shape[0], nrhs), dtype=dtype)
        uhat[b] = np.zeros((int(sk.k[b]), nrhs), dtype=dtype)

    # 4. ifo on levels >= 2
    for b in range(nb):
        if lv[b] < 2:
            continue
        for bj in tree.colleagues[b]:
            u[b] += A(sk.idx[b], sk.idx[bj]) @ qv[bj]
            uhat[b] -= A(sk.skel(b), sk.skel(bj)) @ qhat[bj]

    # 5. ifs: box B with coarse neighbor leaf L_j
    for b in range(nb):
        if lv[b] < 2:
            continue
        for lj in tree.coarse[b]:
            u[b] += A(sk.idx[b], sk.idx[lj]) @ qv[lj]
            uhat[b] -= A(sk.skel(b), sk.idx[lj]) @ qv[lj]

    # 6. tfo: leaf L with fine neighbor B_j
    for b in tree.leaves():
        if lv[b] < 1:
            continue
        for bj in tree.fine[b]:
            u[b] += A(sk.idx[b], sk.idx[bj]) @ qv[bj] - A(sk.idx[b], sk.skel(bj)) @ qhat[bj]

    # 7. level-1 direct sum
    top = tree.boxes_at[1]
    for b in top:
        for bj in top:
            u[b] += A(sk.idx[b], sk.idx[bj]) @ qv[bj]

    # 8. downward pass
    for lvl in range(2, L + 1):
        for b in tree.boxes_at[lvl]:
            p = int(tree.parent[b])
            start = 0
            for c in tree.children[p]:
                if c == b:
                    break
                start += int(sk.k[c])
            uhat[b] += u[p][start:start + int(sk.k[b])]
            u[b][S[b]] += uhat[b]
            u[b][R[b]] += Tmat(b).conj().T @ uhat[b]

    # 9. read the potentials off the leaves
    out = np.zeros((tree.n, nrhs), dtype=dtype)
    for b in tree.leaves():
        out[sk.idx[b]] = u[b]
    return out[:, 0] if squeeze else out
