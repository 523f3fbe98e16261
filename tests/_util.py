"""Shared test helpers (inputs and error measures; no method arithmetic)."""
import numpy as np

from paper_2310_16668_gb300 import workloads as W


def clustered(n, dim, seed, frac=4, sigma=0.01, c=0.41):
    """Uniform points plus a Gaussian cluster: an adaptive tree with coarse and
    fine neighbors."""
    x = W.points_uniform(n, dim, seed)
    rng = np.random.default_rng(seed + 1)
    return np.vstack([x, c + sigma * rng.standard_normal((n // frac, dim))])


def relerr(u, ref):
    """max_i |u_i - ref_i| / max_i |ref_i| (the paper's relerr, Section 5)."""
    u = np.asarray(u)
    ref = np.asarray(ref)
    return float(np.abs(u - ref).max() / np.abs(ref).max())


def skeletons_from_plan(tree, kind, plan, kappa=0.0):
    """An oracle Skeletons object carrying another implementation's IDs
    (requires the same tree), so the oracle's Algorithm 2 can run on them."""
    from oracle import skeleton as osk
    sk = osk.Skeletons.__new__(osk.Skeletons)
    sk.tree, sk.kind, sk.kappa = tree, kind, float(kappa)
    nb = tree.n_boxes
    sk.idx, sk.piv, sk.T = [None] * nb, [None] * nb, [None] * nb
    sk.k = np.array(plan["k"], dtype=np.int64)
    ip, tp = plan["idx_ptr"], plan["T_ptr"]
    for b in range(nb):
        if ip[b + 1] == ip[b]:
            continue
        n = ip[b + 1] - ip[b]
        k = int(plan["k"][b])
        sk.idx[b] = plan["idx"][ip[b]:ip[b + 1]]
        sk.piv[b] = plan["piv"][ip[b]:ip[b + 1]]
        sk.T[b] = np.asarray(plan["T"][tp[b]:tp[b + 1]]).reshape((k, n - k), order="F")
    return sk
