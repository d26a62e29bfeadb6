"""Shared test helpers: oracle/GPU comparisons (no method arithmetic)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def hilbert_index(cell, bits):
    """Position of an integer cell (one coordinate per axis, `bits` bits each)
    along the Hilbert curve, after J. Skilling, "Programming the Hilbert curve"
    (AIP Conf. Proc. 707, 2004): axes to the transposed index, then its bits
    read level by level with axis 0 first."""
    x = [int(v) for v in cell]
    d = len(x)
    q = 1 << (bits - 1)
    while q > 1:
        p = q - 1
        for i in range(d):
            if x[i] & q:
                x[0] ^= p
            else:
                t = (x[0] ^ x[i]) & p
                x[0] ^= t
                x[i] ^= t
        q >>= 1
    for i in range(1, d):
        x[i] ^= x[i - 1]
    t = 0
    q = 1 << (bits - 1)
    while q > 1:
        if x[d - 1] & q:
            t ^= q - 1
        q >>= 1
    x = [v ^ t for v in x]
    h = 0
    for j in range(bits - 1, -1, -1):
        for i in range(d):
            h = (h << 1) | ((x[i] >> j) & 1)
    return h


def morton_cell(m, d, bits):
    """Cell of Morton index m (bit b of axis a at position d*b + a)."""
    return [sum(((m >> (d * b + a)) & 1) << b for b in range(bits)) for a in range(d)]


def leaf_hilbert_perm(otree):
    """The point order of the plan: the oracle's Morton order, with the
    sub-cells three levels below each leaf (four in 2D) put in Hilbert order
    inside the leaf (stable: Morton order inside a sub-cell); leaves deeper
    than M minus that keep the Morton order."""
    d, M = otree.dim, otree.M
    hb = 3 if d == 3 else 4
    nb = 1 << (d * hb)
    rank = np.array([hilbert_index(morton_cell(m, d, hb), hb) for m in range(nb)])
    perm = otree.perm.astype(np.int64).copy()
    keys = otree.key[otree.perm].astype(np.uint64)
    for i in range(len(otree.leaves)):
        s0, c, lev = int(otree.leaf_start[i]), int(otree.leaf_count[i]), int(otree.leaf_level[i])
        if lev + hb > M or c < 2:
            continue
        m = ((keys[s0:s0 + c] >> np.uint64(d * (M - lev - hb))) & np.uint64(nb - 1)).astype(np.int64)
        perm[s0:s0 + c] = perm[s0:s0 + c][np.argsort(rank[m], kind="stable")]
    return perm


def hilbert_order(precision, eps):
    """Plans with FP32 pair terms (MIXED, eps >= 2e-7) order the points inside
    leaves by `leaf_hilbert_perm`; the others keep the Morton order."""
    return precision == 1 and eps >= 2e-7


def assert_tree_equal(gpu_tree, otree, hilbert=False):
    """GPU tree arrays (dmk.Plan.tree()) equal the oracle tree exactly; the
    point order is the oracle's Morton order, or `leaf_hilbert_perm` of it."""
    expect = leaf_hilbert_perm(otree) if hilbert else otree.perm
    assert np.array_equal(gpu_tree["perm"], np.asarray(expect).astype(np.int32))
    L = len(otree.leaves)
    assert len(gpu_tree["leaf_level"]) == L
    assert np.array_equal(gpu_tree["leaf_level"], otree.leaf_level.astype(np.int32))
    assert np.array_equal(gpu_tree["leaf_coords"], otree.leaf_coords)
    assert np.array_equal(gpu_tree["leaf_start"], otree.leaf_start.astype(np.int32))
    assert np.array_equal(gpu_tree["leaf_count"], otree.leaf_count.astype(np.int32))
    off = gpu_tree["near_off"]
    for i in range(L):
        g = {(int(gpu_tree["near_leaf"][e]), tuple(int(v) for v in gpu_tree["near_q"][e]))
             for e in range(off[i], off[i + 1])}
        assert off[i + 1] - off[i] == len(g), f"duplicate near entries in leaf {i}"
        assert g == set(otree.near[i]), f"near list of leaf {i} differs"
