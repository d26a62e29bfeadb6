"""Shared test helpers: oracle/GPU comparisons (no method arithmetic)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_tree_equal(gpu_tree, otree):
    """GPU tree arrays (dmk.Plan.tree()) equal the oracle tree exactly."""
    assert np.array_equal(gpu_tree["perm"], otree.perm.astype(np.int32))
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
