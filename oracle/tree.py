"""Adaptive, level-restricted quad/oct-tree and near lists (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 6.1, Step 1 (a)-(b):
  (a) boxes are split until a leaf holds at most n_s points (the "maximum
      number of points in a leaf node" of Sec. 8); colleagues, coarse and fine
      neighbours are the boxes / leaves sharing a boundary point;
  (b) the tree is level-restricted: two leaves sharing a boundary point are at
      most one level apart.  In the periodic case boxes touch across the
      periodic wrap as well (Fig. 2).
Sec. 6.2: in the periodic case the neighbour lists include periodic images.

Readings used (the paper leaves these open):
  * Coordinates: w = x - lo; in the periodic case w <- w - floor(w) (in-cell
    representative).  Free-space points must satisfy 0 <= w <= 1.  Cell index
    at the finest level M: min(floor(w * 2^M), 2^M - 1), so boxes are
    half-open except that the top face belongs to the last box.
  * Split while count > n_s and level < M (M = 21 in 3D, 31 in 2D).  A leaf at
    level M keeps all its points.
  * Level restriction: refine the coarser leaf until no two touching leaves
    differ by more than one level (the unique minimal balanced refinement).
  * The near list of a leaf B is every leaf X, with a periodic image offset q,
    whose closed box touches B's closed box (B itself included, q = 0 for
    free space).  q is defined so that a pair displacement is
    (w_t - w_s) + q.  This equals the FMM list 1 (remark after Step 4).
  * Child order / Morton order: bit a of the child index is the axis-a bit,
    axis 0 least significant.
"""
import itertools
import numpy as np

MAX_LEVEL = {2: 31, 3: 21}


def in_cell_coords(x, lo, periodic):
    x = np.asarray(x, dtype=np.float64)
    w = x - np.asarray(lo, dtype=np.float64)[: x.shape[1]]
    if periodic:
        w = w - np.floor(w)
    else:
        if np.any(w < 0.0) or np.any(w > 1.0):
            raise ValueError("free-space point outside the unit box")
    return w


def cell_coords(w, M):
    c = np.floor(w * float(2 ** M)).astype(np.int64)
    return np.minimum(c, 2 ** M - 1)


def morton_key(cell, M):
    """Interleave the bits of cell[..., a] (axis 0 least significant)."""
    d = cell.shape[-1]
    key = np.zeros(cell.shape[:-1], dtype=np.uint64)
    for b in range(M):
        for a in range(d):
            bit = (cell[..., a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(d * b + a)
    return key


class Tree:
    def __init__(self, x, n_s, periodic=False, lo=None, max_level=None):
        x = np.asarray(x, dtype=np.float64)
        self.N, self.dim = x.shape
        d = self.dim
        self.M = MAX_LEVEL[d] if max_level is None else int(max_level)
        self.n_s = int(n_s)
        self.periodic = bool(periodic)
        self.lo = np.full(d, -0.5) if lo is None else np.asarray(lo, dtype=np.float64)[:d]
        self.w = in_cell_coords(x, self.lo, self.periodic)
        self.cell = cell_coords(self.w, self.M)
        self.key = morton_key(self.cell, self.M)
        self.perm = np.argsort(self.key, kind="stable")       # sorted -> original
        self.child_offsets = [tuple((j >> a) & 1 for a in range(d)) for j in range(2 ** d)]
        self.directions = [dl for dl in itertools.product((-1, 0, 1), repeat=d)]

        # ---- (a) adaptive refinement: split while count > n_s -------------
        leaves = {}
        stack = [(0, (0,) * d, np.arange(self.N))]
        while stack:
            lev, c, idx = stack.pop()
            if len(idx) > self.n_s and lev < self.M:
                sub = self.cell[idx] >> (self.M - lev - 1)
                for o in self.child_offsets:
                    cc = tuple(2 * c[a] + o[a] for a in range(d))
                    m = np.all(sub == np.array(cc), axis=1)
                    stack.append((lev + 1, cc, idx[m]))
            else:
                leaves[(lev, c)] = True
        self.leafset = leaves

        # ---- (b) level restriction ----------------------------------------
        while True:
            to_split = set()
            for (lev, c) in list(self.leafset):
                for dl in self.directions:
                    if not any(dl):
                        continue
                    nb = self._neighbor(lev, c, dl)
                    if nb is None:
                        continue
                    X = self.containing_leaf(lev, nb[0])
                    if X is not None and X[0] < lev - 1:
                        to_split.add(X)
            if not to_split:
                break
            for (lev, c) in to_split:
                del self.leafset[(lev, c)]
                for o in self.child_offsets:
                    self.leafset[(lev + 1, tuple(2 * c[a] + o[a] for a in range(d)))] = True

        # ---- leaf order, point ranges --------------------------------------
        def anchor_key(L):
            lev, c = L
            return int(morton_key(np.array([c], dtype=np.int64) << (self.M - lev), self.M)[0])
        self.leaves = sorted(self.leafset, key=anchor_key)
        self.leaf_index = {L: i for i, L in enumerate(self.leaves)}
        self.leaf_level = np.array([L[0] for L in self.leaves], dtype=np.int64)
        self.leaf_coords = np.array([L[1] for L in self.leaves], dtype=np.int64)
        # leaves partition the unit box, so the leaf of a point is the last
        # leaf whose anchor key does not exceed the point's key
        self.leaf_anchor_key = np.array([anchor_key(L) for L in self.leaves], dtype=np.uint64)
        skey = self.key[self.perm]
        self.point_leaf_sorted = (np.searchsorted(self.leaf_anchor_key, skey, side="right")
                                  .astype(np.int64) - 1)
        lv = np.array([L[0] for L in self.leaves], dtype=np.int64)[self.point_leaf_sorted]
        lc = np.array([L[1] for L in self.leaves], dtype=np.int64)[self.point_leaf_sorted]
        assert np.all((self.cell[self.perm] >> (self.M - lv)[:, None]) == lc), \
            "point not inside its leaf"
        nl = len(self.leaves)
        self.leaf_count = np.bincount(self.point_leaf_sorted, minlength=nl)
        self.leaf_start = np.concatenate([[0], np.cumsum(self.leaf_count)[:-1]])
        self.point_leaf = np.empty(self.N, dtype=np.int64)     # original order
        self.point_leaf[self.perm] = self.point_leaf_sorted
        self.point_level = self.leaf_level[self.point_leaf]

        # ---- near lists ------------------------------------------------------
        self.near = [self._near_list(L) for L in self.leaves]

    # ------------------------------------------------------------- helpers
    def _neighbor(self, lev, c, dl):
        """Neighbour box position at level lev; returns (wrapped coords, q) or None."""
        n = 2 ** lev
        raw = tuple(c[a] + dl[a] for a in range(self.dim))
        if self.periodic:
            wrapped = tuple(v % n for v in raw)
            s = tuple((raw[a] - wrapped[a]) // n for a in range(self.dim))
            return wrapped, tuple(-v for v in s)
        if any(v < 0 or v >= n for v in raw):
            return None
        return raw, (0,) * self.dim

    def containing_leaf(self, lev, c):
        """Leaf (level <= lev) containing box (lev, c), or None if that box is subdivided."""
        for l in range(lev, -1, -1):
            key = (l, tuple(v >> (lev - l) for v in c))
            if key in self.leafset:
                return key
        return None

    def _near_list(self, B):
        lev, c = B
        out = []
        seen = set()
        for dl in self.directions:
            nb = self._neighbor(lev, c, dl)
            if nb is None:
                continue
            pos, q = nb
            X = self.containing_leaf(lev, pos)
            if X is not None:
                cand = [X]
            else:
                cand = []
                for o in self.child_offsets:
                    if all((dl[a] != 1 or o[a] == 0) and (dl[a] != -1 or o[a] == 1)
                           for a in range(self.dim)):
                        ch = (lev + 1, tuple(2 * pos[a] + o[a] for a in range(self.dim)))
                        assert ch in self.leafset, "tree is not level-restricted"
                        cand.append(ch)
            for X in cand:
                item = (self.leaf_index[X], q)
                if item not in seen:
                    seen.add(item)
                    out.append(item)
        return out

    def locate(self, xt):
        """Separate target points (Sec. 1: sources and targets may differ):
        their in-cell coordinates and the index of the leaf containing each
        (the tree is built from the sources; leaves partition the unit box,
        empty leaves included, so every target has exactly one)."""
        wt = in_cell_coords(xt, self.lo, self.periodic)
        key = morton_key(cell_coords(wt, self.M), self.M)
        leaf = np.searchsorted(self.leaf_anchor_key, key, side="right").astype(np.int64) - 1
        return wt, leaf

    def leaf_points(self, i):
        """Original indices of the points in leaf i (in sorted order)."""
        s = self.leaf_start[i]
        return self.perm[s: s + self.leaf_count[i]]

    def leaf_box(self, i):
        """Closed box of leaf i in units of the finest grid: (lo[d], hi[d])."""
        lev = self.leaf_level[i]
        sz = 2 ** (self.M - lev)
        lo = self.leaf_coords[i] * sz
        return lo, lo + sz
