"""Pins of the Hilbert-curve helper that defines the expected point order
inside leaves (tests/helpers.py): on the 8^3 and 16^2 grids of the leaf
sub-cells it is a bijection onto [0, 2^(d b)), consecutive positions are
face neighbours (the defining property of the curve), it starts at the
origin, and at one bit it is the Gray-code order of the cube's corners."""
import numpy as np
import pytest

from tests.helpers import hilbert_index, morton_cell


@pytest.mark.parametrize("d,bits", [(3, 3), (2, 4), (3, 1), (2, 1), (3, 4)])
def test_hilbert_curve_is_a_bijection_with_unit_steps(d, bits):
    n = 1 << (d * bits)
    cells = [morton_cell(m, d, bits) for m in range(n)]
    h = np.array([hilbert_index(c, bits) for c in cells])
    assert sorted(h.tolist()) == list(range(n))
    order = np.empty((n, d), dtype=np.int64)
    order[h] = np.array(cells)
    steps = np.abs(np.diff(order, axis=0)).sum(axis=1)
    assert np.all(steps == 1)
    assert np.all(order[0] == 0)


def test_one_bit_is_the_gray_code_order():
    # at one level the curve visits the corners in reflected Gray-code order
    h = [hilbert_index(morton_cell(m, 3, 1), 1) for m in range(8)]
    corners = {v: m for m, v in enumerate(h)}
    seq = [morton_cell(corners[i], 3, 1) for i in range(8)]
    # each step flips one axis, as consecutive Gray codes do
    for a, b in zip(seq, seq[1:]):
        assert sum(x != y for x, y in zip(a, b)) == 1
    assert len(set(map(tuple, seq))) == 8


def test_morton_cell_inverts_the_interleave():
    for d, bits in ((3, 3), (2, 4)):
        for m in range(1 << (d * bits)):
            c = morton_cell(m, d, bits)
            back = sum(((c[a] >> b) & 1) << (d * b + a) for b in range(bits) for a in range(d))
            assert back == m
