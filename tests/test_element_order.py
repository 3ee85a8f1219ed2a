"""CPU checks of the library's element renumbering (Sec. III-B, Tab. 1) through the host-only
dg_element_order call: RCM, and the Morton and Hilbert curves of the element centroids.

The curve orders are pinned on lattices of tiny tetrahedra whose centroids fall in distinct
dyadic cells of the 21-bit quantisation grid, so that the library's order must be the curve's
own order of those cells:
- Hilbert: every step between consecutive cells is a unit move along exactly one axis (the
  defining adjacency of the Hilbert curve), starting in the corner cell at the origin;
- Morton: the order of the bit-interleaved cell indices, computed here independently (x in the
  lowest bit).
On a jittered mesh the Hilbert order keeps consecutive elements close, where Morton jumps.
"""
import os

import numpy as np
import pytest

from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(dg.LIB_PATH):
        from paper_2209_01877_gb300 import build
        build.build()
    return dg.load()


def lattice_tets(n, shuffle_seed=7):
    """n^3 separate regular tetrahedra centred on the lattice points (i, j, k), i, j, k < n, with
    exactly representable vertices, listed in a shuffled order; returns (vid, xyz, tag, ijk)."""
    ijk = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(shuffle_seed)
    ijk = ijk[rng.permutation(len(ijk))]
    a = 0.25
    off = np.array([[a, a, a], [-a, a, -a], [a, -a, -a], [-a, -a, a]])   # positive orientation
    xyz = ijk[:, None, :].astype(np.float64) + off[None]
    ne = len(ijk)
    vid = np.arange(4 * ne, dtype=np.int32).reshape(ne, 4)
    tag = np.full((ne, 4), dg.DG_BC_WALL, dtype=np.int8)
    return vid, xyz, tag, ijk


def visit_order(perm):
    """Caller elements in internal order (perm[e] = internal position of e)."""
    order = np.empty_like(perm)
    order[perm] = np.arange(len(perm))
    return order


def test_lattice_tets_are_positively_oriented():
    _, xyz, _, _ = lattice_tets(2)
    J = np.stack([xyz[:, k] - xyz[:, 0] for k in (1, 2, 3)], axis=-1)
    assert (np.linalg.det(J) > 0).all()
    np.testing.assert_array_equal(xyz.mean(axis=1), lattice_tets(2)[3])


@pytest.mark.parametrize("n", [2, 4, 8])
def test_hilbert_order_steps_to_a_face_neighbour_cell(n):
    vid, xyz, tag, ijk = lattice_tets(n)
    perm, _, _ = dg.dg_element_order(vid, xyz, tag, dg.DG_ORDER_HILBERT)
    assert sorted(perm) == list(range(n ** 3))
    path = ijk[visit_order(perm)]
    step = np.abs(np.diff(path, axis=0))
    assert (step.sum(axis=1) == 1).all(), "consecutive cells of a Hilbert curve share a face"
    np.testing.assert_array_equal(path[0], [0, 0, 0])


@pytest.mark.parametrize("n", [4, 8])
def test_morton_order_is_the_bit_interleave(n):
    vid, xyz, tag, ijk = lattice_tets(n)
    perm, _, _ = dg.dg_element_order(vid, xyz, tag, dg.DG_ORDER_MORTON)
    key = np.zeros(len(ijk), dtype=np.int64)
    for b in range(int(np.log2(n))):
        for d in range(3):
            key |= ((ijk[:, d] >> b) & 1) << (3 * b + d)
    np.testing.assert_array_equal(visit_order(perm), np.argsort(key, kind="stable"))


def test_orders_on_a_jittered_mesh():
    m = I.make_periodic_cube(8, jitter=0.1)
    h = 1.0 / 8
    cen = m.tet_xyz.mean(axis=1)
    jump = {}
    bw = {}
    for name, r in (("asis", dg.DG_ORDER_ASIS), ("rcm", dg.DG_ORDER_RCM), ("morton", dg.DG_ORDER_MORTON),
                    ("hilbert", dg.DG_ORDER_HILBERT)):
        perm, b0, b1 = dg.dg_element_order(m.tet_vid, m.tet_xyz, None, r)
        assert np.array_equal(np.sort(perm), np.arange(m.ne))
        c = cen[visit_order(perm)]
        jump[name] = np.linalg.norm(np.diff(c, axis=0), axis=1).max() / h
        bw[name] = (b0, b1)
    assert bw["asis"][0] == bw["asis"][1] == bw["rcm"][0]
    assert bw["rcm"][1] < bw["asis"][0] / 4
    # the Hilbert curve is continuous: no consecutive pair is more than a few cells apart
    assert jump["hilbert"] < 2.0
    assert jump["morton"] > 4.0


def test_element_order_errors():
    vid, xyz, tag, _ = lattice_tets(2)
    with pytest.raises(dg.DGError) as e:
        dg.dg_element_order(vid, xyz, tag, 4)
    assert e.value.status == 1
    with pytest.raises(dg.DGError) as e:       # boundary faces without tags
        dg.dg_element_order(vid, xyz, None, dg.DG_ORDER_HILBERT)
    assert e.value.status == 2
