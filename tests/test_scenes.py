"""The benchmark's synthetic inputs have the sizes and structure their recipe
states (leaf, tet and cell counts, the octree tiling its domain, conforming
meshes, uneven and equal-count pieces, the gear-teeth interleave), and the
seeded generators repeat themselves.  Generated at full size where that
takes seconds (octree, tetrahedral and mixed-cell workloads); the 512^3
grid's piece structure at a reduced size."""
import numpy as np
import pytest

import scenes


@pytest.fixture(scope="module")
def amr():
    return scenes.amr_blobs()


def test_octree_workload_sizes(amr):
    assert amr.finest_cells == 832 and amr.max_level == 2
    assert amr.leaves.shape == (81549, 4) and amr.values.shape == (81549, 9, 9, 9)
    assert amr.values.dtype == np.float32
    np.testing.assert_array_equal(np.bincount(amr.leaves[:, 3]), [14061, 22496, 44992])
    v = amr.views[0]
    assert (v.width, v.height) == (2560, 2560) and amr.step == 0.5


def test_octree_leaves_tile_the_domain_once(amr):
    """Every finest brick (8 finest cells a side) lies in exactly one leaf:
    the leaves cover [0, 832)^3 with no gap and no overlap."""
    nb = amr.finest_cells // 8
    cover = np.zeros(nb ** 3, np.int32)
    for level in range(amr.max_level + 1):
        lv = amr.leaves[amr.leaves[:, 3] == level]
        side = 1 << (amr.max_level - level)              # finest bricks per leaf side
        o = lv[:, :3] // 8
        assert (lv[:, :3] % (8 * side) == 0).all()       # origins aligned to the leaf size
        d = np.arange(side)
        dz, dy, dx = np.meshgrid(d, d, d, indexing="ij")
        bx = (o[:, 0, None] + dx.ravel()[None]).ravel()
        by = (o[:, 1, None] + dy.ravel()[None]).ravel()
        bz = (o[:, 2, None] + dz.ravel()[None]).ravel()
        np.add.at(cover, (bz * nb + by) * nb + bx, 1)
    assert (cover == 1).all()


def test_octree_pieces_uneven_and_contiguous(amr):
    p = amr.piece_of_leaf
    assert p.shape == (81549,) and amr.n_pieces == 72
    counts = np.bincount(p, minlength=72)
    assert (counts > 0).all()
    assert 7.0 <= counts.max() / counts.min() <= 9.0     # sizes in proportion to 8^u, u in [0, 1]
    # contiguous ranges of the Morton order the leaves are stored in
    assert (np.diff(p) >= 0).all() and (np.diff(p) <= 1).all()


def test_octree_generator_repeats_itself():
    a = scenes.amr_blobs(width=32, height=32, base=4, max_level=1, n_pieces=5)
    b = scenes.amr_blobs(width=32, height=32, base=4, max_level=1, n_pieces=5)
    np.testing.assert_array_equal(a.leaves, b.leaves)
    np.testing.assert_array_equal(a.values, b.values)
    np.testing.assert_array_equal(a.piece_of_leaf, b.piece_of_leaf)
    np.testing.assert_array_equal(a.tf, b.tf)


def test_tet_workload_recipe():
    sc = scenes.tet_mesh()
    assert sc.verts.shape == (97 ** 3, 4) and sc.tets.shape == (4423680, 4)
    assert sc.box == (96.0, 96.0, 96.0) and sc.quantum_log2 == 14
    # every tet positively oriented after the positions' rounding
    P = sc.verts[:, :3].astype(np.float64)
    assert (scenes.tet_orient(P, sc.tets.astype(np.int64)) > 0).all()
    # conforming: the neighbour relation is mutual, and the boundary is the
    # box's 6 x 96^2 x 2 triangles
    nb = sc.neighbors
    assert (nb == -1).sum() == 110592
    t, f = np.nonzero(nb >= 0)
    back = nb[nb[t, f]]
    assert (back == t[:, None]).any(axis=1).all()
    # positions on the 2^-14 lattice, boundary vertices on the box faces
    assert (P * 16384.0 == np.rint(P * 16384.0)).all()
    g = np.stack(np.meshgrid(*(np.arange(97.0),) * 3, indexing="ij"), -1).reshape(-1, 3)[:, ::-1]
    jit = P - g
    on_face = (g == 0) | (g == 96)
    assert (jit[on_face] == 0).all()
    assert 0.12 < np.abs(jit[~on_face]).mean() < 0.16    # U[-0.3, 0.3] with the few halved moves
    # 72 pieces of equal tet counts
    np.testing.assert_array_equal(np.bincount(sc.piece_of_tet), np.full(72, 61440))
    assert (sc.views[0].width, sc.views[0].height) == (1024, 1024) and sc.step == 0.5


def test_mixed_cell_workload_recipe():
    sc = scenes.mixed_mesh(n=64, n_pieces=72, width=1024, height=1024)
    t = sc.cell_types
    assert t.shape == (1222408,)
    assert ((t == 4).sum(), (t == 5).sum(), (t == 6).sum()) == (525132, 522048, 175228)
    # every hex of the 64^3 grid became 6 tets, 6 pyramids or 2 prisms
    assert (t == 4).sum() // 6 + (t == 5).sum() // 6 + (t == 6).sum() // 2 == 64 ** 3
    # cells list their vertices, padded with -1 past their type's count
    pad = np.arange(6)[None, :] >= t[:, None]
    assert ((sc.cells < 0) == pad).all()
    counts = np.bincount(sc.piece_of_cell, minlength=72)
    assert counts.min() > 0 and counts.max() - counts.min() <= 1


def test_gear_teeth_interleave():
    K = 8
    sc = scenes.gear_teeth(K)
    assert sc.field.shape == (4 * K * 2 + 1, 513, 513) and sc.n_pieces == K and len(sc.views) == 4
    nb = 512 // 2
    layers = sc.piece_of_brick.reshape(4 * K, nb, nb)
    # layer s belongs to piece s mod K: K - 1 layers of other pieces between two of one
    np.testing.assert_array_equal(layers[:, 0, 0], np.arange(4 * K) % K)
    assert (layers == layers[:, :1, :1]).all()


def test_grid_workload_pieces():
    """The 512^3 grid's piece structure (16^3-cell bricks in 64 jittered
    Morton pieces), at n = 128 so it builds in a moment: every brick has one
    piece and every piece bricks."""
    sc = scenes.blobs512(width=64, height=64, n=128)
    nb = 128 // 16
    assert sc.brick_log2 == 4 and sc.piece_of_brick.shape == (nb ** 3,)
    counts = np.bincount(sc.piece_of_brick, minlength=64)
    assert counts.shape == (64,) and (counts > 0).all() and counts.sum() == nb ** 3
