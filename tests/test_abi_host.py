"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point the header declares, and rejects bad
descriptors before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2501_12581_gb300 as pkg
import scenes
from paper_2501_12581_gb300 import build as pkg_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mboit.h")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return pkg.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^MBOIT_API\s+[\w\s\*]+?\b(mboit_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("mboit_create_volume", "mboit_add_piece", "mboit_render_moments", "mboit_reconstruct_blend",
              "mboit_composite", "mboit_render_frame", "mboit_destroy_volume"):
        assert n in names
    assert set(names) == set(pkg.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert callable(getattr(pkg, name)), name


def test_moment_image_bytes(lib):
    assert pkg.mboit_moment_image_bytes(256, 256) == 20 * 65536
    assert pkg.mboit_moment_image_bytes(7, 3) == 20 * 24       # plane rounded up to 4 pixels
    assert pkg.mboit_moment_image_bytes(0, 3) == 0
    assert pkg.mboit_moment_image_bytes(4, 4, moment_set=9) == 0
    # 6 and 8 power moments: b0 plane, float4 plane of b1..b4, then a float2 / float4 plane
    assert pkg.mboit_moment_image_bytes(7, 3, moment_set=pkg.MBOIT_POWER6) == 28 * 24
    assert pkg.mboit_moment_image_bytes(7, 3, moment_set=pkg.MBOIT_POWER8) == 36 * 24
    assert pkg.mboit_moment_image_bytes(7, 3, moment_set=pkg.MBOIT_POWER8, storage=pkg.MBOIT_STORE_F16) == 0
    assert pkg.mboit_moment_image_bytes(7, 3, moment_set=pkg.MBOIT_TRIG6, storage=pkg.MBOIT_STORE_F16) == 16 * 24


def _desc(**kw):
    d = pkg.mboit_volume_desc()
    d.kind, d.moment_set, d.storage = pkg.MBOIT_GRID, pkg.MBOIT_POWER4, pkg.MBOIT_STORE_F32
    d.field = 0x1000
    d.dims[:] = [9, 9, 9]
    d.brick_log2 = 2
    tf = np.zeros((256, 4), np.float32)
    tf[:, 3] = 0.1
    d._tf = tf
    d.tf_rgba = tf.ctypes.data
    d.tf_range[:] = [0.0, 1.0]
    d.step, d.moment_bias, d.overestimation, d.absorbance_max = 0.5, 5e-5, 0.3, 10.0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad, status", [
    (dict(kind=7), 4),
    (dict(moment_set=5), 4),
    (dict(moment_set=3, storage=1), 4),        # 6 power moments are float32
    (dict(moment_set=4, moment_bias=0.0), 1),  # 8 power moments need a bias
    (dict(field=None), 1),
    (dict(brick_log2=9), 1),
    (dict(step=0.3), 1),
    (dict(step=-0.5), 1),
    (dict(moment_bias=1.5), 1),
    (dict(overestimation=-0.1), 1),
    (dict(absorbance_max=0.0), 1),
    (dict(flags=0x80), 1),
])
def test_create_volume_rejects_bad_descriptors(lib, bad, status):
    d = _desc(**bad)
    h = ctypes.c_void_p()
    rc = lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h))
    assert rc == status
    assert h.value is None
    assert len(pkg.mboit_last_error()) > 0


def test_bad_tf_and_dims_rejected(lib):
    d = _desc()
    d.dims[:] = [1, 9, 9]
    h = ctypes.c_void_p()
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    d = _desc()
    d._tf[5, 3] = 1.0  # opacity 1 has no finite extinction
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    d = _desc()
    d.tf_range[:] = [1.0, 1.0]
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1


def test_null_handles_rejected(lib):
    assert lib.mboit_add_piece(None, None, 0, 0, None) == 1
    assert lib.mboit_render_moments(None, None, 0, None, 0, 1, None, None) == 1
    assert lib.mboit_reconstruct_blend(None, None, 0, None, 0, None, 2, None, None) == 1
    assert lib.mboit_composite(None, 0, 1, 1, 1, 1, None, None, None, None, None) == 1
    assert lib.mboit_render_frame(None, None, 0, None, None, None) == 1
    assert lib.mboit_get_stats(None, None) == 1
    assert lib.mboit_destroy_volume(None) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(pkg.MboitError):
        pkg.load_library(str(tmp_path / "nope.so"))


def _amr_desc(leaves, dims=17, max_level=1):
    d = _desc(kind=pkg.MBOIT_AMR, field=None)
    d.dims[:] = [dims, dims, dims]
    d.brick_log2 = 3
    t = np.ascontiguousarray(leaves, dtype=np.int32)
    d._table = t
    d.leaf_values = 0x2000
    d.leaf_table = t.ctypes.data
    d.n_leaves = t.shape[0]
    d.max_level = max_level
    return d


@pytest.mark.parametrize("leaves, dims, word", [
    ([[0, 0, 0, 0], [8, 0, 0, 1]], 17, "overlap"),          # a level-1 leaf inside the level-0 one
    ([[4, 0, 0, 1]], 17, "lattice"),                        # origin off the 8-cell brick lattice
    ([[8, 8, 8, 0]], 17, "domain"),                         # a 16-cell leaf past the 16-cell domain
    ([[0, 0, 0, 2]], 17, "level"),                          # level above max_level
])
def test_amr_descriptor_validation(lib, leaves, dims, word):
    d = _amr_desc(leaves, dims)
    h = ctypes.c_void_p()
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    assert word in pkg.mboit_last_error()
    assert h.value is None


def test_amr_needs_cubic_domain_and_tables(lib):
    d = _amr_desc([[0, 0, 0, 0]])
    d.dims[:] = [17, 17, 33]
    h = ctypes.c_void_p()
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    d = _amr_desc([[0, 0, 0, 0]])
    d.leaf_table = None
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1


def _tet_desc(sc, **kw):
    d = _desc(kind=pkg.MBOIT_TET, field=None)
    d.dims[:] = [0, 0, 0]
    d.brick_log2 = 0
    keep = {k: np.ascontiguousarray(getattr(sc, k)) for k in ("verts", "tets", "neighbors")}
    for k, v in kw.items():
        keep[k] = v
    d._keep = keep
    d.tet_verts, d.tet_cells, d.tet_neighbors = (keep[k].ctypes.data for k in ("verts", "tets", "neighbors"))
    d.n_verts, d.n_tets = keep["verts"].shape[0], keep["tets"].shape[0]
    d.tet_box[:] = list(sc.box)
    d.quantum_log2 = sc.quantum_log2
    return d


def _tet_scene():
    import scenes
    return scenes.tet_mesh(n=3, n_pieces=2, width=4, height=4)


@pytest.mark.parametrize("mutate, word", [
    (lambda sc: (sc.tets.__setitem__((4, slice(2, 4)), sc.tets[4, [3, 2]]),
                 sc.neighbors.__setitem__((4, slice(2, 4)), sc.neighbors[4, [3, 2]])), "oriented"),
    (lambda sc: sc.tets.__setitem__((2, 1), len(sc.verts)), "vertex id"),
    (lambda sc: sc.neighbors.__setitem__((7, 0), len(sc.tets)), "neighbour id"),
    (lambda sc: sc.verts.__setitem__((5, 0), -0.25), "outside"),
    (lambda sc: sc.neighbors.__setitem__((int(np.nonzero(sc.neighbors[:, 0] >= 0)[0][0]), 0), -1), "reciprocal"),
])
def test_tet_descriptor_validation(lib, mutate, word):
    sc = _tet_scene()
    mutate(sc)
    d = _tet_desc(sc)
    h = ctypes.c_void_p()
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    assert word in pkg.mboit_last_error()
    assert h.value is None


def test_tet_quantum_range_checked(lib):
    sc = _tet_scene()
    h = ctypes.c_void_p()
    d = _tet_desc(sc)
    d.quantum_log2 = 25
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    d = _tet_desc(sc)
    d.quantum_log2 = 24          # 3 * 2^24 quanta would pass the box check, the predicate bound fails
    d.tet_box[:] = [3.0, 3.0, 3.0]
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "64-bit" in pkg.mboit_last_error() or "2^30" in pkg.mboit_last_error()
    d = _tet_desc(sc)
    d.tet_cells = None
    assert lib.mboit_create_volume(ctypes.byref(d), ctypes.byref(h)) == 1


def test_unpack_moments_layouts():
    """The binding's slab unpacking follows the documented planes: b0, the
    float4 plane of b1..b4, then a float2 (6 moments) or float4 (8 moments)
    plane; the plane is the pixel count rounded up to 4."""
    import torch

    class V:
        width, height = 3, 2
    P = 8
    for ms, nm in ((pkg.MBOIT_POWER4, 5), (pkg.MBOIT_POWER6, 7), (pkg.MBOIT_POWER8, 9)):
        buf = torch.arange(2 * nm * P, dtype=torch.float32)
        slabs = pkg.Volume.unpack_moments(buf, [V()], 2, ms)[0]
        for j in range(2):
            s = slabs[j]
            assert s.shape == (6, nm)
            for px in range(6):
                o = j * nm * P
                want = [o + px] + [o + P + 4 * px + c for c in range(4)]
                if nm > 5:
                    want += [o + 5 * P + (nm - 5) * px + c for c in range(nm - 5)]
                assert s[px].tolist() == want


def test_split_cells_matches_oracle_and_rejects_bad_cells(lib):
    """The library's mixed-cell split gives the oracle's tets in the same
    order (both cut quads along the min-id diagonal and orient on the
    snapped vertices) and the face neighbours of the scene module; bad cells
    are rejected before anything is written out."""
    import oracle
    m = scenes.mixed_mesh(n=5, n_pieces=3, width=4, height=4, seed=17)
    t, nb, cot = pkg.mboit_split_cells(m.verts, m.cells, m.cell_types, m.quantum_log2)
    to, co = oracle.split_cells(m)
    np.testing.assert_array_equal(t, to)
    np.testing.assert_array_equal(cot, co)
    np.testing.assert_array_equal(nb, scenes.tet_neighbors(t))
    V = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [1, 1, 1, 0], [2, 0, 0, 0]], np.float32)

    def split(cells, types, q=14):
        return pkg.mboit_split_cells(V, np.array(cells, np.int32).reshape(-1, 6), np.array(types, np.int32), q)
    assert split([0, 1, 2, 3, -1, -1], [4])[0].shape == (1, 4)
    for cells, types in (([0, 1, 2, 3, -1, -1], [7]),          # unknown type
                         ([0, 1, 2, 9, -1, -1], [4]),          # vertex id out of range
                         ([0, 1, 5, 3, -1, -1], [4]),          # flat (0, 1, 5 collinear)
                         ([0, 1, 2, 3, -1, -1] * 3, [4] * 3)):  # one face in three tets
        with pytest.raises(pkg.MboitError):
            split(cells, types)


def test_save_and_load_moments_round_trip(lib, tmp_path):
    """Moment images dumped for a later replay of pass 2 come back with the
    same bits, view sizes and format; a buffer too small for the views is
    refused."""
    import torch
    views = [scenes.ortho_view((16, 16, 16), (0.3, 0.4, 0.86), 7, 5),
             scenes.ortho_view((16, 16, 16), (0.3, 0.4, 0.86), 4, 9)]
    n = sum(pkg.mboit_moment_image_bytes(v.width, v.height) for v in views) // 4
    buf = torch.from_numpy(np.random.default_rng(3).standard_normal(n).astype(np.float32))
    path = tmp_path / "moments.npz"
    pkg.save_moments(str(path), buf, views)
    got, sizes, ms, st, slots = pkg.load_moments(str(path), device="cpu")
    assert torch.equal(got.view(torch.int32), buf.view(torch.int32))
    assert sizes == [(7, 5), (4, 9)] and (ms, st, slots) == (pkg.MBOIT_POWER4, pkg.MBOIT_STORE_F32, 1)
    with pytest.raises(ValueError):
        pkg.save_moments(str(tmp_path / "short.npz"), buf[:10], views)
