"""Tetrahedral meshes on the GPU against the FP64 oracle: exact point
location (per-pixel sample counts equal, also for rays running through
faces, edges and vertices), fused frame, per-piece passes with image sums,
piece subsets, trigonometric moments, sort-last baseline, the host-buffer
frame, and the 4.4M-tet 72-piece 1024x1024 workload on sampled pixels."""
import copy

import numpy as np
import pytest

import oracle
import scenes
from tests import _scenes_small as small
from tests.test_gpu_parity import assert_moments_close, assert_rgba_close, unpack_color, unpack_moments

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    import paper_2501_12581_gb300 as p
    return p


@pytest.fixture(scope="module")
def small_tet(pkg):
    sc = scenes.tet_mesh(n=10, n_pieces=5, width=48, height=40, seed=31)
    ref = oracle.render(sc, want=("moments", "piece_moments", "piece_color", "mboit", "nsamples"))
    vol = pkg.Volume(sc)
    yield sc, ref, vol
    vol.close()


def test_tet_fused_frame(pkg, small_tet):
    import torch
    sc, ref, vol = small_tet
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0], ref["mboit"])
    st = vol.stats()
    assert st["samples_pass1"] == st["samples_pass2"] == int(ref["nsamples"].sum()) > 10000
    # the frame's pass 2 reads the values pass 1 stored; the split calls walk
    # the mesh twice: the same bits either way
    mom2 = pkg.Volume.moment_buffer(v)
    col2 = pkg.Volume.color_buffer(v)
    vol.render_moments(v, mom2)
    vol.reconstruct_blend(v, mom2, col2)
    torch.cuda.synchronize()
    assert torch.equal(mom, mom2) and torch.equal(col, col2)


def test_tet_per_piece_and_composites(pkg, small_tet):
    import torch
    sc, ref, vol = small_tet
    v = sc.views
    K = sc.n_pieces
    per = pkg.Volume.moment_buffer(v, K)
    vol.render_moments(v, per, mode=pkg.MBOIT_MOMENTS_PER_PIECE)
    glob = pkg.Volume.moment_buffer(v)
    vol.composite(pkg.MBOIT_OP_MOMENTS_SUM, v[0].width, v[0].height, 1, K, per, glob)
    pc = pkg.Volume.color_buffer(v, K)
    vol.reconstruct_blend(v, glob, pc, mode=pkg.MBOIT_COLOR_PER_PIECE)
    out = pkg.Volume.color_buffer(v)
    vol.composite(pkg.MBOIT_OP_COLOR_SUM_RESOLVE, v[0].width, v[0].height, 1, K, pc, out, glob)
    torch.cuda.synchronize()
    got = unpack_moments(per, v, K)[0]
    for P in range(K):
        assert_moments_close(got[P], ref["piece_moments"][:, P])
    gpc = unpack_color(pc, v, K)[0]
    for P in range(K):
        assert_rgba_close(gpc[P], ref["piece_color"][:, P])
    assert_rgba_close(unpack_color(out, v)[0][0], ref["mboit"])
    assert vol.stats()["samples_pass2"] == int(ref["nsamples"].sum())


def test_tet_sortlast(pkg, small_tet):
    import torch
    sc, _, vol = small_tet
    v = sc.views
    rgba = pkg.Volume.color_buffer(v)
    segs = torch.zeros(v[0].width * v[0].height, dtype=torch.int32, device="cuda")
    vol.render_sortlast(v, rgba, segs)
    torch.cuda.synchronize()
    ref_rgba, ref_segs = oracle.render_segments(sc)
    np.testing.assert_array_equal(segs.cpu().numpy(), ref_segs)
    assert_rgba_close(rgba.view(-1, 4).cpu().numpy().astype(np.float64), ref_rgba)


@pytest.mark.parametrize("jitter", [0.0, 0.3])
def test_tet_counts_on_faces_edges_vertices(pkg, jitter):
    """Rays along x = i/2, y = j/2 and samples at z = k/2 on an unjittered
    mesh hit faces, edges and vertices exactly; a constant opacity makes b0
    count each pixel's samples, which must equal the oracle's."""
    import torch
    n = 6
    sc = scenes.tet_mesh(n=n, jitter=jitter, n_pieces=3, width=4, height=4, seed=41)
    sc.tf = small.constant_tf(0.05)
    views = [small.axis_view(sc.dims, 2 * n, 2 * n, -5.25, float(n), centre=(2.75, 2.75)),
             small.axis_view(sc.dims, 2 * n + 1, 2 * n - 1, -5.25, float(n), w=(1.0, 0.0, 0.0), u=(0.0, 1.0, 0.0),
                             v=(0.0, 0.0, 1.0), centre=(2.75, 2.75))]
    views[1].eye = np.array([-5.25, 2.75, 2.75], np.float32)
    sc.views = views
    vol = pkg.Volume(sc)
    a = float(np.float32(-np.log1p(-np.float64(np.float32(0.05)))) * np.float32(0.5))
    for v in views:
        mom = pkg.Volume.moment_buffer([v])
        vol.render_moments([v], mom)
        torch.cuda.synchronize()
        ref = oracle.render(sc, view=v, want=("nsamples", "moments"))
        b0 = unpack_moments(mom, [v])[0][0][:, 0]
        np.testing.assert_array_equal(np.rint(b0 / a).astype(np.int64), ref["nsamples"])
        assert ref["nsamples"].sum() > 100
        assert vol.stats()["samples_pass1"] == int(ref["nsamples"].sum())
    vol.close()


def test_tet_piece_subset_and_linear_field(pkg):
    import torch
    sc, _ = small.linear_tets(n=7)
    sc.views = [scenes.perspective_view(sc.dims, (-0.6, 0.45, 0.66), 33, 29, fov_deg=35.0)]
    vol = pkg.Volume(sc)
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    vol.render_moments(v, mom, pieces=[0, 2])
    col = pkg.Volume.color_buffer(v)
    vol.reconstruct_blend(v, mom, col, pieces=[0, 2])
    torch.cuda.synchronize()
    ref = oracle.render(sc, pieces=[0, 2], want=("moments", "mboit", "nsamples"))
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0], ref["mboit"])
    assert vol.stats()["samples_pass1"] == int(ref["nsamples"].sum())
    with pytest.raises(pkg.MboitError):
        vol.set_tuning(1, 0)
    vol.close()


def test_tet_trig_moments(pkg):
    import torch
    sc = scenes.tet_mesh(n=8, n_pieces=3, width=40, height=36, seed=43)
    sc = copy.copy(sc)
    sc.moment_set, sc.storage, sc.moment_bias = "trig6", "f16", 2e-3
    vol = pkg.Volume(sc)
    v = sc.views
    mom = vol.moments_for(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    ref = oracle.render(sc, want=("mboit",))
    assert np.abs(col.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 3e-3
    vol.close()


def test_tet_host_frame_equals_device_frame(pkg, small_tet):
    """mboit_render_frame_host: vertex values from pinned host memory give
    the same image bits as the resident frame."""
    import torch
    sc, _, vol = small_tet
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    torch.cuda.synchronize()
    want = col.cpu().numpy()
    vals = torch.from_numpy(np.ascontiguousarray(sc.verts[:, 3])).pin_memory()
    host = torch.zeros(col.numel(), dtype=torch.float32).pin_memory()
    col2 = pkg.Volume.color_buffer(v)
    pkg.mboit_render_frame_host(vol.handle, vals, v, mom, col2, host)
    np.testing.assert_array_equal(host.numpy(), want)


@pytest.mark.parametrize("max_walk", [None, "1", "2"])
def test_tet_mesh_with_a_hole_and_bin_search(pkg, monkeypatch, max_walk):
    """A mesh with a cavity (tets near a centre point removed, neighbours
    recomputed): walks leave the mesh inside the box and fall back to the
    bin search, points in the cavity belong to no tet.  With the walk capped
    at one or two steps every point is found by the search: the same owners,
    so the same counts and images."""
    import torch
    if max_walk is None:
        monkeypatch.delenv("MBOIT_TET_MAX_WALK", raising=False)
    else:
        monkeypatch.setenv("MBOIT_TET_MAX_WALK", max_walk)
    sc = scenes.tet_mesh(n=8, n_pieces=3, width=40, height=36, seed=51)
    cen = sc.verts[sc.tets, :3].astype(np.float64).mean(axis=1)
    keep = np.linalg.norm(cen - np.array([4.2, 3.7, 4.4]), axis=1) > 2.3
    assert 0 < (~keep).sum() < len(keep)
    sc.tets = np.ascontiguousarray(sc.tets[keep])
    sc.piece_of_tet = np.ascontiguousarray(sc.piece_of_tet[keep])
    sc.neighbors = scenes.tet_neighbors(sc.tets)
    vol = pkg.Volume(sc)
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    ref = oracle.render(sc, want=("moments", "mboit", "nsamples"))
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0], ref["mboit"])
    assert vol.stats()["samples_pass1"] == int(ref["nsamples"].sum())
    vol.close()


def test_tet_full_size_sampled(pkg):
    """4,423,680 tets, 72 pieces, 1024x1024 perspective."""
    import torch
    sc = scenes.tet_mesh()
    vol = pkg.Volume(sc)
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    W = v[0].width
    ys, xs = np.meshgrid(np.arange(11, W, 64), np.arange(23, W, 64), indexing="ij")
    pix = (ys * W + xs).ravel()
    ref = oracle.render(sc, pixels=pix, want=("moments", "mboit"))
    assert_moments_close(unpack_moments(mom, v)[0][0][pix], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0][pix], ref["mboit"])
    assert vol.stats()["samples_pass1"] > 5e7
    vol.close()


def test_mixed_cells_frame_and_pieces(pkg):
    """Tetrahedra, pyramids and prisms (split by the library into a
    conforming tet mesh, pieces by cell): the batched frame's samples equal
    the oracle's (its own split) exactly, moments and image within the
    usual tolerances; per-piece passes add up to the same image."""
    import torch
    m = scenes.mixed_mesh(n=10, n_pieces=4, width=64, height=56)
    vol = pkg.Volume(m)
    v = m.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    ts = oracle.tet_scene_of(m)
    ref = oracle.render(ts, want=("moments", "mboit", "nsamples"))
    assert vol.stats()["samples_pass1"] == int(ref["nsamples"].sum())
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0], ref["mboit"])
    K = m.n_pieces
    per = pkg.Volume.moment_buffer(v, K)
    vol.render_moments(v, per, mode=pkg.MBOIT_MOMENTS_PER_PIECE)
    glob = pkg.Volume.moment_buffer(v)
    vol.composite(pkg.MBOIT_OP_MOMENTS_SUM, v[0].width, v[0].height, 1, K, per, glob)
    pc = pkg.Volume.color_buffer(v, K)
    vol.reconstruct_blend(v, glob, pc, mode=pkg.MBOIT_COLOR_PER_PIECE)
    out = pkg.Volume.color_buffer(v)
    vol.composite(pkg.MBOIT_OP_COLOR_SUM_RESOLVE, v[0].width, v[0].height, 1, K, pc, out, glob)
    torch.cuda.synchronize()
    assert_rgba_close(unpack_color(out, v)[0][0], ref["mboit"])
    vol.close()
