"""Brick-octree (AMR) volumes on the GPU against the FP64 oracle: fused
frame, per-piece passes with image sums, sort-last baseline, and the full
72-piece 2560x2560 workload on sampled pixels."""
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
def small_amr(pkg):
    sc = scenes.amr_blobs(base=4, max_level=2, width=48, height=40, n_pieces=5)
    ref = oracle.render_amr(sc, want=("moments", "piece_moments", "piece_color", "mboit", "nsamples"))
    vol = pkg.Volume(sc)
    yield sc, ref, vol
    vol.close()


def test_amr_fused_frame(pkg, small_amr):
    import torch
    sc, ref, vol = small_amr
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0], ref["mboit"])
    st = vol.stats()
    assert st["samples_pass1"] == st["samples_pass2"] == int(ref["nsamples"].sum())


def test_amr_per_piece_and_composites(pkg, small_amr):
    import torch
    sc, ref, vol = small_amr
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


def test_amr_sortlast(pkg, small_amr):
    import torch
    sc, _, vol = small_amr
    v = sc.views
    rgba = pkg.Volume.color_buffer(v)
    segs = torch.zeros(v[0].width * v[0].height, dtype=torch.int32, device="cuda")
    vol.render_sortlast(v, rgba, segs)
    torch.cuda.synchronize()
    ref_rgba, ref_segs = oracle.render_segments(sc)
    np.testing.assert_array_equal(segs.cpu().numpy(), ref_segs)
    assert_rgba_close(rgba.view(-1, 4).cpu().numpy().astype(np.float64), ref_rgba)


def test_amr_linear_field_and_subset(pkg):
    import torch
    amr, _ = small.linear_amr()
    amr.n_pieces = 2
    amr.piece_of_leaf = (np.arange(len(amr.leaves)) % 2).astype(np.int32)
    v = [scenes.perspective_view(amr.dims, (-0.6, 0.45, 0.66), 33, 29, fov_deg=35.0)]
    amr.views = v
    vol = pkg.Volume(amr)
    mom = pkg.Volume.moment_buffer(v)
    vol.render_moments(v, mom, pieces=[1])
    torch.cuda.synchronize()
    ref = oracle.render_amr(amr, pieces=[1], want=("moments",))
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    with pytest.raises(pkg.MboitError):
        vol.set_tuning(2, 2)
    vol.close()


def test_amr_full_size_sampled(pkg):
    """72 uneven pieces, ~81.5k leaves over three levels, 2560x2560."""
    import torch
    sc = scenes.amr_blobs()
    vol = pkg.Volume(sc)
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    W = v[0].width
    ys, xs = np.meshgrid(np.arange(13, W, 40), np.arange(17, W, 40), indexing="ij")
    pix = (ys * W + xs).ravel()
    ref = oracle.render_amr(sc, pixels=pix, want=("moments", "mboit"))
    assert_moments_close(unpack_moments(mom, v)[0][0][pix], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0][pix], ref["mboit"])
    assert vol.stats()["samples_pass1"] > 1e9
    vol.close()


@pytest.fixture(scope="module")
def adaptive_amr(pkg):
    import copy
    sc = copy.copy(scenes.amr_blobs(base=4, max_level=2, width=48, height=40, n_pieces=5))
    sc.adaptive_step = True
    ref = oracle.render_amr(sc, want=("moments", "piece_moments", "piece_color", "mboit", "nsamples"))
    vol = pkg.Volume(sc)
    yield sc, ref, vol
    vol.close()


def test_amr_adaptive_step_frame(pkg, adaptive_amr):
    """Adaptive dyadic step, batched frame (pass 2 marches again and skips
    the same points): the sample count is the oracle's exactly, moments and
    image within the usual tolerances, and the split calls give the same
    bits."""
    import torch
    sc, ref, vol = adaptive_amr
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    st = vol.stats()
    assert st["samples_pass1"] == st["samples_pass2"] == int(ref["nsamples"].sum())
    assert_moments_close(unpack_moments(mom, v)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0], ref["mboit"])
    mom2 = pkg.Volume.moment_buffer(v)
    col2 = pkg.Volume.color_buffer(v)
    vol.render_moments(v, mom2)
    vol.reconstruct_blend(v, mom2, col2)
    torch.cuda.synchronize()
    assert torch.equal(mom, mom2) and torch.equal(col, col2)


def test_amr_adaptive_step_per_piece_and_sortlast(pkg, adaptive_amr):
    """Per-piece passes and their image sums, and the sort-last baseline's
    segments (runs of consecutive counted points), with the adaptive step."""
    import torch
    sc, ref, vol = adaptive_amr
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
    assert_rgba_close(unpack_color(out, v)[0][0], ref["mboit"])
    rgba = pkg.Volume.color_buffer(v)
    segs = torch.zeros(v[0].width * v[0].height, dtype=torch.int32, device="cuda")
    vol.render_sortlast(v, rgba, segs)
    torch.cuda.synchronize()
    ref_rgba, ref_segs = oracle.render_segments(sc)
    np.testing.assert_array_equal(segs.cpu().numpy(), ref_segs)
    assert_rgba_close(rgba.view(-1, 4).cpu().numpy().astype(np.float64), ref_rgba)


def test_amr_adaptive_step_full_size_sampled(pkg):
    """The 72-piece 2560x2560 octree workload with the adaptive step: sampled
    pixels against the oracle, and about a third of the fixed step's
    samples."""
    import copy
    import torch
    sc = copy.copy(scenes.amr_blobs())
    sc.adaptive_step = True
    vol = pkg.Volume(sc)
    v = sc.views
    mom = pkg.Volume.moment_buffer(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    W = v[0].width
    ys, xs = np.meshgrid(np.arange(11, W, 40), np.arange(23, W, 40), indexing="ij")
    pix = (ys * W + xs).ravel()
    ref = oracle.render_amr(sc, pixels=pix, want=("moments", "mboit"))
    assert_moments_close(unpack_moments(mom, v)[0][0][pix], ref["moments"])
    assert_rgba_close(unpack_color(col, v)[0][0][pix], ref["mboit"])
    n = vol.stats()["samples_pass1"]
    assert 1.0e9 < n < 1.6e9  # 4.05 G with the fixed step
    vol.close()


@pytest.mark.parametrize("ms, st, beta, tol", [("power6", "f32", 5e-5, 1e-3), ("trig6", "f16", 2e-3, 3e-3)])
def test_amr_adaptive_step_other_moment_sets(pkg, ms, st, beta, tol):
    """The adaptive step's sample weight reaches the 6-power-moment and the
    trigonometric bodies too: frame image against the oracle's adaptive
    render within each set's tolerance, sample counts exact."""
    import copy
    import torch
    sc = copy.copy(scenes.amr_blobs(base=4, max_level=2, width=40, height=36, n_pieces=4))
    sc.adaptive_step = True
    sc.moment_set, sc.storage, sc.moment_bias = ms, st, beta
    vol = pkg.Volume(sc)
    v = sc.views
    mom = vol.moments_for(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    ref = oracle.render_amr(sc, want=("mboit", "nsamples"))
    assert vol.stats()["samples_pass1"] == int(ref["nsamples"].sum())
    assert np.abs(col.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= tol
    vol.close()
