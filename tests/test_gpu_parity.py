"""GPU (sm_103a) parity of the CUDA path against the FP64 oracle, through the
C ABI.  Tolerances: RGBA max-abs 2e-4 per channel; moments 1e-5 relative to
the pixel's largest moment; sample counts exact (positions are specified in
float32 and computed identically on both sides)."""
import numpy as np
import pytest

import oracle
import scenes
from tests import _scenes_small as small

pytestmark = pytest.mark.gpu

TOL_RGBA = 2e-4
TOL_MOM = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    import paper_2501_12581_gb300 as p
    return p


def sync():
    import torch
    torch.cuda.synchronize()


def unpack_moments(buf, views, n_slots=1):
    """slab buffer -> list per view of [n_slots][npix][5] float64 arrays."""
    a = buf.cpu().numpy().astype(np.float64)
    out, off = [], 0
    for v in views:
        npx = v.width * v.height
        P = (npx + 3) // 4 * 4
        slabs = []
        for j in range(n_slots):
            s = a[off + j * 5 * P: off + (j + 1) * 5 * P]
            slabs.append(np.concatenate([s[:npx, None], s[P:].reshape(P, 4)[:npx]], axis=1))
        out.append(np.stack(slabs))
        off += n_slots * 5 * P
    return out


def unpack_color(buf, views, n_slots=1):
    a = buf.cpu().numpy().astype(np.float64)
    out, off = [], 0
    for v in views:
        npx = v.width * v.height
        out.append(a[off: off + n_slots * npx * 4].reshape(n_slots, npx, 4))
        off += n_slots * npx * 4
    return out


def assert_moments_close(got, ref):
    scale = np.abs(ref).max(axis=-1, keepdims=True) + 1e-7
    err = np.abs(got - ref) / scale
    assert err.max() <= TOL_MOM, f"moment error {err.max():.3e}"


def assert_rgba_close(got, ref, tol=TOL_RGBA):
    err = np.abs(got - ref).max()
    assert err <= tol, f"rgba max-abs {err:.3e}"


@pytest.fixture(scope="module")
def blobs(pkg):
    sc = scenes.blobs64()
    ref = oracle.render_grid(sc, want=("moments", "piece_moments", "piece_color", "mboit", "raw", "nsamples"))
    vol = pkg.Volume(sc)
    yield sc, ref, vol
    vol.close()


def test_fused_pass1_pass2_match_oracle(pkg, blobs):
    sc, ref, vol = blobs
    views = sc.views
    mom = pkg.Volume.moment_buffer(views)
    vol.render_moments(views, mom)
    col = pkg.Volume.color_buffer(views)
    vol.reconstruct_blend(views, mom, col, mode=pkg.MBOIT_COLOR_RESOLVED)
    sync()
    assert_moments_close(unpack_moments(mom, views)[0][0], ref["moments"])
    assert_rgba_close(unpack_color(col, views)[0][0], ref["mboit"])
    st = vol.stats()
    assert st["samples_pass1"] == st["samples_pass2"] == int(ref["nsamples"].sum())
    col2 = pkg.Volume.color_buffer(views)
    vol.reconstruct_blend(views, mom, col2, mode=pkg.MBOIT_COLOR_REDUCED)
    sync()
    assert_rgba_close(unpack_color(col2, views)[0][0], ref["raw"])


def test_render_frame_graph_matches_oracle_and_is_deterministic(pkg, blobs):
    import torch
    sc, ref, vol = blobs
    views = sc.views
    mom = pkg.Volume.moment_buffer(views)
    a = pkg.Volume.color_buffer(views)
    b = pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, a)
    vol.render_frame(views, mom, b)   # second call replays the captured graph
    vol.synchronize()
    assert torch.equal(a, b)
    assert_rgba_close(unpack_color(a, views)[0][0], ref["mboit"])


def test_frame_sample_cache_equals_split_calls(pkg, blobs):
    """The frame's pass 2 reads the values pass 1 stored in its tile rows; the
    split calls march twice: the same bits, also for ragged views, several
    views in one frame and a view that misses the domain."""
    import torch
    sc, _, vol = blobs
    for views in (sc.views,
                  [scenes.ortho_view(sc.dims, (0.3, -0.8, 0.5), 37, 23),
                   scenes.perspective_view(sc.dims, (-0.5, 0.6, -0.62), 20, 13, fov_deg=40.0),
                   small.axis_view(sc.dims, 9, 5, -10.0, 4.0, centre=(300.0, 300.0))]):
        m1, c1 = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
        vol.render_frame(views, m1, c1)
        vol.render_frame(views, m1, c1)
        m2, c2 = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
        vol.render_moments(views, m2)
        vol.reconstruct_blend(views, m2, c2)
        vol.synchronize()
        sync()
        assert torch.equal(m1, m2) and torch.equal(c1, c2)
        st = vol.stats()
        assert st["samples_pass1"] == st["samples_pass2"]
    m3, c3 = pkg.Volume.moment_buffer(sc.views), pkg.Volume.color_buffer(sc.views)
    vol.render_frame(sc.views, m3, c3)
    st = vol.stats()
    # one launch (the default for this volume): the second event pair is empty
    assert st["frame_pass1_ms"] > 0 and (st["frame_pass2_ms"] > 0 or st["frame_launches"] == 1)


def test_frame_cache_fallback_marches_again(pkg, monkeypatch):
    """Tiles that get no cache rows march the field again in pass 2: with the
    rows capped (none, or a few thousand) the frame's bits do not change."""
    import torch
    sc = scenes.blobs64(width=96, height=80)
    views = sc.views
    want = None
    for cap in (None, "0", "3000"):
        if cap is None:
            monkeypatch.delenv("MBOIT_FRAME_CACHE_ROWS", raising=False)
        else:
            monkeypatch.setenv("MBOIT_FRAME_CACHE_ROWS", cap)
        vol = pkg.Volume(sc)   # a new volume records a new frame graph
        m, c = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
        vol.render_frame(views, m, c)
        vol.synchronize()
        sync()
        if want is None:
            want = (m.clone(), c.clone())
        else:
            assert torch.equal(m, want[0]) and torch.equal(c, want[1])
        st = vol.stats()
        assert st["samples_pass1"] == st["samples_pass2"] > 0
        vol.close()


def test_per_piece_path_and_composites(pkg, blobs):
    sc, ref, vol = blobs
    views = sc.views
    K = sc.n_pieces
    per = pkg.Volume.moment_buffer(views, K)
    vol.render_moments(views, per, mode=pkg.MBOIT_MOMENTS_PER_PIECE)
    glob = pkg.Volume.moment_buffer(views)
    v = views[0]
    vol.composite(pkg.MBOIT_OP_MOMENTS_SUM, v.width, v.height, 1, K, per, glob)
    pc = pkg.Volume.color_buffer(views, K)
    vol.reconstruct_blend(views, glob, pc, mode=pkg.MBOIT_COLOR_PER_PIECE)
    out = pkg.Volume.color_buffer(views)
    vol.composite(pkg.MBOIT_OP_COLOR_SUM_RESOLVE, v.width, v.height, 1, K, pc, out, glob)
    sync()
    got = unpack_moments(per, views, K)[0]
    for P in range(K):
        assert_moments_close(got[P], ref["piece_moments"][:, P])
    assert_moments_close(unpack_moments(glob, views)[0][0], ref["moments"])
    gpc = unpack_color(pc, views, K)[0]
    for P in range(K):
        assert_rgba_close(gpc[P], ref["piece_color"][:, P])
    assert_rgba_close(unpack_color(out, views)[0][0], ref["mboit"])


def test_piece_subset(pkg, blobs):
    sc, ref, vol = blobs
    views = sc.views
    sub = [1, 3]
    r = oracle.render_grid(sc, pieces=sub, want=("moments",))
    mom = pkg.Volume.moment_buffer(views)
    vol.render_moments(views, mom, pieces=sub)
    glob = pkg.Volume.moment_buffer(views)
    vol.render_moments(views, glob)
    col = pkg.Volume.color_buffer(views)
    vol.reconstruct_blend(views, glob, col, pieces=sub, mode=pkg.MBOIT_COLOR_REDUCED)
    sync()
    assert_moments_close(unpack_moments(mom, views)[0][0], r["moments"])
    assert_rgba_close(unpack_color(col, views)[0][0], ref["piece_color"][:, sub].sum(axis=1))


def test_ragged_and_multiple_views(pkg, blobs):
    sc, _, vol = blobs
    views = [scenes.ortho_view(sc.dims, (0.3, -0.8, 0.5), 37, 23),
             scenes.perspective_view(sc.dims, (-0.5, 0.6, -0.62), 20, 13, fov_deg=40.0),
             small.axis_view(sc.dims, 9, 5, -10.0, 4.0, centre=(300.0, 300.0))]   # misses the domain
    mom = pkg.Volume.moment_buffer(views)
    vol.render_moments(views, mom)
    col = pkg.Volume.color_buffer(views)
    vol.reconstruct_blend(views, mom, col, mode=pkg.MBOIT_COLOR_RESOLVED)
    sync()
    gm, gc = unpack_moments(mom, views), unpack_color(col, views)
    for i, v in enumerate(views):
        r = oracle.render_grid(sc, view=v, want=("moments", "mboit"))
        assert_moments_close(gm[i][0], r["moments"])
        assert_rgba_close(gc[i][0], r["mboit"])
    assert np.all(gm[2] == 0) and np.all(gc[2] == 0)


def test_raw_sum_flag(pkg):
    sc = scenes.blobs64(width=40, height=40)
    ref = oracle.render_grid(sc, want=("raw",))
    vol = pkg.Volume(sc, flags=pkg.MBOIT_FLAG_RAW_SUM)
    mom = pkg.Volume.moment_buffer(sc.views)
    col = pkg.Volume.color_buffer(sc.views)
    vol.render_frame(sc.views, mom, col)
    vol.synchronize()
    assert_rgba_close(unpack_color(col, sc.views)[0][0], ref["raw"])
    vol.close()


@pytest.mark.parametrize("name", ["blobs64", "amr"])
def test_fp64_setup_flag(pkg, name):
    """MBOIT_FLAG_FP64_SETUP sets every pixel's frame up in FP64: the same
    images as the float-float set-up to float32 rounding, both within the
    oracle bar, and every pixel with b0 > 0 counted in fp64_pixels."""
    import torch
    if name == "blobs64":
        sc = scenes.blobs64(width=48, height=40)
        ref = oracle.render_grid(sc, want=("mboit",))["mboit"]
    else:
        sc = scenes.amr_blobs(base=4, max_level=2, width=45, height=38, n_pieces=5)
        ref = oracle.render_amr(sc, want=("mboit",))["mboit"]
    out = []
    for flags in (0, pkg.MBOIT_FLAG_FP64_SETUP):
        vol = pkg.Volume(sc, flags=flags)
        mom, col = pkg.Volume.moment_buffer(sc.views), pkg.Volume.color_buffer(sc.views)
        vol.render_frame(sc.views, mom, col)
        vol.synchronize()
        st = vol.stats()
        npx = sc.views[0].width * sc.views[0].height
        hit = int((mom[:npx] > 0).sum())
        out.append((col.view(-1, 4).double().cpu().numpy(), st["fp64_pixels"], hit))
        vol.close()
    (c_ff, n_ff, hit), (c_64, n_64, hit64) = out
    assert hit == hit64 > 0 and n_64 == hit and n_ff < hit
    assert np.abs(c_ff - c_64).max() <= 2e-6
    assert np.abs(c_64 - ref).max() <= 2e-4


@pytest.mark.parametrize("atoms, weights, in_front", [
    ((-0.875,), (0.5,), 0.5),                 # one absorber in front of the slab
    ((0.875,), (0.75,), 0.0),                 # one absorber behind it
    ((-0.875, 0.875), (0.5, 1.25), 0.5),      # slab between two absorbers
    ((-0.875, -0.5), (0.5, 0.25), 0.75),      # both in front
])
def test_singular_moment_branches_closed_form(pkg, atoms, weights, in_front):
    """Zero bias and global moments of one or two absorbers (dyadic values,
    exact in float32), so the Hankel matrix is exactly singular; blending a
    slab whose warped depths lie in (0.19, 0.39) must give
    T = exp(-optical depth of the absorbers in front)."""
    import torch
    n = 17
    field = np.ones((n, n, n), np.float32)
    bz = np.repeat(np.arange(n - 1), (n - 1) ** 2)
    pob = np.where((bz >= 6) & (bz < 10), 0, 1).astype(np.int32)
    sc = scenes.GridScene("slab", field, 0, pob, 2, small.constant_tf(0.2), (np.float32(0), np.float32(2)), 0.5, [])
    sc.moment_bias = 0.0
    view = small.axis_view(sc.dims, 8, 8, -6.0, 8.0, near=2.0, far=40.0)
    npx = view.width * view.height
    m = np.zeros(5)
    for x, a in zip(atoms, weights):
        m += a * np.array([x ** j for j in range(5)])
    P = (npx + 3) // 4 * 4
    slab = np.zeros(5 * P, np.float32)
    slab[:npx] = m[0]
    slab[P:].reshape(P, 4)[:npx] = m[1:]
    assert np.all(slab[P:].reshape(P, 4)[0].astype(np.float64) == m[1:])   # exact in float32
    mom = torch.from_numpy(slab).cuda()
    vol = pkg.Volume(sc)
    col = pkg.Volume.color_buffer([view])
    vol.reconstruct_blend([view], mom, col, pieces=[0], mode=pkg.MBOIT_COLOR_REDUCED)
    sync()
    st = vol.stats()
    assert st["singular_pixels"] == npx
    c = unpack_color(col, [view])[0][0]
    sigma = -np.log1p(-np.float64(np.float32(0.2)))
    a = sigma * 0.5
    expect = np.exp(-in_front) * (1 - np.exp(-a)) * 8     # 8 samples in z in [6, 10)
    np.testing.assert_allclose(c[:, 3], expect, rtol=2e-5)
    vol.close()


def test_full_size_workload_sampled(pkg):
    """512^3 field, 64 pieces, 2048^2 perspective view, batched frame as the
    benchmark runs it; every 16th row and column checked against the oracle."""
    sc = scenes.blobs512()
    vol = pkg.Volume(sc)
    views = sc.views
    mom = pkg.Volume.moment_buffer(views)
    col = pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    W = views[0].width
    ys, xs = np.meshgrid(np.arange(3, W, 16), np.arange(5, W, 16), indexing="ij")
    pix = (ys * W + xs).ravel()
    ref = oracle.render_grid(sc, pixels=pix, want=("moments", "mboit"))
    assert_moments_close(unpack_moments(mom, views)[0][0][pix], ref["moments"])
    assert_rgba_close(unpack_color(col, views)[0][0][pix], ref["mboit"])
    assert vol.stats()["samples_pass1"] > 1e9
    vol.close()


def test_error_paths(pkg):
    import torch
    sc = small.slab_scene()
    vol = pkg.Volume(sc)
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_add_piece(vol.handle, np.array([0, 1], np.int32))   # already owned
    assert e.value.status == 1
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_add_piece(vol.handle, np.array([10 ** 6], np.int32))
    assert e.value.status == 1
    view = small.axis_view(sc.dims, 4, 4, -10.0, 4.0)
    mom = pkg.Volume.moment_buffer([view])
    with pytest.raises(pkg.MboitError):
        vol.render_moments([view] * 17, mom)
    with pytest.raises(pkg.MboitError):
        vol.render_moments([view], mom, pieces=[5])
    bad = small.axis_view(sc.dims, 4, 4, -10.0, 4.0, near=5.0, far=1.0)
    with pytest.raises(pkg.MboitError):
        vol.render_moments([bad], mom)
    vol.synchronize()
    vol.close()
    # a volume without pieces is not renderable yet
    d = pkg.mboit_volume_desc()
    d.kind, d.moment_set, d.storage = 0, 0, 0
    f = torch.zeros(8 ** 3, device="cuda")
    d.field = f.data_ptr()
    d.dims[:] = [8, 8, 8]
    d.brick_log2 = 2
    tf = small.constant_tf(0.1)
    d.tf_rgba = tf.ctypes.data
    d.tf_range[:] = [0, 1]
    d.step, d.moment_bias, d.overestimation, d.absorbance_max = 0.5, 5e-5, 0.3, 10.0
    h = pkg.mboit_create_volume(d)
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_render_moments(h, [view], mom)
    assert e.value.status == 5
    pkg.mboit_destroy_volume(h)


def test_replay_pass2_from_saved_moments(pkg, tmp_path):
    """Pass 2 replayed from moments dumped to a file gives the frame's image."""
    import torch
    sc = scenes.blobs64(width=40, height=32)
    vol = pkg.Volume(sc)
    views = sc.views
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    pkg.save_moments(str(tmp_path / "m.npz"), mom, views)
    buf, sizes, ms, st, slots = pkg.load_moments(str(tmp_path / "m.npz"))
    assert sizes == [(v.width, v.height) for v in views] and slots == 1
    col2 = pkg.Volume.color_buffer(views)
    vol.reconstruct_blend(views, buf, col2)
    vol.synchronize()
    assert torch.equal(col, col2)
    vol.close()
