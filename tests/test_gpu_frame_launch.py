"""The one-launch frame (each warp blends its ray tile right after marching
it, Sec. 4.1-4.2 per tile) against the two-launch frame: the same moments
and images bit for bit, on grids in every window configuration, for several
and ragged views, with a brick mask, with the sample cache capped (tiles
that get no rows march the field again) and at the full 512^3 / 2048^2
size, and on octrees (fixed and adaptive step) and tetrahedral meshes; the
two-launch frame's parity against the oracle is tested elsewhere, and here
once more for the form the autotuner picks."""
import dataclasses

import numpy as np
import pytest

import oracle
import scenes
from tests import _scenes_small as small

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


def frame(pkg, vol, views, launches, tuning=None):
    import torch
    vol.set_frame_launches(launches)
    if tuning is not None:
        vol.set_tuning(*tuning)
    m, c = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    vol.render_frame(views, m, c)
    vol.render_frame(views, m, c)      # the replayed graph
    vol.synchronize()
    torch.cuda.synchronize()
    st = vol.stats()
    assert st["frame_launches"] == launches
    assert st["samples_pass1"] == st["samples_pass2"]
    return m, c, st


def test_one_launch_equals_two_launches_every_tuning(pkg):
    import torch
    sc = scenes.blobs64(width=96, height=80)
    views = [sc.views[0],
             scenes.ortho_view(sc.dims, (0.3, -0.8, 0.5), 37, 23),
             scenes.perspective_view(sc.dims, (-0.5, 0.6, -0.62), 61, 37, fov_deg=40.0),
             small.axis_view(sc.dims, 9, 5, -10.0, 4.0, centre=(300.0, 300.0))]   # misses the domain
    vol = pkg.Volume(sc)
    for cfg in range(pkg.MBOIT_NUM_TUNINGS):
        m2, c2, s2 = frame(pkg, vol, views, 2, (cfg, cfg))
        m1, c1, s1 = frame(pkg, vol, views, 1, (cfg, cfg))
        assert torch.equal(m1, m2), f"moments differ in configuration {cfg}"
        assert torch.equal(c1, c2), f"image differs in configuration {cfg}"
        assert s1["samples_pass1"] == s2["samples_pass1"] > 0
        assert s1["frame_pass1_ms"] > 0
    vol.close()


def test_one_launch_with_a_brick_mask(pkg):
    """A volume whose pieces leave bricks unowned: the kernel variant that
    tests each sample's brick."""
    import torch
    sc = scenes.blobs64(width=64, height=48)
    pob = np.asarray(sc.piece_of_brick).copy()
    pob[pob == sc.n_pieces - 1] = -1
    sc = dataclasses.replace(sc, piece_of_brick=pob, n_pieces=sc.n_pieces - 1)
    vol = pkg.Volume(sc)
    m2, c2, _ = frame(pkg, vol, sc.views, 2)
    m1, c1, _ = frame(pkg, vol, sc.views, 1)
    assert torch.equal(m1, m2) and torch.equal(c1, c2)
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(c1.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 2e-4
    vol.close()


def test_one_launch_cache_fallback(pkg, monkeypatch):
    import torch
    sc = scenes.blobs64(width=96, height=80)
    want = None
    for cap in (None, "0", "3000"):
        if cap is None:
            monkeypatch.delenv("MBOIT_FRAME_CACHE_ROWS", raising=False)
        else:
            monkeypatch.setenv("MBOIT_FRAME_CACHE_ROWS", cap)
        vol = pkg.Volume(sc)
        m, c, st = frame(pkg, vol, sc.views, 1)
        assert st["samples_pass1"] > 0
        if want is None:
            want = (m.clone(), c.clone())
        else:
            assert torch.equal(m, want[0]) and torch.equal(c, want[1])
        vol.close()


def test_one_launch_full_size(pkg):
    """512^3 field, 64 pieces, 2048^2: the two forms agree bit for bit."""
    import torch
    sc = scenes.blobs512()
    vol = pkg.Volume(sc)
    m2, c2, s2 = frame(pkg, vol, sc.views, 2, (3, 3))
    m1, c1, s1 = frame(pkg, vol, sc.views, 1, (3, 3))
    assert torch.equal(m1, m2) and torch.equal(c1, c2)
    assert s1["samples_pass1"] == s2["samples_pass1"] > 1e9
    vol.close()


def test_autotune_form_matches_oracle(pkg):
    sc = scenes.blobs64(width=64, height=48)
    vol = pkg.Volume(sc)
    mom, col = pkg.Volume.moment_buffer(sc.views), pkg.Volume.color_buffer(sc.views)
    p1, p2, pk = vol.autotune(sc.views, mom, col)
    st = vol.stats()
    assert st["frame_launches"] in (1, 2)
    assert (st["tuning_pass1"], st["tuning_pass2"], st["packet"]) == (p1, p2, pk)
    vol.render_frame(sc.views, mom, col)
    vol.synchronize()
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(col.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 2e-4
    vol.close()


@pytest.mark.parametrize("kind", ["amr", "amr_adaptive", "tets"])
def test_one_launch_units_equal_two_launches(pkg, kind, monkeypatch):
    """Octrees and meshes: the same bits in one launch and in two, also with the
    cache capped so that some tiles march again."""
    import torch
    if kind == "tets":
        sc = scenes.tet_mesh(n=8, n_pieces=3, width=43, height=29, seed=7)
    else:
        sc = scenes.amr_blobs(base=4, max_level=2, width=45, height=38, n_pieces=5)
        sc.adaptive_step = kind == "amr_adaptive"
    for cap in (None, "40"):
        if cap is None:
            monkeypatch.delenv("MBOIT_FRAME_CACHE_ROWS", raising=False)
        else:
            monkeypatch.setenv("MBOIT_FRAME_CACHE_ROWS", cap)
        vol = pkg.Volume(sc)
        m2, c2, s2 = frame(pkg, vol, sc.views, 2)
        m1, c1, s1 = frame(pkg, vol, sc.views, 1)
        assert torch.equal(m1, m2) and torch.equal(c1, c2)
        assert s1["samples_pass1"] == s2["samples_pass1"] > 0
        vol.close()


def test_one_launch_refused_outside_its_scope(pkg):
    sc = scenes.blobs64(width=32, height=24)
    sc.moment_set, sc.storage = "power6", "f32"
    vol = pkg.Volume(sc)
    assert vol.stats()["frame_launches"] == 2
    with pytest.raises(pkg.MboitError) as e:
        vol.set_frame_launches(1)
    assert e.value.status == 4                  # MBOIT_ERR_UNSUPPORTED
    vol.set_frame_launches(2)
    vol.close()
    g = pkg.Volume(scenes.blobs64(width=16, height=16))
    for bad in (0, 3, -1):
        with pytest.raises(pkg.MboitError) as e:
            g.set_frame_launches(bad)
        assert e.value.status == 1              # MBOIT_ERR_INVALID_ARG
    g.close()


def test_one_launch_with_singular_frames_in_every_warp(pkg):
    """Zero bias, and rays that cross one absorber (a plane at z = 8), two (a
    second plane at z = 12 for x < 6), many (a block for y >= 10) or none
    (x >= 12): every 8 x 4 warp holds generic, one- and two-atom and empty
    frames, so the one-launch kernel takes its blend loop that tests each
    sample's frame kind.  The transfer function is opaque only above 0.9 and
    the lattice meets the planes exactly (eye at z = -6.25, step 0.5)."""
    import torch
    n = 17
    field = np.zeros((n, n, n), np.float32)
    field[8, :, :12] = 1.0
    field[12, :, :6] = 1.0
    field[2:15, 10:, :] = 1.0
    B = 4
    nb = (n - 1) // B
    bz = np.repeat(np.arange(nb), nb * nb)
    pob = (bz >= 2).astype(np.int32)
    tf = small.constant_tf(0.0)
    tf[230:, 3] = 0.3
    sc = scenes.GridScene("planes", field, 2, pob, 2, tf, (np.float32(0.0), np.float32(1.0)), 0.5, [])
    sc.moment_bias = 0.0
    view = small.axis_view(sc.dims, 16, 16, -6.25, 16.0, near=2.0, far=40.0)
    vol = pkg.Volume(sc)
    m2, c2, s2 = frame(pkg, vol, [view], 2)
    m1, c1, s1 = frame(pkg, vol, [view], 1)
    assert torch.equal(m1, m2) and torch.equal(c1, c2)
    assert s1["singular_pixels"] == s2["singular_pixels"] > 0
    sc.views = [view]
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(c1.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 2e-4
    vol.close()


def test_one_launch_sixteen_views(pkg):
    """The most views one frame takes (16), ragged sizes, both projections:
    the two forms agree bit for bit and every view's pixels are sampled."""
    import torch
    sc = scenes.blobs64(width=32, height=24)
    views = []
    for i in range(16):
        ang = 2.0 * np.pi * i / 16.0
        w = (float(np.cos(ang)) * 0.8, 0.35, float(np.sin(ang)) * 0.8 + 0.05)
        if i % 2:
            views.append(scenes.perspective_view(sc.dims, w, 13 + i, 7 + i, fov_deg=35.0))
        else:
            views.append(scenes.ortho_view(sc.dims, w, 9 + 2 * i, 11 + i))
    vol = pkg.Volume(sc)
    m2, c2, s2 = frame(pkg, vol, views, 2)
    m1, c1, s1 = frame(pkg, vol, views, 1)
    assert torch.equal(m1, m2) and torch.equal(c1, c2)
    assert s1["samples_pass1"] == s2["samples_pass1"] > 0
    off = 0
    for v in views:   # every view has some opaque pixel
        npx = v.width * v.height
        a = c1[4 * off:4 * (off + npx)].view(-1, 4)[:, 3]
        assert float(a.max()) > 0.0
        off += npx
    vol.close()


@pytest.mark.parametrize("name", ["blobs64", "amr", "tets"])
def test_cost_ordered_tiles_bit_identical(pkg, name):
    """Ray tiles dequeued longest first (mboit_set_tile_order(1)): every tile
    is still marched once, so moments and images keep their bits, in both
    frame forms and with several ragged views."""
    import torch
    if name == "blobs64":
        sc = scenes.blobs64(width=61, height=37)
        views = [sc.views[0], scenes.perspective_view(sc.dims, (-0.5, 0.6, -0.62), 48, 40, fov_deg=40.0)]
    elif name == "amr":
        sc = scenes.amr_blobs(base=4, max_level=2, width=45, height=38, n_pieces=5)
        views = sc.views
    else:
        sc = scenes.tet_mesh(n=8, n_pieces=3, width=43, height=29, seed=7)
        views = sc.views
    vol = pkg.Volume(sc)
    for launches in (1, 2):
        vol.set_tile_order(0)
        m0, c0, s0 = frame(pkg, vol, views, launches)
        vol.set_tile_order(1)
        m1, c1, s1 = frame(pkg, vol, views, launches)
        assert s0["tile_order"] == 0 and s1["tile_order"] == 1
        assert torch.equal(m0, m1) and torch.equal(c0, c1)
        assert s0["samples_pass1"] == s1["samples_pass1"] > 0
    with pytest.raises(pkg.MboitError):
        vol.set_tile_order(2)
    vol.close()
