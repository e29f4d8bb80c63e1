"""Window configurations of the fused passes: every configuration gives
bit-identical moments and images (the same float32 operations in the same
order per ray), the 16-byte-load configurations are refused where they do
not apply, and the autotuner picks valid ones."""
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


def frame(pkg, vol, views, tuning):
    import torch
    vol.set_tuning(*tuning)
    mom = pkg.Volume.moment_buffer(views)
    col = pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    return mom, col


@pytest.mark.parametrize("name", ["blobs64", "blobs512"])
def test_all_tunings_bit_identical(pkg, name):
    import torch
    sc = scenes.blobs64() if name == "blobs64" else scenes.blobs512()
    views = list(sc.views)
    if name == "blobs64":
        views += [scenes.perspective_view(sc.dims, (-0.5, 0.6, -0.62), 61, 37, fov_deg=40.0),
                  scenes.ortho_view(sc.dims, (0.1, 0.2, 0.97), 30, 30)]
    vol = pkg.Volume(sc)
    ref_m, ref_c = frame(pkg, vol, views, (0, 0))
    for cfg in range(1, pkg.MBOIT_NUM_TUNINGS):
        m, c = frame(pkg, vol, views, (cfg, cfg))
        assert torch.equal(m, ref_m), f"moments differ for tuning {cfg}"
        assert torch.equal(c, ref_c), f"image differs for tuning {cfg}"
        assert vol.stats()["tuning_pass1"] == cfg
    vol.close()


@pytest.mark.parametrize("name", ["blobs64", "amr", "tets"])
def test_packets_bit_identical(pkg, name):
    """A warp's 32 rays as 8 x 4 or 4 x 8 pixels: every ray is marched alone,
    so moments and images keep their bits (ragged views included)."""
    import torch
    if name == "blobs64":
        sc = scenes.blobs64(width=61, height=37)
    elif name == "amr":
        sc = scenes.amr_blobs(base=4, max_level=2, width=45, height=38, n_pieces=5)
    else:
        sc = scenes.tet_mesh(n=8, n_pieces=3, width=43, height=29, seed=7)
    vol = pkg.Volume(sc)
    out = []
    for packet in (pkg.MBOIT_PACKET_8X4, pkg.MBOIT_PACKET_4X8):
        vol.set_packet(packet)
        m, c = pkg.Volume.moment_buffer(sc.views), pkg.Volume.color_buffer(sc.views)
        vol.render_frame(sc.views, m, c)
        m2, c2 = pkg.Volume.moment_buffer(sc.views), pkg.Volume.color_buffer(sc.views)
        vol.render_moments(sc.views, m2)
        vol.reconstruct_blend(sc.views, m2, c2)
        vol.synchronize()
        torch.cuda.synchronize()
        assert vol.stats()["packet"] == packet
        out.append((m, c, m2, c2))
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)
    with pytest.raises(pkg.MboitError):
        vol.set_packet(2)
    vol.close()


def test_vector_tunings_refused_when_rows_unaligned(pkg):
    sc = small.linear_scene()          # nx = 17
    view = scenes.ortho_view(sc.dims, (0.36, 0.48, 0.8), 12, 10)
    sc.views = [view]
    vol = pkg.Volume(sc)
    for cfg in (2, 3, 4):
        with pytest.raises(pkg.MboitError) as e:
            vol.set_tuning(cfg, 0)
        assert e.value.status == 1
    m, c = frame(pkg, vol, [view], (1, 1))
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(c.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 2e-4
    assert pkg.mboit_autotune(vol.handle, [view], m, c)[0] in (0, 1)
    vol.close()


def test_autotune_then_frame_matches_oracle(pkg):
    sc = scenes.blobs64(width=64, height=48)
    vol = pkg.Volume(sc)
    mom = pkg.Volume.moment_buffer(sc.views)
    col = pkg.Volume.color_buffer(sc.views)
    p1, p2, pk = vol.autotune(sc.views, mom, col)
    assert 0 <= p1 < pkg.MBOIT_NUM_TUNINGS and 0 <= p2 < pkg.MBOIT_NUM_TUNINGS and pk in (0, 1)
    st = vol.stats()
    assert (st["tuning_pass1"], st["tuning_pass2"], st["packet"]) == (p1, p2, pk)
    vol.render_frame(sc.views, mom, col)
    vol.synchronize()
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(col.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 2e-4
    vol.close()


def test_autotune_choice_is_kept_per_configuration(pkg):
    """The autotuner's choice is kept for the process by (volume
    configuration, views, SM count): a second volume of the same
    configuration takes it without timing; other views are another key."""
    import time
    pkg.mboit_clear_tuning_cache()
    sc = scenes.blobs64(width=64, height=48)
    a, b = pkg.Volume(sc), pkg.Volume(sc)
    views = sc.views
    m, c = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    t0 = time.perf_counter()
    ca = a.autotune(views, m, c)
    t1 = time.perf_counter()
    cb = b.autotune(views, m, c)
    t2 = time.perf_counter()
    assert ca == cb
    sa, sb = a.stats(), b.stats()
    for k in ("tuning_pass1", "tuning_pass2", "packet", "frame_launches", "tile_order"):
        assert sa[k] == sb[k], k
    assert t2 - t1 < 0.5 * (t1 - t0)             # no timing runs the second time
    # the kept choice renders as the timed one did
    a.render_frame(views, m, c)
    ref = c.clone()
    b.render_frame(views, m, c)
    b.synchronize()
    assert (ref == c).all()
    # another view is another key, and a cleared cache times again
    other = [scenes.ortho_view(sc.dims, (0.1, 0.2, 0.97), 40, 30)]
    m2, c2 = pkg.Volume.moment_buffer(other), pkg.Volume.color_buffer(other)
    p1, p2, pk = b.autotune(other, m2, c2)
    assert 0 <= p1 < pkg.MBOIT_NUM_TUNINGS and 0 <= p2 < pkg.MBOIT_NUM_TUNINGS and pk in (0, 1)
    pkg.mboit_clear_tuning_cache()
    t3 = time.perf_counter()
    assert a.autotune(views, m, c)[2] in (0, 1)
    assert time.perf_counter() - t3 > t2 - t1
    a.close()
    b.close()
