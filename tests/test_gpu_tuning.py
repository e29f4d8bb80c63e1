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
    p1, p2 = vol.autotune(sc.views, mom, col)
    assert 0 <= p1 < pkg.MBOIT_NUM_TUNINGS and 0 <= p2 < pkg.MBOIT_NUM_TUNINGS
    st = vol.stats()
    assert (st["tuning_pass1"], st["tuning_pass2"]) == (p1, p2)
    vol.render_frame(sc.views, mom, col)
    vol.synchronize()
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(col.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= 2e-4
    vol.close()
