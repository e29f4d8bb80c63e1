"""Failure detection through the device error word (mboit_synchronize).

Every octree or mesh render first checks the library-owned index tables as a
whole (octree leaf ids in the finest-brick map, mesh tet ids in face
neighbours and bin lists, bin ranges); a bad entry is reported in the volume's
error word and the kernels that read those tables return at entry.  Here a
table is corrupted on the host after validation (mboit_debug_corrupt), the
volume renders, and mboit_synchronize must report MBOIT_ERR_DEVICE_ASSERT
once; no kernel reads outside the tables, so the context stays usable.

The grid kernels' one wait, the TMA window load of tuning configurations 5
and 6, is bounded: the hook arms the barrier without issuing the copy (a completion that
nothing delivers, no copy in flight), every wait runs to its limit, and
mboit_synchronize must report MBOIT_ERR_TIMEOUT."""
import time

import numpy as np
import pytest

import scenes
from tests import _scenes_small as small

pytestmark = pytest.mark.gpu

STATE = 5
TIMEOUT = 6
DEVICE_ASSERT = 7


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    import paper_2501_12581_gb300 as p
    return p


def _frame_then_check(pkg, sc, what, text):
    vol = pkg.Volume(sc)
    views = sc.views
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, col)
    vol.synchronize()                       # clean before the corruption
    good = col.clone()
    pkg.mboit_debug_corrupt(vol.handle, what)
    vol.render_frame(views, mom, col)
    with pytest.raises(pkg.MboitError) as e:
        vol.synchronize()
    assert e.value.status == DEVICE_ASSERT and text in str(e.value)
    vol.synchronize()                       # reported once, then cleared
    # the split calls check the same indices
    vol.render_moments(views, mom)
    with pytest.raises(pkg.MboitError) as e:
        vol.synchronize()
    assert e.value.status == DEVICE_ASSERT
    vol.close()
    # the context is still usable: a fresh volume renders the good image again
    vol = pkg.Volume(sc)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    assert np.array_equal(col.cpu().numpy(), good.cpu().numpy())
    vol.close()


def test_corrupt_octree_map_is_reported(pkg):
    amr, _ = small.linear_amr()
    amr.views = [scenes.perspective_view(amr.dims, (0.57, 0.49, 0.66), 64, 48)]
    _frame_then_check(pkg, amr, 1, "leaf id")


def test_corrupt_mesh_neighbours_are_reported(pkg):
    sc = scenes.tet_mesh(n=8, n_pieces=4, width=48, height=40)
    _frame_then_check(pkg, sc, 2, "tet id")


def test_corrupt_hook_rejects_wrong_kind(pkg):
    sc = scenes.blobs64(width=16, height=16)
    vol = pkg.Volume(sc)
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_debug_corrupt(vol.handle, 1)
    assert e.value.status == 1
    vol.close()


@pytest.mark.parametrize("cfg", [5, 6])
@pytest.mark.parametrize("launches", [1, 2])
def test_tma_wait_limit_is_reported(pkg, launches, cfg):
    sc = scenes.blobs64(width=48, height=40)
    views = sc.views
    vol = pkg.Volume(sc)
    vol.set_tuning(cfg, 3)
    vol.set_frame_launches(launches)
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    good = col.clone()
    pkg.mboit_debug_corrupt(vol.handle, 3)
    t0 = time.perf_counter()
    vol.render_frame(views, mom, col)
    with pytest.raises(pkg.MboitError) as e:
        vol.synchronize()
    waited = time.perf_counter() - t0
    assert e.value.status == TIMEOUT and "TMA" in str(e.value)
    assert waited < 60.0                    # two bounded waits per warp, the warps side by side
    vol.synchronize()                       # reported once, then cleared
    vol.close()
    vol = pkg.Volume(sc)
    vol.set_tuning(cfg, 3)
    vol.set_frame_launches(launches)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    assert np.array_equal(col.cpu().numpy(), good.cpu().numpy())
    vol.close()


def test_tma_hook_rejects_wrong_kind(pkg):
    sc = scenes.tet_mesh(n=4, n_pieces=2, width=8, height=8)
    vol = pkg.Volume(sc)
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_debug_corrupt(vol.handle, 3)
    assert e.value.status == 1
    vol.close()


def test_second_stream_while_busy_is_refused(pkg):
    """One volume, one stream at a time: a frame on another stream while the
    first stream's frame still runs is refused with MBOIT_ERR_STATE and
    enqueues nothing; once that stream is done, the other stream may go."""
    import torch
    sc = scenes.blobs512(width=2048, height=2048)
    vol = pkg.Volume(sc)
    views = sc.views
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    vol.render_frame(views, mom, col, stream=sa)      # records the frame graph
    sa.synchronize()
    ref = col.clone()
    refused = 0
    for _ in range(3):
        for _ in range(4):
            vol.render_frame(views, mom, col, stream=sa)   # ~7 ms each, queued
        try:
            vol.render_frame(views, mom, col, stream=sb)
        except pkg.MboitError as e:
            assert e.status == STATE
            refused += 1
        sa.synchronize()
        sb.synchronize()
    assert refused == 3
    vol.render_frame(views, mom, col, stream=sb)      # stream a is idle now
    sb.synchronize()
    assert torch.equal(col, ref)
    vol.close()
