"""Failure detection through the device error word (mboit_synchronize).

The kernels test every table-derived index (octree leaf ids from the
finest-brick map, mesh tet ids from face neighbours and bin lists, bin ranges)
before the access it would make; a bad one is reported in the volume's error
word and the access is skipped.  Here a library-owned table is corrupted on
the host after validation (mboit_debug_corrupt), the volume renders, and
mboit_synchronize must report MBOIT_ERR_DEVICE_ASSERT once; no kernel reads
outside the tables, so the context stays usable."""
import numpy as np
import pytest

import scenes
from tests import _scenes_small as small

pytestmark = pytest.mark.gpu

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
