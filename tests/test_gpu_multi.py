"""Several volumes in one frame (mboit_render_frame_multi): one
persistent launch per pass over the ray tiles of every volume's views.  Each
view's moments and image must equal, bit for bit, its volume's own
mboit_render_frame (the per-tile code is the same); the calls' argument
checks reject what one launch cannot serve."""
import dataclasses

import numpy as np
import pytest

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


def _variant(sc, seed, name):
    """The scene with another field of the same shape, transfer function and
    step (its value range, and so its table mapping, its own)."""
    rng = np.random.default_rng(seed)
    f = np.ascontiguousarray(np.flip(sc.field, axis=int(rng.integers(0, 3))) * np.float32(0.7 + 0.2 * rng.random()))
    f = f.astype(np.float32)
    return dataclasses.replace(sc, name=name, field=f, tf_range=(np.float32(f.min()), np.float32(f.max())),
                               moment_bias=sc.moment_bias * 2.0)


def _slices(views, mom, col):
    """Per view: its moment slab and its RGBA image (as laid out for all views)."""
    out, mo, co = [], 0, 0
    for v in views:
        npx = v.width * v.height
        nm = 5 * ((npx + 3) // 4 * 4)
        out.append((mom[mo:mo + nm].clone(), col[co:co + 4 * npx].clone()))
        mo += nm
        co += 4 * npx
    return out


def _check_multi(pkg, scs, views, owner):
    import torch
    vols = [pkg.Volume(sc) for sc in scs]
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    pkg.Volume.render_frame_multi(vols, views, owner, mom, col)
    torch.cuda.synchronize()
    got = _slices(views, mom, col)
    st = vols[0].stats()
    total = 0
    for i, v in enumerate(vols):
        mine = [j for j in range(len(views)) if owner[j] == i]
        if not mine:
            continue
        sub = [views[j] for j in mine]
        m1, c1 = pkg.Volume.moment_buffer(sub), pkg.Volume.color_buffer(sub)
        v.set_frame_launches(2)
        v.render_frame(sub, m1, c1)
        v.synchronize()
        total += v.stats()["samples_pass1"]
        for (rm, rc), j in zip(_slices(sub, m1, c1), mine):
            assert torch.equal(got[j][0], rm), f"moments of view {j} differ"
            assert torch.equal(got[j][1], rc), f"image of view {j} differs"
    assert st["samples_pass1"] == total > 0
    for v in vols:
        v.close()


def test_multi_volume_frame_equals_each_volume_vector_windows(pkg):
    a = scenes.blobs64(width=61, height=37)
    b = _variant(a, 3, "blobs64_b")
    c = _variant(a, 5, "blobs64_c")
    views = [a.views[0],
             scenes.perspective_view(a.dims, (-0.5, 0.6, -0.62), 48, 40, fov_deg=40.0),
             scenes.ortho_view(a.dims, (0.1, 0.2, 0.97), 33, 29),
             small.axis_view(a.dims, 9, 5, -10.0, 4.0, centre=(300.0, 300.0)),   # misses the domain
             scenes.perspective_view(a.dims, (0.3, -0.8, 0.5), 40, 24)]
    _check_multi(pkg, [a, b, c], views, [0, 1, 2, 0, 1])


def test_multi_volume_frame_equals_each_volume_scalar_windows(pkg):
    # dims[0] % 4 != 0: the multi-volume launch takes configuration 0's windows
    a = small.linear_scene(dims=(17, 13, 11))
    b = _variant(a, 7, "linear_b")
    views = [small.axis_view(a.dims, 21, 17, -8.0, 20.0),
             scenes.perspective_view(a.dims, (0.57, 0.49, 0.66), 30, 26),
             scenes.ortho_view(a.dims, (-0.3, 0.2, 0.93), 19, 23)]
    _check_multi(pkg, [a, b], views, [1, 0, 1])


def test_multi_volume_frame_rejects(pkg):
    a = scenes.blobs64(width=16, height=16)
    b = _variant(a, 3, "blobs64_b")
    other_tf = dataclasses.replace(b, tf=np.ascontiguousarray(b.tf[::-1]))
    amr = scenes.amr_blobs(base=4, max_level=1, width=16, height=16, n_pieces=3)
    va, vb, vt, vm = pkg.Volume(a), pkg.Volume(b), pkg.Volume(other_tf), pkg.Volume(amr)
    views = a.views
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    cases = [([va, vt], [0], 1),       # another transfer function
             ([va, va], [0], 1),       # a volume listed twice
             ([va, vb], [2], 1),       # view_volume out of range
             ([va, vm], [0], 1)]       # a grid and an octree
    for vols, owner, status in cases:
        with pytest.raises(pkg.MboitError) as e:
            pkg.Volume.render_frame_multi(vols, views, owner, mom, col)
        assert e.value.status == status
    for v in (va, vb, vt, vm):
        v.close()
    # the adaptive step is not batched across volumes
    ad = dataclasses.replace(amr)
    ad.adaptive_step = True
    vad = pkg.Volume(ad)
    with pytest.raises(pkg.MboitError) as e:
        pkg.Volume.render_frame_multi([vad], views, [0], mom, col)
    assert e.value.status == 4
    vad.close()


def _amr_variant(sc, scale, name):
    v = np.ascontiguousarray(sc.values * np.float32(scale)).astype(np.float32)
    return dataclasses.replace(sc, name=name, values=v, tf_range=(np.float32(v.min()), np.float32(v.max())))


def test_multi_octree_frame_equals_each_volume(pkg):
    a = scenes.amr_blobs(base=4, max_level=2, width=45, height=38, n_pieces=5, seed=11)
    b = _amr_variant(scenes.amr_blobs(base=4, max_level=2, width=8, height=8, n_pieces=3, seed=12), 0.8, "amr_b")
    views = [a.views[0],
             scenes.perspective_view(a.dims, (-0.5, 0.6, -0.62), 40, 33, fov_deg=40.0),
             scenes.ortho_view(a.dims, (0.1, 0.2, 0.97), 29, 31)]
    _check_multi(pkg, [a, b], views, [0, 1, 1])


def test_multi_octree_with_holes(pkg):
    # an octree with holes among the volumes: the checked kernels
    amr, _ = small.linear_amr()
    amr.views = [scenes.perspective_view(amr.dims, (0.57, 0.49, 0.66), 30, 24)]
    holes = dataclasses.replace(amr, name="holes", leaves=amr.leaves[:-3], values=amr.values[:-3],
                                piece_of_leaf=amr.piece_of_leaf[:-3])
    views = [amr.views[0], scenes.ortho_view(amr.dims, (0.3, -0.8, 0.5), 27, 21)]
    _check_multi(pkg, [amr, holes], views, [1, 0])
