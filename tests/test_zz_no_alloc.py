"""The allocation-free pass 1, mboit_render_moments_noalloc.

It exists for embedders that must not allocate device memory: an in-situ
adaptor inside a simulation whose memory pool owns the device, a plugin whose
host application forbids side allocations, or a loop that cannot take the
implicit synchronisation of an allocation.  Its scratch is a fixed array
inside the library (at most 1,048,576 bricks).  These tests call it through
the C ABI and compare it with mboit_render_moments (REDUCED), which uses a
volume's allocated scratch, within the moment tolerance of the other GPU
tests.  Calls follow one another on one stream with a brick mask, without
one, and with another transfer function, so that nothing the shared array
keeps from a previous call (the mask, the table, the queue head) can pass
unnoticed.  This file is collected last on purpose."""
import copy

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

TOL_MOM = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    import paper_2501_12581_gb300 as pkg
    sc = scenes.blobs64(width=96, height=80)
    yield torch, pkg, sc


def _pixels(buf, view):
    a = buf.cpu().numpy().astype(np.float64)
    npx = view.width * view.height
    P = (npx + 3) // 4 * 4
    return np.concatenate([a[:npx, None], a[P:5 * P].reshape(P, 4)[:npx]], axis=1)


def _close(got, ref):
    scale = np.abs(ref).max(axis=-1, keepdims=True) + 1e-7
    err = np.abs(got - ref) / scale
    assert np.all(np.isfinite(got))
    assert err.max() <= TOL_MOM, f"moment error {err.max():.3e}"


def _reference(torch, pkg, sc, pieces):
    """mboit_render_moments of a volume built from the same inputs."""
    vol = pkg.Volume(sc)
    ref = pkg.Volume.moment_buffer(sc.views)
    vol.render_moments(sc.views, ref, pieces=pieces)
    torch.cuda.synchronize()
    want = _pixels(ref, sc.views[0])
    vol.close()
    assert want[:, 0].max() > 0
    return want


def test_noalloc_pass1_matches_render_moments(env):
    torch, pkg, sc = env
    other = copy.copy(sc)
    tf2 = sc.tf.copy()
    tf2[:, 3] = np.clip(tf2[:, 3] * 1.7 + 0.01, 0.0, 0.9)   # another opacity table
    tf2[:, :3] = tf2[::-1, :3]
    other.tf = tf2.astype(np.float32)
    # (scene, selected pieces) in call order: masked, unmasked, masked again,
    # another transfer function without a mask, then the first scene again
    calls = [(sc, [1, 3]), (sc, None), (sc, [0, 2]), (other, None), (sc, None)]
    field = torch.from_numpy(np.ascontiguousarray(sc.field)).cuda()
    for scene, pieces in calls:
        want = _reference(torch, pkg, scene, pieces)
        desc, keep = pkg.grid_desc(scene, field)
        mask = None if pieces is None else np.isin(scene.piece_of_brick, pieces).astype(np.uint8)
        out = pkg.Volume.moment_buffer(scene.views).fill_(float("nan"))
        pkg.mboit_render_moments_noalloc(desc, scene.views, out, brick_selected=mask)
        torch.cuda.synchronize()
        _close(_pixels(out, scene.views[0]), want)
        del keep


def test_noalloc_two_calls_in_a_row(env):
    """Two calls back to back on one stream, synchronised only at the end."""
    torch, pkg, sc = env
    want = _reference(torch, pkg, sc, None)
    field = torch.from_numpy(np.ascontiguousarray(sc.field)).cuda()
    desc, keep = pkg.grid_desc(sc, field)
    outs = [pkg.Volume.moment_buffer(sc.views).fill_(float("nan")) for _ in range(2)]
    for out in outs:
        pkg.mboit_render_moments_noalloc(desc, sc.views, out)
    torch.cuda.synchronize()
    for out in outs:
        _close(_pixels(out, sc.views[0]), want)
    del keep


def test_noalloc_rejects_bad_arguments(env):
    torch, pkg, sc = env
    field = torch.from_numpy(np.ascontiguousarray(sc.field)).cuda()
    desc, keep = pkg.grid_desc(sc, field)
    out = pkg.Volume.moment_buffer(sc.views)
    with pytest.raises(ValueError):
        pkg.mboit_render_moments_noalloc(desc, sc.views, out, brick_selected=np.ones(7, np.uint8))
    bad, keep_bad = pkg.grid_desc(sc, field)
    bad.overestimation = 1.5
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_render_moments_noalloc(bad, sc.views, out)
    assert e.value.status == 1 and "overestimation" in str(e.value)
    big, keep_big = pkg.grid_desc(sc, field)
    big.dims[:] = [1 << 12, 1 << 12, 2]   # 2^22 one-cell bricks > 2^20
    big.brick_log2 = 0
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_render_moments_noalloc(big, sc.views, out)
    assert e.value.status == 1 and "at most" in str(e.value)
    del keep, keep_bad, keep_big
