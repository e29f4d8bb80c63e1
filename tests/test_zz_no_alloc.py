"""The allocation-free pass 1, mboit_render_moments_noalloc.

It exists for embedders that must not allocate device memory: an in-situ
adaptor inside a simulation whose memory pool owns the device, a plugin whose
host application forbids side allocations, or a loop that cannot take the
implicit synchronisation of an allocation.  Its scratch is a fixed array
inside the library (at most 1,048,576 bricks).  These tests call it through
the C ABI and compare it with mboit_render_moments (REDUCED), which uses a
volume's allocated scratch, within the moment tolerance of the other GPU
tests, on two calls in a row (the array keeps the previous call's contents).
This file is collected last on purpose."""
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
    vol = pkg.Volume(sc)
    yield torch, pkg, sc, vol
    vol.close()


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


@pytest.mark.parametrize("pieces", [None, [1, 3]])
def test_noalloc_pass1_matches_render_moments(env, pieces):
    torch, pkg, sc, vol = env
    views = sc.views
    ref = pkg.Volume.moment_buffer(views)
    vol.render_moments(views, ref, pieces=pieces)
    torch.cuda.synchronize()
    want = _pixels(ref, views[0])
    assert want[:, 0].max() > 0
    desc, keep = pkg.grid_desc(sc, vol.field)
    mask = None if pieces is None else np.isin(sc.piece_of_brick, pieces).astype(np.uint8)
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        pkg.mboit_render_moments_noalloc(desc, views, out, brick_selected=mask)
        torch.cuda.synchronize()
        _close(_pixels(out, views[0]), want)
    del keep


def test_noalloc_rejects_volumes_beyond_its_scratch(env):
    torch, pkg, sc, vol = env
    desc, keep = pkg.grid_desc(sc, vol.field)
    desc.dims[:] = [1 << 12, 1 << 12, 2]   # 2^22 one-cell bricks > 2^20
    desc.brick_log2 = 0
    out = pkg.Volume.moment_buffer(sc.views)
    with pytest.raises(pkg.MboitError) as e:
        pkg.mboit_render_moments_noalloc(desc, sc.views, out)
    assert e.value.status == 1 and "at most" in str(e.value)
    del keep
