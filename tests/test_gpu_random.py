"""Seeded random scenes of every volume kind against the FP64 oracle: grid
shapes with ragged sizes (dims[0] % 4 of every residue), brick sizes, piece
counts, sampling steps, both projections in random directions, ragged image
sizes and the raw-sum flag; octrees of one and two refinement levels; meshes
of random resolutions.  Each frame must match the oracle within the 2e-4 bar
of four power moments, take exactly the oracle's samples, and equal the split
calls bit for bit."""
import numpy as np
import pytest

import oracle
import scenes

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


def _direction(s):
    while True:
        w = s.uniform(3, -1.0, 1.0)
        if np.linalg.norm(w) > 0.3:
            return tuple(float(x) for x in w / np.linalg.norm(w))


def _view(s, dims):
    w, h = 5 + int(s.uniform(1)[0] * 60), 5 + int(s.uniform(1)[0] * 60)
    if s.uniform(1)[0] < 0.5:
        return scenes.ortho_view(dims, _direction(s), w, h)
    return scenes.perspective_view(dims, _direction(s), w, h, fov_deg=20.0 + 30.0 * float(s.uniform(1)[0]))


def random_grid(seed):
    s = scenes.Stream(seed)
    dims = tuple(9 + int(x) for x in s.uniform(3) * 32)
    bl = 1 + int(s.uniform(1)[0] * 3)
    f = scenes.blob_field(dims, 4, 2.0, 8.0, s)
    tf = scenes.tf_table(s, 0.25)
    bd = tuple((n - 1 + (1 << bl) - 1) >> bl for n in dims)
    k = 1 + int(s.uniform(1)[0] * min(6, int(np.prod(bd))))
    piece = scenes.morton_pieces(bd, k, s)
    step = 0.5 if s.uniform(1)[0] < 0.7 else 0.25
    sc = scenes.GridScene(f"random_grid_{seed}", f, bl, piece, k, tf,
                          (np.float32(f.min()), np.float32(f.max())), step, [])
    sc.views = [_view(s, sc.dims)]
    return sc, s.uniform(1)[0] < 0.3


def _check(pkg, sc, ref, flags, want):
    import torch
    vol = pkg.Volume(sc, flags=flags)
    views = sc.views
    mom, col = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    vol.render_frame(views, mom, col)
    vol.synchronize()
    st = vol.stats()
    m2, c2 = pkg.Volume.moment_buffer(views), pkg.Volume.color_buffer(views)
    vol.render_moments(views, m2)
    vol.reconstruct_blend(views, m2, c2)
    vol.synchronize()
    torch.cuda.synchronize()
    vol.close()
    got = col.view(-1, 4).double().cpu().numpy()
    assert np.abs(got - ref[want]).max() <= 2e-4
    assert st["samples_pass1"] == int(ref["nsamples"].sum()) == st["samples_pass2"]
    assert torch.equal(mom, m2) and torch.equal(col, c2)


@pytest.mark.parametrize("seed", range(12))
def test_random_grid_matches_oracle(pkg, seed):
    sc, raw = random_grid(7000 + seed)
    want = "raw" if raw else "mboit"
    ref = oracle.render_grid(sc, want=(want, "nsamples"))
    _check(pkg, sc, ref, pkg.MBOIT_FLAG_RAW_SUM if raw else 0, want)


@pytest.mark.parametrize("seed", range(6))
def test_random_octree_matches_oracle(pkg, seed):
    s = scenes.Stream(8000 + seed)
    base, max_level = 2 + int(s.uniform(1)[0] * 3), 1 + int(s.uniform(1)[0] * 2)
    sc = scenes.amr_blobs(width=16, height=16, n_pieces=1 + int(s.uniform(1)[0] * 5), seed=8000 + seed,
                          base=base, max_level=max_level)
    sc.views = [_view(s, sc.dims)]
    ref = oracle.render_amr(sc, want=("mboit", "nsamples"))
    _check(pkg, sc, ref, 0, "mboit")


@pytest.mark.parametrize("seed", range(6))
def test_random_mesh_matches_oracle(pkg, seed):
    s = scenes.Stream(9000 + seed)
    sc = scenes.tet_mesh(n=4 + int(s.uniform(1)[0] * 4), n_pieces=1 + int(s.uniform(1)[0] * 4), width=16,
                         height=16, seed=9000 + seed)
    sc.views = [_view(s, sc.dims)]
    ref = oracle.render_amr(sc, want=("mboit", "nsamples"))
    _check(pkg, sc, ref, 0, "mboit")
