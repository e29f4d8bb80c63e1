"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, brute-force enumeration on tiny inputs, the moment-bound theory the
reconstruction rests on, or invariants the paper states (Sec. 4.1: moment
addition commutes, so per-piece moments sum to the single-node ones; Sec. 5.2:
APC reproduces single-node MBOIT; Fig. 6: per-rank partial images add up).
"""
import math

import numpy as np
import pytest

import oracle
import scenes
from tests import _scenes_small as small

W0 = 0.3  # overestimation used in the paper's evaluation (Sec. 5)


def raw_moments(x, a):
    x = np.asarray(x, float)
    a = np.asarray(a, float)
    return np.array([np.sum(a * x ** j) for j in range(5)])


# --------------------------------------------------------------------------
# Alg. 3: the moment bound


@pytest.mark.parametrize("x", [-0.7, 0.0, 0.42])
def test_one_absorber_exact(x):
    """One absorber, no bias: T(z) = 1 before it and e^-a after it."""
    a = 1.7
    m = raw_moments([x], [a])
    for z in np.linspace(-1, 1, 41):
        if abs(z - x) < 1e-9:
            continue
        A, branch = oracle.mboit_bound(m, z, 0.0, W0)
        assert branch == 1
        T = math.exp(-m[0] * A)
        assert T == pytest.approx(1.0 if z < x else math.exp(-a), abs=1e-12)


def test_two_absorbers_exact():
    """Two absorbers, no bias: T(z) = exp(-sum of the absorbances in front)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = np.sort(rng.uniform(-1, 1, 2))
        if x[1] - x[0] < 0.05:
            continue
        a = rng.uniform(0.05, 3.0, 2)
        m = raw_moments(x, a)
        for z in rng.uniform(-1, 1, 8):
            if np.min(np.abs(z - x)) < 1e-6:
                continue
            A, branch = oracle.mboit_bound(m, z, 0.0, W0)
            assert branch == 2
            assert math.exp(-m[0] * A) == pytest.approx(math.exp(-a[x < z].sum()), abs=1e-10)


def test_three_absorbers_canonical():
    """Generic branch.  A three-atom measure is the unique canonical
    representation through each of its atoms, so at z0 = x_j the bound is
    exactly (sum_{x_i < x_j} a_i + w0 a_j) / sum a."""
    rng = np.random.default_rng(2)
    n = 0
    while n < 500:
        x = np.sort(rng.uniform(-1, 1, 3))
        if np.diff(x).min() < 0.1:
            continue
        a = rng.uniform(0.1, 2.0, 3)
        w0 = rng.uniform(0, 1)
        m = raw_moments(x, a)
        for j in range(3):
            A, branch = oracle.mboit_bound(m, x[j], 0.0, w0)
            assert branch == 0
            assert A == pytest.approx((a[x < x[j]].sum() + w0 * a[j]) / a.sum(), abs=1e-11)
        n += 1


def test_full_bias_is_bias_vector_measure():
    """With mix amount 1 the moments become the bias vector (0, 3/8, 0, 3/8),
    the moments of the measure {-1: 3/16, 0: 5/8, 1: 3/16}."""
    m = raw_moments([0.3, -0.2, 0.9], [0.5, 1.0, 0.2])
    for w0 in (0.0, 0.3, 1.0):
        assert oracle.mboit_bound(m, -1.0, 1.0, w0)[0] == pytest.approx(w0 * 3 / 16, abs=1e-14)
        assert oracle.mboit_bound(m, 0.0, 1.0, w0)[0] == pytest.approx(3 / 16 + w0 * 5 / 8, abs=1e-14)
        assert oracle.mboit_bound(m, 1.0, 1.0, w0)[0] == pytest.approx(13 / 16 + w0 * 3 / 16, abs=1e-14)


def test_bound_containment():
    """Chebyshev-Markov-Stieltjes: with w0 = 0 the bound is a lower bound on
    the mass strictly in front of z, with w0 = 1 an upper bound on the mass
    up to and including z, for every measure with these moments."""
    rng = np.random.default_rng(3)
    for _ in range(300):
        k = rng.integers(3, 12)
        x = rng.uniform(-1, 1, k)
        a = rng.uniform(0.01, 1.0, k)
        m = raw_moments(x, a)
        for z in rng.uniform(-1, 1, 10):
            lo = oracle.mboit_bound(m, z, 0.0, 0.0)[0]
            hi = oracle.mboit_bound(m, z, 0.0, 1.0)[0]
            before = a[x < z].sum() / a.sum()
            upto = a[x <= z].sum() / a.sum()
            assert lo <= before + 1e-9
            assert upto <= hi + 1e-9


def test_bound_monotone_and_in_range():
    """A(z) = (1 - w0) * lower + w0 * upper is non-decreasing in z, in [0, 1]."""
    rng = np.random.default_rng(4)
    zs = np.linspace(-1, 1, 201)
    for _ in range(100):
        k = rng.integers(1, 20)
        m = raw_moments(rng.uniform(-1, 1, k), rng.uniform(0.01, 2.0, k))
        beta = 10 ** rng.uniform(-6, -1)
        A = np.array([oracle.mboit_bound(m, z, beta, W0)[0] for z in zs])
        assert np.all(A >= -1e-9) and np.all(A <= 1 + 1e-9)
        assert np.all(np.diff(A) >= -1e-7)


def test_log_warp_closed_form():
    n, f = 3.0, 48.0
    assert oracle.log_warp(n, n, f) == pytest.approx(-1.0, abs=1e-15)
    assert oracle.log_warp(f, n, f) == pytest.approx(1.0, abs=1e-15)
    assert oracle.log_warp(math.sqrt(n * f), n, f) == pytest.approx(0.0, abs=1e-14)
    assert oracle.log_warp(0.5, n, f) == -1.0
    assert oracle.log_warp(100.0, n, f) == 1.0


# --------------------------------------------------------------------------
# sampling, Alg. 2, stage one


def _f32_fma(a, b, c):
    # a*b of two float32 is exact in float64; the one rounding to float32
    # that follows matches fmaf except at exact float32 midpoints.
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _brute_samples(view, dims, step, px, py, kmax=6000):
    """Lattice points of one orthographic ray inside the domain, by enumeration."""
    f32 = np.float32
    fx, fy = f32(px) + f32(0.5), f32(py) + f32(0.5)
    sx = (fx / f32(view.width) - f32(0.5)) * view.scale_u
    sy = (fy / f32(view.height) - f32(0.5)) * view.scale_v
    o = [(view.eye[c] + sx * view.u[c]) + sy * view.v[c] for c in range(3)]
    d = [view.w[c] for c in range(3)]
    out = []
    for k in range(kmax):
        t = (f32(k) + f32(0.5)) * f32(step)
        p = [_f32_fma(t, d[c], o[c]) for c in range(3)]
        if all(f32(0) <= p[c] < f32(dims[c] - 1) for c in range(3)):
            out.append((float(t), [float(q) for q in p]))
    return out


def test_linear_field_brute_force():
    """Trilinear interpolation reproduces a linear field, and a linear sigma
    table is reproduced by linear lookup, so b_j = sum sigma(f(p_k)) step
    z(t_k)^j over the enumerated lattice points (catches axis transposition,
    lost or extra samples, wrong warp or power)."""
    sc = small.linear_scene()
    dims = sc.dims
    view = small.axis_view(dims, 7, 6, -9.0, 14.0, w=(0.36, 0.48, 0.8), u=(0.8, -0.6, 0.0),
                           v=(0.48, 0.64, -0.6), near=4.0, far=40.0, centre=(6.0, 7.0))
    view.eye = np.array([2.0, 1.0, -9.0], np.float32)
    sc.views = [view]
    r = oracle.render_grid(sc, want=("moments", "exact", "nsamples"))
    vmin, vmax = float(sc.tf_range[0]), float(sc.tf_range[1])
    hit = 0
    for py in range(view.height):
        for px in range(view.width):
            idx = py * view.width + px
            S = _brute_samples(view, dims, sc.step, px, py)
            assert r["nsamples"][idx] == len(S)
            m = np.zeros(5)
            acc = np.zeros(3)
            tau = 0.0
            for t, p in S:
                val = 0.25 + p[0] / 16 + p[1] / 32 + p[2] / 8
                xn = (val - vmin) / (vmax - vmin)
                a = (0.05 + 0.3 * xn) * sc.step
                z = min(max(2 * math.log(t / 4.0) / math.log(10.0) - 1, -1), 1)
                m += a * z ** np.arange(5)
                alpha = 1 - math.exp(-a)
                acc += math.exp(-tau) * alpha * np.array([xn, 1 - xn, 0.5])
                tau += a
            hit += len(S) > 0
            np.testing.assert_allclose(r["moments"][idx], m, rtol=2e-6, atol=1e-9)
            np.testing.assert_allclose(r["exact"][idx, :3], acc, rtol=2e-6, atol=1e-9)
            assert r["exact"][idx, 3] == pytest.approx(1 - math.exp(-tau), rel=2e-6, abs=1e-9)
    assert hit > 20


def test_constant_slab_zeroth_moment():
    """Field = 1, constant opacity, the slab is one z-layer of bricks, rays
    along +z with lattice points on the slab faces' half-step offsets: b0 =
    sigma L exactly; b_j is the midpoint rule of the integral of
    sigma z(t)^j, within its O(step^2) error bound."""
    alpha = 0.1
    sc = small.slab_scene(alpha=alpha)
    sigma = -math.log(1 - np.float64(np.float32(alpha)))
    view = small.axis_view(sc.dims, 8, 8, -10.0, 16.0, near=5.0, far=60.0)
    sc.views = [view]
    r = oracle.render_grid(sc, pieces=[1], want=("moments", "nsamples"))
    L = 8.0  # one 8-cell brick layer, z in [8, 16)
    assert np.all(r["nsamples"] == 16)
    np.testing.assert_allclose(r["moments"][:, 0], sigma * L, rtol=1e-14)
    # midpoint rule of int_{18}^{26} sigma z(t)^j dt (t from the eye plane)
    ln = math.log(60.0 / 5.0)
    t = np.linspace(18.0, 26.0, 20001)
    for j in range(1, 5):
        g = sigma * (2 * np.log(t / 5.0) / ln - 1) ** j
        integ = np.trapezoid(g, t)
        g2 = np.abs(np.gradient(np.gradient(g, t), t)).max()
        bound = 8.0 * 0.5 ** 2 / 24 * g2 * 1.5 + 1e-9
        assert abs(r["moments"][0, j] - integ) <= bound


def test_oblique_slab_zeroth_moment():
    """Oblique rays: b0 is within sigma*step of sigma times the chord."""
    alpha = 0.1
    sc = small.slab_scene(alpha=alpha)
    sigma = -math.log(1 - np.float64(np.float32(alpha)))
    w = np.array([0.3, 0.2, 1.0])
    w /= np.linalg.norm(w)
    u = np.cross(w, [0, 1, 0])
    u /= np.linalg.norm(u)
    v = np.cross(u, w)
    view = small.axis_view(sc.dims, 6, 6, -10.0, 6.0, w=w, u=u, v=v)
    sc.views = [view]
    r = oracle.render_grid(sc, pieces=[1], want=("moments",))
    chord = 8.0 / w[2]
    assert np.all(np.abs(r["moments"][:, 0] - sigma * chord) <= sigma * 0.5 + 1e-12)


# --------------------------------------------------------------------------
# stage one / two invariants (Sec. 4.1, 4.2, 5.2, Fig. 6)


def _one_piece(sc):
    import copy
    s1 = copy.copy(sc)
    s1.piece_of_brick = np.zeros_like(sc.piece_of_brick)
    s1.n_pieces = 1
    return s1


def test_union_equals_sum(blobs64):
    """Per-piece moment images summed equal the single-node moments."""
    r = oracle.render_grid(blobs64, want=("piece_moments", "moments"))
    u = oracle.render_grid(_one_piece(blobs64), want=("moments",))
    s = r["piece_moments"].sum(axis=1)
    scale = np.abs(u["moments"]).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(s - u["moments"]) / scale) <= 1e-12
    # every piece contributes somewhere: the partition is really used
    assert np.all(np.abs(r["piece_moments"][:, :, 0]).sum(axis=0) > 0)


def test_piece_order_independence(blobs64):
    """Relabelling pieces (a different reduction order) changes nothing."""
    import copy
    perm = np.array([2, 0, 3, 1], np.int32)
    s2 = copy.copy(blobs64)
    s2.piece_of_brick = perm[blobs64.piece_of_brick]
    a = oracle.render_grid(blobs64, want=("moments", "mboit"))
    b = oracle.render_grid(s2, want=("moments", "mboit"))
    np.testing.assert_allclose(a["moments"], b["moments"], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(a["mboit"], b["mboit"], rtol=1e-12, atol=1e-14)


def test_alpha_identity_and_sortlast(blobs64):
    """Renormalised MBOIT alpha = exact alpha = 1 - e^-b0; per-piece segments
    sorted and blended equal the global front-to-back march."""
    r = oracle.render_grid(blobs64, want=("moments", "mboit", "exact", "sortlast"))
    np.testing.assert_allclose(r["mboit"][:, 3], r["exact"][:, 3], atol=1e-12)
    np.testing.assert_allclose(r["mboit"][:, 3], 1 - np.exp(-r["moments"][:, 0]), atol=1e-15)
    np.testing.assert_allclose(r["sortlast"], r["exact"], atol=1e-12)
    # MBOIT is an approximation of the exact blend, not a copy of it
    assert 1e-4 < np.abs(r["mboit"] - r["exact"]).max() < 0.2


def test_sandwich_partials_add_up():
    """Fig. 6: three ranks of interleaved slices; the per-rank partial images
    rendered with the global moments sum to the single-node MBOIT image."""
    sc = small.sandwich_scene()
    sc.views = [scenes.ortho_view(sc.dims, (0.3, 0.25, 0.92), 24, 24)]
    r = oracle.render_grid(sc, want=("piece_color", "raw", "mboit"))
    u = oracle.render_grid(_one_piece(sc), want=("raw", "mboit"))
    np.testing.assert_allclose(r["piece_color"].sum(axis=1), u["raw"], atol=1e-12)
    np.testing.assert_allclose(r["mboit"], u["mboit"], atol=1e-12)
    for P in range(3):
        assert r["piece_color"][:, P, 3].max() > 1e-3


def test_sortlast_segments_of_interleaved_slabs():
    """Fig. 6 geometry: six z-slabs dealt to three pieces in turn; a ray along
    +z crosses six slabs, so each piece contributes two segments."""
    sc = small.sandwich_scene()
    sc.views = [small.axis_view(sc.dims, 6, 6, -10.0, 10.0, near=5.0, far=60.0)]
    rgba, nseg = oracle.render_segments(sc)
    assert np.all(nseg == 6)
    np.testing.assert_allclose(rgba, oracle.render_grid(sc, want=("exact",))["exact"], atol=1e-12)


def test_empty_and_missing_rays():
    """Rays that miss the domain produce zero moments and a zero image."""
    sc = small.slab_scene()
    sc.views = [small.axis_view(sc.dims, 4, 4, -10.0, 4.0, centre=(100.0, 100.0))]
    r = oracle.render_grid(sc, want=("moments", "mboit", "exact", "nsamples"))
    assert np.all(r["nsamples"] == 0)
    assert np.all(r["moments"] == 0) and np.all(r["mboit"] == 0) and np.all(r["exact"] == 0)


# --------------------------------------------------------------------------
# brick octree (AMR) sampling


def test_amr_linear_field_equals_finest_grid():
    """Trilinear interpolation reproduces a linear field at every level, so
    the octree render equals the finest regular grid's (pins leaf lookup,
    local coordinates, level scaling and vertex layout)."""
    amr, grid = small.linear_amr()
    assert set(np.unique(amr.leaves[:, 3])) == {0, 1, 2}
    views = [scenes.ortho_view(amr.dims, (0.4, 0.5, 0.77), 24, 20),
             scenes.perspective_view(amr.dims, (-0.6, 0.45, 0.66), 18, 16, fov_deg=35.0)]
    for v in views:
        a = oracle.render_amr(amr, view=v, want=("moments", "mboit", "exact", "nsamples"))
        g = oracle.render_grid(grid, view=v, want=("moments", "mboit", "exact", "nsamples"))
        np.testing.assert_array_equal(a["nsamples"], g["nsamples"])
        np.testing.assert_allclose(a["moments"], g["moments"], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(a["mboit"], g["mboit"], atol=1e-12)
        np.testing.assert_allclose(a["exact"], g["exact"], atol=1e-12)


def test_amr_pieces_sum_and_sortlast():
    sc = scenes.amr_blobs(base=4, max_level=2, width=32, height=28, n_pieces=5)
    r = oracle.render_amr(sc, want=("piece_moments", "moments", "exact", "sortlast", "mboit"))
    np.testing.assert_allclose(r["piece_moments"].sum(axis=1), r["moments"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["sortlast"], r["exact"], atol=1e-12)
    assert np.abs(r["mboit"] - r["exact"]).max() > 1e-4
    assert (r["moments"][:, 0] > 0).mean() > 0.3


def test_amr_overlapping_leaves_rejected():
    amr, _ = small.linear_amr()
    import copy
    bad = copy.copy(amr)
    bad.leaves = np.concatenate([amr.leaves, amr.leaves[:1]])
    bad.values = np.concatenate([amr.values, amr.values[:1]])
    bad.piece_of_leaf = np.zeros(len(bad.leaves), np.int32)
    bad.views = [scenes.ortho_view(amr.dims, (0.4, 0.5, 0.77), 4, 4)]
    with pytest.raises(ValueError):
        oracle.render_amr(bad)


def test_amr_leaf_lookup_brute_force():
    """A different constant in every leaf, a linear extinction table: each
    ray's b0 and b1 must equal the sums over the enumerated lattice points of
    the containing leaf's extinction, the leaf found by testing every box."""
    amr, _ = small.linear_amr()
    n = len(amr.leaves)
    const = (np.arange(n) % 7) / 8.0 + 0.125
    amr.values = np.broadcast_to(const[:, None, None, None], (n, 9, 9, 9)).astype(np.float32).copy()
    amr.tf_range = (np.float32(0.0), np.float32(1.0))
    view = small.axis_view(amr.dims, 9, 7, -20.0, 60.0, w=(0.36, 0.48, 0.8), u=(0.8, -0.6, 0.0),
                           v=(0.48, 0.64, -0.6), near=4.0, far=300.0, centre=(40.0, 44.0))
    view.eye = np.array([30.0, 20.0, -20.0], np.float32)
    r = oracle.render_amr(amr, view=view, want=("moments", "nsamples"))
    size = (8 << amr.max_level) >> amr.leaves[:, 3]
    lo, hi = amr.leaves[:, :3].astype(np.float64), amr.leaves[:, :3] + size[:, None]
    dims = amr.dims
    hit = 0
    for py in range(view.height):
        for px in range(view.width):
            S = _brute_samples(view, dims, amr.step, px, py)
            m0 = m1 = 0.0
            for t, p in S:
                inside = np.all((lo <= p) & (np.array(p) < hi), axis=1)
                assert inside.sum() == 1
                val = const[np.argmax(inside)]
                a = (0.04 + 0.2 * val) * amr.step
                z = min(max(2 * math.log(t / 4.0) / math.log(300.0 / 4.0) - 1, -1), 1)
                m0 += a
                m1 += a * z
            idx = py * view.width + px
            assert r["nsamples"][idx] == len(S)
            np.testing.assert_allclose(r["moments"][idx, :2], [m0, m1], rtol=2e-6, atol=1e-9)
            hit += len(S) > 0
    assert hit > 30


def test_amr_adaptive_step_brute_force():
    """Adaptive dyadic step: a lattice point k in a leaf of level L counts
    only if k is a multiple of 2^(max_level - L), with absorbance
    sigma * step * 2^(max_level - L).  Each ray's sample count, b0 and b1
    against the enumerated lattice points, the leaf found by testing every
    box."""
    import copy
    amr, _ = small.linear_amr()
    n = len(amr.leaves)
    const = (np.arange(n) % 7) / 8.0 + 0.125
    amr.values = np.broadcast_to(const[:, None, None, None], (n, 9, 9, 9)).astype(np.float32).copy()
    amr.tf_range = (np.float32(0.0), np.float32(1.0))
    amr = copy.copy(amr)
    amr.adaptive_step = True
    view = small.axis_view(amr.dims, 9, 7, -20.0, 60.0, w=(0.36, 0.48, 0.8), u=(0.8, -0.6, 0.0),
                           v=(0.48, 0.64, -0.6), near=4.0, far=300.0, centre=(40.0, 44.0))
    view.eye = np.array([30.0, 20.0, -20.0], np.float32)
    r = oracle.render_amr(amr, view=view, want=("moments", "nsamples"))
    size = (8 << amr.max_level) >> amr.leaves[:, 3]
    lo, hi = amr.leaves[:, :3].astype(np.float64), amr.leaves[:, :3] + size[:, None]
    hit = skipped = 0
    for py in range(view.height):
        for px in range(view.width):
            S = _brute_samples(view, amr.dims, amr.step, px, py)
            m0 = m1 = 0.0
            count = 0
            for t, p in S:
                k = int(round(t / amr.step - 0.5))
                inside = np.all((lo <= p) & (np.array(p) < hi), axis=1)
                leaf = np.argmax(inside)
                stride = 1 << (amr.max_level - int(amr.leaves[leaf, 3]))
                if k % stride:
                    skipped += 1
                    continue
                a = (0.04 + 0.2 * const[leaf]) * amr.step * stride
                z = min(max(2 * math.log(t / 4.0) / math.log(300.0 / 4.0) - 1, -1), 1)
                m0 += a
                m1 += a * z
                count += 1
            idx = py * view.width + px
            assert r["nsamples"][idx] == count
            np.testing.assert_allclose(r["moments"][idx, :2], [m0, m1], rtol=2e-6, atol=1e-9)
            hit += count > 0
    assert hit > 30 and skipped > 100


def test_amr_adaptive_step_single_level_and_pieces():
    """With one level the nested lattice is the full one (adaptive = fixed,
    bit for bit); on a three-level octree the pieces' moments still add up
    to the global ones, the sort-last route still equals the exact blend of
    the same samples, and fewer samples are taken."""
    import copy
    one = scenes.amr_blobs(base=4, max_level=0, width=24, height=20, n_pieces=3)
    ad = copy.copy(one)
    ad.adaptive_step = True
    a = oracle.render_amr(ad, want=("moments", "mboit", "nsamples"))
    f = oracle.render_amr(one, want=("moments", "mboit", "nsamples"))
    np.testing.assert_array_equal(a["nsamples"], f["nsamples"])
    np.testing.assert_array_equal(a["moments"], f["moments"])
    np.testing.assert_array_equal(a["mboit"], f["mboit"])
    sc = scenes.amr_blobs(base=4, max_level=2, width=32, height=28, n_pieces=5)
    ad = copy.copy(sc)
    ad.adaptive_step = True
    r = oracle.render_amr(ad, want=("piece_moments", "moments", "exact", "sortlast", "nsamples"))
    fixed = oracle.render_amr(sc, want=("nsamples",))
    np.testing.assert_allclose(r["piece_moments"].sum(axis=1), r["moments"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["sortlast"], r["exact"], atol=1e-12)
    assert r["nsamples"].sum() < 0.8 * fixed["nsamples"].sum()
    assert np.all(r["nsamples"] <= fixed["nsamples"])


def test_gear_teeth_layout_and_segments():
    """Sec. 5 stress test: piece p owns layers p, p + K, p + 2K, p + 3K (one
    brick thick), so a ray along the stacking axis meets exactly 4K segments
    of alternating pieces; the sort-last route equals the exact blend and the
    pieces' moments add up."""
    K = 3
    sc = scenes.gear_teeth(n_pieces=K, footprint=16, width=8, height=8, n_views=1)
    nb = sc.brick_dims
    layers = sc.piece_of_brick.reshape(nb[2], nb[1], nb[0])
    assert np.all(layers == (np.arange(nb[2]) % K)[:, None, None])
    for p in range(K):
        assert np.flatnonzero(layers[:, 0, 0] == p).tolist() == [p, p + K, p + 2 * K, p + 3 * K]
    view = small.axis_view(sc.dims, 6, 6, -10.0, 12.0, near=5.0, far=60.0)
    r = oracle.render_grid(sc, view=view, want=("exact", "sortlast", "moments", "piece_moments"))
    _, segs = oracle.render_segments(sc, view=view)
    assert np.all(segs == 4 * K)
    np.testing.assert_allclose(r["sortlast"], r["exact"], atol=1e-12)
    np.testing.assert_allclose(r["piece_moments"].sum(axis=1), r["moments"], rtol=1e-12, atol=1e-14)
    # b0 = sigma * depth on these axis-aligned rays (24 cells, 48 samples)
    sigma = -np.log1p(-np.float64(sc.tf[0, 3]))
    np.testing.assert_allclose(r["moments"][:, 0], sigma * 0.5 * 48, rtol=1e-9)


# --------------------------------------------------------------------------
# trigonometric moments (Sec. 4.3, Fig. 3: "different moments")


def trig_moments(phis, a, n):
    t = [np.sum(a * np.exp(1j * j * np.asarray(phis))) for j in range(n + 1)]
    return np.array([t[0].real] + sum([[t[j].real, t[j].imag] for j in range(1, n + 1)], []))


@pytest.mark.parametrize("n", [3, 4])
def test_trig_n_plus_one_atoms_canonical(n):
    """n+1 atoms on the circle are their own Szego representation through
    each atom: A(phi_j) = (sum_{phi_i < phi_j} a_i + w0 a_j) / sum a."""
    rng = np.random.default_rng(10 + n)
    done = 0
    while done < 200:
        phis = np.sort(rng.uniform(-0.9 * np.pi, 0.9 * np.pi, n + 1))
        if np.diff(phis).min() < 0.25:
            continue
        a = rng.uniform(0.1, 2.0, n + 1)
        w0 = rng.uniform(0, 1)
        m = trig_moments(phis, a, n)
        for j in range(n + 1):
            A, st, ws = oracle.trig_bound(m, n, phis[j], 0.0, w0)
            assert st == 0
            assert ws == pytest.approx(1.0, abs=1e-11)
            assert A == pytest.approx((a[phis < phis[j]].sum() + w0 * a[j]) / a.sum(), abs=1e-10)
        done += 1


@pytest.mark.parametrize("n", [3, 4])
def test_trig_full_bias_is_uniform_measure(n):
    """Mix amount 1 leaves the uniform measure: the nodes through u0 are the
    (n+1)-th roots of unity times u0, each of weight 1/(n+1)."""
    m = trig_moments([0.4, -1.1], np.array([1.0, 0.5]), n)
    for phi0 in np.linspace(-2.8, 2.8, 9):
        nodes = np.angle(np.exp(1j * (phi0 + 2 * np.pi * np.arange(1, n + 1) / (n + 1))))
        A, st, ws = oracle.trig_bound(m, n, phi0, 1.0, 0.3)
        assert A == pytest.approx((0.3 + np.sum(nodes < phi0)) / (n + 1), abs=1e-12)


@pytest.mark.parametrize("n", [3, 4])
def test_trig_representation_reproduces_moments(n):
    """For any biased moments and any u0 the representation is exact: its
    nodes lie on the circle, its weights are positive and sum to 1, and
    sum_i rho_i u_i^j equals the biased normalised moment tau'_j; the bound
    lies in [0, 1]."""
    rng = np.random.default_rng(20 + n)
    for _ in range(60):
        k = rng.integers(1, 15)
        m = trig_moments(rng.uniform(-0.9 * np.pi, 0.9 * np.pi, k), rng.uniform(0.05, 2, k), n)
        beta = 10 ** rng.uniform(-4, -1)
        tau = (1 - beta) * (m[1::2] + 1j * m[2::2]) / m[0]
        for phi0 in rng.uniform(-0.9 * np.pi, 0.9 * np.pi, 5):
            u, w, st = oracle.trig_nodes(m, n, phi0, beta)
            assert st == 0
            np.testing.assert_allclose(np.abs(u), 1.0, atol=1e-12)
            assert np.all(w > 0) and w.sum() == pytest.approx(1.0, abs=1e-10)
            for j in range(1, n + 1):
                assert np.sum(w * u ** j) == pytest.approx(tau[j - 1], abs=1e-9)
            A = oracle.trig_bound(m, n, phi0, beta, 0.3)[0]
            assert -1e-12 <= A <= 1 + 1e-12


def test_trig_storage_rounding_matches_numpy():
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-1, 1, 2000), rng.uniform(-1e-3, 1e-3, 500), [0.0, 1.0, -1.0, 0.1]])
    for x in xs:
        assert oracle.store_round(x, "f16") == float(np.float16(np.float32(x)))
        u = np.array([np.float32(x)]).view(np.uint32).astype(np.uint64)
        u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
        assert oracle.store_round(x, "bf16") == float(u.view(np.float32)[0])


def test_trig_render_quantised_storage_changes_little():
    """The 16-bit stored moments give images close to the float64 ones."""
    import copy
    sc = scenes.blobs64(width=48, height=48)
    out = {}
    for st, beta in (("f32", 1e-5), ("f16", 2e-3), ("bf16", 2e-2)):
        s2 = copy.copy(sc)
        s2.moment_set, s2.storage, s2.moment_bias = "trig6", st, beta
        out[st] = oracle.render_grid(s2, want=("mboit", "exact"))
    for st in ("f16", "bf16"):
        assert np.abs(out[st]["mboit"] - out["f32"]["mboit"]).max() < 0.1
    assert np.sqrt(((out["f32"]["mboit"] - out["f32"]["exact"]) ** 2).mean()) < 0.02


@pytest.mark.parametrize("n", [3, 4])
def test_trig_node_just_behind_is_not_counted(n):
    """Two atoms 0.03 rad apart among n+1: at the front one, the one just
    behind must not count (and at the back one, the front one must)."""
    rng = np.random.default_rng(30 + n)
    for _ in range(50):
        base = np.sort(rng.uniform(-0.8 * np.pi, 0.7 * np.pi, n))
        if np.diff(base).min() < 0.3:
            continue
        phis = np.sort(np.concatenate([base, [base[0] + 0.03]]))
        a = rng.uniform(0.2, 2.0, n + 1)
        m = trig_moments(phis, a, n)
        for j in range(n + 1):
            A = oracle.trig_bound(m, n, phis[j], 0.0, 0.5)[0]
            assert A == pytest.approx((a[phis < phis[j]].sum() + 0.5 * a[j]) / a.sum(), abs=1e-6)


# --------------------------------------------------------------------------
# Alg. 3 with 6 and 8 power moments (the moment-count variants of Sec. 4.3 /
# Fig. 3): the bound of order n uses b0..b_2n and a (n+1) x (n+1) Hankel matrix


def power_moments(x, a, n):
    x = np.asarray(x, float)
    a = np.asarray(a, float)
    return np.array([np.sum(a * x ** j) for j in range(2 * n + 1)])


def arcsine_moments(n):
    """b1..b2n of the arcsine law on [-1, 1]: b_2k = C(2k, k) / 4^k."""
    return np.array([0.0 if j % 2 else math.comb(j, j // 2) / 4.0 ** (j // 2) for j in range(1, 2 * n + 1)])


def test_power_bias_is_arcsine_law():
    for n in (3, 4):
        np.testing.assert_allclose(oracle.power_bias(n), arcsine_moments(n), rtol=0, atol=1e-15)


def test_power_order_two_equals_four_moment_routine():
    """The order-n routine at n = 2 (bias (0, 3/8, 0, 3/8)) reproduces the
    4-moment routine on generic and one-/two-atom measures."""
    rng = np.random.default_rng(40)
    for _ in range(1000):
        k = rng.integers(1, 12)
        m = power_moments(rng.uniform(-1, 1, k), rng.uniform(0.01, 1, k), 2)
        z0, beta, w0 = rng.uniform(-1, 1), rng.choice([0.0, 5e-5, 1e-2]), rng.uniform(0, 1)
        A4, b4 = oracle.mboit_bound(m, z0, beta, w0)
        An, bn, _ = oracle.power_bound(m, 2, z0, beta, w0, bias=oracle.BIAS_VECTOR_POWER4)
        assert bn == b4
        assert An == pytest.approx(A4, abs=1e-11)


@pytest.mark.parametrize("n", [3, 4])
def test_power_few_atoms_exact(n):
    """k <= n absorbers, no bias: the Hankel matrix is singular, the measure
    is recovered and T(z) = exp(-sum of the absorbances in front)."""
    rng = np.random.default_rng(41 + n)
    for k in range(1, n + 1):
        done = 0
        while done < 60:
            x = np.sort(rng.uniform(-1, 1, k))
            if k > 1 and np.diff(x).min() < 0.05:
                continue
            a = rng.uniform(0.05, 3.0, k)
            m = power_moments(x, a, n)
            for z in rng.uniform(-1, 1, 6):
                if np.min(np.abs(z - x)) < 1e-4:
                    continue
                A, branch, nodes = oracle.power_bound(m, n, z, 0.0, rng.uniform(0, 1))
                assert branch == k
                np.testing.assert_allclose(nodes[:k], x, atol=1e-7)
                assert math.exp(-m[0] * A) == pytest.approx(math.exp(-a[x < z].sum()), abs=1e-9)
            done += 1


@pytest.mark.parametrize("n", [3, 4])
def test_power_n_plus_one_atoms_canonical(n):
    """Generic branch.  n+1 atoms are the canonical representation through
    each of their atoms, so at z0 = x_j the bound is exactly
    (sum_{x_i < x_j} a_i + w0 a_j) / sum a."""
    rng = np.random.default_rng(50 + n)
    done = 0
    while done < 200:
        x = np.sort(rng.uniform(-1, 1, n + 1))
        if np.diff(x).min() < 0.1:
            continue
        a = rng.uniform(0.1, 2.0, n + 1)
        w0 = rng.uniform(0, 1)
        m = power_moments(x, a, n)
        for j in range(n + 1):
            A, branch, _ = oracle.power_bound(m, n, x[j], 0.0, w0)
            assert branch == 0
            assert A == pytest.approx((a[x < x[j]].sum() + w0 * a[j]) / a.sum(), abs=1e-8)
        done += 1


@pytest.mark.parametrize("n", [3, 4])
def test_power_full_bias_is_arcsine_gauss_rule(n):
    """Mix amount 1 leaves the arcsine law, whose (n+1)-point Gauss rule has
    nodes cos((2k - 1) pi / (2n + 2)) and weights 1/(n+1) and integrates
    degree 2n+1 exactly: through one of its nodes it is the canonical
    representation, so A = (w0 + nodes in front) / (n + 1)."""
    m = power_moments([0.3, -0.2, 0.9], [0.5, 1.0, 0.2], n)
    g = np.sort(np.cos((2 * np.arange(1, n + 2) - 1) * np.pi / (2 * n + 2)))
    for j, z0 in enumerate(g):
        for w0 in (0.0, 0.3, 1.0):
            A, branch, nodes = oracle.power_bound(m, n, z0, 1.0, w0)
            assert branch == 0
            np.testing.assert_allclose(np.sort(nodes), g, atol=1e-9)
            assert A == pytest.approx((w0 + j) / (n + 1), abs=1e-10)


@pytest.mark.parametrize("n", [3, 4])
def test_power_representation_christoffel_weights(n):
    """The support points are a quadrature exact to degree 2n: with the
    Christoffel weights 1 / K(x, x) (K(x, y) = v(x)^T H^-1 v(y), H the biased
    Hankel matrix) they reproduce every biased moment b0'..b2n', and the
    bound equals w0 rho(z0) + the weights of the points in front."""
    rng = np.random.default_rng(60 + n)
    for _ in range(100):
        k = rng.integers(n + 1, 25)
        m = power_moments(rng.uniform(-1, 1, k), rng.uniform(0.01, 1, k), n)
        beta = rng.choice([0.0, 1e-3, 5e-2])
        b = np.concatenate([[1.0], (1 - beta) * m[1:] / m[0] + beta * arcsine_moments(n)])
        H = np.array([[b[i + j] for j in range(n + 1)] for i in range(n + 1)])
        Hinv = np.linalg.inv(H)
        for z0 in rng.uniform(-1, 1, 4):
            w0 = rng.uniform(0, 1)
            A, branch, x = oracle.power_bound(m, n, z0, beta, w0)
            assert branch == 0 and x[0] == z0
            rho = np.array([1.0 / (x[i] ** np.arange(n + 1) @ Hinv @ x[i] ** np.arange(n + 1)) for i in range(n + 1)])
            assert np.all(rho > 0)
            for j in range(2 * n + 1):
                assert np.sum(rho * x ** j) == pytest.approx(b[j], abs=1e-8)
            assert A == pytest.approx(w0 * rho[0] + rho[1:][x[1:] < z0].sum(), abs=1e-8)


def test_power_bounds_nest_and_contain():
    """Chebyshev-Markov-Stieltjes with more moments: the lower bound (w0 = 0)
    rises and the upper bound (w0 = 1) falls as n goes 2 -> 3 -> 4, and both
    keep containing the true mass in front of z."""
    rng = np.random.default_rng(70)
    for _ in range(400):
        k = rng.integers(6, 30)
        x = rng.uniform(-1, 1, k)
        a = rng.uniform(0.01, 1.0, k)
        z = rng.uniform(-1, 1)
        lo, hi = [], []
        for n in (2, 3, 4):
            m = power_moments(x, a, n)
            bias = oracle.BIAS_VECTOR_POWER4 if n == 2 else None
            lo.append(oracle.power_bound(m, n, z, 0.0, 0.0, bias=bias)[0])
            hi.append(oracle.power_bound(m, n, z, 0.0, 1.0, bias=bias)[0])
        before, upto = a[x < z].sum() / a.sum(), a[x <= z].sum() / a.sum()
        e = 1e-9
        assert lo[0] <= lo[1] + e and lo[1] <= lo[2] + e and lo[2] <= before + e
        assert upto <= hi[2] + e and hi[2] <= hi[1] + e and hi[1] <= hi[0] + e


@pytest.mark.parametrize("n", [3, 4])
def test_power_bound_equals_linear_program(n):
    """Brute force: over all non-negative measures on a fine grid with the
    given 2n+1 moments, the largest mass in (-inf, z0] is the bound with
    w0 = 1 and the smallest mass in (-inf, z0) the bound with w0 = 0 (up to
    the grid's resolution)."""
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(80 + n)
    done = 0
    while done < 6:
        k = rng.integers(n + 2, 10)
        x = np.round(rng.uniform(-1, 1, k), 3)
        z0 = round(float(rng.uniform(-0.8, 0.8)), 3)
        if np.min(np.abs(x - z0)) < 0.01:
            continue
        a = rng.uniform(0.05, 1.0, k)
        m = power_moments(x, a, n)
        b = m / m[0]
        hi = oracle.power_bound(m, n, z0, 0.0, 1.0)[0]
        lo, _, nodes = oracle.power_bound(m, n, z0, 0.0, 0.0)
        R = max(1.0, float(np.nanmax(np.abs(nodes)))) + 0.25
        grid = np.unique(np.concatenate([np.linspace(-R, R, int(2 * R / 5e-4) + 1), [z0], x]))
        # equality constraints in the Chebyshev basis of [-R, R] (well scaled)
        V = np.polynomial.chebyshev.chebvander(grid / R, 2 * n).T
        C = np.zeros((2 * n + 1, 2 * n + 1))
        for j in range(2 * n + 1):
            c = np.polynomial.chebyshev.cheb2poly(np.eye(2 * n + 1)[j])
            C[j, :len(c)] = c / R ** np.arange(len(c))
        rhs = C @ b
        r_hi = opt.linprog(-(grid <= z0).astype(float), A_eq=V, b_eq=rhs, bounds=(0, None), method="highs")
        r_lo = opt.linprog((grid < z0).astype(float), A_eq=V, b_eq=rhs, bounds=(0, None), method="highs")
        if r_hi.status != 0 or r_lo.status != 0:
            continue
        assert -r_hi.fun == pytest.approx(hi, abs=2e-4)
        assert r_lo.fun == pytest.approx(lo, abs=2e-4)
        done += 1


@pytest.mark.parametrize("n", [3, 4])
def test_power_bound_monotone_and_in_range(n):
    rng = np.random.default_rng(90 + n)
    zs = np.linspace(-1, 1, 201)
    for _ in range(60):
        k = rng.integers(1, 20)
        m = power_moments(rng.uniform(-1, 1, k), rng.uniform(0.01, 2.0, k), n)
        beta = 10 ** rng.uniform(-5, -1)
        A = np.array([oracle.power_bound(m, n, z, beta, W0)[0] for z in zs])
        assert np.all(A >= -1e-9) and np.all(A <= 1 + 1e-9)
        assert np.all(np.diff(A) >= -1e-7)


def test_power_render_more_moments_closer_to_exact():
    """Rendering with 6 and 8 power moments: the moment images of the pieces
    add up to the global ones, alpha is exact, and the image moves towards the
    exact blend as moments are added (Fig. 3)."""
    import copy
    sc = scenes.blobs64(width=40, height=40)
    rmse, first5 = {}, None
    for ms, beta in (("power4", 5e-5), ("power6", 5e-5), ("power8", 5e-5)):
        s2 = copy.copy(sc)
        s2.moment_set, s2.moment_bias = ms, beta
        out = oracle.render_grid(s2, want=("mboit", "exact", "moments", "piece_moments"))
        nm = {"power4": 5, "power6": 7, "power8": 9}[ms]
        mo = out["moments"].reshape(-1, out["moments"].shape[-1])
        assert mo.shape[-1] == nm
        np.testing.assert_allclose(out["piece_moments"].sum(axis=-2), out["moments"], rtol=1e-12, atol=1e-12)
        # the same samples: b0..b4 agree across the sets; every pixel's
        # normalised Hankel matrix is positive semidefinite (|z| <= 1 too)
        if first5 is None:
            first5 = mo[:, :5]
        np.testing.assert_allclose(mo[:, :5], first5, rtol=1e-12, atol=1e-12)
        hit = mo[:, 0] > 1e-3
        b = mo[hit] / mo[hit, :1]
        h = (nm - 1) // 2
        H = np.stack([np.stack([b[:, i + j] for j in range(h + 1)], -1) for i in range(h + 1)], -2)
        assert np.linalg.eigvalsh(H).min() > -1e-9
        assert np.all(np.abs(b) <= 1 + 1e-12)
        np.testing.assert_allclose(out["mboit"][..., 3], out["exact"][..., 3], atol=1e-12)
        rmse[ms] = float(np.sqrt(((out["mboit"] - out["exact"]) ** 2).mean()))
    assert rmse["power8"] < rmse["power6"] < rmse["power4"]


# --------------------------------------------------------------------------
# tetrahedral meshes (Sec. 5: unstructured pieces)


def _special_points(sc):
    """Vertices, edge midpoints and face centroids of every tet."""
    V = sc.verts[:, :3].astype(np.float64)
    T = sc.tets
    e = [(V[T[:, i]] + V[T[:, j]]) / 2 for i in range(4) for j in range(i + 1, 4)]
    f = [(V[T[:, a]] + V[T[:, b]] + V[T[:, c]]) / 3 for a, b, c in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))]
    return np.concatenate([V] + e + f).astype(np.float32)


def test_tet_mesh_is_conforming_and_oriented():
    sc = scenes.tet_mesh(n=5, n_pieces=3, width=4, height=4)
    assert sc.tets.shape == (5 * 125, 4)
    assert np.all(scenes.tet_orient(sc.verts[:, :3], sc.tets) > 0)
    # every interior face is shared by exactly two tets: 2 n^2 boundary triangles per box face
    assert (sc.neighbors < 0).sum() == 2 * 6 * 25
    for t in range(0, len(sc.tets), 7):
        for i in range(4):
            u = sc.neighbors[t, i]
            if u >= 0:
                assert t in sc.neighbors[u]
                assert set(np.delete(sc.tets[t], i)) <= set(sc.tets[u])


def test_tet_location_partitions_the_box():
    """Exactly one tet owns every point of [0, n)^3, on faces, edges and
    vertices included (the symbolic perturbation), none owns a point outside;
    the owner's barycentric coordinates (solved independently in numpy) are
    all >= 0, and the binned search equals testing every tet."""
    n = 5
    sc = scenes.tet_mesh(n=n, n_pieces=3, width=4, height=4, seed=5)
    rng = np.random.default_rng(1)
    pts = np.concatenate([(rng.random((3000, 3)) * n).astype(np.float32), _special_points(sc)])
    inside = np.all((pts >= 0) & (pts < n), axis=1)
    owner, npass, val = oracle.tet_locate(sc, pts)
    np.testing.assert_array_equal(npass[inside], 1)
    assert np.all(owner[~inside] < 0) or np.all(npass[~inside] <= 1)
    ob, npb, _ = oracle.tet_locate(sc, pts, brute_force=True)
    np.testing.assert_array_equal(ob, owner)
    np.testing.assert_array_equal(npb, npass)
    V = sc.verts[:, :3].astype(np.float64)
    Qs = 2.0 ** sc.quantum_log2
    q = np.rint(pts[inside].astype(np.float64) * Qs) / Qs
    T = sc.tets[owner[inside]]
    A = np.stack([V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]], V[T[:, 3]] - V[T[:, 0]]], axis=2)
    lam = np.linalg.solve(A, (q - V[T[:, 0]])[:, :, None])[:, :, 0]
    bary = np.concatenate([1 - lam.sum(1, keepdims=True), lam], 1)
    assert bary.min() > -1e-9
    # points on the upper box faces belong to no tet (the box is half-open)
    top = np.array([[n, 1.5, 2.5], [2.25, n, 0.5], [0.5, 0.5, n], [0.0, 0.0, 0.0]], np.float32)
    o2, n2, _ = oracle.tet_locate(sc, top)
    np.testing.assert_array_equal(n2, [0, 0, 0, 1])


def test_tet_point_inside_known_tet():
    """Points built from barycentric coordinates >= 1/20 are owned by the
    tet they were built in, with the linear value of that combination."""
    sc = scenes.tet_mesh(n=4, n_pieces=2, width=4, height=4, seed=9)
    rng = np.random.default_rng(3)
    ts = rng.integers(0, len(sc.tets), 400)
    lam = rng.random((400, 4)) + 0.2
    lam /= lam.sum(1, keepdims=True)
    V = sc.verts[:, :3].astype(np.float64)
    P = np.einsum("ni,nik->nk", lam, V[sc.tets[ts]])
    P = (np.rint(P * 2.0 ** sc.quantum_log2) / 2.0 ** sc.quantum_log2).astype(np.float32)
    owner, npass, val = oracle.tet_locate(sc, P)
    np.testing.assert_array_equal(owner, ts)
    # the value is linear in the snapped point: re-solve its barycentric coordinates
    T = sc.tets[ts]
    A = np.stack([V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]], V[T[:, 3]] - V[T[:, 0]]], axis=2)
    mu = np.linalg.solve(A, (P.astype(np.float64) - V[T[:, 0]])[:, :, None])[:, :, 0]
    bary = np.concatenate([1 - mu.sum(1, keepdims=True), mu], 1)
    assert np.abs(bary - lam).max() < 1e-3
    want = np.einsum("ni,ni->n", bary, sc.verts[T, 3].astype(np.float64))
    np.testing.assert_allclose(val, want, rtol=1e-12, atol=1e-13)


def test_tet_linear_field_equals_grid():
    """Barycentric interpolation reproduces a linear field on any mesh, so a
    tet render equals the regular grid's up to the 2^-14 position snap."""
    sc, grid = small.linear_tets()
    P = sc.verts[:, :3].astype(np.float64)
    owner, npass, val = oracle.tet_locate(sc, (np.random.default_rng(2).random((500, 3)) * 6).astype(np.float32))
    views = [scenes.ortho_view(sc.dims, (0.4, 0.5, 0.77), 20, 18),
             scenes.perspective_view(sc.dims, (-0.6, 0.45, 0.66), 16, 14, fov_deg=35.0)]
    for v in views:
        a = oracle.render(sc, view=v, want=("moments", "mboit", "exact", "nsamples"))
        g = oracle.render_grid(grid, view=v, want=("moments", "mboit", "exact", "nsamples"))
        assert np.abs(a["nsamples"] - g["nsamples"]).max() <= 1
        assert (a["nsamples"] == g["nsamples"]).mean() > 0.95
        same = a["nsamples"] == g["nsamples"]
        np.testing.assert_allclose(a["moments"][same], g["moments"][same], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(a["mboit"][same], g["mboit"][same], atol=1e-5)
        np.testing.assert_allclose(a["exact"], g["exact"], atol=0.05)
        assert a["nsamples"].sum() > 100


def test_tet_pieces_sum_and_sortlast():
    sc = scenes.tet_mesh(n=6, n_pieces=4, width=20, height=18, seed=13)
    r = oracle.render(sc, want=("piece_moments", "moments", "exact", "sortlast", "mboit", "nsamples"))
    np.testing.assert_allclose(r["piece_moments"].sum(axis=1), r["moments"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["sortlast"], r["exact"], atol=1e-12)
    assert np.abs(r["mboit"] - r["exact"]).max() > 1e-4
    assert (r["moments"][:, 0] > 0).mean() > 0.3
    sub = oracle.render(sc, pieces=[1, 3], want=("moments",))
    pm = r["piece_moments"][:, [1, 3]].sum(axis=1)
    np.testing.assert_allclose(sub["moments"], pm, rtol=1e-12, atol=1e-14)


def test_tet_inverted_mesh_rejected():
    sc = scenes.tet_mesh(n=3, n_pieces=2, width=4, height=4)
    sc.tets[5, [2, 3]] = sc.tets[5, [3, 2]]
    with pytest.raises(ValueError):
        oracle.tet_locate(sc, np.zeros((1, 3), np.float32))


# --------------------------------------------------------------------------
# mixed cells (Sec. 5: the FUN3D pieces hold tetrahedra, pyramids and prisms)


def test_mixed_split_is_conforming():
    """Pyramids split into 2 tets, prisms into 3, along the quad diagonals
    through the smallest vertex id: every tet is positively oriented, each
    cell keeps its volume, the only unpaired faces are the 2 triangles of
    each boundary quad, and exactly one tet owns every point of the box
    (faces, edges and vertices included)."""
    n = 5
    m = scenes.mixed_mesh(n=n, n_pieces=3, width=4, height=4, seed=41)
    assert set(np.unique(m.cell_types)) == {4, 5, 6}
    tets, cot = oracle.split_cells(m)
    np.testing.assert_array_equal(np.bincount(cot, minlength=len(m.cells)), m.cell_types - 3)
    P = m.verts[:, :3].astype(np.float64)
    vol = np.linalg.det(np.stack([P[tets[:, i]] - P[tets[:, 0]] for i in (1, 2, 3)], 2)) / 6.0
    assert vol.min() > 0
    cell_vol = np.bincount(cot, weights=vol)
    want = np.where(m.cell_types == 5, 1.0 / 6.0, np.where(m.cell_types == 6, 0.5, 1.0 / 6.0))
    np.testing.assert_allclose(cell_vol, want, rtol=1e-12)
    nb = scenes.tet_neighbors(tets)
    assert (nb < 0).sum() == 12 * n * n
    ts = oracle.tet_scene_of(m)
    rng = np.random.default_rng(4)
    pts = np.concatenate([(rng.random((3000, 3)) * n).astype(np.float32), _special_points(ts)])
    inside = np.all((pts >= 0) & (pts < n), axis=1)
    owner, npass, _ = oracle.tet_locate(ts, pts, brute_force=True)
    np.testing.assert_array_equal(npass[inside], 1)


def test_mixed_linear_field_equals_grid():
    """Linear interpolation on the split tets reproduces a linear field, and
    the mixed mesh's vertices sit exactly on the lattice, so its render
    equals the regular grid's: the same samples, and moments equal up to
    the mesh path's 2^-14 snap of sample positions (at most 3.1e-5 in each
    coordinate, 4e-6 in this field's value: 2e-4 of the pixel's largest moment)."""
    n = 5
    lin = lambda x, y, z: 0.25 + x / 16.0 + y / 32.0 + z / 8.0  # noqa: E731
    m = scenes.mixed_mesh(n=n, n_pieces=3, width=4, height=4, seed=43)
    P = m.verts[:, :3].astype(np.float64)
    m.verts[:, 3] = lin(P[:, 0], P[:, 1], P[:, 2])
    g = np.arange(n + 1.0)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    field = lin(X, Y, Z).astype(np.float32)
    tf = small.linear_tf(0.05, 0.3)
    vr = (np.float32(field.min()), np.float32(field.max()))
    m.tf, m.tf_range = tf, vr
    grid = scenes.GridScene("lin", field, 1, np.zeros(((n + 1) // 2) ** 3, np.int32), 1, tf, vr, 0.5, [])
    ts = oracle.tet_scene_of(m)
    for v in [scenes.ortho_view(ts.dims, (0.4, 0.5, 0.77), 20, 18),
              scenes.perspective_view(ts.dims, (-0.6, 0.45, 0.66), 16, 14, fov_deg=35.0)]:
        a = oracle.render(ts, view=v, want=("moments", "mboit", "nsamples"))
        b = oracle.render_grid(grid, view=v, want=("moments", "mboit", "nsamples"))
        np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
        scale = np.abs(b["moments"]).max(axis=1, keepdims=True) + 1e-12  # odd moments cancel: per-pixel scale
        assert (np.abs(a["moments"] - b["moments"]) / scale).max() <= 2e-4
        np.testing.assert_allclose(a["mboit"], b["mboit"], atol=1e-4)
        assert a["nsamples"].sum() > 100



# --------------------------------------------------------------------------
# Alg. 1 loop 2 and the resolve (Sec. 4.2, 4.3) at render level


def _absorber_values(name, step=0.5, amax=10.0):
    """(a, alpha, rgb) of absorber A or B from its table plateau (R6/R7:
    sigma = -ln(1 - alpha_TF) per voxel, a = min(sigma * step, A_max),
    opacity 1 - e^-a)."""
    alpha_tf, rgb = small.ABSORBER_A if name == "A" else small.ABSORBER_B
    sigma = -math.log1p(-float(np.float32(alpha_tf)))
    a = min(sigma * step, amax)
    return a, -math.expm1(-a), np.array([float(np.float32(c)) for c in rgb])


def _closed_form_raw(absorbers, w0):
    """Alg. 1 loop 2 with the exact canonical bound of one or two atoms:
    sample k sees T = exp(-sum_{j<k} a_j - w0 a_k) (the atoms in front count
    fully, its own atom with the overestimation weight), and adds
    T alpha_k (r, g, b, 1)."""
    C = np.zeros(4)
    front = 0.0
    for name in absorbers:
        a, alpha, rgb = _absorber_values(name)
        T = math.exp(-front - w0 * a)
        C[:3] += T * alpha * rgb
        C[3] += T * alpha
        front += a
    return C, front


@pytest.mark.parametrize("w0", [0.0, W0, 1.0])
def test_render_one_and_two_absorbers_closed_form(w0):
    """Rays through one or two absorbing lattice points (depths warped to
    exactly -1 and +1, zero bias): the raw sum, the renormalised image and the
    moments equal their closed forms; with w0 = 0 the raw sum is the exact
    front-to-back blend in all four channels.  A blend with the absorbance a
    in place of the opacity alpha, a transmittance taken at the next sample's
    depth, or a resolve that drops the (1 - e^-b0) / C.a factor fails here."""
    sc, pix, absorbers = small.two_absorber_scene(w0)
    r = oracle.render_grid(sc, pixels=pix, want=("moments", "raw", "mboit", "exact", "nsamples"))
    assert np.all(r["nsamples"] == 30)   # z = 0.25, 0.75, ..., 14.75: the domain depth [0, 15) at step 0.5
    for n, ab in enumerate(absorbers):
        C, b0 = _closed_form_raw(ab, w0)
        np.testing.assert_allclose(r["raw"][n], C, rtol=0, atol=1e-13)
        # stage one: b_j = sum_k a_k z_k^j with z = -1 (front), +1 (back)
        a = [_absorber_values(x)[0] for x in ab]
        z = [-1.0, 1.0][:len(ab)]
        m = [sum(ak * zk ** j for ak, zk in zip(a, z)) for j in range(5)]
        np.testing.assert_allclose(r["moments"][n], m, rtol=0, atol=1e-13)
        # resolve (Sec. 4.3): colour renormalised to the alpha of the zeroth moment
        A = -math.expm1(-b0)
        np.testing.assert_allclose(r["mboit"][n, :3], C[:3] * A / C[3], rtol=0, atol=1e-13)
        assert r["mboit"][n, 3] == pytest.approx(A, abs=1e-15)
        if w0 == 0.0:
            np.testing.assert_allclose(r["raw"][n], r["exact"][n], rtol=0, atol=1e-13)
    # the closed form really distinguishes the cases: swapped order changes colour
    if w0 == W0:
        assert np.abs(r["raw"][0] - r["raw"][absorbers.index(("B", "A"))]).max() > 0.05


@pytest.mark.parametrize("w0", [0.0, W0])
def test_stage_two_from_given_moments(w0):
    """Stage two from given global moments: the closed-form moments of the
    one- and two-absorber rays reproduce the closed-form image, and moments
    of other absorbers change it as the bound says (here: the absorbers'
    weights swapped between front and back)."""
    sc, pix, absorbers = small.two_absorber_scene(w0)
    given = []
    for ab in absorbers:
        a = [_absorber_values(x)[0] for x in ab]
        z = [-1.0, 1.0][:len(ab)]
        given.append([sum(ak * zk ** j for ak, zk in zip(a, z)) for j in range(5)])
    given = np.array(given)
    r = oracle.render_grid_given(sc, given, pixels=pix)
    for n, ab in enumerate(absorbers):
        C, b0 = _closed_form_raw(ab, w0)
        np.testing.assert_allclose(r["raw"][n], C, rtol=0, atol=1e-13)
    # two-absorber rays with the front / back absorbances swapped in the moments:
    # the front sample now sees w0 a_back, the back one a_back + w0 a_front
    n2 = [n for n, ab in enumerate(absorbers) if len(ab) == 2]
    sw = given.copy()
    for n in n2:
        a = [_absorber_values(x)[0] for x in absorbers[n]]
        sw[n] = [sum(ak * zk ** j for ak, zk in zip(a[::-1], [-1.0, 1.0])) for j in range(5)]
    r2 = oracle.render_grid_given(sc, sw, pixels=pix)
    for n in n2:
        (fa, falpha, frgb), (ba, balpha, brgb) = [_absorber_values(x) for x in absorbers[n]]
        Tf = math.exp(-w0 * ba)
        Tb = math.exp(-ba - w0 * fa)
        want = Tf * falpha * np.append(frgb, 1.0) + Tb * balpha * np.append(brgb, 1.0)
        np.testing.assert_allclose(r2["raw"][n], want, rtol=0, atol=1e-13)
