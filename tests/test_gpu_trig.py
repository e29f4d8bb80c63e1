"""Trigonometric moments (3 / 4 complex moments in float16 / bfloat16) on the
GPU against the FP64 oracle.

Tolerances.  (1) Pass 2 alone on exactly representable stored moments: the
FP32 device arithmetic of the bound agrees with the oracle's FP64 bound to
|dA| <= 2e-4 (CPU emulation over concentrated and spread measures), so
T = exp(-b0 A) agrees to a relative b0 * 2e-4; the test allows 1e-3.
(2) End to end, pass 1 accumulates in FP32 and rounds t_j / b0 to the 16-bit
format, the oracle in FP64: the stored values may differ by one unit in the
last place of the format (2^-11 for float16 at |tau| < 1, 2^-8 for bfloat16),
which moves A by about that much and the renormalised colour by at most
b0 times it: the images must agree to 3e-3 (float16) and 2e-2 (bfloat16),
b0 is float32 in both, and the moment planes within one 16-bit unit.
(3) The two error sources apart: the oracle's stage two run on the GPU's own
stored 16-bit moments (oracle.render_grid_given) leaves only the FP32
arithmetic of the bound, |dA| <= 2e-4, so each T_k moves by a relative
b0 * 2e-4 at most and the renormalised colour, a ratio of two T-weighted sums
times the exact alpha, by at most twice that: |d rgb| <= 4e-4 b0 per pixel
(alpha exact), for both formats."""
import copy

import numpy as np
import pytest

import oracle
import scenes
from tests import _scenes_small as small

pytestmark = pytest.mark.gpu

IMG_TOL = {"f16": 3e-3, "bf16": 2e-2}
BETA = {"f16": 2e-3, "bf16": 2e-2}
ULP = {"f16": 2.0 ** -10, "bf16": 2.0 ** -7}   # one unit at |tau| in [0.5, 1): bounds all |tau| <= 1


@pytest.fixture(scope="module")
def pkg():
    import torch
    import __graft_entry__
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    import paper_2501_12581_gb300 as p
    return p


def trig_scene(sc, ms, st):
    s2 = copy.copy(sc)
    s2.moment_set, s2.storage, s2.moment_bias = ms, st, BETA[st]
    return s2


def unpack_trig(buf, view, n):
    a = buf.cpu().numpy()
    npx = view.width * view.height
    P = (npx + 3) // 4 * 4
    b0 = a[:npx].astype(np.float64)
    return b0, a.view(np.uint8)[4 * P: 4 * P + 4 * n * P]


def dequant(raw, n, P, npx, st):
    out = []
    for j in range(n):
        plane = raw[4 * P * j: 4 * P * j + 4 * npx]
        if st == "f16":
            v = plane.view(np.float16).astype(np.float64).reshape(npx, 2)
        else:
            u = plane.view(np.uint16).astype(np.uint32) << 16
            v = u.view(np.float32).astype(np.float64).reshape(npx, 2)
        out.append(v[:, 0] + 1j * v[:, 1])
    return np.stack(out, 1)


@pytest.mark.parametrize("ms, n", [("trig6", 3), ("trig8", 4)])
@pytest.mark.parametrize("st", ["f16", "bf16"])
def test_trig_pass2_on_exact_moments(pkg, ms, n, st):
    """Stored moments that are exact in both 16-bit formats; the slab's
    8 samples at known depths must give sum alpha T(z_k) with T from the
    oracle's bound."""
    import torch
    rng = np.random.default_rng(7)
    beta = BETA[st]
    while True:
        k = rng.integers(3, 8)
        phis = rng.uniform(-2.5, 2.5, k)
        a = rng.uniform(0.2, 1.0, k)
        tau = np.array([np.sum(a * np.exp(1j * j * phis)) for j in range(1, n + 1)]) / a.sum()
        tau = np.round(tau.real * 256) / 256 + 1j * np.round(tau.imag * 256) / 256
        T = np.eye(n + 1, dtype=complex)
        for r in range(n + 1):
            for c in range(n + 1):
                if c > r:
                    T[r, c] = (1 - beta) * tau[c - r - 1]
                elif c < r:
                    T[r, c] = np.conj((1 - beta) * tau[r - c - 1])
        if np.linalg.eigvalsh(T).min() > 1e-3:
            break
    b0 = 1.5
    n_ = 17
    field = np.ones((n_, n_, n_), np.float32)
    bz = np.repeat(np.arange(n_ - 1), (n_ - 1) ** 2)
    pob = np.where((bz >= 6) & (bz < 10), 0, 1).astype(np.int32)
    sc = scenes.GridScene("slab", field, 0, pob, 2, small.constant_tf(0.2), (np.float32(0), np.float32(2)), 0.5, [])
    sc.moment_set, sc.storage, sc.moment_bias = ms, st, beta
    view = small.axis_view(sc.dims, 8, 8, -6.0, 8.0, near=2.0, far=40.0)
    npx = 64
    P = 64
    slab = np.zeros(P * (1 + n), np.float32)
    slab[:npx] = b0
    raw = slab.view(np.uint8)
    for j in range(n):
        pair = np.array([tau[j].real, tau[j].imag], np.float32)
        if st == "f16":
            bits = pair.astype(np.float16).view(np.uint8)
        else:
            bits = (pair.view(np.uint32) >> 16).astype(np.uint16).view(np.uint8)
        for p in range(npx):
            raw[4 * P * (1 + j) + 4 * p: 4 * P * (1 + j) + 4 * p + 4] = bits
    vol = pkg.Volume(sc)
    mom = torch.from_numpy(slab).cuda()
    col = pkg.Volume.color_buffer([view])
    vol.reconstruct_blend([view], mom, col, pieces=[0], mode=pkg.MBOIT_COLOR_REDUCED)
    torch.cuda.synchronize()
    got = col.view(-1, 4).cpu().numpy()[:, 3].astype(np.float64)
    m = np.concatenate([[b0], np.stack([b0 * tau.real, b0 * tau.imag], 1).ravel()])
    sigma = -np.log1p(-np.float64(np.float32(0.2)))
    alpha = 1 - np.exp(-sigma * 0.5)
    want = 0.0
    for kk in range(8):
        t = 12.25 + 0.5 * kk
        z = oracle.log_warp(t, 2.0, 40.0)
        A = oracle.trig_bound(m, n, z * 0.9 * np.pi, beta, sc.overestimation)[0]
        want += alpha * np.exp(-b0 * A)
    np.testing.assert_allclose(got, want, rtol=1e-3)
    vol.close()


@pytest.mark.parametrize("ms, n", [("trig6", 3), ("trig8", 4)])
@pytest.mark.parametrize("st", ["f16", "bf16"])
def test_trig_frame_matches_oracle(pkg, ms, n, st):
    import torch
    sc = trig_scene(scenes.blobs64(width=96, height=80), ms, st)
    vol = pkg.Volume(sc)
    v = sc.views
    mom = vol.moments_for(v)
    col = pkg.Volume.color_buffer(v)
    vol.render_frame(v, mom, col)
    vol.synchronize()
    torch.cuda.synchronize()
    ref = oracle.render_grid(sc, want=("moments", "mboit"))
    npx = v[0].width * v[0].height
    P = (npx + 3) // 4 * 4
    b0, raw = unpack_trig(mom, v[0], n)
    np.testing.assert_allclose(b0, ref["moments"][:, 0], rtol=1e-5, atol=1e-6)
    tau = dequant(raw, n, P, npx, st)
    hit = ref["moments"][:, 0] > 0
    tau_ref = (ref["moments"][:, 1::2] + 1j * ref["moments"][:, 2::2])[hit] / ref["moments"][hit, 0:1]
    assert np.abs(tau[hit] - tau_ref).max() <= 1.5 * ULP[st]
    img = col.view(-1, 4).cpu().numpy().astype(np.float64)
    err = np.abs(img - ref["mboit"]).max()
    assert err <= IMG_TOL[st], err
    # stage two of the oracle on the GPU's stored moments: the arithmetic alone
    given = np.zeros((npx, 1 + 2 * n))
    given[:, 0] = b0
    given[:, 1::2] = (tau * b0[:, None]).real
    given[:, 2::2] = (tau * b0[:, None]).imag
    same = oracle.render_grid_given(sc, given)["mboit"]
    bound = 4e-4 * b0[:, None] + 1e-6
    assert np.all(np.abs(img - same) <= bound), np.abs(img - same).max()
    vol.close()


def test_trig_per_piece_path_and_octree(pkg):
    import torch
    sc = trig_scene(scenes.blobs64(width=64, height=48), "trig6", "f16")
    vol = pkg.Volume(sc)
    v = sc.views
    K = sc.n_pieces
    per = vol.moments_for(v, K)
    vol.render_moments(v, per, mode=pkg.MBOIT_MOMENTS_PER_PIECE)
    glob = vol.moments_for(v)
    vol.composite(pkg.MBOIT_OP_MOMENTS_SUM, v[0].width, v[0].height, 1, K, per, glob)
    pc = pkg.Volume.color_buffer(v, K)
    vol.reconstruct_blend(v, glob, pc, mode=pkg.MBOIT_COLOR_PER_PIECE)
    out = pkg.Volume.color_buffer(v)
    vol.composite(pkg.MBOIT_OP_COLOR_SUM_RESOLVE, v[0].width, v[0].height, 1, K, pc, out, glob)
    torch.cuda.synchronize()
    ref = oracle.render_grid(sc, want=("mboit",))
    assert np.abs(out.view(-1, 4).cpu().numpy() - ref["mboit"]).max() <= IMG_TOL["f16"]
    vol.close()
    amr = trig_scene(scenes.amr_blobs(base=4, max_level=2, width=40, height=36, n_pieces=4), "trig8", "bf16")
    avol = pkg.Volume(amr)
    mom = avol.moments_for(amr.views)
    col = pkg.Volume.color_buffer(amr.views)
    avol.render_frame(amr.views, mom, col)
    avol.synchronize()
    aref = oracle.render_amr(amr, want=("mboit",))
    assert np.abs(col.view(-1, 4).cpu().numpy() - aref["mboit"]).max() <= IMG_TOL["bf16"]
    avol.close()
