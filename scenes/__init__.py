"""Seeded synthetic inputs for the MBOIT puzzle-piece render.

This module only *describes* workloads: scalar fields, brick partitions into
pieces, RGBA transfer-function tables and camera specifications.  It holds
none of the method's arithmetic (no ray set-up, sampling, opacity conversion,
moments or reconstruction).  Both the FP64 oracle (`oracle/`) and the CUDA
library consume the arrays it returns, so the two sides see bit-identical
inputs.

Coordinates: the field is a float32 array ``field[z][y][x]`` of vertex values;
vertex (x, y, z) sits at point (x, y, z), so the domain is the box
[0, nx-1] x [0, ny-1] x [0, nz-1] and cell (i, j, k) spans [i, i+1) etc.
Bricks are cubes of ``2**brick_log2`` cells; brick (bx, by, bz) has id
``(bz*nby + by)*nbx + bx``.  A piece is a set of bricks (Morton-order ranges,
as p4est partitions a Morton curve, §3), so pieces are disjoint and jagged.

Views are given in the same index space.  All camera numbers are float32 so
both sides read the same bits.  ``near``/``far`` bound the logarithmic depth
warp of the view (Alg. 2): they bracket the domain's bounding sphere.
"""
from dataclasses import dataclass, field as dc_field
from typing import List

import numpy as np

from .rng import Stream

ORTHO = 0
PERSPECTIVE = 1


@dataclass
class View:
    eye: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    width: int
    height: int
    projection: int
    scale_u: np.float32
    scale_v: np.float32
    near: np.float32
    far: np.float32


@dataclass
class GridScene:
    name: str
    field: np.ndarray            # float32 [nz][ny][nx]
    brick_log2: int
    piece_of_brick: np.ndarray   # int32 [nbz*nby*nbx]
    n_pieces: int
    tf: np.ndarray               # float32 [256][4]: r, g, b, alpha (opacity per unit length)
    tf_range: tuple              # (vmin, vmax) float32
    step: float                  # sample spacing along the ray, voxel units (power of two)
    views: List[View] = dc_field(default_factory=list)
    moment_bias: float = 5e-5
    overestimation: float = 0.3
    absorbance_max: float = 10.0

    @property
    def dims(self):
        nz, ny, nx = self.field.shape
        return (nx, ny, nz)

    @property
    def brick_dims(self):
        b = 1 << self.brick_log2
        return tuple((n - 1 + b - 1) // b for n in self.dims)

    def piece_bricks(self, p):
        return np.nonzero(self.piece_of_brick == p)[0].astype(np.int32)


# ---------------------------------------------------------------------------
# fields

def _axis_gauss(n, centres, sigmas):
    x = np.arange(n, dtype=np.float64)
    return np.exp(-((x[None, :] - centres[:, None]) ** 2) / (2.0 * sigmas[:, None] ** 2))


def blob_field(shape_xyz, n_blobs, sigma_lo, sigma_hi, stream):
    """Sum of isotropic Gaussians A*exp(-|x-c|^2/(2 s^2)), evaluated at vertices."""
    nx, ny, nz = shape_xyz
    c = stream.uniform(3 * n_blobs).reshape(n_blobs, 3) * np.array([nx, ny, nz], dtype=np.float64)
    s = stream.uniform(n_blobs, sigma_lo, sigma_hi)
    a = stream.uniform(n_blobs, 0.3, 1.0)
    gx = _axis_gauss(nx, c[:, 0], s) * a[:, None]
    gy = _axis_gauss(ny, c[:, 1], s)
    gz = _axis_gauss(nz, c[:, 2], s)
    out = np.empty((nz, ny, nx), dtype=np.float32)
    chunk = max(1, (1 << 22) // (ny * nx) * 8)
    for z0 in range(0, nz, chunk):
        z1 = min(nz, z0 + chunk)
        zy = (gz[:, z0:z1, None] * gy[:, None, :]).reshape(n_blobs, -1)  # [blob][(z,y)]
        out[z0:z1] = (zy.T @ gx).reshape(z1 - z0, ny, nx).astype(np.float32)
    return out


def _lerp_matrix(n, spacing):
    """[n][L] weights of piecewise-linear interpolation from a lattice of the given spacing."""
    L = int(np.ceil((n - 1) / spacing)) + 1
    x = np.arange(n, dtype=np.float64) / spacing
    i = np.minimum(np.floor(x).astype(np.int64), L - 2)
    f = x - i
    W = np.zeros((n, L))
    W[np.arange(n), i] = 1.0 - f
    W[np.arange(n), i + 1] += f
    return W


def value_noise(shape_xyz, spacing, stream):
    """Lattice value noise: U[0,1) values on a lattice, trilinearly interpolated."""
    nx, ny, nz = shape_xyz
    Wx, Wy, Wz = (_lerp_matrix(n, spacing) for n in (nx, ny, nz))
    V = stream.uniform(Wz.shape[1] * Wy.shape[1] * Wx.shape[1]).reshape(Wz.shape[1], Wy.shape[1], Wx.shape[1])
    t = np.einsum("abc,xc->abx", V, Wx)
    t = np.einsum("abx,yb->ayx", t, Wy).reshape(Wz.shape[1], -1)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for z0 in range(0, nz, 64):
        z1 = min(nz, z0 + 64)
        out[z0:z1] = (Wz[z0:z1] @ t).reshape(z1 - z0, ny, nx)
    return out


# ---------------------------------------------------------------------------
# partitions

def morton3(bx, by, bz, bits):
    code = np.zeros(np.shape(bx), dtype=np.int64)
    for b in range(bits):
        code |= ((bx >> b) & 1) << (3 * b)
        code |= ((by >> b) & 1) << (3 * b + 1)
        code |= ((bz >> b) & 1) << (3 * b + 2)
    return code


def morton_pieces(brick_dims, n_pieces, stream, jitter=0.45, weights=None):
    """Split the Morton-ordered brick list into contiguous ranges, one per piece.

    Interior split points are moved by round(U[-jitter, jitter] * range), so
    pieces straddle Morton octants and are non-convex.  `weights` (optional)
    gives relative piece sizes before jitter.
    """
    nbx, nby, nbz = brick_dims
    bz, by, bx = np.meshgrid(np.arange(nbz), np.arange(nby), np.arange(nbx), indexing="ij")
    bits = int(np.ceil(np.log2(max(nbx, nby, nbz, 2))))
    code = morton3(bx.ravel(), by.ravel(), bz.ravel(), bits)
    order = np.argsort(code, kind="stable")
    n = order.size
    if weights is None:
        weights = np.ones(n_pieces)
    cum = np.concatenate([[0.0], np.cumsum(weights) / np.sum(weights)]) * n
    nominal = np.diff(cum)
    j = stream.uniform(n_pieces - 1, -jitter, jitter)
    splits = [0]
    for i in range(1, n_pieces):
        s = int(round(cum[i] + j[i - 1] * min(nominal[i - 1], nominal[i])))
        splits.append(min(max(s, splits[-1] + 1), n - (n_pieces - i)))
    splits.append(n)
    piece = np.empty(n, dtype=np.int32)
    for p in range(n_pieces):
        piece[order[splits[p]:splits[p + 1]]] = p
    return piece


# ---------------------------------------------------------------------------
# transfer function

def tf_table(stream, alpha_max, n_ctrl=6):
    """256-entry piecewise-linear RGBA table from n_ctrl seeded control points.

    Control positions are 0, 1 and n_ctrl-2 sorted U(0,1) draws; colours are
    U[0,1); alpha is U[0, alpha_max) (opacity of one voxel of material).
    """
    pos = np.concatenate([[0.0], np.sort(stream.uniform(n_ctrl - 2)), [1.0]])
    rgb = stream.uniform(3 * n_ctrl).reshape(n_ctrl, 3)
    alpha = stream.uniform(n_ctrl, 0.0, alpha_max)
    x = np.arange(256, dtype=np.float64) / 255.0
    tab = np.stack([np.interp(x, pos, rgb[:, 0]), np.interp(x, pos, rgb[:, 1]),
                    np.interp(x, pos, rgb[:, 2]), np.interp(x, pos, alpha)], axis=1)
    return tab.astype(np.float32)


# ---------------------------------------------------------------------------
# cameras

def _basis(wdir):
    w = np.asarray(wdir, dtype=np.float64)
    w = w / np.linalg.norm(w)
    up = np.array([0.0, 0.0, 1.0])
    u = np.cross(w, up)
    u /= np.linalg.norm(u)
    v = np.cross(u, w)
    return u, v, w


def _f32(a):
    return np.asarray(a, dtype=np.float32)


def ortho_view(dims, wdir, width, height, margin=1.02):
    """Orthographic view whose window covers the domain's bounding sphere.

    The view plane sits one domain diagonal in front of the sphere's near
    side, so depth is positive everywhere and the log warp is defined.
    """
    ext = np.array(dims, dtype=np.float64) - 1.0
    c = ext / 2.0
    diag = float(np.linalg.norm(ext))
    r = diag / 2.0
    u, v, w = _basis(wdir)
    dist = r + diag
    eye = c - dist * w
    size = 2.0 * r * margin
    return View(_f32(eye), _f32(u), _f32(v), _f32(w), width, height, ORTHO,
                np.float32(size * width / max(width, height)), np.float32(size * height / max(width, height)),
                np.float32(dist - r), np.float32(dist + r))


def perspective_view(dims, wdir, width, height, fov_deg=30.0, dist_diag=1.8):
    ext = np.array(dims, dtype=np.float64) - 1.0
    c = ext / 2.0
    diag = float(np.linalg.norm(ext))
    r = diag / 2.0
    u, v, w = _basis(wdir)
    dist = dist_diag * diag
    eye = c - dist * w
    th = np.tan(np.radians(fov_deg) / 2.0)
    aspect = width / height
    return View(_f32(eye), _f32(u), _f32(v), _f32(w), width, height, PERSPECTIVE,
                np.float32(th * aspect), np.float32(th),
                np.float32(max(dist - r, 0.25)), np.float32(dist + r))


# ---------------------------------------------------------------------------
# named workloads

# Per-workload alpha_max: chosen so the median zeroth moment b0 over hit
# pixels is about 3 (a semi-transparent volume), measured with the oracle.
ALPHA_MAX = {"blobs64": 0.13, "blobs512": 0.053}


def blobs64(width=256, height=256, n_pieces=4, seed=1001):
    """64^3 float32 field = 8 Gaussian blobs (sigma 4-12 voxels, amplitude
    U[0.3,1]); 8^3-cell bricks split into 4 jittered Morton pieces; 6-point
    transfer function; orthographic view, step 0.5 voxel."""
    s = Stream(seed)
    dims = (64, 64, 64)
    f = blob_field(dims, 8, 4.0, 12.0, s)
    tf = tf_table(s, ALPHA_MAX["blobs64"])
    bl = 3
    bd = tuple((n - 1 + (1 << bl) - 1) >> bl for n in dims)
    piece = morton_pieces(bd, n_pieces, s)
    view = ortho_view(dims, (0.62, 0.48, 0.62), width, height)
    return GridScene("blobs64", f, bl, piece, n_pieces, tf,
                     (np.float32(f.min()), np.float32(f.max())), 0.5, [view])


def blobs512(width=2048, height=2048, n_pieces=64, seed=1002, n=512):
    """512^3 float32 field = 64 Gaussian blobs (sigma 32-96 voxels) plus
    3-octave value noise (lattice spacing 64, 32, 16 voxels, weight 0.15 *
    0.5^octave); 16^3-cell bricks split into 64 jittered Morton pieces;
    perspective view (fov 30 degrees, eye 1.8 diagonals from the centre),
    step 0.5 voxel.  `n` shrinks the grid for tests (sizes scale with n)."""
    s = Stream(seed)
    dims = (n, n, n)
    k = n / 64.0
    f = blob_field(dims, 64, 4.0 * k, 12.0 * k, s).astype(np.float64)
    for o in range(3):
        f += 0.15 * 0.5 ** o * value_noise(dims, max(2.0, 64.0 * k / 8.0 / 2 ** o), s)
    f = f.astype(np.float32)
    tf = tf_table(s, ALPHA_MAX["blobs512"] * 512.0 / n)
    bl = 4
    bd = tuple((m - 1 + (1 << bl) - 1) >> bl for m in dims)
    piece = morton_pieces(bd, n_pieces, s)
    view = perspective_view(dims, (0.57, 0.49, 0.66), width, height)
    return GridScene("blobs512" if n == 512 else f"blobs{n}", f, bl, piece, n_pieces, tf,
                     (np.float32(f.min()), np.float32(f.max())), 0.5, [view])


def gear_teeth(n_pieces=8, layers_per_piece=4, layer_cells=2, footprint=512, width=512, height=512, n_views=4,
               tilt_deg=20.0, b0_target=3.0):
    """Weak-scaling stress test of Sec. 5 ("gear teeth", Fig. 7): every one of
    K = n_pieces pieces owns `layers_per_piece` layers of footprint x
    footprint x layer_cells cells, interleaved so that K - 1 layers of other
    pieces lie between two layers of a piece (layer s belongs to piece
    s mod K).  A ray through the stack meets 4K segments of alternating
    pieces, so an exact sort-last compositor sorts 4K fragments per pixel.

    Field: per layer the value (piece + 1/2) / K (a piece colour through the
    table) plus a gentle in-plane wobble; vertex plane z takes the value of
    layer floor(z / layer_cells).  Bricks of layer_cells^3 cells, so a layer
    is one brick thick.  Constant opacity with sigma * depth = b0_target
    (a semi-transparent stack at every K).  n_views perspective views on an
    orbit tilted `tilt_deg` from the stacking axis."""
    K = n_pieces
    n_layers = layers_per_piece * K
    nz = n_layers * layer_cells + 1
    nx = ny = footprint + 1
    bl = int(layer_cells).bit_length() - 1
    assert (1 << bl) == layer_cells and footprint % layer_cells == 0
    x = np.arange(nx, dtype=np.float64)
    wob = (0.03 * np.sin(2 * np.pi * x / 128.0)[None, :] * np.sin(2 * np.pi * x / 96.0)[:, None]).astype(np.float32)
    layer = np.minimum(np.arange(nz) // layer_cells, n_layers - 1)
    base = ((layer % K) + 0.5) / K * 0.8 + 0.1
    field = np.empty((nz, ny, nx), np.float32)
    for z in range(nz):
        field[z] = np.float32(base[z]) + wob
    nb = footprint // layer_cells
    pob = np.repeat((np.arange(n_layers) % K).astype(np.int32), nb * nb)
    sigma = b0_target / float(n_layers * layer_cells)
    xs = np.arange(256) / 255.0
    tf = np.stack([0.5 + 0.5 * np.cos(2 * np.pi * (xs + 0.0)), 0.5 + 0.5 * np.cos(2 * np.pi * (xs + 1 / 3)),
                   0.5 + 0.5 * np.cos(2 * np.pi * (xs + 2 / 3)), np.full(256, 1.0 - np.exp(-sigma))], 1)
    dims = (nx, ny, nz)
    t = np.radians(tilt_deg)
    views = [perspective_view(dims, (np.sin(t) * np.cos(a), np.sin(t) * np.sin(a), np.cos(t)), width, height)
             for a in np.radians(45.0 + 90.0 * np.arange(n_views))]
    return GridScene(f"gear_teeth{K}", field, bl, pob, K, tf.astype(np.float32), (np.float32(0.0), np.float32(1.0)),
                     0.5, views)


@dataclass
class MixedScene:
    """Unstructured mesh of tetrahedra, pyramids and prisms (the cell mix of
    the paper's FUN3D data) filling the box [0, n]^3.  cells[i] lists the
    vertex ids of cell i, padded with -1: a tet (4), a pyramid (5: base quad
    in cyclic order, then the apex) or a prism (6: bottom triangle, then the
    top triangle with vertex j + 3 above vertex j); cell_types[i] is that
    count."""
    name: str
    verts: np.ndarray           # float32 [nv][4]: x, y, z, value
    cells: np.ndarray           # int32 [nc][6]
    cell_types: np.ndarray      # int32 [nc]: 4, 5 or 6
    box: tuple
    quantum_log2: int
    piece_of_cell: np.ndarray   # int32 [nc]
    n_pieces: int
    tf: np.ndarray
    tf_range: tuple
    step: float
    views: List[View] = dc_field(default_factory=list)
    moment_bias: float = 5e-5
    overestimation: float = 0.3
    absorbance_max: float = 10.0

    @property
    def dims(self):
        return tuple(int(b) + 1 for b in self.box)


def mixed_mesh(n=24, n_pieces=8, width=256, height=256, seed=1006, alpha_max=None):
    """n^3 hex grid whose every hex becomes, at random: 6 tets around its main
    diagonal (Kuhn), 2 prisms (cut by the vertical plane through its (0, 0)
    and (1, 1) edges), or 6 pyramids on its faces with an apex at its centre.
    Vertex ids grow with x, then y, then z, so every quad face these cells
    share is cut, when split into tets along the diagonal through its
    smallest vertex id, the same way from both sides.  Values: the 64^3
    workload's 8 blobs scaled to n; pieces: equal-count ranges of the Morton
    order of cell centroids; a perspective view; step 0.5."""
    s = Stream(seed)
    nv1 = n + 1
    g = np.arange(nv1, dtype=np.float64)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    P = [np.stack([X, Y, Z], -1).reshape(-1, 3)]
    vid = lambda x, y, z: (z * nv1 + y) * nv1 + x  # noqa: E731
    kind = np.floor(s.uniform(n ** 3) * 3).astype(np.int64)
    cells, types, cen = [], [], []
    n_extra = 0
    for h in range(n ** 3):
        x, y, z = h % n, (h // n) % n, h // (n * n)
        c = {(a, b, e): vid(x + a, y + b, z + e) for a in (0, 1) for b in (0, 1) for e in (0, 1)}
        centre = (x + 0.5, y + 0.5, z + 0.5)
        if kind[h] == 0:      # Kuhn: paths v000 -> +e_a -> +e_a + e_b -> v111
            for a, b in ((0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)):
                u = [0, 0, 0]
                u[a] = 1
                w = list(u)
                w[b] = 1
                cells.append([c[(0, 0, 0)], c[tuple(u)], c[tuple(w)], c[(1, 1, 1)], -1, -1])
                types.append(4)
                cen.append(centre)
        elif kind[h] == 1:    # two prisms, vertical cut through (0, 0)-(1, 1)
            for tri in (((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))):
                cells.append([c[(a, b, 0)] for a, b in tri] + [c[(a, b, 1)] for a, b in tri])
                types.append(6)
                cen.append(centre)
        else:                 # six pyramids around a centre vertex
            apex = nv1 ** 3 + n_extra
            n_extra += 1
            P.append(np.array([centre]))
            faces = [[(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)], [(0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)],
                     [(0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)], [(0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1)],
                     [(0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1)], [(1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)]]
            for f in faces:
                cells.append([c[q] for q in f] + [apex, -1])
                types.append(5)
                cen.append(centre)
    P = np.concatenate(P, 0)
    k = n / 64.0
    cb = s.uniform(24).reshape(8, 3) * n
    sg = s.uniform(8, 4.0 * k, 12.0 * k)
    am = s.uniform(8, 0.3, 1.0)
    val = np.zeros(len(P))
    for i in range(8):
        val += am[i] * np.exp(-((P - cb[i]) ** 2).sum(1) / (2 * sg[i] ** 2))
    verts = np.concatenate([P, val[:, None]], 1).astype(np.float32)
    cen = np.array(cen)
    q = np.clip((cen / n * 1023).astype(np.int64), 0, 1023)
    order = np.argsort(morton3(q[:, 0], q[:, 1], q[:, 2], 10), kind="stable")
    piece = np.empty(len(cells), np.int32)
    bounds = np.linspace(0, len(cells), n_pieces + 1).round().astype(np.int64)
    for p in range(n_pieces):
        piece[order[bounds[p]:bounds[p + 1]]] = p
    tf = tf_table(Stream(seed + 7), alpha_max if alpha_max is not None else min(0.13 * 64.0 / n, 0.4))
    view = perspective_view((n + 1,) * 3, (0.57, 0.49, 0.66), width, height)
    vf = verts[:, 3]
    return MixedScene(f"mixed{n}", verts, np.array(cells, np.int32), np.array(types, np.int32), (float(n),) * 3, 14,
                      piece, n_pieces, tf, (np.float32(vf.min()), np.float32(vf.max())), 0.5, [view])


# ---------------------------------------------------------------------------
# AMR brick octree

@dataclass
class AmrScene:
    """Leaves of a brick octree.  Leaf i covers origin_i + [0, 8 * 2^(max_level -
    level_i))^3 in finest-cell units and stores 9^3 vertex-centred values of
    the field at its own resolution, values[i][z][y][x].  The domain is
    [0, D]^3 with D = base_bricks * 8 * 2^max_level finest cells."""
    name: str
    leaves: np.ndarray          # int32 [n][4]: origin x, y, z (finest cells), level
    values: np.ndarray          # float32 [n][9][9][9]
    max_level: int
    finest_cells: int           # D
    piece_of_leaf: np.ndarray   # int32 [n]
    n_pieces: int
    tf: np.ndarray
    tf_range: tuple
    step: float
    views: List[View] = dc_field(default_factory=list)
    moment_bias: float = 5e-5
    overestimation: float = 0.3
    absorbance_max: float = 10.0
    brick_log2: int = 3
    adaptive_step: bool = False  # nested lattice of 2^(max_level - level) steps per leaf

    @property
    def dims(self):
        return (self.finest_cells + 1,) * 3

    @property
    def n_units(self):
        return self.leaves.shape[0]


class AnalyticField:
    """The 512^3 workload's field as a function of position (Gaussian blobs
    plus lattice value noise, trilinear between lattice values), so it can be
    sampled at any resolution."""

    def __init__(self, seed=1002, n=512):
        s = Stream(seed)
        k = n / 64.0
        nb = 64
        self.c = s.uniform(3 * nb).reshape(nb, 3) * n
        self.s = s.uniform(nb, 4.0 * k, 12.0 * k)
        self.a = s.uniform(nb, 0.3, 1.0)
        self.noise = []
        for o in range(3):
            sp = max(2.0, 64.0 * k / 8.0 / 2 ** o)
            L = int(np.ceil((n - 1) / sp)) + 1
            V = s.uniform(L * L * L).reshape(L, L, L)   # [z][y][x]
            self.noise.append((0.15 * 0.5 ** o, sp, V))

    def grid_values(self, xs, ys, zs):
        """Values on the tensor grid xs x ys x zs (1-D arrays, coordinates of
        the 512^3 vertex space), returned [z][y][x]."""
        gx = np.exp(-(xs[None, :] - self.c[:, 0:1]) ** 2 / (2 * self.s[:, None] ** 2)) * self.a[:, None]
        gy = np.exp(-(ys[None, :] - self.c[:, 1:2]) ** 2 / (2 * self.s[:, None] ** 2))
        gz = np.exp(-(zs[None, :] - self.c[:, 2:3]) ** 2 / (2 * self.s[:, None] ** 2))
        out = np.einsum("bz,by,bx->zyx", gz, gy, gx)
        for w, sp, V in self.noise:
            L = V.shape[0]
            def lerp_w(q):
                x = q / sp
                i = np.minimum(np.floor(x).astype(np.int64), L - 2)
                f = x - i
                W = np.zeros((q.size, L))
                W[np.arange(q.size), i] = 1.0 - f
                W[np.arange(q.size), i + 1] += f
                return W
            Wx, Wy, Wz = lerp_w(xs), lerp_w(ys), lerp_w(zs)
            out += w * np.einsum("zc,yb,xa,cba->zyx", Wz, Wy, Wx, V, optimize=True)
        return out


def _leaf_values(field, origins_f, size_f, scale, batch=2048):
    """9^3 samples of each leaf (finest-unit origins, one finest-unit size for
    all) of the analytic field, whose coordinates are finest units * scale."""
    n = len(origins_f)
    out = np.empty((n, 9, 9, 9), np.float32)
    h = float(size_f[0]) / 8.0 if n else 1.0
    j = np.arange(9, dtype=np.float64)
    for b0 in range(0, n, batch):
        o = origins_f[b0:b0 + batch].astype(np.float64)
        X = (o[:, 0:1] + j * h) * scale           # [B][9] coordinates per axis
        Y = (o[:, 1:2] + j * h) * scale
        Z = (o[:, 2:3] + j * h) * scale
        B = len(o)
        # Gaussian blobs, separable: [B][blob][9] per axis, then (z,y) x x products
        gx = np.exp(-(X[:, None, :] - field.c[None, :, 0:1]) ** 2 / (2 * field.s[None, :, None] ** 2)) * field.a[None, :, None]
        gy = np.exp(-(Y[:, None, :] - field.c[None, :, 1:2]) ** 2 / (2 * field.s[None, :, None] ** 2))
        gz = np.exp(-(Z[:, None, :] - field.c[None, :, 2:3]) ** 2 / (2 * field.s[None, :, None] ** 2))
        zy = (gz[:, :, :, None] * gy[:, :, None, :]).reshape(B, gx.shape[1], 81)
        v = np.matmul(zy.transpose(0, 2, 1), gx).reshape(B, 9, 9, 9)
        # value noise: trilinear weights restricted to a 4x4x4 lattice block per leaf
        for w, sp, V in field.noise:
            L = V.shape[0]
            nb = min(L, int(np.ceil(8 * h * scale / sp)) + 2)   # lattice block covering one leaf

            def local(q):
                x = q / sp
                idx = np.minimum(np.floor(x).astype(np.int64), L - 2)
                i0 = np.clip(idx[:, 0], 0, L - nb)
                f = x - idx
                W = np.zeros((q.shape[0], 9, nb))
                rel = idx - i0[:, None]
                bi = np.arange(q.shape[0])[:, None]
                ji = np.arange(9)[None, :]
                W[bi, ji, rel] = 1.0 - f
                W[bi, ji, rel + 1] += f
                return W, i0
            Wx, ix = local(X)
            Wy, iy = local(Y)
            Wz, iz = local(Z)
            r = np.arange(nb)
            blk = V[(iz[:, None] + r)[:, :, None, None], (iy[:, None] + r)[:, None, :, None], (ix[:, None] + r)[:, None, None, :]]
            v += w * np.einsum("bzc,byd,bxe,bcde->bzyx", Wz, Wy, Wx, blk, optimize=True)
        out[b0:b0 + batch] = v.astype(np.float32)
    return out


def _max_gradient(vals, h):
    g = np.zeros(vals.shape[0])
    for ax in (1, 2, 3):
        d = np.abs(np.diff(vals, axis=ax)) / h[:, None, None, None]
        g = np.maximum(g, d.reshape(d.shape[0], -1).max(axis=1))
    return g


def amr_blobs(width=2560, height=2560, n_pieces=72, seed=1003, base=26, max_level=2, refine_frac=0.2,
              alpha_max=None):
    """Brick octree over the 512^3 workload's field: 26^3 base bricks of 8^3
    cells, refined twice (the top 20 % of bricks by maximum gradient
    magnitude each time), ~81.6k leaves / ~41.8M cells; 72 pieces of uneven
    size (ratio 8) by Morton order of leaf origins; perspective view; step
    0.5 finest voxel.  Smaller `base` / `max_level` shrink it for tests."""
    field = AnalyticField()
    D = base * 8 * (1 << max_level)
    scale = 511.0 / D
    bsz0 = 8 * (1 << max_level)
    o = np.stack(np.meshgrid(np.arange(base), np.arange(base), np.arange(base), indexing="ij"), -1).reshape(-1, 3)
    cur = o[:, ::-1] * bsz0                      # (x, y, z) finest-unit origins of level-0 bricks
    leaves, values = [], []
    for level in range(max_level + 1):
        size = bsz0 >> level
        vals = _leaf_values(field, cur, np.full(len(cur), size, np.float64), scale)
        if level == max_level:
            refine = np.zeros(len(cur), bool)
        else:
            g = _max_gradient(vals.astype(np.float64), np.full(len(cur), size / 8.0 * scale))
            k = int(round(refine_frac * len(cur)))
            refine = np.zeros(len(cur), bool)
            refine[np.argsort(-g, kind="stable")[:k]] = True
        keep = ~refine
        leaves.append(np.concatenate([cur[keep], np.full((keep.sum(), 1), level)], axis=1))
        values.append(vals[keep])
        half = size // 2
        kids = []
        for dz in (0, half):
            for dy in (0, half):
                for dx in (0, half):
                    kids.append(cur[refine] + np.array([dx, dy, dz]))
        cur = np.concatenate(kids) if kids and refine.any() else np.zeros((0, 3), np.int64)
    leaves = np.concatenate(leaves).astype(np.int32)
    values = np.concatenate(values).astype(np.float32)
    s = Stream(seed)
    bits = int(np.ceil(np.log2(D)))
    code = morton3(leaves[:, 0].astype(np.int64), leaves[:, 1].astype(np.int64), leaves[:, 2].astype(np.int64), bits)
    order = np.argsort(code, kind="stable")
    leaves, values = leaves[order], values[order]
    u = s.uniform(n_pieces)
    u = (u - u.min()) / (u.max() - u.min()) if n_pieces > 1 else np.zeros(1)
    piece = morton_pieces_linear(len(leaves), n_pieces, 8.0 ** u, s)
    vmin, vmax = float(values.min()), float(values.max())
    am = alpha_max if alpha_max is not None else 0.053 * 512.0 / D
    tf = tf_table(Stream(1002 + 7), am)
    dims = (D + 1,) * 3
    view = perspective_view(dims, (0.57, 0.49, 0.66), width, height)
    return AmrScene("amr_blobs" if base == 26 else f"amr_blobs{base}", leaves, values, max_level, D, piece,
                    n_pieces, tf, (np.float32(vmin), np.float32(vmax)), 0.5, [view])


def morton_pieces_linear(n, n_pieces, weights, stream, jitter=0.0):
    """Contiguous ranges of an already Morton-sorted list with relative sizes `weights`."""
    cum = np.concatenate([[0.0], np.cumsum(weights) / np.sum(weights)]) * n
    splits = [0]
    for i in range(1, n_pieces):
        splits.append(min(max(int(round(cum[i])), splits[-1] + 1), n - (n_pieces - i)))
    splits.append(n)
    piece = np.empty(n, dtype=np.int32)
    for p in range(n_pieces):
        piece[splits[p]:splits[p + 1]] = p
    return piece


# ---------------------------------------------------------------------------
# tetrahedral mesh

@dataclass
class TetScene:
    """Conforming tetrahedral mesh of the box [0, n]^3: vertices (x, y, z,
    value) float32, tets (4 vertex ids, positively oriented), neighbours
    (the tet across the face opposite vertex i, -1 on the boundary)."""
    name: str
    verts: np.ndarray           # float32 [nv][4]
    tets: np.ndarray            # int32 [nt][4]
    neighbors: np.ndarray       # int32 [nt][4]
    box: tuple                  # the domain is [0, box) per axis
    quantum_log2: int           # positions snap to multiples of 2^-quantum_log2
    piece_of_tet: np.ndarray    # int32 [nt]
    n_pieces: int
    tf: np.ndarray
    tf_range: tuple
    step: float
    views: List[View] = dc_field(default_factory=list)
    moment_bias: float = 5e-5
    overestimation: float = 0.3
    absorbance_max: float = 10.0

    @property
    def dims(self):
        return tuple(int(b) + 1 for b in self.box)


# corner indices (dx, dy, dz) of the 5-tet split; even hexes use the first
# set, odd hexes its mirror, so neighbouring hexes split shared faces alike
_TET5_EVEN = [((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)), ((1, 1, 0), (0, 1, 0), (1, 0, 0), (1, 1, 1)),
              ((1, 0, 1), (0, 0, 1), (1, 1, 1), (1, 0, 0)), ((0, 1, 1), (1, 1, 1), (0, 0, 1), (0, 1, 0)),
              ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1))]
_TET5_ODD = [tuple((1 - a, b, c) for a, b, c in t) for t in _TET5_EVEN]


def tet_neighbors(tets):
    """Tet across each face (face i is opposite vertex i); -1 on the boundary."""
    nt = tets.shape[0]
    faces = np.stack([np.delete(tets, i, axis=1) for i in range(4)], axis=1).reshape(-1, 3)
    faces = np.sort(faces, axis=1).astype(np.int64)
    key = (faces[:, 0] << 42) | (faces[:, 1] << 21) | faces[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    nb = np.full(nt * 4, -1, np.int64)
    a, b = order[same], order[same + 1]
    nb[a] = b // 4
    nb[b] = a // 4
    return nb.reshape(nt, 4).astype(np.int32)


def tet_orient(P, tets):
    """Six signed volumes of the tets, exact for coordinates on the 2^-16 lattice (or a coarser one)."""
    Q = np.rint(np.asarray(P, np.float64) * 65536.0).astype(np.int64)
    a, b, c, d = (Q[tets[:, i]] for i in range(4))
    u, v, w = b - a, c - a, d - a
    return (u[:, 0] * (v[:, 1] * w[:, 2] - v[:, 2] * w[:, 1]) - u[:, 1] * (v[:, 0] * w[:, 2] - v[:, 2] * w[:, 0])
            + u[:, 2] * (v[:, 0] * w[:, 1] - v[:, 1] * w[:, 0]))


def hex_tets(n):
    """Vertex ids of the 5-tet split of an n^3 hex grid ((n+1)^3 vertices,
    x fastest), 5 tets per hex in hex order (parity-alternating split)."""
    nv1 = n + 1
    hz, hy, hx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hx, hy, hz = hx.ravel(), hy.ravel(), hz.ravel()
    even = ((hx + hy + hz) % 2) == 0
    tets = np.empty((n ** 3, 5, 4), np.int64)
    for t in range(5):
        for corner in range(4):
            e, o = _TET5_EVEN[t][corner], _TET5_ODD[t][corner]
            tets[:, t, corner] = np.where(even, ((hz + e[2]) * nv1 + (hy + e[1])) * nv1 + (hx + e[0]),
                                          ((hz + o[2]) * nv1 + (hy + o[1])) * nv1 + (hx + o[0]))
    return tets.reshape(-1, 4)


def tet_mesh(n=96, jitter=0.3, n_pieces=72, width=1024, height=1024, seed=1004, alpha_max=None):
    """Jittered n^3 hex grid, 5 tets per hex, the scalar of the 64^3 blob
    workload (8 blobs, scaled to n) at the vertices, 72 pieces in equal-count
    ranges of the Morton order of tet centroids, a perspective view, step 0.5.

    Vertices move by U[-jitter, jitter] cells per axis (boundary vertices only
    along the box faces, so the mesh fills the box exactly); a vertex whose
    move would leave a tet with under 5% of its unjittered volume has its
    move halved until none does; positions are then rounded to multiples of
    2^-14 (the lattice the exact point location snaps to)."""
    s = Stream(seed)
    nv1 = n + 1
    g = np.arange(nv1, dtype=np.float64)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    P0 = np.stack([X, Y, Z], -1).reshape(-1, 3)
    J = s.uniform(P0.size).reshape(-1, 3) * (2 * jitter) - jitter
    J[(P0 == 0) | (P0 == n)] = 0.0
    tets = hex_tets(n)
    v0 = tet_orient(P0, tets)
    flip = v0 < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    v0 = np.abs(v0)
    while True:
        P = np.rint((P0 + J) * 16384.0) / 16384.0
        bad = tet_orient(P, tets) < 0.05 * v0
        if not bad.any():
            break
        J[np.unique(tets[bad].ravel())] *= 0.5
    # value: 8 blobs as in the 64^3 workload, scaled to n
    k = n / 64.0
    c = s.uniform(24).reshape(8, 3) * n
    sg = s.uniform(8, 4.0 * k, 12.0 * k)
    am = s.uniform(8, 0.3, 1.0)
    val = np.zeros(len(P))
    for i in range(8):
        val += am[i] * np.exp(-((P - c[i]) ** 2).sum(1) / (2 * sg[i] ** 2))
    verts = np.concatenate([P, val[:, None]], 1).astype(np.float32)
    tets = tets.astype(np.int32)
    nb = tet_neighbors(tets)
    cen = P[tets].mean(axis=1)
    q = np.clip((cen / n * 1023).astype(np.int64), 0, 1023)
    order = np.argsort(morton3(q[:, 0], q[:, 1], q[:, 2], 10), kind="stable")
    piece = np.empty(len(tets), np.int32)
    bounds = np.linspace(0, len(tets), n_pieces + 1).round().astype(np.int64)
    for p in range(n_pieces):
        piece[order[bounds[p]:bounds[p + 1]]] = p
    tf = tf_table(Stream(seed + 7), alpha_max if alpha_max is not None else min(0.13 * 64.0 / n, 0.4))
    dims = (n + 1,) * 3
    view = perspective_view(dims, (0.57, 0.49, 0.66), width, height)
    vf = verts[:, 3]
    return TetScene("tets" if n == 96 else f"tets{n}", verts, tets, nb, (float(n),) * 3, 14, piece, n_pieces, tf,
                    (np.float32(vf.min()), np.float32(vf.max())), 0.5, [view])
