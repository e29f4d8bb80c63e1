"""Small hand-built scenes for pins and edge cases (inputs only, no method arithmetic)."""
import numpy as np

import scenes


def axis_view(dims, width, height, eye_z, scale, w=(0.0, 0.0, 1.0), u=(1.0, 0.0, 0.0), v=(0.0, 1.0, 0.0),
              near=5.0, far=60.0, centre=None):
    nx, ny, nz = dims
    c = centre if centre is not None else ((nx - 1) / 2.0, (ny - 1) / 2.0)
    return scenes.View(np.array([c[0], c[1], eye_z], np.float32), np.array(u, np.float32),
                       np.array(v, np.float32), np.array(w, np.float32), width, height, scenes.ORTHO,
                       np.float32(scale), np.float32(scale), np.float32(near), np.float32(far))


def constant_tf(alpha, rgb=(0.8, 0.4, 0.2)):
    tf = np.zeros((256, 4), np.float32)
    tf[:, 0:3] = rgb
    tf[:, 3] = alpha
    return tf


def linear_tf(s0, s1):
    """sigma_j = s0 + s1*j/255 (opacity alpha_j = 1 - exp(-sigma_j)); r = j/255,
    g = 1 - j/255, b = 0.5, so every channel is linear in the normalised value."""
    j = np.arange(256) / 255.0
    tf = np.zeros((256, 4), np.float64)
    tf[:, 0] = j
    tf[:, 1] = 1.0 - j
    tf[:, 2] = 0.5
    tf[:, 3] = 1.0 - np.exp(-(s0 + s1 * j))
    return tf.astype(np.float32)


def slab_scene(alpha=0.1, n=33, brick_log2=3, slab_layer=1):
    """Constant field; piece 1 = the bricks of one z-layer, piece 0 = the rest."""
    field = np.ones((n, n, n), np.float32)
    B = 1 << brick_log2
    nb = (n - 1 + B - 1) // B
    bz = np.repeat(np.arange(nb), nb * nb)
    piece = (bz == slab_layer).astype(np.int32)
    return scenes.GridScene("slab", field, brick_log2, piece, 2, constant_tf(alpha),
                            (np.float32(0.0), np.float32(2.0)), 0.5, [])


def linear_scene(dims=(17, 13, 11), brick_log2=2, n_pieces=3, seed=7):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    field = (0.25 + x / 16.0 + y / 32.0 + z / 8.0).astype(np.float32)
    B = 1 << brick_log2
    bd = tuple((m - 1 + B - 1) // B for m in dims)
    piece = scenes.morton_pieces(bd, n_pieces, scenes.Stream(seed))
    return scenes.GridScene("linear", field, brick_log2, piece, n_pieces, linear_tf(0.05, 0.3),
                            (np.float32(field.min()), np.float32(field.max())), 0.5, [])


def sandwich_scene(n=25, brick_log2=2, ranks=3, seed=11):
    """Fig. 6: each of `ranks` pieces owns interleaved z-slices of one cube."""
    s = scenes.Stream(seed)
    field = scenes.blob_field((n, n, n), 4, 3.0, 8.0, s)
    B = 1 << brick_log2
    nb = (n - 1 + B - 1) // B
    bz = np.repeat(np.arange(nb), nb * nb)
    piece = (bz % ranks).astype(np.int32)
    return scenes.GridScene("sandwich", field, brick_log2, piece, ranks, scenes.tf_table(s, 0.35),
                            (np.float32(field.min()), np.float32(field.max())), 0.5, [])


def linear_amr(base=3, max_level=2, refine=((0, 0, 0), (1, 2, 1))):
    """Brick octree with a dyadic linear field (exact in float32 at every
    vertex): base^3 level-0 bricks of 8^3 cells; the listed level-0 bricks are
    refined once, and the first child of each is refined again.  Returns the
    octree scene and the finest regular grid holding the same field."""
    bsz = 8 << max_level
    D = base * bsz
    lin = lambda x, y, z: 0.25 + x / 64.0 + y / 128.0 + z / 32.0  # noqa: E731
    leaves = []

    def add(o, level):
        leaves.append((o[0], o[1], o[2], level))

    for bz in range(base):
        for by in range(base):
            for bx in range(base):
                o0 = (bx * bsz, by * bsz, bz * bsz)
                if (bx, by, bz) not in refine:
                    add(o0, 0)
                    continue
                half = bsz // 2
                kids = [(o0[0] + dx, o0[1] + dy, o0[2] + dz) for dz in (0, half) for dy in (0, half) for dx in (0, half)]
                for i, kidx in enumerate(kids):
                    if i == 0 and max_level >= 2:
                        q = half // 2
                        for dz in (0, q):
                            for dy in (0, q):
                                for dx in (0, q):
                                    add((kidx[0] + dx, kidx[1] + dy, kidx[2] + dz), 2)
                    else:
                        add(kidx, 1)
    leaves = np.array(leaves, np.int32)
    j = np.arange(9.0)
    vals = np.empty((len(leaves), 9, 9, 9), np.float32)
    for i, (ox, oy, oz, L) in enumerate(leaves):
        h = (bsz >> L) / 8.0
        z, y, x = np.meshgrid(oz + j * h, oy + j * h, ox + j * h, indexing="ij")
        vals[i] = lin(x, y, z)
    tf = linear_tf(0.04, 0.2)
    g = np.arange(D + 1.0)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    field = lin(X, Y, Z).astype(np.float32)
    vmin, vmax = np.float32(field.min()), np.float32(field.max())
    amr = scenes.AmrScene("linear_amr", leaves, vals, max_level, D, np.zeros(len(leaves), np.int32), 1, tf,
                          (vmin, vmax), 0.5, [])
    grid = scenes.GridScene("linear_grid", field, 3, np.zeros(((D + 7) // 8) ** 3, np.int32), 1, tf, (vmin, vmax), 0.5, [])
    return amr, grid


def linear_tets(n=6, n_pieces=3, seed=21):
    """Jittered n^3 tetrahedral mesh with the dyadic linear field of
    linear_amr at its vertices (barycentric interpolation reproduces it), and
    the (n+1)^3 regular grid holding the same field."""
    lin = lambda x, y, z: 0.25 + x / 16.0 + y / 32.0 + z / 8.0  # noqa: E731
    sc = scenes.tet_mesh(n=n, n_pieces=n_pieces, width=4, height=4, seed=seed)
    P = sc.verts[:, :3].astype(np.float64)
    sc.verts[:, 3] = lin(P[:, 0], P[:, 1], P[:, 2])
    g = np.arange(n + 1.0)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    field = lin(X, Y, Z).astype(np.float32)
    vmin, vmax = np.float32(field.min()), np.float32(field.max())
    tf = linear_tf(0.05, 0.3)
    sc.tf, sc.tf_range = tf, (vmin, vmax)
    B = 2
    nb = (n + B - 1) // B
    grid = scenes.GridScene("linear_grid", field, 1, np.zeros(nb ** 3, np.int32), 1, tf, (vmin, vmax), 0.5, [])
    return sc, grid


# Transfer function of the two-absorber scene: three plateaus of constant
# (r, g, b, alpha) over the table entries, zero opacity outside them.  A
# sample whose table coordinate lies inside a plateau (both neighbouring
# entries in it) takes the plateau's values exactly.
ABSORBER_A = (0.35, (0.9, 0.3, 0.1))     # alpha, rgb over entries 185..200
ABSORBER_B = (0.6, (0.1, 0.4, 0.95))     # alpha, rgb over entries 221..255


def absorber_tf():
    tf = np.zeros((256, 4), np.float32)
    tf[:, 0:3] = 0.5
    tf[185:201, 3] = ABSORBER_A[0]
    tf[185:201, 0:3] = ABSORBER_A[1]
    tf[221:256, 3] = ABSORBER_B[0]
    tf[221:256, 0:3] = ABSORBER_B[1]
    return tf


def two_absorber_scene(overestimation, moment_bias=0.0):
    """Every ray crosses one or two absorbing lattice points, at known depths,
    with known colours, and nothing else absorbs.

    Field: varies with z only inside three x-bands of vertices (0..5, 6..11,
    12..17); zero except two z-levels of vertices.  An orthographic view looks
    along +z from z = -8 with step 0.5, so the lattice points sit at
    z = j + 1/4 and z = j + 3/4 and the trilinear values there are 3/4 and 1/4
    blends of two vertex values.  Band 1 (g(8) = 1, g(9) = 0.6): lattice values
    0.75 at z = 7.75 (table coordinate 191.25: absorber A) and 0.9 at 8.25
    (229.5: absorber B), every other one below table coordinate 185 (zero
    opacity).  Band 2 (g(7) = 0.6, g(8) = 1): B at 7.75, then A at 8.25.
    Band 3 (g(8) = 1, g(9) = 0.2): A at 7.75 only (0.8 at 8.25 falls in the
    zero-opacity gap 201..220).  The log-depth warp's near / far (15.9375,
    16.0625) lie between the two lattice depths t = 15.75 and 16.25, so the
    front point warps to exactly -1 and the back one to exactly +1.  Bricks of
    2 cells; the two points fall in bricks of different z, dealt to 4 pieces.

    Returns (scene, pixels, absorbers): the pixels whose rays stay inside one
    band, and per pixel the front-to-back list of absorbers ("A" / "B")."""
    nx, ny, nz = 18, 4, 16
    field = np.zeros((nz, ny, nx), np.float32)
    field[8, :, 0:6], field[9, :, 0:6] = 1.0, 0.6
    field[7, :, 6:12], field[8, :, 6:12] = 0.6, 1.0
    field[8, :, 12:18], field[9, :, 12:18] = 1.0, 0.2
    B = 2
    nb = [(n - 1 + B - 1) // B for n in (nx, ny, nz)]
    bz, by, bx = np.meshgrid(np.arange(nb[2]), np.arange(nb[1]), np.arange(nb[0]), indexing="ij")
    pob = ((bz % 2) + 2 * (bx % 2)).astype(np.int32).ravel()
    sc = scenes.GridScene("two_absorbers", field, 1, pob, 4, absorber_tf(), (np.float32(0.0), np.float32(1.0)),
                          0.5, [], moment_bias=moment_bias, overestimation=overestimation)
    W, H = nx - 1, ny - 1
    # o = eye + ((px + 1/2) / W - 1/2) * W * u: rays at x = px + 1/2, y = py + 1/2
    view = scenes.View(np.array([W / 2.0, H / 2.0, -8.0], np.float32), np.array([1, 0, 0], np.float32),
                       np.array([0, 1, 0], np.float32), np.array([0, 0, 1], np.float32), W, H, scenes.ORTHO,
                       np.float32(W), np.float32(H), np.float32(15.9375), np.float32(16.0625))
    sc.views = [view]
    pixels, absorbers = [], []
    for py in range(H):
        for px in range(W):
            if px in (5, 11):
                continue   # the ray's cell mixes two bands
            pixels.append(py * W + px)
            absorbers.append(("A", "B") if px < 5 else ("B", "A") if px < 11 else ("A",))
    return sc, np.array(pixels, np.int64), absorbers
