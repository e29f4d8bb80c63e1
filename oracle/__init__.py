"""FP64 CPU oracle of the MBOIT puzzle-piece render (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package.  The product library never does: it shares no code
with the oracle.  The C source (``mboit_oracle.c``) is compiled with the host
C compiler on first use (or by ``build()``) and called through ctypes.

Functions that are "parity unpinned": none; every routine here is pinned by
``tests/test_oracle_pins.py`` (closed forms, brute force, invariants).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mboit_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmboit_oracle.so")
_lock = threading.Lock()
_lib = None

BIAS_VECTOR_POWER4 = (0.0, 0.375, 0.0, 0.375)


class _View(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("u", ctypes.c_float * 3), ("v", ctypes.c_float * 3),
                ("w", ctypes.c_float * 3), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("projection", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("scale_u", ctypes.c_float), ("scale_v", ctypes.c_float),
                ("znear", ctypes.c_float), ("zfar", ctypes.c_float)]


class _Grid(ctypes.Structure):
    _fields_ = [("field", ctypes.c_void_p), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("brick_log2", ctypes.c_int32),
                ("piece_of_brick", ctypes.c_void_p), ("n_pieces", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("piece_selected", ctypes.c_void_p),
                ("tf", ctypes.c_void_p), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double),
                ("step", ctypes.c_double), ("moment_bias", ctypes.c_double),
                ("overestimation", ctypes.c_double), ("absorbance_max", ctypes.c_double),
                ("bias_vector", ctypes.c_double * 4), ("moment_set", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("trig_zone", ctypes.c_double)]


class _Amr(ctypes.Structure):
    _fields_ = [("values", ctypes.c_void_p), ("leaves", ctypes.c_void_p), ("n_leaves", ctypes.c_int32),
                ("max_level", ctypes.c_int32), ("finest_cells", ctypes.c_int32), ("brick_log2", ctypes.c_int32),
                ("piece_of_leaf", ctypes.c_void_p), ("n_pieces", ctypes.c_int32), ("adaptive_step", ctypes.c_int32),
                ("piece_selected", ctypes.c_void_p), ("tf", ctypes.c_void_p), ("vmin", ctypes.c_double),
                ("vmax", ctypes.c_double), ("step", ctypes.c_double), ("moment_bias", ctypes.c_double),
                ("overestimation", ctypes.c_double), ("absorbance_max", ctypes.c_double),
                ("bias_vector", ctypes.c_double * 4), ("moment_set", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("trig_zone", ctypes.c_double)]

class _Tet(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("tets", ctypes.c_void_p), ("n_verts", ctypes.c_int64),
                ("n_tets", ctypes.c_int64), ("box", ctypes.c_double * 3), ("quantum_log2", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("piece_of_tet", ctypes.c_void_p), ("n_pieces", ctypes.c_int32),
                ("reserved2", ctypes.c_int32), ("piece_selected", ctypes.c_void_p), ("tf", ctypes.c_void_p),
                ("vmin", ctypes.c_double), ("vmax", ctypes.c_double), ("step", ctypes.c_double),
                ("moment_bias", ctypes.c_double), ("overestimation", ctypes.c_double),
                ("absorbance_max", ctypes.c_double), ("bias_vector", ctypes.c_double * 4),
                ("moment_set", ctypes.c_int32), ("storage", ctypes.c_int32), ("trig_zone", ctypes.c_double)]


MOMENT_SETS = {"power4": 0, "trig6": 3, "trig8": 4, "power6": 6, "power8": 8}
STORAGES = {"f32": 0, "f16": 1, "bf16": 2}
TRIG_ZONE = 0.1


def _nm(scene):
    n = MOMENT_SETS[getattr(scene, "moment_set", "power4")]
    return 1 + 2 * n if n in (3, 4) else 1 + (n or 4)


def _set_moment_fields(st, scene):
    st.moment_set = MOMENT_SETS[getattr(scene, "moment_set", "power4")]
    st.storage = STORAGES[getattr(scene, "storage", "f32")]
    st.trig_zone = float(getattr(scene, "trig_zone", TRIG_ZONE))


def build(force=False):
    """Compile the oracle with the host C compiler (no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mboit_oracle.h"))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["cc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_mboit_bound.restype = ctypes.c_double
            lib.orc_mboit_bound.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
            lib.orc_power_bound.restype = ctypes.c_double
            lib.orc_power_bound.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_power_bias.restype = None
            lib.orc_power_bias.argtypes = [ctypes.c_int, ctypes.c_void_p]
            lib.orc_split_cells.restype = ctypes.c_int
            lib.orc_split_cells.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p]
            lib.orc_log_warp.restype = ctypes.c_double
            lib.orc_log_warp.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.orc_render_grid.restype = ctypes.c_int
            lib.orc_render_grid.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + \
                [ctypes.c_void_p] * 8
            lib.orc_trig_nodes.restype = ctypes.c_int
            lib.orc_trig_nodes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_store_round.restype = ctypes.c_double
            lib.orc_store_round.argtypes = [ctypes.c_double, ctypes.c_int]
            lib.orc_trig_bound.restype = ctypes.c_double
            lib.orc_trig_bound.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_render_amr.restype = ctypes.c_int
            lib.orc_render_amr.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + \
                [ctypes.c_void_p] * 9
            lib.orc_render_tet.restype = ctypes.c_int
            lib.orc_render_tet.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + \
                [ctypes.c_void_p] * 9
            lib.orc_tet_locate.restype = ctypes.c_int
            lib.orc_tet_locate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
            lib.orc_render_grid_given.restype = ctypes.c_int
            lib.orc_render_grid_given.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_render_grid_segments.restype = ctypes.c_int
            lib.orc_render_grid_segments.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def mboit_bound(m, z0, moment_bias, overestimation, bias_vector=BIAS_VECTOR_POWER4):
    """Alg. 3's absorbance fraction A(z0); returns (A, branch) with branch 0
    generic, 1 one-atom, 2 two-atom."""
    lib = _load()
    m = np.ascontiguousarray(m, dtype=np.float64)
    bv = np.ascontiguousarray(bias_vector, dtype=np.float64)
    fl = ctypes.c_int(0)
    A = lib.orc_mboit_bound(m.ctypes.data, float(z0), float(moment_bias), bv.ctypes.data,
                            float(overestimation), ctypes.byref(fl))
    return A, fl.value


def power_bias(n):
    """b1..b2n of the bias measure of the 2n-power-moment sets (arcsine law)."""
    out = np.zeros(2 * n)
    _load().orc_power_bias(int(n), out.ctypes.data)
    return out


def power_bound(m, n, z0, moment_bias, overestimation, bias=None):
    """Alg. 3 with 2n power moments m = b0..b2n: returns (A, branch, nodes);
    branch 0 generic (nodes = z0 and the n roots), k = a k-atom measure
    (nodes = its atoms, the rest NaN)."""
    lib = _load()
    m = np.ascontiguousarray(m, dtype=np.float64)
    bv = np.ascontiguousarray(power_bias(n) if bias is None else bias, dtype=np.float64)
    fl = ctypes.c_int(0)
    nodes = np.full(n + 1, np.nan)
    A = lib.orc_power_bound(m.ctypes.data, int(n), float(z0), float(moment_bias), bv.ctypes.data,
                            float(overestimation), ctypes.byref(fl), nodes.ctypes.data)
    return A, fl.value, nodes


def split_cells(scene):
    """A mixed-cell scene (tets, pyramids, prisms) split into tetrahedra by
    the oracle's own rule: returns (tets [m][4] int32, cell_of_tet [m] int64)."""
    import numpy as _np
    verts = _np.ascontiguousarray(scene.verts, dtype=_np.float32)
    cells = _np.ascontiguousarray(scene.cells, dtype=_np.int32)
    types = _np.ascontiguousarray(scene.cell_types, dtype=_np.int32)
    cap = 3 * len(cells)
    tets = _np.zeros((cap, 4), _np.int32)
    cot = _np.zeros(cap, _np.int64)
    n = ctypes.c_int64(0)
    if _load().orc_split_cells(verts.ctypes.data, len(verts), cells.ctypes.data, types.ctypes.data, len(cells),
                               int(scene.quantum_log2), tets.ctypes.data, cot.ctypes.data, cap, ctypes.byref(n)) != 0:
        raise ValueError("oracle rejected the cells (bad ids or types, or a flat tet)")
    return tets[:n.value].copy(), cot[:n.value].copy()


def tet_scene_of(scene):
    """The oracle's tetrahedral scene of a mixed-cell scene (its own split;
    face neighbours from the scene module)."""
    import scenes as _scenes
    tets, cot = split_cells(scene)
    return _scenes.TetScene(scene.name + "_tets", scene.verts, tets, _scenes.tet_neighbors(tets), scene.box,
                            scene.quantum_log2, scene.piece_of_cell[cot].astype(np.int32), scene.n_pieces, scene.tf,
                            scene.tf_range, scene.step, list(scene.views), scene.moment_bias, scene.overestimation,
                            scene.absorbance_max)


def trig_nodes(m, n, phi0, moment_bias):
    """Nodes (complex, node 0 = e^{i phi0}) and weights of the canonical representation."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    nodes = np.zeros(2 * (n + 1))
    w = np.zeros(n + 1)
    st = _load().orc_trig_nodes(m.ctypes.data, int(n), float(phi0), float(moment_bias), nodes.ctypes.data,
                                w.ctypes.data)
    return nodes[0::2] + 1j * nodes[1::2], w, st


def store_round(x, storage):
    """float64 -> float32 -> float16 / bfloat16 (nearest even), as stored."""
    return _load().orc_store_round(float(x), STORAGES[storage] if isinstance(storage, str) else int(storage))


def trig_bound(m, n, phi0, moment_bias, overestimation):
    """Trigonometric moment bound: (A, status, sum of the representation's weights)."""
    lib = _load()
    m = np.ascontiguousarray(m, dtype=np.float64)
    st = ctypes.c_int(0)
    ws = ctypes.c_double(0.0)
    A = lib.orc_trig_bound(m.ctypes.data, int(n), float(phi0), float(moment_bias), float(overestimation),
                           ctypes.byref(st), ctypes.byref(ws))
    return A, st.value, ws.value


def transmittance(m, z0, moment_bias, overestimation, bias_vector=BIAS_VECTOR_POWER4):
    A, _ = mboit_bound(m, z0, moment_bias, overestimation, bias_vector)
    return float(np.clip(np.exp(-m[0] * A), 0.0, 1.0))


def log_warp(t, znear, zfar):
    return _load().orc_log_warp(float(t), float(znear), float(zfar))


def _view_struct(v):
    s = _View()
    for name in ("eye", "u", "v", "w"):
        arr = np.asarray(getattr(v, name), dtype=np.float32)
        getattr(s, name)[:] = [float(x) for x in arr]
    s.width, s.height, s.projection = int(v.width), int(v.height), int(v.projection)
    s.scale_u, s.scale_v = float(v.scale_u), float(v.scale_v)
    s.znear, s.zfar = float(v.near), float(v.far)
    return s


def _grid_struct(scene, pieces):
    K = scene.n_pieces
    keep = dict(field=np.ascontiguousarray(scene.field, dtype=np.float32),
                pob=np.ascontiguousarray(scene.piece_of_brick, dtype=np.int32),
                tf=np.ascontiguousarray(scene.tf, dtype=np.float32), sel=None)
    if pieces is not None:
        keep["sel"] = np.zeros(K, dtype=np.uint8)
        keep["sel"][np.asarray(list(pieces), dtype=np.int64)] = 1
    g = _Grid()
    nx, ny, nz = scene.dims
    g.field, g.nx, g.ny, g.nz, g.brick_log2 = keep["field"].ctypes.data, nx, ny, nz, scene.brick_log2
    g.piece_of_brick, g.n_pieces = keep["pob"].ctypes.data, K
    g.piece_selected = _ptr(keep["sel"])
    g.tf = keep["tf"].ctypes.data
    g.vmin, g.vmax = float(scene.tf_range[0]), float(scene.tf_range[1])
    g.step = float(scene.step)
    g.moment_bias, g.overestimation = float(scene.moment_bias), float(scene.overestimation)
    g.absorbance_max = float(scene.absorbance_max)
    g.bias_vector[:] = list(getattr(scene, "bias_vector", BIAS_VECTOR_POWER4))
    _set_moment_fields(g, scene)
    return g, keep


def _amr_struct(scene, pieces):
    K = scene.n_pieces
    keep = dict(values=np.ascontiguousarray(scene.values, dtype=np.float32),
                leaves=np.ascontiguousarray(scene.leaves, dtype=np.int32),
                pol=np.ascontiguousarray(scene.piece_of_leaf, dtype=np.int32),
                tf=np.ascontiguousarray(scene.tf, dtype=np.float32), sel=None)
    if pieces is not None:
        keep["sel"] = np.zeros(K, dtype=np.uint8)
        keep["sel"][np.asarray(list(pieces), dtype=np.int64)] = 1
    a = _Amr()
    a.values, a.leaves, a.n_leaves = keep["values"].ctypes.data, keep["leaves"].ctypes.data, scene.leaves.shape[0]
    a.max_level, a.finest_cells, a.brick_log2 = scene.max_level, scene.finest_cells, scene.brick_log2
    a.piece_of_leaf, a.n_pieces = keep["pol"].ctypes.data, K
    a.adaptive_step = 1 if getattr(scene, "adaptive_step", False) else 0
    a.piece_selected = _ptr(keep["sel"])
    a.tf = keep["tf"].ctypes.data
    a.vmin, a.vmax = float(scene.tf_range[0]), float(scene.tf_range[1])
    a.step = float(scene.step)
    a.moment_bias, a.overestimation = float(scene.moment_bias), float(scene.overestimation)
    a.absorbance_max = float(scene.absorbance_max)
    a.bias_vector[:] = list(getattr(scene, "bias_vector", BIAS_VECTOR_POWER4))
    _set_moment_fields(a, scene)
    return a, keep


def _tet_struct(scene, pieces):
    K = scene.n_pieces
    keep = dict(verts=np.ascontiguousarray(scene.verts, dtype=np.float32),
                tets=np.ascontiguousarray(scene.tets, dtype=np.int32),
                pot=np.ascontiguousarray(scene.piece_of_tet, dtype=np.int32),
                tf=np.ascontiguousarray(scene.tf, dtype=np.float32), sel=None)
    if pieces is not None:
        keep["sel"] = np.zeros(K, dtype=np.uint8)
        keep["sel"][np.asarray(list(pieces), dtype=np.int64)] = 1
    m = _Tet()
    m.verts, m.tets = keep["verts"].ctypes.data, keep["tets"].ctypes.data
    m.n_verts, m.n_tets = keep["verts"].shape[0], keep["tets"].shape[0]
    m.box[:] = [float(b) for b in scene.box]
    m.quantum_log2 = int(scene.quantum_log2)
    m.piece_of_tet, m.n_pieces = keep["pot"].ctypes.data, K
    m.piece_selected = _ptr(keep["sel"])
    m.tf = keep["tf"].ctypes.data
    m.vmin, m.vmax = float(scene.tf_range[0]), float(scene.tf_range[1])
    m.step = float(scene.step)
    m.moment_bias, m.overestimation = float(scene.moment_bias), float(scene.overestimation)
    m.absorbance_max = float(scene.absorbance_max)
    m.bias_vector[:] = list(getattr(scene, "bias_vector", BIAS_VECTOR_POWER4))
    _set_moment_fields(m, scene)
    return m, keep


def _is_amr(scene):
    return hasattr(scene, "leaves")


def _is_tet(scene):
    return hasattr(scene, "tets")


def tet_locate(scene, points, brute_force=False):
    """Exact point location in a tetrahedral scene: (owner tet [n] int32, -1
    none; tets passing the test [n] int32; interpolated value [n] float64)."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    n = pts.shape[0]
    owner = np.zeros(n, np.int32)
    npass = np.zeros(n, np.int32)
    val = np.zeros(n)
    m, keep = _tet_struct(scene, None)
    if lib.orc_tet_locate(ctypes.byref(m), pts.ctypes.data, n, owner.ctypes.data, npass.ctypes.data,
                          val.ctypes.data, int(bool(brute_force))) != 0:
        raise ValueError("oracle rejected the mesh (orientation, box or quantum)")
    return owner, npass, val


def render_amr(scene, view=0, pixels=None, pieces=None, want=("mboit",)):
    """render_grid for a brick-octree scene (`scenes.AmrScene`) or a
    tetrahedral scene (`scenes.TetScene`); `want` may also name "nsegments"."""
    lib = _load()
    v = scene.views[view] if isinstance(view, int) else view
    pix = np.arange(v.width * v.height, dtype=np.int64) if pixels is None else \
        np.ascontiguousarray(pixels, dtype=np.int64)
    n, K, nm = pix.size, scene.n_pieces, _nm(scene)
    shapes = {"moments": (n, nm), "piece_moments": (n, K, nm), "piece_color": (n, K, 4), "mboit": (n, 4),
              "raw": (n, 4), "exact": (n, 4), "sortlast": (n, 4)}
    out = {k: np.zeros(shapes[k]) for k in want if k in shapes}
    for k in ("nsamples", "nsegments"):
        if k in want:
            out[k] = np.zeros(n, dtype=np.int64)
    if "nsegments" in out and "sortlast" not in out:
        out["sortlast"] = np.zeros((n, 4))
    if _is_tet(scene):
        a, keep = _tet_struct(scene, pieces)
        fn = lib.orc_render_tet
    else:
        a, keep = _amr_struct(scene, pieces)
        fn = lib.orc_render_amr
    vs = _view_struct(v)
    rc = fn(ctypes.byref(a), ctypes.byref(vs), pix.ctypes.data, n,
                            _ptr(out.get("moments")), _ptr(out.get("piece_moments")), _ptr(out.get("piece_color")),
                            _ptr(out.get("mboit")), _ptr(out.get("raw")), _ptr(out.get("exact")),
                            _ptr(out.get("sortlast")), _ptr(out.get("nsamples")), _ptr(out.get("nsegments")))
    if rc != 0:
        raise ValueError("oracle rejected its arguments (bad or overlapping leaves or tets?)")
    return out


def render(scene, view=0, pixels=None, pieces=None, want=("mboit",)):
    """render_grid or render_amr, by scene type."""
    f = render_amr if (_is_amr(scene) or _is_tet(scene)) else render_grid
    return f(scene, view=view, pixels=pixels, pieces=pieces, want=want)


def render_segments(scene, view=0, pixels=None, pieces=None):
    """Sort-last route only: (rgba [n][4] float64, segments per pixel [n] int64)."""
    if _is_amr(scene) or _is_tet(scene):
        r = render_amr(scene, view=view, pixels=pixels, pieces=pieces, want=("sortlast", "nsegments"))
        return r["sortlast"], r["nsegments"]
    lib = _load()
    v = scene.views[view] if isinstance(view, int) else view
    pix = np.arange(v.width * v.height, dtype=np.int64) if pixels is None else \
        np.ascontiguousarray(pixels, dtype=np.int64)
    g, keep = _grid_struct(scene, pieces)
    rgba = np.zeros((pix.size, 4))
    nseg = np.zeros(pix.size, dtype=np.int64)
    vs = _view_struct(v)
    if lib.orc_render_grid_segments(ctypes.byref(g), ctypes.byref(vs), pix.ctypes.data, pix.size,
                                    rgba.ctypes.data, nseg.ctypes.data) != 0:
        raise ValueError("oracle rejected its arguments")
    return rgba, nseg


def render_grid_given(scene, moments, view=0, pixels=None, pieces=None):
    """Stage two of a grid scene from given global moments (Alg. 1 loop 2):
    `moments` [n][nm] per listed pixel in the order render_grid returns them
    (b0, b1.. or b0, Re t1, Im t1, ..; t_j not normalised).  Returns
    {"mboit", "raw"} [n][4]."""
    lib = _load()
    v = scene.views[view] if isinstance(view, int) else view
    pix = np.arange(v.width * v.height, dtype=np.int64) if pixels is None else \
        np.ascontiguousarray(pixels, dtype=np.int64)
    given = np.ascontiguousarray(moments, dtype=np.float64).reshape(pix.size, _nm(scene))
    g, keep = _grid_struct(scene, pieces)
    out = {"mboit": np.zeros((pix.size, 4)), "raw": np.zeros((pix.size, 4))}
    vs = _view_struct(v)
    if lib.orc_render_grid_given(ctypes.byref(g), ctypes.byref(vs), pix.ctypes.data, pix.size, given.ctypes.data,
                                 out["mboit"].ctypes.data, out["raw"].ctypes.data) != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def render_grid(scene, view=0, pixels=None, pieces=None, want=("mboit",)):
    """Runs the oracle on the listed pixels (flat indices y*W + x; None = all).

    `pieces`: iterable of selected piece ids (None = all).  `want` picks the
    outputs among: moments, piece_moments, piece_color, mboit, raw, exact,
    sortlast, nsamples.  Returns a dict of float64 arrays (nsamples int64);
    moments have 5 entries (power) or 1 + 2n (n trigonometric moments).
    """
    lib = _load()
    v = scene.views[view] if isinstance(view, int) else view
    npx = v.width * v.height
    pix = np.arange(npx, dtype=np.int64) if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    n, K, nm = pix.size, scene.n_pieces, _nm(scene)
    g, keep = _grid_struct(scene, pieces)
    shapes = {"moments": (n, nm), "piece_moments": (n, K, nm), "piece_color": (n, K, 4), "mboit": (n, 4),
              "raw": (n, 4), "exact": (n, 4), "sortlast": (n, 4)}
    out = {k: np.zeros(shapes[k]) for k in want if k in shapes}
    if "nsamples" in want:
        out["nsamples"] = np.zeros(n, dtype=np.int64)
    vs = _view_struct(v)
    rc = lib.orc_render_grid(ctypes.byref(g), ctypes.byref(vs), pix.ctypes.data, n,
                             _ptr(out.get("moments")), _ptr(out.get("piece_moments")),
                             _ptr(out.get("piece_color")), _ptr(out.get("mboit")), _ptr(out.get("raw")),
                             _ptr(out.get("exact")), _ptr(out.get("sortlast")), _ptr(out.get("nsamples")))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out
