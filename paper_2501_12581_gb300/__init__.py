"""GB300 MBOIT puzzle-piece renderer (Approximate Puzzlepiece Compositing,
arXiv 2501.12581): Python binding of the C ABI in ``include/mboit.h``.

The functions ``mboit_*`` below have the names of the C entry points and only
marshal arguments (torch CUDA tensors -> device pointers, the current torch
stream -> cudaStream_t, views -> ``mboit_view`` structs); every step of the
render runs in the CUDA library ``_lib/libmboit.so``.  There is no CPU path:
if the library is missing or fails to load, every call raises.

``Volume`` wraps a volume handle for the common case of a regular grid built
from a ``scenes.GridScene``-like object.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmboit.so")

MBOIT_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "UNSUPPORTED", 5: "STATE",
                6: "TIMEOUT", 7: "DEVICE_ASSERT"}
MBOIT_GRID, MBOIT_AMR, MBOIT_TET = 0, 1, 2
MBOIT_POWER4, MBOIT_TRIG6, MBOIT_TRIG8, MBOIT_POWER6, MBOIT_POWER8 = 0, 1, 2, 3, 4
MBOIT_STORE_F32, MBOIT_STORE_F16, MBOIT_STORE_BF16 = 0, 1, 2
MOMENT_SET_IDS = {"power4": MBOIT_POWER4, "trig6": MBOIT_TRIG6, "trig8": MBOIT_TRIG8, "power6": MBOIT_POWER6,
                  "power8": MBOIT_POWER8}
STORAGE_IDS = {"f32": MBOIT_STORE_F32, "f16": MBOIT_STORE_F16, "bf16": MBOIT_STORE_BF16}
MBOIT_ORTHO, MBOIT_PERSPECTIVE = 0, 1
MBOIT_PACKET_8X4, MBOIT_PACKET_4X8 = 0, 1
MBOIT_MOMENTS_PER_PIECE, MBOIT_MOMENTS_REDUCED = 0, 1
MBOIT_COLOR_PER_PIECE, MBOIT_COLOR_REDUCED, MBOIT_COLOR_RESOLVED = 0, 1, 2
MBOIT_OP_MOMENTS_SUM, MBOIT_OP_COLOR_SUM_RESOLVE = 0, 1
MBOIT_FLAG_RAW_SUM, MBOIT_FLAG_DETERMINISTIC, MBOIT_FLAG_ADAPTIVE_STEP, MBOIT_FLAG_FP64_SETUP = 0x1, 0x2, 0x4, 0x8

EXPORTED = ["mboit_last_error", "mboit_moment_image_bytes", "mboit_create_volume", "mboit_destroy_volume",
            "mboit_add_piece", "mboit_render_moments", "mboit_reconstruct_blend", "mboit_composite",
            "mboit_render_frame", "mboit_render_frame_host", "mboit_render_frame_multi", "mboit_synchronize",
            "mboit_get_stats",
            "mboit_render_moments_noalloc", "mboit_set_tuning", "mboit_set_packet", "mboit_set_frame_launches",
            "mboit_set_tile_order", "mboit_autotune", "mboit_clear_tuning_cache",
            "mboit_render_sortlast", "mboit_split_cells", "mboit_debug_corrupt"]
MBOIT_NUM_TUNINGS = 7


class MboitError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mboit_view(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("u", ctypes.c_float * 3), ("v", ctypes.c_float * 3),
                ("w", ctypes.c_float * 3), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("projection", ctypes.c_int32), ("reserved", ctypes.c_int32), ("scale_u", ctypes.c_float),
                ("scale_v", ctypes.c_float), ("near", ctypes.c_float), ("far", ctypes.c_float)]


class mboit_volume_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("moment_set", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("field", ctypes.c_void_p), ("dims", ctypes.c_int32 * 3),
                ("brick_log2", ctypes.c_int32), ("tf_rgba", ctypes.c_void_p), ("tf_range", ctypes.c_float * 2),
                ("step", ctypes.c_float), ("moment_bias", ctypes.c_float), ("overestimation", ctypes.c_float),
                ("absorbance_max", ctypes.c_float), ("leaf_values", ctypes.c_void_p), ("leaf_table", ctypes.c_void_p),
                ("n_leaves", ctypes.c_int32), ("max_level", ctypes.c_int32), ("tet_verts", ctypes.c_void_p),
                ("tet_cells", ctypes.c_void_p), ("tet_neighbors", ctypes.c_void_p), ("n_verts", ctypes.c_int64),
                ("n_tets", ctypes.c_int64), ("tet_box", ctypes.c_float * 3), ("quantum_log2", ctypes.c_int32)]


class mboit_stats(ctypes.Structure):
    _fields_ = [("samples_pass1", ctypes.c_int64), ("samples_pass2", ctypes.c_int64),
                ("singular_pixels", ctypes.c_int64), ("n_pieces", ctypes.c_int32), ("device", ctypes.c_int32),
                ("tuning_pass1", ctypes.c_int32), ("tuning_pass2", ctypes.c_int32),
                ("sortlast_segments", ctypes.c_int64), ("sortlast_max_segments", ctypes.c_int32),
                ("fp64_pixels", ctypes.c_int32), ("frame_pass1_ms", ctypes.c_float), ("frame_pass2_ms", ctypes.c_float),
                ("packet", ctypes.c_int32), ("frame_launches", ctypes.c_int32), ("tile_order", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def load_library(path=LIB_PATH):
    """Loads libmboit.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise MboitError(3, f"CUDA library {path} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "mboit_last_error": (ctypes.c_char_p, []),
        "mboit_moment_image_bytes": (ctypes.c_size_t, [I32, I32, I32, I32]),
        "mboit_create_volume": (ctypes.c_int, [P, P]),
        "mboit_destroy_volume": (ctypes.c_int, [P]),
        "mboit_add_piece": (ctypes.c_int, [P, P, I64, I32, P]),
        "mboit_render_moments": (ctypes.c_int, [P, P, I32, P, I32, I32, P, P]),
        "mboit_reconstruct_blend": (ctypes.c_int, [P, P, I32, P, I32, P, I32, P, P]),
        "mboit_composite": (ctypes.c_int, [P, I32, I32, I32, I32, I32, P, P, P, P, P]),
        "mboit_render_frame": (ctypes.c_int, [P, P, I32, P, P, P]),
        "mboit_render_frame_host": (ctypes.c_int, [P, P, P, I32, P, P, P, P]),
        "mboit_render_frame_multi": (ctypes.c_int, [P, I32, P, P, I32, P, P, P]),
        "mboit_synchronize": (ctypes.c_int, [P, P]),
        "mboit_get_stats": (ctypes.c_int, [P, P]),
        "mboit_render_moments_noalloc": (ctypes.c_int, [P, P, P, I32, P, P]),
        "mboit_set_tuning": (ctypes.c_int, [P, I32, I32]),
        "mboit_set_packet": (ctypes.c_int, [P, I32]),
        "mboit_set_frame_launches": (ctypes.c_int, [P, I32]),
        "mboit_set_tile_order": (ctypes.c_int, [P, I32]),
        "mboit_clear_tuning_cache": (None, []),
        "mboit_autotune": (ctypes.c_int, [P, P, I32, P, P, P, P]),
        "mboit_render_sortlast": (ctypes.c_int, [P, P, I32, P, P, P]),
        "mboit_split_cells": (ctypes.c_int, [P, I64, P, P, I64, I32, P, P, P, I64, P]),
        "mboit_debug_corrupt": (ctypes.c_int, [P, I32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != MBOIT_OK:
        raise MboitError(status, load_library().mboit_last_error().decode(errors="replace"))


def _ptr(t):
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensors passed to libmboit must be contiguous")
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def make_view(v):
    """``scenes.View``-like object (or an mboit_view) -> mboit_view."""
    if isinstance(v, mboit_view):
        return v
    s = mboit_view()
    for name in ("eye", "u", "v", "w"):
        getattr(s, name)[:] = [float(x) for x in np.asarray(getattr(v, name), dtype=np.float32)]
    s.width, s.height, s.projection = int(v.width), int(v.height), int(v.projection)
    s.scale_u, s.scale_v = float(v.scale_u), float(v.scale_v)
    s.near, s.far = float(v.near), float(v.far)
    return s


def _views(views):
    views = list(views)
    arr = (mboit_view * len(views))()
    for i, v in enumerate(views):
        arr[i] = make_view(v)
    return arr, len(views)


def _pieces(pieces):
    if pieces is None:
        return None, 0, None
    a = np.ascontiguousarray(np.asarray(list(pieces), dtype=np.int32))
    return a.ctypes.data, a.size, a


# ---------------------------------------------------------------------------
# the C entry points, same names


def mboit_last_error():
    return load_library().mboit_last_error().decode(errors="replace")


def mboit_split_cells(verts, cells, cell_types, quantum_log2):
    """Mixed cells (4 tet, 5 pyramid, 6 prism) -> (tets [m][4] int32,
    neighbours [m][4] int32, cell_of_tet [m] int64), split by the library."""
    verts = np.ascontiguousarray(verts, dtype=np.float32)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    types = np.ascontiguousarray(cell_types, dtype=np.int32)
    cap = 3 * len(cells)
    tets = np.zeros((cap, 4), np.int32)
    nbrs = np.zeros((cap, 4), np.int32)
    cot = np.zeros(cap, np.int64)
    n = ctypes.c_int64(0)
    _check(load_library().mboit_split_cells(verts.ctypes.data, len(verts), cells.ctypes.data, types.ctypes.data,
                                            len(cells), int(quantum_log2), tets.ctypes.data, nbrs.ctypes.data,
                                            cot.ctypes.data, cap, ctypes.byref(n)))
    m = n.value
    return tets[:m].copy(), nbrs[:m].copy(), cot[:m].copy()


def mboit_moment_image_bytes(width, height, moment_set=MBOIT_POWER4, storage=MBOIT_STORE_F32):
    return int(load_library().mboit_moment_image_bytes(width, height, moment_set, storage))


def mboit_create_volume(desc):
    h = ctypes.c_void_p()
    _check(load_library().mboit_create_volume(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def mboit_destroy_volume(v):
    _check(load_library().mboit_destroy_volume(v))


def mboit_add_piece(v, ids, ids_on_device=None):
    if ids_on_device is None:
        ids_on_device = bool(hasattr(ids, "is_cuda") and ids.is_cuda)
    keep = ids if hasattr(ids, "data_ptr") else np.ascontiguousarray(ids, dtype=np.int32)
    if hasattr(keep, "dtype") and str(keep.dtype) not in ("int32", "torch.int32"):
        raise ValueError("brick ids must be int32")
    out = ctypes.c_int32(-1)
    n = keep.numel() if hasattr(keep, "numel") else keep.size
    _check(load_library().mboit_add_piece(v, _ptr(keep), n, int(ids_on_device), ctypes.byref(out)))
    return out.value


def mboit_render_moments(v, views, moments, pieces=None, mode=MBOIT_MOMENTS_REDUCED, stream=None):
    arr, n = _views(views)
    pp, npc, _keep = _pieces(pieces)
    _check(load_library().mboit_render_moments(v, arr, n, pp, npc, mode, _ptr(moments), _stream(stream)))


def mboit_reconstruct_blend(v, views, global_moments, color, pieces=None, mode=MBOIT_COLOR_RESOLVED, stream=None):
    arr, n = _views(views)
    pp, npc, _keep = _pieces(pieces)
    _check(load_library().mboit_reconstruct_blend(v, arr, n, pp, npc, _ptr(global_moments), mode, _ptr(color),
                                                  _stream(stream)))


def mboit_composite(v, op, width, height, n_views, n_inputs, inp, out, global_moments=None, bg=None, stream=None):
    bgp = None
    if bg is not None:
        bga = (ctypes.c_float * 4)(*[float(x) for x in bg])
        bgp = ctypes.cast(bga, ctypes.c_void_p).value
    _check(load_library().mboit_composite(v, op, width, height, n_views, n_inputs, _ptr(inp), _ptr(out),
                                          _ptr(global_moments), bgp, _stream(stream)))


def mboit_render_frame(v, views, moments_scratch, rgba, stream=None):
    arr, n = _views(views)
    _check(load_library().mboit_render_frame(v, arr, n, _ptr(moments_scratch), _ptr(rgba), _stream(stream)))


def mboit_render_frame_multi(vols, views, view_volume, moments_scratch, rgba, stream=None):
    """One frame over several grid volumes: view i samples vols[view_volume[i]]."""
    vols = list(vols)
    handles = (ctypes.c_void_p * len(vols))(*vols)
    arr, n = _views(views)
    vv = list(view_volume)
    if len(vv) != n:
        raise ValueError(f"view_volume has {len(vv)} entries for {n} views")
    owner = (ctypes.c_int32 * n)(*vv)
    _check(load_library().mboit_render_frame_multi(handles, len(vols), arr, owner, n, _ptr(moments_scratch),
                                                   _ptr(rgba), _stream(stream)))


def mboit_render_frame_host(v, field_host, views, moments_scratch, rgba_device, rgba_host, stream=None):
    arr, n = _views(views)
    _check(load_library().mboit_render_frame_host(v, _ptr(field_host), arr, n, _ptr(moments_scratch),
                                                  _ptr(rgba_device), _ptr(rgba_host), _stream(stream)))


def mboit_synchronize(v, stream=None):
    _check(load_library().mboit_synchronize(v, _stream(stream)))


def mboit_get_stats(v):
    s = mboit_stats()
    _check(load_library().mboit_get_stats(v, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in mboit_stats._fields_}


def mboit_set_tuning(v, pass1, pass2):
    _check(load_library().mboit_set_tuning(v, int(pass1), int(pass2)))


def mboit_set_packet(v, packet):
    _check(load_library().mboit_set_packet(v, int(packet)))


def mboit_set_frame_launches(v, launches):
    _check(load_library().mboit_set_frame_launches(v, int(launches)))


def mboit_clear_tuning_cache():
    load_library().mboit_clear_tuning_cache()


def mboit_set_tile_order(v, order):
    _check(load_library().mboit_set_tile_order(v, int(order)))


def mboit_autotune(v, views, moments_scratch, rgba, stream=None):
    """Returns (pass-1 configuration, pass-2 configuration, ray packet)."""
    arr, n = _views(views)
    out = (ctypes.c_int32 * 3)()
    _check(load_library().mboit_autotune(v, arr, n, _ptr(moments_scratch), _ptr(rgba), _stream(stream), out))
    return int(out[0]), int(out[1]), int(out[2])


def mboit_render_sortlast(v, views, rgba, segments_per_pixel=None, stream=None):
    arr, n = _views(views)
    _check(load_library().mboit_render_sortlast(v, arr, n, _ptr(rgba), _ptr(segments_per_pixel), _stream(stream)))


def grid_desc(scene, field, flags=0):
    """mboit_volume_desc for a regular-grid scene whose field is the CUDA
    tensor `field`; returns (desc, keepalive) - keep both while in use."""
    tf = np.ascontiguousarray(scene.tf, dtype=np.float32)
    d = mboit_volume_desc()
    d.kind, d.moment_set, d.storage, d.flags = MBOIT_GRID, MBOIT_POWER4, MBOIT_STORE_F32, flags
    d.field = field.data_ptr()
    nz, ny, nx = scene.field.shape
    d.dims[:] = [nx, ny, nz]
    d.brick_log2 = scene.brick_log2
    d.tf_rgba = tf.ctypes.data
    d.tf_range[:] = [float(scene.tf_range[0]), float(scene.tf_range[1])]
    d.step, d.moment_bias = float(scene.step), float(scene.moment_bias)
    d.overestimation, d.absorbance_max = float(scene.overestimation), float(scene.absorbance_max)
    return d, (tf, field)


def mboit_render_moments_noalloc(desc, views, moments, brick_selected=None, stream=None):
    """Pass 1 without any device allocation (see include/mboit.h).

    brick_selected: None (every brick) or one byte per brick of the grid,
    nbx * nby * nbz with nb = ceil((dims - 1) / 2^brick_log2) per axis."""
    arr, n = _views(views)
    sel = None
    if brick_selected is not None:
        sel = np.ascontiguousarray(brick_selected, dtype=np.uint8).ravel()
        B = 1 << int(desc.brick_log2)
        nbricks = 1
        for c in range(3):
            nbricks *= (int(desc.dims[c]) - 1 + B - 1) // B
        if sel.size != nbricks:
            raise ValueError(f"brick_selected has {sel.size} entries; the grid has {nbricks} bricks")
    _check(load_library().mboit_render_moments_noalloc(ctypes.byref(desc), _ptr(sel), arr, n, _ptr(moments),
                                                       _stream(stream)))


def mboit_debug_corrupt(handle, what):
    """Test hook of the failure detection (see include/mboit.h): overwrites a
    library-owned table of the volume (1: an octree map entry, 2: mesh face
    neighbours) so that later renders report MBOIT_ERR_DEVICE_ASSERT, or (3,
    grids) makes every TMA window load wait for a copy never issued, so that
    renders in window configurations 5 and 6 report MBOIT_ERR_TIMEOUT."""
    _check(load_library().mboit_debug_corrupt(handle, int(what)))


# ---------------------------------------------------------------------------
# convenience wrapper


class Volume:
    """A volume on the current CUDA device built from a scene: a regular grid
    (``field``, ``brick_log2``, ``piece_of_brick``), a brick octree
    (``leaves``, ``values``, ``max_level``, ``piece_of_leaf``) or a
    tetrahedral mesh (``verts``, ``tets``, ``neighbors``, ``box``,
    ``quantum_log2``, ``piece_of_tet``), plus ``n_pieces``, ``tf``,
    ``tf_range``, ``step``, ``moment_bias``, ``overestimation``,
    ``absorbance_max``.  Keeps the device data alive."""

    def __init__(self, scene, field=None, flags=0):
        import torch
        load_library()
        self.scene = scene
        if hasattr(scene, "cells"):
            # mixed cells: the library's split into tets, pieces by cell
            tets, nbrs, cot = mboit_split_cells(scene.verts, scene.cells, scene.cell_types, scene.quantum_log2)
            import copy as _copy
            mixed = scene
            scene = _copy.copy(scene)
            scene.tets, scene.neighbors = tets, nbrs
            scene.piece_of_tet = np.asarray(mixed.piece_of_cell)[cot].astype(np.int32)
        amr = hasattr(scene, "leaves")
        tet = hasattr(scene, "tets")
        if tet:
            self.field = None
        else:
            data = scene.values if amr else scene.field
            self.field = field if field is not None else torch.from_numpy(np.ascontiguousarray(data)).cuda()
        tf = np.ascontiguousarray(scene.tf, dtype=np.float32)
        d = mboit_volume_desc()
        d.kind = MBOIT_TET if tet else MBOIT_AMR if amr else MBOIT_GRID
        self.moment_set = MOMENT_SET_IDS[getattr(scene, "moment_set", "power4")]
        self.storage = STORAGE_IDS[getattr(scene, "storage", "f32")]
        if amr and getattr(scene, "adaptive_step", False):
            flags |= MBOIT_FLAG_ADAPTIVE_STEP
        d.moment_set, d.storage, d.flags = self.moment_set, self.storage, flags
        if tet:
            verts = np.ascontiguousarray(scene.verts, dtype=np.float32)
            cells = np.ascontiguousarray(scene.tets, dtype=np.int32)
            nbrs = np.ascontiguousarray(scene.neighbors, dtype=np.int32)
            d.tet_verts, d.tet_cells, d.tet_neighbors = verts.ctypes.data, cells.ctypes.data, nbrs.ctypes.data
            d.n_verts, d.n_tets = verts.shape[0], cells.shape[0]
            d.tet_box[:] = [float(b) for b in scene.box]
            d.quantum_log2 = int(scene.quantum_log2)
        elif amr:
            table = np.ascontiguousarray(scene.leaves, dtype=np.int32)
            d.leaf_values, d.leaf_table = self.field.data_ptr(), table.ctypes.data
            d.n_leaves, d.max_level = table.shape[0], scene.max_level
            d.dims[:] = list(scene.dims)
        else:
            d.field = self.field.data_ptr()
            nz, ny, nx = scene.field.shape
            d.dims[:] = [nx, ny, nz]
        d.brick_log2 = 0 if tet else scene.brick_log2
        d.tf_rgba = tf.ctypes.data
        d.tf_range[:] = [float(scene.tf_range[0]), float(scene.tf_range[1])]
        d.step, d.moment_bias = float(scene.step), float(scene.moment_bias)
        d.overestimation, d.absorbance_max = float(scene.overestimation), float(scene.absorbance_max)
        self.handle = mboit_create_volume(d)
        pob = np.asarray(scene.piece_of_tet if tet else scene.piece_of_leaf if amr else scene.piece_of_brick)
        for p in range(scene.n_pieces):
            mboit_add_piece(self.handle, np.nonzero(pob == p)[0].astype(np.int32))

    def close(self):
        if getattr(self, "handle", None):
            mboit_destroy_volume(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def moment_buffer(views, n_slots=1, moment_set=MBOIT_POWER4, storage=MBOIT_STORE_F32):
        """Zeroed device buffer (float32 words) for n_slots moment slabs per view."""
        import torch
        total = sum(mboit_moment_image_bytes(v.width, v.height, moment_set, storage) for v in views) * n_slots
        return torch.zeros(total // 4, dtype=torch.float32, device="cuda")

    def moments_for(self, views, n_slots=1):
        """moment_buffer in this volume's moment format."""
        return Volume.moment_buffer(views, n_slots, self.moment_set, self.storage)

    @staticmethod
    def color_buffer(views, n_slots=1):
        import torch
        total = sum(v.width * v.height * 4 for v in views) * n_slots
        return torch.zeros(total, dtype=torch.float32, device="cuda")

    @staticmethod
    def unpack_moments(buf, views, n_slots=1, moment_set=MBOIT_POWER4):
        """Device slab buffer of power moments -> list per view of
        [n_slots][H*W][2n + 1] float32 tensors (b0..b2n; n = 2, 3 or 4)."""
        nm = {MBOIT_POWER4: 5, MBOIT_POWER6: 7, MBOIT_POWER8: 9}[moment_set]
        out, off = [], 0
        for v in views:
            npx = v.width * v.height
            P = (npx + 3) // 4 * 4
            slabs = []
            for j in range(n_slots):
                s = buf[off + j * nm * P: off + (j + 1) * nm * P]
                slabs.append(torch_cat_moments(s, P, npx, nm))
            out.append(slabs)
            off += n_slots * nm * P
        return out

    def render_moments(self, views, moments, pieces=None, mode=MBOIT_MOMENTS_REDUCED, stream=None):
        mboit_render_moments(self.handle, views, moments, pieces, mode, stream)

    def reconstruct_blend(self, views, global_moments, color, pieces=None, mode=MBOIT_COLOR_RESOLVED, stream=None):
        mboit_reconstruct_blend(self.handle, views, global_moments, color, pieces, mode, stream)

    def composite(self, op, width, height, n_views, n_inputs, inp, out, global_moments=None, bg=None, stream=None):
        mboit_composite(self.handle, op, width, height, n_views, n_inputs, inp, out, global_moments, bg, stream)

    def render_frame(self, views, moments_scratch, rgba, stream=None):
        mboit_render_frame(self.handle, views, moments_scratch, rgba, stream)

    @staticmethod
    def render_frame_multi(volumes, views, view_volume, moments_scratch, rgba, stream=None):
        """One frame over several grid volumes (view i samples volumes[view_volume[i]])."""
        mboit_render_frame_multi([v.handle for v in volumes], views, view_volume, moments_scratch, rgba, stream)

    def synchronize(self, stream=None):
        mboit_synchronize(self.handle, stream)

    def render_sortlast(self, views, rgba, segments_per_pixel=None, stream=None):
        mboit_render_sortlast(self.handle, views, rgba, segments_per_pixel, stream)

    def set_tuning(self, pass1, pass2):
        mboit_set_tuning(self.handle, pass1, pass2)

    def set_packet(self, packet):
        mboit_set_packet(self.handle, packet)

    def set_frame_launches(self, launches):
        mboit_set_frame_launches(self.handle, launches)

    def set_tile_order(self, order):
        mboit_set_tile_order(self.handle, order)

    def autotune(self, views, moments_scratch, rgba, stream=None):
        return mboit_autotune(self.handle, views, moments_scratch, rgba, stream)

    def stats(self):
        return mboit_get_stats(self.handle)


def save_moments(path, moments, views, moment_set=MBOIT_POWER4, storage=MBOIT_STORE_F32, n_slots=1):
    """Writes a moment buffer (as render_moments or render_frame leave it) to
    `path` (.npz): its raw 32-bit words and the views' sizes and the moment
    format, so that pass 2 (reconstruct_blend) can be replayed from it later."""
    import numpy as np
    import torch
    words = moments.detach().cpu().contiguous().view(-1)
    sizes = np.array([[v.width, v.height] for v in views], np.int32)
    expect = sum(mboit_moment_image_bytes(int(w), int(h), moment_set, storage) for w, h in sizes) * n_slots
    if words.numel() * 4 < expect:
        raise ValueError(f"the buffer holds {words.numel() * 4} bytes, the views need {expect}")
    np.savez(path, words=words.view(torch.int32).numpy(), sizes=sizes,
             fmt=np.array([moment_set, storage, n_slots], np.int32))


def load_moments(path, device="cuda"):
    """Reads save_moments' file: (buffer as float32 words on `device`, view
    sizes [(width, height)], moment set, storage, slots)."""
    import numpy as np
    import torch
    z = np.load(path)
    buf = torch.from_numpy(z["words"]).view(torch.float32).to(device)
    ms, st, slots = (int(x) for x in z["fmt"])
    return buf, [tuple(int(a) for a in r) for r in z["sizes"]], ms, st, slots


def torch_cat_moments(slab, P, npx, nm=5):
    """One power-moment slab (nm * P floats: b0 plane, float4 plane of b1..b4,
    then a float2 plane (nm = 7) or float4 plane (nm = 9)) -> [npx][nm]."""
    import torch
    parts = [slab[:P][:npx, None], slab[P:5 * P].view(P, 4)[:npx]]
    if nm > 5:
        parts.append(slab[5 * P:nm * P].view(P, nm - 5)[:npx])
    return torch.cat(parts, dim=1)