/*
 * mboit.h -- C ABI of the GB300 library for Approximate Puzzlepiece
 * Compositing: the two-pass moment-based order-independent transparency
 * (MBOIT) volume render of non-convex subdomains ("puzzle pieces").
 *
 * Method (arXiv 2501.12581):
 *   Sec. 4.1 / Alg. 2   pass 1: every piece ray-marches its own samples and
 *                       accumulates per-pixel power moments of the warped
 *                       depth, b_j += absorbance * z^j (j = 0..4);
 *   Sec. 4.1            the per-piece moment images are summed
 *                       (the paper's MPI_Allreduce add);
 *   Sec. 4.2 / Alg. 3   pass 2: every piece re-marches its samples, gets the
 *                       transmittance T(z) from the summed moments (Hankel /
 *                       Cholesky moment bound with bias) and adds
 *                       T * alpha * (r, g, b, 1);
 *   Sec. 4.2, 4.3       the colour images are summed (MPI_Reduce add) and
 *                       renormalised so that total opacity = 1 - e^-b0.
 * On one GPU all pieces live on the device; both reductions are on-device.
 *
 * Conventions shared by every entry point
 *   - Every function returns an mboit_status; MBOIT_OK = 0.  On failure
 *     mboit_last_error() returns a message (thread-local, valid until the
 *     next call on the same thread).  Arguments are validated before any
 *     work is enqueued; nothing is enqueued when a call fails validation.
 *   - "device" pointers are CUDA global-memory addresses on the volume's
 *     device; "host" pointers are ordinary CPU memory.  The library never
 *     frees memory it did not allocate.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Render calls are asynchronous on that stream; errors raised
 *     inside kernels (a wait limit or an index check) are reported by
 *     mboit_synchronize().  One volume serves one stream at a time: a
 *     render call (passes, frame, host frame, multi-volume frame, sort-last,
 *     autotuner)
 *     on another stream while work of the volume's previous call may still
 *     run returns MBOIT_ERR_STATE and enqueues nothing (an event recorded
 *     after each call's work tells; calls made while a stream is being
 *     captured into a graph are not tracked).  Calls from several host
 *     threads on one volume are serialised by its lock.
 *   - Images are row-major, pixel index y * width + x, x to the right.
 *   - Moment images: per (view[, piece]) one slab, P = width * height rounded
 *     up to a multiple of 4.  Power moments: b0 as P float32, then (b1, b2,
 *     b3, b4) as P float4 (20 * P bytes); with 6 power moments then (b5, b6)
 *     as P float2 (28 * P bytes), with 8 then (b5, .., b8) as P float4
 *     (36 * P bytes).  Trigonometric moments: b0 as P
 *     float32, then for j = 1..n a plane of P 16-bit pairs (Re, Im of
 *     t_j / b0) ((4 + 4 n) * P bytes).  mboit_moment_image_bytes() gives the
 *     slab size.
 *   - Colour images: float32 RGBA [height][width][4] per (view[, piece]),
 *     premultiplied (sum of T * alpha * (r, g, b) and sum of T * alpha).
 */
#ifndef MBOIT_H
#define MBOIT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MBOIT_API __attribute__((visibility("default")))
#else
#define MBOIT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBOIT_OK = 0,
    MBOIT_ERR_INVALID_ARG = 1,
    MBOIT_ERR_OUT_OF_MEMORY = 2,
    MBOIT_ERR_CUDA = 3,
    MBOIT_ERR_UNSUPPORTED = 4,
    MBOIT_ERR_STATE = 5,
    MBOIT_ERR_TIMEOUT = 6,
    MBOIT_ERR_DEVICE_ASSERT = 7
} mboit_status;

typedef enum { MBOIT_GRID = 0, MBOIT_AMR = 1, MBOIT_TET = 2 } mboit_volume_kind;
/* Moment sets (Sec. 4.3, Fig. 3): 4, 6 or 8 power moments of the warped depth
 * z (Alg. 2: b_j = sum a z^j; Alg. 3 with a 3x3, 4x4 or 5x5 Hankel matrix), or
 * 3 / 4 complex trigonometric moments ("6 / 8 trigonometric moments") of the
 * angle phi = z (1 - 0.1) pi (a wrapping zone of 0.2 pi separates far from
 * near).  The 6- and 8-moment sets mix the normalised moments with those of
 * the arcsine law on [-1, 1] (b_2k = C(2k, k) / 4^k, odd moments 0) and need
 * moment_bias > 0. */
typedef enum {
    MBOIT_POWER4 = 0,
    MBOIT_TRIG6 = 1,
    MBOIT_TRIG8 = 2,
    MBOIT_POWER6 = 3,
    MBOIT_POWER8 = 4
} mboit_moment_set;
/* Moment storage: power moments in float32; trigonometric moments normalised
 * by b0 (kept in float32) in float16 or bfloat16 (nearest-even rounding). */
typedef enum { MBOIT_STORE_F32 = 0, MBOIT_STORE_F16 = 1, MBOIT_STORE_BF16 = 2 } mboit_storage;
typedef enum { MBOIT_ORTHO = 0, MBOIT_PERSPECTIVE = 1 } mboit_projection;
/* Ray packet of one warp (32 rays): 8 x 4 or 4 x 8 neighbouring pixels. */
typedef enum { MBOIT_PACKET_8X4 = 0, MBOIT_PACKET_4X8 = 1 } mboit_packet;

/* pass-1 output layout */
typedef enum {
    MBOIT_MOMENTS_PER_PIECE = 0, /* one slab per (view, selected piece): the per-rank local images */
    MBOIT_MOMENTS_REDUCED = 1    /* one slab per view: pieces summed on the fly */
} mboit_moment_out;

/* pass-2 output layout */
typedef enum {
    MBOIT_COLOR_PER_PIECE = 0, /* one RGBA image per (view, selected piece): the per-rank partials */
    MBOIT_COLOR_REDUCED = 1,   /* one RGBA image per view: partials summed on the fly */
    MBOIT_COLOR_RESOLVED = 2   /* one RGBA image per view, summed and renormalised (final image) */
} mboit_color_out;

typedef enum {
    MBOIT_OP_MOMENTS_SUM = 0,      /* n_inputs moment slabs per view -> one (the Allreduce add) */
    MBOIT_OP_COLOR_SUM_RESOLVE = 1 /* n_inputs colour images per view -> final RGBA (the Reduce add) */
} mboit_composite_op;

/* volume flags */
#define MBOIT_FLAG_RAW_SUM 0x1u       /* resolve without renormalisation: out = sum T*alpha*(c, 1) */
#define MBOIT_FLAG_DETERMINISTIC 0x2u /* accepted; every path here is run-to-run deterministic */
/* Octrees only: adaptive dyadic step.  A lattice point k in a leaf of level L
 * is sampled only if k is a multiple of 2^(max_level - L), and that sample's
 * absorbance covers the longer interval (sigma * step * 2^(max_level - L)):
 * coarse leaves are sampled at their own resolution on a nested lattice, so
 * pieces still partition the samples and their moments still add up. */
#define MBOIT_FLAG_ADAPTIVE_STEP 0x4u
/* Every pixel's reconstruction frame (four power moments) set up in FP64,
 * as the paper's reading of Alg. 3 does in double precision; without it
 * the set-up is float-float FP32 and only near-singular Hankel matrices
 * take FP64 (mboit_stats.fp64_pixels counts them).  For comparison: both
 * give the same images to float32 rounding. */
#define MBOIT_FLAG_FP64_SETUP 0x8u

typedef struct mboit_volume_s* mboit_volume;

typedef struct {
    int32_t kind;               /* mboit_volume_kind */
    int32_t moment_set;         /* mboit_moment_set */
    int32_t storage;            /* mboit_storage */
    uint32_t flags;             /* MBOIT_FLAG_* */
    /* regular grid: float32 vertex values field[z][y][x] (device pointer,
     * BORROWED: it must stay valid and unchanged while the volume renders).
     * Vertex (x, y, z) sits at point (x, y, z); the domain is
     * [0, nx-1] x [0, ny-1] x [0, nz-1]; cells are half-open unit cubes. */
    const float* field;
    int32_t dims[3];            /* nx, ny, nz >= 2 */
    int32_t brick_log2;         /* bricks are cubes of 2^brick_log2 cells (0..7) */
    /* transfer function: 256 entries of (r, g, b, alpha) float32, HOST
     * pointer, COPIED.  alpha in [0, 1) is the opacity of one voxel of
     * material; the value range [tf_range[0], tf_range[1]] maps linearly onto
     * the table, values outside are clamped. */
    const float* tf_rgba;
    float tf_range[2];
    float step;                 /* sample spacing in voxels, a power of two (Sec. 5.3: fixed step);
                                 * lattice point k sits at t = (k + 1/2) step from the eye, and only
                                 * k < 2^22 is sampled (t exact in float32) */
    float moment_bias;          /* mix amount of the bias vector (Alg. 3 "mix"), in [0, 1); for
                                 * trigonometric moments the mix is with the uniform measure and
                                 * must be >= 2e-3 (float16) / 2e-2 (bfloat16); 6 and 8 power
                                 * moments need it > 0 */
    float overestimation;       /* weight of the sample's own depth (Alg. 3), paper: 0.3 */
    float absorbance_max;       /* ABSORBANCE_MAX_VALUE of Alg. 2, > 0 */
    /* MBOIT_AMR (brick octree) only; `field` is then unused.  dims = finest
     * cells per axis + 1 (the domain is [0, dims-1] in finest-cell units, all
     * three equal); brick_log2 = log2 of a leaf's cells per side.  Leaf i of
     * level L covers origin_i + [0, 2^(brick_log2 + max_level - L)) per axis
     * and stores nv = 2^brick_log2 + 1 vertex values per side at its own
     * resolution.  Leaves must not overlap; origins are multiples of
     * 2^brick_log2.  Pieces are lists of leaf ids. */
    const float* leaf_values;   /* DEVICE float32 [n_leaves][nv][nv][nv] ([z][y][x]), borrowed */
    const int32_t* leaf_table;  /* HOST int32 [n_leaves][4]: origin x, y, z (finest cells), level; copied */
    int32_t n_leaves;
    int32_t max_level;          /* 0..10 */
    /* MBOIT_TET (tetrahedral mesh, Sec. 5's unstructured pieces) only;
     * field, dims and brick_log2 are then unused.  The mesh must be a
     * conforming tetrahedralisation lying in the box [0, tet_box] (the
     * sampled domain is [0, tet_box) per axis).  Point location is exact:
     * vertex and sample positions snap to multiples of 2^-quantum_log2
     * (nearest-even), and a snapped point q belongs to the one tet that
     * contains q + (e, e^2, e^3) for an infinitesimal e > 0, so faces, edges
     * and vertices are owned exactly once.  A sample takes the linear
     * (barycentric) interpolation of its tet's four vertex values.  Pieces
     * are lists of tet ids.  Checked: ids in range, every tet positively
     * oriented after snapping, vertices inside the box, neighbours
     * reciprocal, and the snapped coordinates small enough for exact 64-bit
     * predicates (6 E^2 Q < 2^62 with E the largest tet extent and Q the box,
     * both in quanta). */
    const float* tet_verts;     /* HOST float32 [n_verts][4]: x, y, z, value; copied */
    const int32_t* tet_cells;   /* HOST int32 [n_tets][4]: vertex ids; copied */
    const int32_t* tet_neighbors; /* HOST int32 [n_tets][4]: the tet across the face opposite corner i,
                                   * -1 on the boundary; copied */
    int64_t n_verts;
    int64_t n_tets;             /* 1 .. 2^31 - 1 */
    float tet_box[3];
    int32_t quantum_log2;       /* 0 .. 24; 2^quantum_log2 * tet_box < 2^30 */
} mboit_volume_desc;

typedef struct {
    float eye[3];               /* ortho: centre of the view window; perspective: eye point */
    float u[3], v[3], w[3];     /* right, up, forward (w need not be unit for ortho: ray direction = w) */
    int32_t width, height;
    int32_t projection;         /* mboit_projection */
    int32_t reserved;
    /* ortho: window extents along u and v; perspective: tan(fov/2)*aspect and tan(fov/2) */
    float scale_u, scale_v;
    /* the log-depth warp maps ray parameter t in [near, far] to [-1, 1]
     * (Alg. 2 logDepthWarp); must bracket the volume, 0 < near < far */
    float near, far;
} mboit_view;

typedef struct {
    int64_t samples_pass1;      /* owned samples marched by the last render_moments */
    int64_t samples_pass2;      /* owned samples marched by the last reconstruct_blend */
    int64_t singular_pixels;    /* pixels of the last pass 2 whose Hankel matrix took a 1- or 2-atom branch */
    int32_t n_pieces;
    int32_t device;
    int32_t tuning_pass1;       /* window configuration of the fused passes (see mboit_set_tuning) */
    int32_t tuning_pass2;
    int64_t sortlast_segments;  /* segments of the last mboit_render_sortlast */
    int32_t sortlast_max_segments; /* most segments on one pixel in it */
    int32_t fp64_pixels;        /* pixels of the last pass 2 whose reconstruction frame (four power moments) was
                                 * set up in FP64: a variance or Schur complement of the biased Hankel matrix
                                 * within 1e-4 of b2 or b4 (near-singular); every other pixel is set up in
                                 * float-float FP32 arithmetic */
    float frame_pass1_ms;       /* device time of pass 1 in the last mboit_render_frame (CUDA events
                                 * recorded in its graph); -1 before the first frame */
    float frame_pass2_ms;       /* the same for pass 2 */
    int32_t packet;             /* mboit_packet in use (see mboit_set_packet) */
    int32_t frame_launches;     /* kernel launches of mboit_render_frame (see mboit_set_frame_launches);
                                 * with 1, frame_pass1_ms is that launch and frame_pass2_ms about 0 */
    int32_t tile_order;         /* 1: frames dequeue ray tiles longest first (see mboit_set_tile_order) */
    int32_t reserved;
} mboit_stats;

/* Number of window configurations of the fused passes.  Each fused kernel
 * stages, per warp, the block of the field its 32 rays traverse over the
 * next S lattice steps in shared memory; configurations differ in block
 * shape, S and load width.  All give bit-identical results. */
#define MBOIT_NUM_TUNINGS 7

/* Message of the last failing call on this thread ("" if none). */
MBOIT_API const char* mboit_last_error(void);

/* Bytes of one moment slab for a width x height image (P = w*h rounded up to
 * 4): 20 P, 28 P or 36 P for 4, 6 or 8 power moments (float32), (4 + 4 n) P
 * for n complex trigonometric moments (16-bit); 0 for an invalid pair. */
MBOIT_API size_t mboit_moment_image_bytes(int32_t width, int32_t height, int32_t moment_set, int32_t storage);

/* Mixed unstructured cells (Sec. 5: the FUN3D pieces hold tetrahedra,
 * pyramids and prisms) as the tetrahedral mesh MBOIT_TET volumes take.  All
 * pointers are HOST memory; nothing is kept.
 *   verts [n_verts][4]: x, y, z, value (as tet_verts);
 *   cells [n_cells][6]: vertex ids, padded with -1; cell_types[i] = 4 (tet),
 *     5 (pyramid: base quad in cyclic order, then the apex) or 6 (prism:
 *     bottom triangle, then the top triangle with vertex j + 3 above j).
 * Every quad face is cut along its diagonal through the smallest vertex id,
 * so cells that share a face cut it alike (a conforming mesh); a pyramid
 * gives 2 tets, a prism 3.  Each tet is oriented positively on the vertices
 * snapped to 2^-quantum_log2 (its last two vertices swapped if needed).
 * Outputs: tets_out [max_tets][4] and neighbors_out [max_tets][4] (the tet
 * across the face opposite vertex i, -1 on the boundary: ready for
 * tet_cells / tet_neighbors), cell_of_tet [max_tets] (for piece ids), and
 * *n_tets.  At most 3 tets per cell.  INVALID_ARG for a bad id or type, a
 * flat tet, a face shared by more than two tets, or max_tets too small. */
MBOIT_API mboit_status mboit_split_cells(const float* verts, int64_t n_verts, const int32_t* cells,
                                         const int32_t* cell_types, int64_t n_cells, int32_t quantum_log2,
                                         int32_t* tets_out, int32_t* neighbors_out, int64_t* cell_of_tet,
                                         int64_t max_tets, int64_t* n_tets);

/* Creates a volume on the current CUDA device.  Validates the descriptor,
 * copies the transfer function (converted to extinction sigma = -ln(1-alpha)
 * per voxel), allocates the brick-ownership table.  The field stays
 * borrowed.  *out is set only on success. */
MBOIT_API mboit_status mboit_create_volume(const mboit_volume_desc* desc, mboit_volume* out);

/* Releases everything the volume owns (not the field).  NULL is a no-op.
 * Synchronises the volume's device first. */
MBOIT_API mboit_status mboit_destroy_volume(mboit_volume v);

/* Adds one piece: `ids` lists brick ids ((bz*nby + by)*nbx + bx) of the
 * piece (leaf ids of an octree, tet ids of a mesh); copied.  `ids_on_device` = 1 if ids is a device pointer.  Pieces
 * must not overlap (Sec. 6: reconstruction requires non-overlapping
 * volumes); a brick already owned -> MBOIT_ERR_INVALID_ARG and the volume is
 * unchanged.  Piece ids are 0, 1, ... in call order.  Bricks that belong to
 * no piece are never sampled.  Synchronous. */
MBOIT_API mboit_status mboit_add_piece(mboit_volume v, const int32_t* ids, int64_t n, int32_t ids_on_device,
                             int32_t* piece_id_out);

/* Pass 1 (Sec. 4.1, Alg. 2).  views: HOST array of n_views views.  pieces:
 * HOST array of n_pieces selected piece ids, or NULL = all pieces (then
 * n_pieces is ignored).  moments: DEVICE buffer of n_views * S bytes
 * (REDUCED) or n_views * n_pieces * S bytes (PER_PIECE), S =
 * mboit_moment_image_bytes(); fully overwritten. */
MBOIT_API mboit_status mboit_render_moments(mboit_volume v, const mboit_view* views, int32_t n_views,
                                  const int32_t* pieces, int32_t n_pieces, int32_t mode, void* moments,
                                  void* stream);

/* Pass 2 (Sec. 4.2, Alg. 1 loop 2, Alg. 3).  global_moments: DEVICE
 * buffer of n_views REDUCED slabs (the summed moments of ALL pieces).
 * color: DEVICE float32 RGBA, n_views (REDUCED, RESOLVED) or n_views *
 * n_pieces (PER_PIECE) images; fully overwritten.  RESOLVED applies the
 * renormalisation of mboit_composite with a zero background. */
MBOIT_API mboit_status mboit_reconstruct_blend(mboit_volume v, const mboit_view* views, int32_t n_views,
                                     const int32_t* pieces, int32_t n_pieces, const void* global_moments,
                                     int32_t mode, float* color, void* stream);

/* Image-space reductions (the paper's Allreduce add and Reduce add).
 *   MOMENTS_SUM: in = n_views * n_inputs moment slabs of width x height,
 *     out = n_views slabs; compensated (Neumaier) float32 sum in input order.
 *   COLOR_SUM_RESOLVE: in = n_views * n_inputs RGBA images; out = n_views RGBA
 *     images: C = sum of inputs (compensated); alpha = 1 - e^-b0 from
 *     global_moments; rgb = C.rgb * alpha / C.a (0 if C.a = 0); then
 *     out += e^-b0 * bg.  With MBOIT_FLAG_RAW_SUM on the volume, out = C
 *     (the plain sum of Alg. 1) and global_moments may be NULL.
 * All buffers are DEVICE pointers; bg is a HOST float[4] or NULL (zero). */
MBOIT_API mboit_status mboit_composite(mboit_volume v, int32_t op, int32_t width, int32_t height, int32_t n_views,
                             int32_t n_inputs, const void* in, void* out, const void* global_moments,
                             const float* bg, void* stream);

/* Whole frame, batched: pass 1 (REDUCED) -> pass 2 (RESOLVED) for all pieces
 * and all views, recorded once into a CUDA graph per (views, stream kind)
 * and replayed.  moments_scratch: DEVICE buffer of n_views moment slabs
 * (kept, so the caller can inspect the global moments); rgba: DEVICE
 * float32 RGBA n_views images.  Pass 1 also stores every lattice point's
 * sample value in a library-owned cache (4 bytes per lattice point inside
 * the domain, sized exactly when a graph is recorded, e.g. 6.4 GB for 1.6 G
 * points) and pass 2 reads it instead of sampling the volume again (the
 * same values: images are bit-identical to the separate pass calls).  If
 * the device lacks that memory with 1 GiB to spare, pass 2 samples again
 * (so does every ray tile past the row count in the environment variable
 * MBOIT_FRAME_CACHE_ROWS, read when a graph is recorded, if it is set).
 * The first call for a set of views synchronises once to size the cache.
 * The frame runs as one kernel launch (each warp takes its ray tile through
 * pass 1 and then pass 2) or as two (see mboit_set_frame_launches); both
 * give the same bits. */
MBOIT_API mboit_status mboit_render_frame(mboit_volume v, const mboit_view* views, int32_t n_views, void* moments_scratch,
                                float* rgba, void* stream);

/* Whole frame over several volumes at once (the batching pattern of Sec. 4
 * applied across independent volumes): one persistent launch per pass takes
 * the ray tiles of every view, and view i samples volume
 * vols[view_volume[i]].  The volumes are all MBOIT_GRID or all MBOIT_AMR
 * (fixed step), with MBOIT_POWER4 and MBOIT_STORE_F32 (another kind, set,
 * storage or the adaptive step: MBOIT_ERR_UNSUPPORTED; kinds mixed:
 * MBOIT_ERR_INVALID_ARG), on one device, listed once, and share one transfer
 * function and sampling step (else MBOIT_ERR_INVALID_ARG); fields, domains,
 * moment bias, overestimation and flags stay each volume's own.
 * 1 <= n_vols <= 8, 1 <= n_views <= 16.  moments_scratch and rgba are laid
 * out as for mboit_render_frame over the n_views views; every image equals,
 * bit for bit, its volume's own mboit_render_frame.  Pass 1 stores the
 * sample cache of vols[0] (sized for all views; synchronises once per call
 * to size it) and pass 2 blends from it; grid windows take configuration 3
 * when every field qualifies (dims[0] % 4, alignment), else 0; octrees have
 * their tables checked first, each into its own error word
 * (mboit_synchronize on that volume reports a failure; that volume's tiles
 * are skipped).  Counters (mboit_get_stats) land in vols[0].  Two launches
 * on `stream`, not captured into a graph; takes every volume's lock.  The
 * paper has no counterpart (its pieces are one volume's). */
MBOIT_API mboit_status mboit_render_frame_multi(const mboit_volume* vols, int32_t n_vols, const mboit_view* views,
                                                const int32_t* view_volume, int32_t n_views, void* moments_scratch,
                                                float* rgba, void* stream);

/* End-to-end frame from HOST memory: copies `field_host` (nx*ny*nz
 * float32 for a grid, the leaf values for an octree, n_verts vertex values
 * for a tet mesh; preferably pinned) into the volume's device values,
 * renders the frame as mboit_render_frame, and copies the RGBA images to
 * `rgba_host` (n_views * width * height * 4 float32).  Returns after the
 * image has arrived on the host. */
MBOIT_API mboit_status mboit_render_frame_host(mboit_volume v, const float* field_host, const mboit_view* views,
                                     int32_t n_views, void* moments_scratch, float* rgba_device,
                                     float* rgba_host, void* stream);

/* Waits for `stream` and reports kernel-side errors recorded by this
 * volume's launches since the last call: MBOIT_ERR_DEVICE_ASSERT when a
 * table check found an entry out of range (an octree finest-brick map entry
 * that is no leaf id, a mesh face neighbour or bin-list entry that is no tet
 * id, a mesh bin range outside the bin list).  Every render of an octree or
 * mesh first runs these checks over the whole tables on its stream (a few
 * microseconds to tens of microseconds); when one fails, the passes launched
 * after it return at entry, so no out-of-range index is ever used and the
 * images of that render are not valid.  The error word is cleared when
 * reported.  MBOIT_ERR_TIMEOUT (reported first when both apply) when a
 * grid kernel's TMA window load (tuning configurations 5, 6) did not complete
 * within its wait limit, about a second: the warp that gave up waits once
 * more, bounded, for the copy in flight and stops, so the images of that
 * render are not valid.  The paper has no counterpart. */
MBOIT_API mboit_status mboit_synchronize(mboit_volume v, void* stream);

/* Test hook of the failure detection above; the paper has no counterpart.
 * Overwrites a table the library owns, after the volume was validated:
 * what = 1 (octree) sets every finest-brick map entry to a value that is no
 * leaf id; what = 2 (mesh) sets every tet's neighbour
 * across face 0 to a value that is no tet id; renders then report
 * MBOIT_ERR_DEVICE_ASSERT from mboit_synchronize.  what = 3 (grid) makes
 * every TMA window load (tuning configurations 5, 6) arm its barrier without
 * issuing the copy, so each wait runs to its limit (a completion that
 * nothing delivers; no copy is left in flight); renders with configuration
 * 5 then report MBOIT_ERR_TIMEOUT.  The volume stays corrupt (destroy it
 * afterwards).  MBOIT_ERR_INVALID_ARG for another kind or `what`.
 * Synchronous. */
MBOIT_API mboit_status mboit_debug_corrupt(mboit_volume v, int32_t what);

/* Counters of the last passes (synchronises the stream of the last render). */
MBOIT_API mboit_status mboit_get_stats(mboit_volume v, mboit_stats* out);

/* GPU exact sort-last baseline (the segment-layer compositor the paper
 * compares against, Sec. 5; no moments, exact front-to-back result).  Every
 * piece turns each maximal run of consecutive lattice points it owns into
 * one segment (premultiplied colour and opacity of the run, keyed by its
 * first lattice index); per pixel the segments of all pieces are sorted by
 * key and composited with "over".  rgba: DEVICE float32 RGBA, n_views
 * images (premultiplied colour, alpha = 1 - transmittance, no background).
 * segments_per_pixel: DEVICE int32 [pixels of all views] or NULL (the
 * segment-density image).  Uses library-owned buffers that grow to the
 * largest frame seen; synchronises `stream` once (to size the segment
 * buffer), so it cannot be captured into a graph. */
MBOIT_API mboit_status mboit_render_sortlast(mboit_volume v, const mboit_view* views, int32_t n_views, float* rgba,
                                             int32_t* segments_per_pixel, void* stream);

/* Selects the window configuration (0 .. MBOIT_NUM_TUNINGS-1) of the fused
 * pass 1 and pass 2.  Configurations 2-6 read 16-byte chunks and need
 * dims[0] % 4 == 0 and a 16-byte aligned field; configurations 5 and 6 fill
 * pass 1's window by one TMA tensor copy per warp (cp.async.bulk.tensor.3d
 * from the field's tensor map, completed on an mbarrier; pass 2 takes
 * configuration 3): 5 with configuration 3's 16 x 8 x 8 floats, 6 with 12 x
 * 11 x 8, whose dense layout spreads shared-memory banks; both also need the
 * driver's tensor-map encoder; otherwise MBOIT_ERR_INVALID_ARG and nothing
 * changes.  Every configuration gives the same bits.  Takes effect for the
 * next call; captured frame graphs are re-recorded. */
MBOIT_API mboit_status mboit_set_tuning(mboit_volume v, int32_t pass1, int32_t pass2);

/* Number of kernel launches of mboit_render_frame: 2 (pass 1, then pass 2
 * over the whole frame) or 1 (Sec. 4.1-4.2 per ray tile: the warp that
 * marched every selected piece of its 32 rays holds their summed moments, so
 * it blends those rays at once, from the sample values it just stored; grid
 * window configuration: pass 1's).  Both give bit-identical images and
 * moments.  Default: 1 for MBOIT_GRID volumes with MBOIT_POWER4, else 2
 * (mboit_autotune times both forms).  1 is for MBOIT_POWER4 volumes (every
 * kind) only, else MBOIT_ERR_UNSUPPORTED; other values MBOIT_ERR_INVALID_ARG.
 * Captured frame graphs are re-recorded. */
MBOIT_API mboit_status mboit_set_frame_launches(mboit_volume v, int32_t launches);

/* Dequeue order of the ray tiles in mboit_render_frame (the batching
 * pattern's cost-ordered work items): 0 = tile order (views in turn, rows
 * of tiles top to bottom), 1 = longest first: when a frame graph is
 * recorded, one small kernel counts each ray tile's lattice rows (the rows
 * its warp walks in lockstep, the tile's cost) and the tiles are sorted by
 * it, so the persistent kernels start the long tiles early and end on
 * short ones.  The order lives with the recorded graph.  Results do not
 * depend on it; mboit_autotune times both.  Other calls keep tile order.
 * MBOIT_ERR_INVALID_ARG for another value.  Captured frame graphs are
 * re-recorded. */
MBOIT_API mboit_status mboit_set_tile_order(mboit_volume v, int32_t order);

/* Selects the ray packet of every pass (mboit_packet).  Results do not
 * depend on it (every ray is marched alone); speed does.  Captured frame
 * graphs are re-recorded. */
MBOIT_API mboit_status mboit_set_packet(mboit_volume v, int32_t packet);

/* Autotuner (the batching pattern's tuner): for each ray packet, times every
 * eligible window configuration of pass 1 and of pass 2 on these views (3
 * launches each, CUDA events on `stream`, after one warm launch) and takes
 * the fastest of each.  For volumes with four power moments it then times,
 * on the same packet and with the frame's sample cache, the frame in those
 * two launches against one launch (mboit_set_frame_launches) in each
 * eligible configuration, and keeps the packet and form of the fastest
 * frame (in one launch, the configuration found there is pass 1's); for
 * other moment sets, the packet with the smallest sum of its pass-1 and
 * pass-2 times; with four power moments it also times the fastest frame
 * with its ray tiles dequeued longest first (mboit_set_tile_order).  Writes
 * pass 1's, pass 2's configuration and the packet to chosen[0..2] (HOST,
 * may be NULL); the form and the order are in mboit_stats.frame_launches and
 * tile_order.  The buffers are as for mboit_render_frame and are
 * overwritten.  Synchronous.  The choice is kept for the process, keyed by
 * the volume's configuration (kind, shape, brick size, sampling step, moment
 * set and storage, flags, leaf / tet / piece counts, the window
 * configurations it can take), the views and the device's SM count: a later
 * call with the same key, for this or another volume, takes it without
 * timing anything (mboit_clear_tuning_cache forgets every choice). */
MBOIT_API mboit_status mboit_autotune(mboit_volume v, const mboit_view* views, int32_t n_views, void* moments_scratch,
                                      float* rgba, void* stream, int32_t* chosen);

/* Forgets the autotuner's kept choices (the next mboit_autotune times again).
 * Volumes keep the tuning they have. */
MBOIT_API void mboit_clear_tuning_cache(void);

/* Pass 1 for callers that must not allocate device memory.  The paper has
 * no counterpart; it serves embedders such as an in-situ adaptor linked into
 * a simulation whose memory pool owns the whole device, a plugin whose host
 * application forbids side allocations, or a latency-critical loop that
 * cannot afford the implicit synchronisation a cudaMalloc/cudaFree may
 * cause.  Every other entry point needs a volume, and creating one
 * allocates.
 *
 * Computes exactly what mboit_render_moments(MBOIT_MOMENTS_REDUCED) computes
 * for a volume described by `desc` whose selected bricks are those with
 * brick_selected[b] != 0 (HOST array of nbx*nby*nbz bytes; NULL = every
 * brick), with no volume object.  The caller passes everything else: desc
 * (field DEVICE pointer, borrowed; transfer function HOST pointer, read
 * during the call), views (HOST), moments (DEVICE, n_views REDUCED slabs).
 *
 * Its scratch (work-queue head and counters, the converted transfer
 * function, the brick mask) lives in one fixed device array of
 * 256 + 4096 + 1,048,576 bytes inside the library, which every device that
 * loads the library keeps until the process exits.  Limit: at most
 * 1,048,576 bricks (MBOIT_ERR_INVALID_ARG beyond).  The call makes no
 * cudaMalloc, cudaFree or other allocating call.  Every call looks up the
 * array's device address in the current context (a lookup, so a context
 * re-created after cudaDeviceReset gets its own copy); the first call on a
 * device also loads the library's kernels there (set-up) and should come
 * before any stream capture on that device.  The transfer function travels
 * by value in a kernel argument, so the caller's table is free once the
 * call returns.  The brick mask is copied from the caller's memory by a
 * copy on `stream`: pinned memory is read when that copy runs and must stay
 * unchanged until then.  All calls share the array: calls whose work
 * overlaps on the GPU (two streams, or two host threads) race and give
 * wrong results; order them on one stream.  Argument checks are those of
 * mboit_create_volume for a grid (MBOIT_ERR_INVALID_ARG). */
MBOIT_API mboit_status mboit_render_moments_noalloc(const mboit_volume_desc* desc, const uint8_t* brick_selected,
                                                    const mboit_view* views, int32_t n_views, void* moments,
                                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif
