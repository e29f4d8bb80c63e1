// Internal launch interface between the C ABI (mboit_api.cu) and the
// kernels (mboit_grid.cu, mboit_units.cu, mboit_kernels.cu).  Not part of
// the public ABI.
#pragma once
#include <cuda.h>   // CUtensorMap (the type only; the library calls the driver through the runtime's entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include "mboit_device.cuh"

namespace mb {

constexpr int kMaxViews = 16;

struct ViewSlot {
    ViewD v;
    int32_t tile_base;      // first global tile index of this view
    int32_t ntx;            // tiles per row
    int64_t moment_off;     // byte offset of this view's first moment slab
    int64_t color_off;      // float offset of this view's first RGBA image
    int32_t plane;          // pixels per moment plane (w*h rounded up to 4)
    int32_t tw_log2;        // a warp's ray tile (packet) is 2^tw_log2 x 2^(5 - tw_log2) pixels: 8 x 4 or 4 x 8
    int32_t vol;            // multi-volume frames: the view's volume in the GridTable (else 0)
    int32_t pad;
};

// Pixel of lane `lane` in tile `lt` of a view (tiles row-major, ntx per row).
MB_HD void tile_pixel(const ViewSlot& S, int lt, int lane, int& px, int& py) {
    const int tw = 1 << S.tw_log2;
    px = (lt % S.ntx) * tw + (lane & (tw - 1));
    py = (lt / S.ntx) * (32 >> S.tw_log2) + (lane >> S.tw_log2);
}

struct ViewTable {
    int32_t n;
    int32_t total_tiles;
    // dequeue order: the queue's i-th pop takes tile order[i] (a permutation of
    // the tiles, longest first); NULL: tiles in order (views in turn, rows of
    // tiles top to bottom)
    const int32_t* order;
    ViewSlot s[kMaxViews];
};

// Bits of Counters::error: a kernel found a table entry out of range,
// skipped the access it would have made and went on with a safe substitute.
constexpr int32_t kErrLeafId = 0x2;   // an octree finest-brick map entry is not a leaf id (nor -1)
constexpr int32_t kErrTetId = 0x4;    // a mesh face neighbour or bin-list entry is not a tet id
constexpr int32_t kErrBinRange = 0x8; // a mesh bin's range of the bin list leaves the list
constexpr int32_t kErrTmaTimeout = 0x10;  // a TMA window load did not complete within its wait limit

// Device counters owned by a volume.
struct Counters {
    int32_t tile_next[4];            // work-queue heads, one per concurrent pass
    int32_t error;                   // kErr* bits of the kernel-side checks that failed since the last read
    int32_t pad;
    unsigned long long samples[2];   // pass 1, pass 2
    unsigned long long singular;     // pixels on a 1-/2-atom branch
    unsigned long long segments;     // sort-last segments of the last baseline frame
    int32_t max_segments;            // most segments on one pixel
    int32_t pad2;
    unsigned long long cache_rows;   // rows of the frame's sample cache handed out so far
    unsigned long long fp64_pixels;  // pixels whose reconstruction frame was set up in FP64
};

struct PieceBox {
    float lo[3], hi[3];              // voxel-space box covering the piece's bricks
};

enum ColorMode : int32_t { kColorPerPiece = 0, kColorReduced = 1, kColorResolved = 2 };

// Brick octree (AMR) as the kernels see it.  `g` carries the domain
// [0, hx) x [0, hy) x [0, hz) in finest cells and every sampling and
// transfer-function parameter (its field/brick members are unused).
struct AmrD {
    GridD g;
    const float* values;    // [n_leaves][nv^3] vertex values, [z][y][x]
    const int4* leaves;     // origin x, y, z (finest cells), level
    const float4* leaf_box; // the same origin as floats, and 2^-(max_level - level) = 1 / cell size
    const int32_t* fmap;    // [fdim^3] finest brick (2^brick_log2 cells) -> leaf, -1 none
    int32_t fdim, nv, max_level;
    int32_t complete;       // 1: every finest brick has a leaf (no holes)
    int32_t n_leaves;       // leaf ids are 0 .. n_leaves - 1 (checked where the map is read)
    int32_t pad;
    int32_t* err;           // the volume's Counters::error
};

// Tetrahedral mesh as the kernels see it.  `g` carries the box
// [0, hx) x [0, hy) x [0, hz) and every sampling and transfer-function
// parameter (its field/brick members are unused).  Coordinates are integers
// in quanta of 2^-quantum_log2; a point snaps by nearest-even rounding of
// p * qscale.
struct TetD {
    GridD g;
    const int4* corners;       // per tet its 4 corners (positively oriented): snapped x, y, z and the
                               //   value's float32 bits
    const int4* nbrs;          // per tet: the tet across the face opposite each corner (-1 on the boundary)
    const int32_t* bin_start;  // [nbins + 1]: bins of 2^bin_shift quanta, CSR over
    const int32_t* bin_tets;   //   the tets whose snapped bounding box meets the bin
    int32_t bdim[3];
    int32_t bin_shift;
    float qscale;              // 2^quantum_log2
    int32_t max_walk;          // walk steps before a bin search takes over
    int32_t narrow;            // 1: every tet spans < 2^15 quanta, so face normals fit in 32 bits
    int32_t n_tets;            // tet ids are 0 .. n_tets - 1 (checked before every tet load)
    int32_t n_bin_tets;        // entries of bin_tets (bin ranges are checked against it)
    int32_t pad;
    int32_t* err;              // the volume's Counters::error
};

// The kernels' view of a mesh, with the normal width as a type.
template <bool kNarrow>
struct TetT : TetD {};

// Sample values of one batched frame, shared by its two passes.  A warp's
// 8 x 4 ray tile owns rows kmin..kmax (its lattice indices); row r holds 32
// floats, one per lane, at vals[(tile_base[tile] + r - kmin) * 32 + lane]
// (NaN: not sampled).  Pass 1 takes the tile's rows from ctr->cache_rows and
// stores; pass 2 reads.  A tile that found no room (tile_base -1) is marched
// again in pass 2.  vals NULL: no cache.
struct TileCache {
    float* vals;
    long long* tile_base;
    long long rows_cap;
};

// Number of shared-memory window configurations of the fused passes (the
// autotuner's choices).  Configurations 2-6 use 16-byte loads and need
// nx % 4 == 0 and a 16-byte aligned field; 0 and 1 work everywhere.
// Configurations 5 and 6 fill pass 1's window by a TMA tensor copy (pass 2
// takes configuration 3); they need the field's tensor maps.
constexpr int kNumStageConfigs = 7;
bool stage_config_eligible(const GridD& g, int cfg);

// Loads all kernels and caches launch shapes (call before any capture).
cudaError_t prepare_kernels();
// Fused pass 1 over all selected pieces, REDUCED output.  `brick_sel` NULL
// means every brick is sampled.  An ineligible `cfg` falls back to 0.
cudaError_t launch_pass1_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               void* moments, Counters* ctr, cudaStream_t s, int cfg = 0,
                               TileCache cache = TileCache{}, const CUtensorMap* tmap = nullptr);
// Fused pass 2 over all selected pieces, REDUCED or RESOLVED output.
cudaError_t launch_pass2_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                               int cfg = 0, TileCache cache = TileCache{});
// One-launch frame (four power moments, regular grid): each warp takes its
// ray tile through pass 1 and then pass 2, RESOLVED or REDUCED colour; the
// cache rows are handed out as in the two-launch frame (no room: pass 2
// marches again).  Results equal launch_pass1_fused + launch_pass2_fused.
cudaError_t launch_frame_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s, int cfg,
                               TileCache cache, const CUtensorMap* tmap = nullptr);
// The field's tensor map for TMA windows (dims nx, ny, nz floats, box of
// configuration 5's window); false when the driver offers no encoder or the
// field does not qualify (nx % 4, alignment).
bool encode_field_maps(const GridD& g, CUtensorMap out[2]);
// Several grid volumes in one persistent launch per pass (four power
// moments, one transfer function): view slot i samples volume vt.s[i].vol.
constexpr int kMaxVolumes = 8;
struct GridTable {
    GridD g[kMaxVolumes];
};
// The multi-volume frame's two passes: `vec` selects configuration 3's
// window (every volume has nx % 4 == 0 and a 16-byte aligned field), else
// configuration 0's.  Pass 1 stores the tile cache when cache.vals is set and
// pass 2 then blends from it; results equal each volume's own frame.
cudaError_t launch_pass1_multi(const GridTable& gt, const float4* tf, const ViewTable& vt, void* moments,
                               Counters* ctr, cudaStream_t s, bool vec, TileCache cache);
cudaError_t launch_pass2_multi(const GridTable& gt, const float4* tf, const ViewTable& vt, const void* moments,
                               float* color, Counters* ctr, cudaStream_t s, bool vec, TileCache cache);
cudaError_t prepare_multi_kernels();
// Rows a frame's tile cache needs over the domain box of `g` (sum over the
// ray tiles of kmax - kmin + 1), added to *rows.
// With per_tile set, also writes each tile's row count (its cost: the warp
// walks those rows in lockstep) to per_tile[tile].
cudaError_t launch_tile_rows(const GridD& g, const ViewTable& vt, unsigned long long* rows, cudaStream_t s,
                             int32_t* per_tile = nullptr);
// Plain per-piece passes: one launch = one piece, its own slab.
cudaError_t launch_pass1_piece(const GridD& g, const float4* tf, const int32_t* piece_of_brick, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               void* moments, Counters* ctr, cudaStream_t s);
cudaError_t launch_pass2_piece(const GridD& g, const float4* tf, const int32_t* piece_of_brick, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               const void* moments, float* color, Counters* ctr, cudaStream_t s);
// GPU exact sort-last baseline: per-piece segment count / fill marches,
// offsets (per-pixel totals, exclusive scan, per-(piece, pixel) starts),
// per-pixel sort and blend.  counts/starts: [pixels of all views][n_slots]
// laid out per view as [slot][pixel].
cudaError_t launch_sortlast_march(bool fill, const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s);
cudaError_t launch_sortlast_offsets(const ViewTable& vt, int32_t n_slots, const int32_t* counts, int32_t* totals,
                                   int64_t* base, int64_t* bsum, int64_t* starts, int64_t total_px, cudaStream_t s);
cudaError_t launch_sortlast_blend(const int64_t* base, int32_t* seg_key, float4* seg_col, float* rgba, int64_t total_px,
                                  Counters* ctr, cudaStream_t s);
// Octree versions of the passes (direct gathers; same output layouts).
// `cache` (vals NULL: none): pass 1 stores the frame's samples, pass 2 reads them.
cudaError_t launch_pass1_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, Counters* ctr, cudaStream_t s, TileCache cache = TileCache{});
cudaError_t launch_pass2_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache = TileCache{});
// One-launch frame (four power moments), as launch_frame_fused.
cudaError_t launch_frame_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache);
cudaError_t launch_pass1_piece(const AmrD& a, const float4* tf, const int32_t* piece_of_unit, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               void* moments, Counters* ctr, cudaStream_t s);
cudaError_t launch_pass2_piece(const AmrD& a, const float4* tf, const int32_t* piece_of_unit, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               const void* moments, float* color, Counters* ctr, cudaStream_t s);
cudaError_t launch_sortlast_march(bool fill, const AmrD& a, const float4* tf, const int32_t* piece_of_unit,
                                  int32_t piece, const PieceBox& box, const ViewTable& vt, int32_t slot,
                                  int32_t n_slots, int32_t* counts, const int64_t* starts, int32_t* seg_key,
                                  float4* seg_col, cudaStream_t s);
// Tetrahedral-mesh versions (walks between face neighbours; same layouts).
// `cache` (vals NULL: none): pass 1 stores the frame's samples, pass 2 reads them.
cudaError_t launch_pass1_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, Counters* ctr, cudaStream_t s, TileCache cache = TileCache{});
cudaError_t launch_pass2_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache = TileCache{});
cudaError_t launch_frame_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache);
cudaError_t launch_pass1_piece(const TetD& m, const float4* tf, const int32_t* piece_of_unit, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               void* moments, Counters* ctr, cudaStream_t s);
cudaError_t launch_pass2_piece(const TetD& m, const float4* tf, const int32_t* piece_of_unit, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               const void* moments, float* color, Counters* ctr, cudaStream_t s);
cudaError_t launch_sortlast_march(bool fill, const TetD& m, const float4* tf, const int32_t* piece_of_unit,
                                  int32_t piece, const PieceBox& box, const ViewTable& vt, int32_t slot,
                                  int32_t n_slots, int32_t* counts, const int64_t* starts, int32_t* seg_key,
                                  float4* seg_col, cudaStream_t s);
// Writes vertex values (values[vertex id]) into the .w words of the tets'
// corner records.
cudaError_t launch_tet_values(int4* corners, const int4* cells, int64_t n_tets, const float* values, cudaStream_t s);

// Table checks before a render's passes (failure detection): octree
// finest-brick map entries are leaf ids or -1; mesh face neighbours are tet
// ids or -1, bin offsets are ordered and inside the bin list, bin-list entries
// are tet ids.  A failure sets kErr* bits in the volume's error word, and the
// passes launched after it on the stream return at entry.
cudaError_t launch_check_tables(const AmrD& a, cudaStream_t s);
cudaError_t launch_check_tables(const TetD& m, cudaStream_t s);

// Image-space reductions.
cudaError_t launch_moments_sum(const GridD& g, const ViewTable& vt, int32_t n_inputs, const void* in, void* out,
                               cudaStream_t s);
cudaError_t launch_color_resolve(const ViewTable& vt, int32_t n_inputs, const float* in, float* out,
                                 const void* moments, float4 bg, int32_t raw_sum, cudaStream_t s);

}  // namespace mb
