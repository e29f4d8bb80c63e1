// C ABI of the MBOIT puzzle-piece renderer (see include/mboit.h).
//
// Host side only: argument validation, the volume registry (transfer
// function, brick ownership, piece boxes), view tables, CUDA-graph capture of
// the batched frame, and error reporting.  Every step of the render runs in
// the kernels of mboit_grid.cu, mboit_units.cu and mboit_kernels.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "mboit.h"
#include "mboit_internal.h"
#include "mboit_multi.h"

namespace {

thread_local std::string g_err;

mboit_status fail(mboit_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define MB_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(MBOIT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Makes the volume's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite3(const float* a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

// An NVTX range around an entry point, so that profilers show each call's
// span beside its kernels (no cost without an attached tool).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct GraphEntry {
    std::vector<char> key;
    cudaGraphExec_t exec = nullptr;
    int32_t* d_order = nullptr;   // the graph's tile order (cost-ordered dequeue), or NULL
};

}  // namespace

struct mboit_volume_s {
    int device = 0;
    mboit_volume_desc desc{};
    int32_t kind = MBOIT_GRID;
    mb::GridD grid{};
    mb::AmrD amr{};             // octree volumes: amr.g aliases the sampling parameters
    int4* d_leaves = nullptr;
    float4* d_leaf_box = nullptr;
    int32_t* d_fmap = nullptr;
    std::vector<int32_t> leaf_table;
    mb::TetD tet{};             // tetrahedral meshes: amr-like parameters plus the device tables below
    int4* d_tcorners = nullptr;
    int4* d_tnbrs = nullptr;
    int4* d_tcells = nullptr;
    float* d_tcvals = nullptr;  // tile-row sample cache of the batched frame (grow only)
    long long* d_tile_base = nullptr;
    unsigned long long* d_rows = nullptr;
    size_t cap_tcvals = 0, cap_tile_base = 0;
    int32_t* d_bin_start = nullptr;
    int32_t* d_bin_tets = nullptr;
    float* d_tvals = nullptr;   // staging of host vertex values (mboit_render_frame_host)
    std::vector<int32_t> tet_cells;
    std::vector<float> tet_xyz;
    int64_t nbricks = 0;
    size_t field_bytes = 0;
    float4* d_tf = nullptr;
    std::vector<float4> tf_host;   // the converted table as uploaded (multi-volume frames compare them)
    int32_t* d_pob = nullptr;
    uint8_t* d_sel = nullptr;
    mb::Counters* d_ctr = nullptr;
    std::vector<int32_t> pob;
    std::vector<mb::PieceBox> boxes;
    int64_t owned = 0;
    std::vector<uint8_t> sel_host;
    bool sel_uploaded = false;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t frame_ev[3] = {nullptr, nullptr, nullptr};  // recorded around the passes of every frame graph
    bool frame_timed = false;
    std::vector<GraphEntry> graphs;
    int32_t tune1 = 0, tune2 = 0;
    CUtensorMap field_map[2];   // grids: the field's tensor maps for TMA windows (configurations 5 and 6)
    bool has_field_map = false;
    int32_t packet = MBOIT_PACKET_8X4;
    int32_t tile_order = 0;     // 1: frames dequeue their ray tiles longest first (mboit_set_tile_order)
    // one volume, one stream at a time: the stream of the last call that
    // launched work and an event recorded after that work
    cudaEvent_t done_ev = nullptr;
    cudaStream_t last_stream = nullptr;
    bool done_recorded = false;
    int32_t frame_launches = 2;  // 1: one launch per frame (four power moments)
    // sort-last baseline buffers (grow only)
    int32_t* sl_counts = nullptr;
    int64_t* sl_starts = nullptr;
    int32_t* sl_totals = nullptr;
    int64_t* sl_base = nullptr;
    int64_t* sl_bsum = nullptr;
    int32_t* sl_key = nullptr;
    float4* sl_col = nullptr;
    size_t cap_counts = 0, cap_starts = 0, cap_totals = 0, cap_base = 0, cap_bsum = 0, cap_seg = 0, cap_col = 0;
    int64_t sl_segments = 0;
    std::mutex mu;
};

namespace {

constexpr double kTrigZone = 0.1;  // wrapping zone: phi = z (1 - zeta) pi

// Angle map and the coefficients of s^m in (s + i)^k (s - i)^(n-k).
void fill_trig(mb::TrigTables& T, int32_t moment_set, int32_t storage, float beta) {
    std::memset(&T, 0, sizeof T);
    T.n = moment_set == MBOIT_TRIG6 ? 3 : moment_set == MBOIT_TRIG8 ? 4 : 0;
    T.sel = T.n ? T.n : moment_set == MBOIT_POWER6 ? 6 : moment_set == MBOIT_POWER8 ? 8 : 0;
    T.storage = storage;
    T.beta = beta;
    T.zone_scale = (float)((1.0 - kTrigZone) * 3.14159265358979323846);
    for (int k = 0; k <= T.n; ++k) {
        double cr[6] = {1, 0, 0, 0, 0, 0}, ci[6] = {0, 0, 0, 0, 0, 0};
        for (int f = 0; f < T.n; ++f) {
            const double rim = f < k ? 1.0 : -1.0;  // factor (s + i) or (s - i)
            double nr[6] = {0, 0, 0, 0, 0, 0}, ni[6] = {0, 0, 0, 0, 0, 0};
            for (int m = 0; m <= f; ++m) {
                nr[m + 1] += cr[m];
                ni[m + 1] += ci[m];
                nr[m] += -ci[m] * rim;  // c * (i * rim)
                ni[m] += cr[m] * rim;
            }
            for (int m = 0; m <= f + 1; ++m) {
                cr[m] = nr[m];
                ci[m] = ni[m];
            }
        }
        for (int m = 0; m <= T.n; ++m) {
            T.er[k][m] = (float)cr[m];
            T.ei[k][m] = (float)ci[m];
        }
    }
}

bool is_trig(int32_t moment_set) { return moment_set == MBOIT_TRIG6 || moment_set == MBOIT_TRIG8; }

// Scalar sampling parameters every volume kind shares (tf_range, step,
// moment_bias, overestimation, absorbance_max): checked the same way by
// mboit_create_volume and mboit_render_moments_noalloc.
mboit_status check_sampling(const mboit_volume_desc* d) {
    if (!d->tf_rgba) return fail(MBOIT_ERR_INVALID_ARG, "tf_rgba is NULL");
    if (!std::isfinite(d->tf_range[0]) || !std::isfinite(d->tf_range[1]) || !(d->tf_range[1] > d->tf_range[0]))
        return fail(MBOIT_ERR_INVALID_ARG, "tf_range must be finite with tf_range[1] > tf_range[0]");
    int ex = 0;
    if (!(d->step > 0.0f) || !std::isfinite(d->step) || std::frexp(d->step, &ex) != 0.5f)
        return fail(MBOIT_ERR_INVALID_ARG, "step must be a positive power of two");
    if (!(d->moment_bias >= 0.0f && d->moment_bias < 1.0f)) return fail(MBOIT_ERR_INVALID_ARG, "moment_bias must be in [0, 1)");
    if (!(d->overestimation >= 0.0f && d->overestimation <= 1.0f))
        return fail(MBOIT_ERR_INVALID_ARG, "overestimation must be in [0, 1]");
    if (!(d->absorbance_max > 0.0f) || !std::isfinite(d->absorbance_max))
        return fail(MBOIT_ERR_INVALID_ARG, "absorbance_max must be positive");
    return MBOIT_OK;
}

// The 256 transfer-function entries as the kernels read them: (r, g, b,
// absorbance of one sample = sigma * step) with sigma = -ln(1 - alpha) per
// voxel (Alg. 2: absorbance = -log of the sample's transmittance).
mboit_status convert_tf(const mboit_volume_desc* d, float4* tf) {
    for (int j = 0; j < 256; ++j) {
        const float* e = d->tf_rgba + 4 * j;
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(e[c])) return fail(MBOIT_ERR_INVALID_ARG, "non-finite transfer-function entry");
        if (!(e[3] >= 0.0f && e[3] < 1.0f)) return fail(MBOIT_ERR_INVALID_ARG, "transfer-function alpha must be in [0, 1)");
        const double sigma = -std::log1p(-(double)e[3]);
        tf[j] = make_float4(e[0], e[1], e[2], (float)(sigma * (double)d->step));
    }
    return MBOIT_OK;
}

// Grid geometry and sampling parameters of a descriptor (validated).
void fill_grid(const mboit_volume_desc* d, mb::GridD& g) {
    const int B = 1 << d->brick_log2;
    g.field = d->field;
    g.nx = d->dims[0];
    g.ny = d->dims[1];
    g.nz = d->dims[2];
    g.brick_log2 = d->brick_log2;
    g.nbx = (g.nx - 1 + B - 1) / B;
    g.nby = (g.ny - 1 + B - 1) / B;
    g.nbz = (g.nz - 1 + B - 1) / B;
    g.hx = (float)(g.nx - 1);
    g.hy = (float)(g.ny - 1);
    g.hz = (float)(g.nz - 1);
    g.step = d->step;
    g.tf_scale = (float)(255.0 / ((double)d->tf_range[1] - (double)d->tf_range[0]));
    g.tf_bias = (float)(-(double)d->tf_range[0] * 255.0 / ((double)d->tf_range[1] - (double)d->tf_range[0]));
    g.absorbance_max = d->absorbance_max;
    g.moment_bias = d->moment_bias;
    g.overestimation = d->overestimation;
    g.bias_vector[0] = 0.0f;
    g.bias_vector[1] = 0.375f;
    g.bias_vector[2] = 0.0f;
    g.bias_vector[3] = 0.375f;
    g.flags = d->flags;
}

int64_t slab_bytes_per_px(int32_t moment_set) {
    switch (moment_set) {
        case MBOIT_TRIG6: return 16;
        case MBOIT_TRIG8: return 20;
        case MBOIT_POWER6: return 28;
        case MBOIT_POWER8: return 36;
        default: return 20;
    }
}

template <class T>
cudaError_t ensure_capacity(T*& p, size_t& cap, size_t n) {
    if (n <= cap) return cudaSuccess;
    cudaFree(p);  // waits for work that may still read the old buffer
    p = nullptr;
    cap = 0;
    const cudaError_t e = cudaMalloc(&p, (n > 0 ? n : 1) * sizeof(T));
    if (e == cudaSuccess) cap = n;
    return e;
}

void drop_graphs(mboit_volume v) {
    for (auto& g : v->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        cudaFree(g.d_order);   // after the graph: cudaFree waits for work that may still read it
    }
    v->graphs.clear();
}

// The volume's queue heads, counters and frame cache serve one stream at a
// time: a call on another stream while work of the volume's last call may
// still run is refused (MBOIT_ERR_STATE).
mboit_status claim_stream(mboit_volume v, cudaStream_t s) {
    if (v->done_recorded && s != v->last_stream) {
        const cudaError_t q = cudaEventQuery(v->done_ev);
        if (q == cudaErrorNotReady)
            return fail(MBOIT_ERR_STATE, "the volume's last call still runs on another stream; synchronise that "
                                         "stream first (one volume, one stream at a time)");
        if (q != cudaSuccess) cudaGetLastError();
    }
    return MBOIT_OK;
}

// Marks the end of this call's work on `s` (nothing to mark while `s` is
// being captured into a graph: the caller's graph orders it).
void release_stream(mboit_volume v, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        v->done_recorded = false;
        return;
    }
    if (cudaEventRecord(v->done_ev, s) == cudaSuccess) {
        v->done_recorded = true;
        v->last_stream = s;
    } else {
        cudaGetLastError();
        v->done_recorded = false;
    }
}

mboit_status check_volume(mboit_volume v) {
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (v->boxes.empty()) return fail(MBOIT_ERR_STATE, "volume has no pieces (mboit_add_piece first)");
    return MBOIT_OK;
}

// Validates views and lays out tiles and output offsets.
mboit_status build_views(const mboit_view* views, int32_t n_views, mb::ViewTable& vt, int64_t bpp = 20,
                         int32_t packet = MBOIT_PACKET_8X4) {
    if (!views) return fail(MBOIT_ERR_INVALID_ARG, "views is NULL");
    if (n_views < 1 || n_views > mb::kMaxViews)
        return fail(MBOIT_ERR_INVALID_ARG, "n_views must be in [1, " + std::to_string(mb::kMaxViews) + "]");
    std::memset(&vt, 0, sizeof vt);
    vt.n = n_views;
    int64_t tiles = 0, moff = 0, coff = 0;
    for (int i = 0; i < n_views; ++i) {
        const mboit_view& V = views[i];
        const std::string at = "view " + std::to_string(i) + ": ";
        if (V.width < 1 || V.height < 1 || V.width > 32768 || V.height > 32768)
            return fail(MBOIT_ERR_INVALID_ARG, at + "width and height must be in [1, 32768]");
        if (V.projection != MBOIT_ORTHO && V.projection != MBOIT_PERSPECTIVE)
            return fail(MBOIT_ERR_INVALID_ARG, at + "unknown projection");
        if (!finite3(V.eye) || !finite3(V.u) || !finite3(V.v) || !finite3(V.w) || !std::isfinite(V.scale_u) ||
            !std::isfinite(V.scale_v))
            return fail(MBOIT_ERR_INVALID_ARG, at + "non-finite camera parameter");
        if (V.w[0] == 0.0f && V.w[1] == 0.0f && V.w[2] == 0.0f)
            return fail(MBOIT_ERR_INVALID_ARG, at + "w (ray direction) is zero");
        if (!(V.near > 0.0f) || !(V.far > V.near) || !std::isfinite(V.far))
            return fail(MBOIT_ERR_INVALID_ARG, at + "need 0 < near < far");
        mb::ViewSlot& S = vt.s[i];
        for (int c = 0; c < 3; ++c) {
            S.v.eye[c] = V.eye[c];
            S.v.u[c] = V.u[c];
            S.v.v[c] = V.v[c];
            S.v.w[c] = V.w[c];
        }
        S.v.width = V.width;
        S.v.height = V.height;
        S.v.projection = V.projection;
        S.v.scale_u = V.scale_u;
        S.v.scale_v = V.scale_v;
        // z = 2 (ln t - ln n) / (ln f - ln n) - 1 = warp_a * log2(t) + warp_b
        const double ln_n = std::log((double)V.near), ln_f = std::log((double)V.far);
        S.v.warp_a = (float)(2.0 * std::log(2.0) / (ln_f - ln_n));
        S.v.warp_b = (float)(-2.0 * ln_n / (ln_f - ln_n) - 1.0);
        S.tw_log2 = packet == MBOIT_PACKET_4X8 ? 2 : 3;
        const int tw = 1 << S.tw_log2, th = 32 >> S.tw_log2;
        S.ntx = (V.width + tw - 1) / tw;
        const int64_t nty = (V.height + th - 1) / th;
        S.tile_base = (int32_t)tiles;
        tiles += (int64_t)S.ntx * nty;
        S.plane = (int32_t)((((int64_t)V.width * V.height) + 3) / 4 * 4);
        S.moment_off = moff;
        S.color_off = coff;
        moff += bpp * S.plane;
        coff += (int64_t)4 * V.width * V.height;
    }
    if (tiles >= (int64_t)1 << 31) return fail(MBOIT_ERR_INVALID_ARG, "too many pixels in one call");
    vt.total_tiles = (int32_t)tiles;
    return MBOIT_OK;
}

// Image-only table for the composite op (offsets of n_views equal images).
mboit_status build_images(int32_t width, int32_t height, int32_t n_views, mb::ViewTable& vt, int64_t bpp = 20) {
    if (n_views < 1 || n_views > mb::kMaxViews) return fail(MBOIT_ERR_INVALID_ARG, "n_views out of range");
    if (width < 1 || height < 1 || width > 32768 || height > 32768)
        return fail(MBOIT_ERR_INVALID_ARG, "width and height must be in [1, 32768]");
    std::memset(&vt, 0, sizeof vt);
    vt.n = n_views;
    for (int i = 0; i < n_views; ++i) {
        mb::ViewSlot& S = vt.s[i];
        S.v.width = width;
        S.v.height = height;
        S.plane = (int32_t)((((int64_t)width * height) + 3) / 4 * 4);
        S.moment_off = (int64_t)i * bpp * S.plane;
        S.color_off = (int64_t)i * 4 * width * height;
    }
    return MBOIT_OK;
}

// Piece list -> selection; returns the brick mask to use (nullptr = every brick).
mboit_status select_pieces(mboit_volume v, const int32_t* pieces, int32_t n_pieces, std::vector<int32_t>& list,
                           const uint8_t** mask) {
    const int32_t K = (int32_t)v->boxes.size();
    list.clear();
    if (!pieces) {
        for (int32_t p = 0; p < K; ++p) list.push_back(p);
    } else {
        if (n_pieces < 1) return fail(MBOIT_ERR_INVALID_ARG, "n_pieces must be >= 1 when pieces is given");
        for (int32_t i = 0; i < n_pieces; ++i) {
            if (pieces[i] < 0 || pieces[i] >= K)
                return fail(MBOIT_ERR_INVALID_ARG, "piece id " + std::to_string(pieces[i]) + " out of range");
            list.push_back(pieces[i]);
        }
    }
    std::vector<uint8_t> want_piece(K, 0);
    for (int32_t p : list) want_piece[p] = 1;
    bool all = true;
    for (int32_t p = 0; p < K; ++p) all = all && want_piece[p];
    if (all && v->owned == v->nbricks) {
        *mask = nullptr;
        return MBOIT_OK;
    }
    std::vector<uint8_t> sel((size_t)v->nbricks);
    for (int64_t b = 0; b < v->nbricks; ++b) sel[b] = v->pob[b] >= 0 && want_piece[v->pob[b]];
    if (!v->sel_uploaded || sel != v->sel_host) {
        // the mask is read by kernels still in flight: wait for them first
        MB_CUDA(cudaDeviceSynchronize());
        MB_CUDA(cudaMemcpy(v->d_sel, sel.data(), sel.size(), cudaMemcpyHostToDevice));
        v->sel_host.swap(sel);
        v->sel_uploaded = true;
        drop_graphs(v);
    }
    *mask = v->d_sel;
    return MBOIT_OK;
}

// Host tables of a tetrahedral mesh: snapped vertex records, cells,
// neighbours and the bin lists, after checking everything the exact
// predicates rely on.
struct TetHost {
    std::vector<int4> verts, cells, nbrs, corners;
    bool narrow = false;
    std::vector<int32_t> bin_start, bin_tets;
    int32_t bdim[3] = {0, 0, 0};
    int32_t bin_shift = 0;
};

mboit_status prepare_tets(const mboit_volume_desc* d, TetHost& h) {
    if (!d->tet_verts || !d->tet_cells || !d->tet_neighbors)
        return fail(MBOIT_ERR_INVALID_ARG, "tet_verts, tet_cells and tet_neighbors are required");
    if (d->n_verts < 4 || d->n_verts > INT32_MAX) return fail(MBOIT_ERR_INVALID_ARG, "n_verts must be in [4, 2^31)");
    if (d->n_tets < 1 || d->n_tets > INT32_MAX) return fail(MBOIT_ERR_INVALID_ARG, "n_tets must be in [1, 2^31)");
    if (d->quantum_log2 < 0 || d->quantum_log2 > 24) return fail(MBOIT_ERR_INVALID_ARG, "quantum_log2 must be in [0, 24]");
    const int s = d->quantum_log2;
    double qmax = 0.0;
    for (int c = 0; c < 3; ++c) {
        if (!(d->tet_box[c] > 0.0f) || !std::isfinite(d->tet_box[c]))
            return fail(MBOIT_ERR_INVALID_ARG, "tet_box must be positive and finite");
        qmax = std::max(qmax, std::ldexp((double)d->tet_box[c], s));
    }
    if (qmax >= 1073741824.0) return fail(MBOIT_ERR_INVALID_ARG, "tet_box * 2^quantum_log2 must be below 2^30");
    const int64_t nv = d->n_verts, nt = d->n_tets;
    h.verts.resize((size_t)nv);
    for (int64_t i = 0; i < nv; ++i) {
        const float* P = d->tet_verts + 4 * i;
        int q[3];
        for (int c = 0; c < 3; ++c) {
            if (!(P[c] >= 0.0f && P[c] <= d->tet_box[c]))
                return fail(MBOIT_ERR_INVALID_ARG, "vertex " + std::to_string(i) + " lies outside [0, tet_box]");
            q[c] = (int)std::nearbyint(std::ldexp((double)P[c], s));
        }
        if (!std::isfinite(P[3])) return fail(MBOIT_ERR_INVALID_ARG, "vertex " + std::to_string(i) + ": non-finite value");
        int w;
        std::memcpy(&w, &P[3], sizeof w);
        h.verts[i] = make_int4(q[0], q[1], q[2], w);
    }
    h.cells.resize((size_t)nt);
    h.nbrs.resize((size_t)nt);
    int64_t emax = 0;
    double esum = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* C = d->tet_cells + 4 * t;
        const int32_t* N = d->tet_neighbors + 4 * t;
        for (int i = 0; i < 4; ++i) {
            if (C[i] < 0 || C[i] >= nv) return fail(MBOIT_ERR_INVALID_ARG, "tet " + std::to_string(t) + ": vertex id out of range");
            if (N[i] < -1 || N[i] >= nt) return fail(MBOIT_ERR_INVALID_ARG, "tet " + std::to_string(t) + ": neighbour id out of range");
        }
        h.cells[t] = make_int4(C[0], C[1], C[2], C[3]);
        h.nbrs[t] = make_int4(N[0], N[1], N[2], N[3]);
        int64_t ext = 0;
        for (int c = 0; c < 3; ++c) {
            int lo = INT32_MAX, hi = INT32_MIN;
            for (int i = 0; i < 4; ++i) {
                const int4& V = h.verts[C[i]];
                const int x = c == 0 ? V.x : c == 1 ? V.y : V.z;
                lo = std::min(lo, x);
                hi = std::max(hi, x);
            }
            ext = std::max(ext, (int64_t)hi - lo);
        }
        emax = std::max(emax, ext);
        esum += (double)ext;
    }
    h.narrow = emax <= 32767;  // 2 E^2 < 2^31: normals fit in 32 bits
    // |n_i| <= 2 E^2 per component and |q - b| <= Q: every D_i fits in 64 bits
    if (6.0 * (double)emax * (double)emax * (qmax + 2.0) >= 4.6e18)
        return fail(MBOIT_ERR_INVALID_ARG, "tets too large for exact 64-bit predicates at this quantum_log2 "
                                           "(use a smaller quantum_log2)");
    for (int64_t t = 0; t < nt; ++t) {
        const int4 c = h.cells[t];
        const int4 a = h.verts[c.x], b = h.verts[c.y], e = h.verts[c.z], f = h.verts[c.w];
        const long long ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
        const long long vx = e.x - a.x, vy = e.y - a.y, vz = e.z - a.z;
        const long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        if (nx * (f.x - a.x) + ny * (f.y - a.y) + nz * (f.z - a.z) <= 0)
            return fail(MBOIT_ERR_INVALID_ARG, "tet " + std::to_string(t) + " is not positively oriented after snapping");
        const int32_t* C = d->tet_cells + 4 * t;
        const int32_t* N = d->tet_neighbors + 4 * t;
        for (int i = 0; i < 4; ++i) {
            const int32_t u = N[i];
            if (u < 0) continue;
            const int32_t* CU = d->tet_cells + 4 * (int64_t)u;
            const int32_t* NU = d->tet_neighbors + 4 * (int64_t)u;
            int j = 0;
            while (j < 4 && NU[j] != t) ++j;
            bool ok = j < 4;
            for (int k = 0; ok && k < 4; ++k) {
                if (k == i) continue;
                bool found = false;
                for (int l = 0; l < 4; ++l) found = found || (l != j && CU[l] == C[k]);
                ok = found;
            }
            if (!ok)
                return fail(MBOIT_ERR_INVALID_ARG, "tets " + std::to_string(t) + " and " + std::to_string(u) +
                                                       ": neighbours not reciprocal or not sharing the face");
        }
    }
    // bins: a power of two no smaller than the mean tet extent, at most ~4 per tet
    const double eavg = std::max(1.0, esum / (double)nt);
    int bs = 0;
    while (bs < 30 && std::ldexp(1.0, bs) < eavg) ++bs;
    for (;; ++bs) {
        int64_t nb = 1;
        for (int c = 0; c < 3; ++c) nb *= ((int64_t)std::nearbyint(std::ldexp((double)d->tet_box[c], s)) >> bs) + 1;
        if (nb <= 4 * nt + 64 && nb <= (int64_t(1) << 26)) break;
    }
    h.bin_shift = bs;
    for (int c = 0; c < 3; ++c) h.bdim[c] = (int32_t)(((int64_t)std::nearbyint(std::ldexp((double)d->tet_box[c], s)) >> bs) + 1);
    const int64_t nbins = (int64_t)h.bdim[0] * h.bdim[1] * h.bdim[2];
    std::vector<int64_t> start((size_t)nbins + 1, 0);
    for (int sweep = 0; sweep < 2; ++sweep) {
        if (sweep == 1) {
            for (int64_t b = 0; b < nbins; ++b) start[b + 1] += start[b];
            if (start[nbins] > INT32_MAX) return fail(MBOIT_ERR_INVALID_ARG, "mesh too large for the bin lists");
            h.bin_tets.resize((size_t)start[nbins]);
        }
        std::vector<int64_t> fill;
        if (sweep == 1) fill.assign(start.begin(), start.end() - 1);
        for (int64_t t = 0; t < nt; ++t) {
            const int4 c = h.cells[t];
            const int4 V[4] = {h.verts[c.x], h.verts[c.y], h.verts[c.z], h.verts[c.w]};
            int lo[3], hi[3];
            lo[0] = std::min(std::min(V[0].x, V[1].x), std::min(V[2].x, V[3].x)) >> bs;
            lo[1] = std::min(std::min(V[0].y, V[1].y), std::min(V[2].y, V[3].y)) >> bs;
            lo[2] = std::min(std::min(V[0].z, V[1].z), std::min(V[2].z, V[3].z)) >> bs;
            hi[0] = std::max(std::max(V[0].x, V[1].x), std::max(V[2].x, V[3].x)) >> bs;
            hi[1] = std::max(std::max(V[0].y, V[1].y), std::max(V[2].y, V[3].y)) >> bs;
            hi[2] = std::max(std::max(V[0].z, V[1].z), std::max(V[2].z, V[3].z)) >> bs;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        const int64_t b = ((int64_t)z * h.bdim[1] + y) * h.bdim[0] + x;
                        if (sweep == 0) ++start[b + 1];
                        else h.bin_tets[(size_t)fill[b]++] = (int32_t)t;
                    }
        }
    }
    h.bin_start.assign(start.begin(), start.end());
    h.corners.resize(4 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int4 c = h.cells[t];
        h.corners[4 * t] = h.verts[c.x];
        h.corners[4 * t + 1] = h.verts[c.y];
        h.corners[4 * t + 2] = h.verts[c.z];
        h.corners[4 * t + 3] = h.verts[c.w];
    }
    return MBOIT_OK;
}

// The batched (fused, persistent) passes of the volume's kind.  `cache`:
// mesh sample values shared by the two passes of one frame.
// The field's tensor map of a grid volume, or NULL (no TMA windows).
const CUtensorMap* field_map_of(mboit_volume v, int cfg) {
    return v->has_field_map && (cfg == 5 || cfg == 6) ? &v->field_map[cfg - 5] : nullptr;
}

// Whether window configuration cfg can run on this volume.
bool config_usable(mboit_volume v, int cfg) {
    return mb::stage_config_eligible(v->grid, cfg) && ((cfg != 5 && cfg != 6) || v->has_field_map);
}

// Checks the octree's or mesh's index tables on stream s before passes that
// read them (grids have none).
cudaError_t check_tables(mboit_volume v, cudaStream_t s) {
    if (v->kind == MBOIT_AMR) return mb::launch_check_tables(v->amr, s);
    if (v->kind == MBOIT_TET) return mb::launch_check_tables(v->tet, s);
    return cudaSuccess;
}

cudaError_t pass1_batched(mboit_volume v, const uint8_t* mask, const mb::ViewTable& vt, void* moments, cudaStream_t s,
                          mb::TileCache tc = mb::TileCache{}) {
    const cudaError_t e = check_tables(v, s);
    if (e != cudaSuccess) return e;
    if (v->kind == MBOIT_AMR) return mb::launch_pass1_amr(v->amr, v->d_tf, mask, vt, moments, v->d_ctr, s, tc);
    if (v->kind == MBOIT_TET) return mb::launch_pass1_tet(v->tet, v->d_tf, mask, vt, moments, v->d_ctr, s, tc);
    return mb::launch_pass1_fused(v->grid, v->d_tf, mask, vt, moments, v->d_ctr, s, v->tune1, tc,
                                  field_map_of(v, v->tune1));
}

cudaError_t pass2_batched(mboit_volume v, const uint8_t* mask, const mb::ViewTable& vt, const void* moments,
                          float* color, int32_t mode, cudaStream_t s, mb::TileCache tc = mb::TileCache{}) {
    const cudaError_t e = check_tables(v, s);
    if (e != cudaSuccess) return e;
    if (v->kind == MBOIT_AMR)
        return mb::launch_pass2_amr(v->amr, v->d_tf, mask, vt, moments, color, mode, v->d_ctr, s, tc);
    if (v->kind == MBOIT_TET)
        return mb::launch_pass2_tet(v->tet, v->d_tf, mask, vt, moments, color, mode, v->d_ctr, s, tc);
    return mb::launch_pass2_fused(v->grid, v->d_tf, mask, vt, moments, color, mode, v->d_ctr, s, v->tune2, tc);
}

// The one-launch frame of the volume's kind (four power moments).
cudaError_t frame_batched(mboit_volume v, const uint8_t* mask, const mb::ViewTable& vt, void* moments, float* color,
                          cudaStream_t s, int cfg, mb::TileCache tc) {
    const cudaError_t e = check_tables(v, s);
    if (e != cudaSuccess) return e;
    if (v->kind == MBOIT_AMR)
        return mb::launch_frame_amr(v->amr, v->d_tf, mask, vt, moments, color, mb::kColorResolved, v->d_ctr, s, tc);
    if (v->kind == MBOIT_TET)
        return mb::launch_frame_tet(v->tet, v->d_tf, mask, vt, moments, color, mb::kColorResolved, v->d_ctr, s, tc);
    return mb::launch_frame_fused(v->grid, v->d_tf, mask, vt, moments, color, mb::kColorResolved, v->d_ctr, s, cfg, tc,
                                  field_map_of(v, cfg));
}

// The tile-row sample cache of a frame: its exact row count for these views
// (one small kernel, synchronous; done once per recorded frame graph), then
// grow-only buffers.  Left off (c.vals NULL, pass 2 marches again) when the
// device lacks the memory with 1 GiB to spare.
mboit_status cache_buffers(mboit_volume v, unsigned long long rows, int32_t total_tiles, mb::TileCache& c);

mboit_status tile_cache(mboit_volume v, const mb::ViewTable& vt, mb::TileCache& c) {
    c = mb::TileCache{};
    cudaStream_t cs = v->cap_stream;
    if (!v->d_rows) MB_CUDA(cudaMalloc(&v->d_rows, sizeof(unsigned long long)));
    MB_CUDA(cudaMemsetAsync(v->d_rows, 0, sizeof(unsigned long long), cs));
    MB_CUDA(mb::launch_tile_rows(v->grid, vt, v->d_rows, cs));
    unsigned long long rows = 0;
    MB_CUDA(cudaMemcpyAsync(&rows, v->d_rows, sizeof rows, cudaMemcpyDeviceToHost, cs));
    MB_CUDA(cudaStreamSynchronize(cs));
    return cache_buffers(v, rows, vt.total_tiles, c);
}

// The frame's cost-ordered dequeue: every ray tile's row count (the rows its
// warp walks in lockstep, k_tile_rows), then the tiles sorted by it, longest
// first (ties in tile order), in a new device buffer the caller owns.
// Synchronous; for graph recording and the autotuner.
mboit_status make_tile_order(mboit_volume v, const mb::ViewTable& vt, int32_t** out) {
    *out = nullptr;
    const size_t n = (size_t)std::max(vt.total_tiles, 1);
    cudaStream_t cs = v->cap_stream;
    int32_t* d_rows = nullptr;
    MB_CUDA(cudaMalloc(&d_rows, n * sizeof(int32_t)));
    if (!v->d_rows) {
        const cudaError_t e = cudaMalloc(&v->d_rows, sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(d_rows);
            return fail(MBOIT_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    std::vector<int32_t> rows(n, 0);
    cudaError_t e = cudaMemsetAsync(d_rows, 0, n * sizeof(int32_t), cs);
    if (e == cudaSuccess) e = mb::launch_tile_rows(v->grid, vt, v->d_rows, cs, d_rows);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rows.data(), d_rows, n * sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    cudaFree(d_rows);
    if (e != cudaSuccess) return fail(MBOIT_ERR_CUDA, std::string("tile order: ") + cudaGetErrorString(e));
    std::vector<int32_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return rows[a] > rows[b]; });
    int32_t* d = nullptr;
    MB_CUDA(cudaMalloc(&d, n * sizeof(int32_t)));
    e = cudaMemcpy(d, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return fail(MBOIT_ERR_CUDA, std::string("tile order upload: ") + cudaGetErrorString(e));
    }
    *out = d;
    return MBOIT_OK;
}

// Grow-only cache buffers of `v` for `rows` rows over `total_tiles` tiles
// (left off, c.vals NULL, without 1 GiB to spare).
mboit_status cache_buffers(mboit_volume v, unsigned long long rows, int32_t total_tiles, mb::TileCache& c) {
    c = mb::TileCache{};
    const size_t nvals = (size_t)rows * 32, ntiles = (size_t)std::max(total_tiles, 1);
    size_t free_b = 0, total_b = 0;
    MB_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t grow = (nvals > v->cap_tcvals ? nvals * sizeof(float) : 0) +
                        (ntiles > v->cap_tile_base ? ntiles * sizeof(long long) : 0);
    if (grow + (size_t(1) << 30) > free_b) return MBOIT_OK;
    float* b1 = v->d_tcvals;
    long long* b2 = v->d_tile_base;
    MB_CUDA(ensure_capacity(v->d_tcvals, v->cap_tcvals, std::max<size_t>(nvals, 32)));
    MB_CUDA(ensure_capacity(v->d_tile_base, v->cap_tile_base, ntiles));
    if (v->d_tcvals != b1 || v->d_tile_base != b2) drop_graphs(v);
    c.vals = v->d_tcvals;
    c.tile_base = v->d_tile_base;
    c.rows_cap = (long long)(v->cap_tcvals / 32);
    // MBOIT_FRAME_CACHE_ROWS caps the rows handed out (0: every tile marches
    // again in pass 2), to exercise and measure the fallback
    if (const char* cap = std::getenv("MBOIT_FRAME_CACHE_ROWS")) c.rows_cap = std::min(c.rows_cap, std::atoll(cap));
    return MBOIT_OK;
}

}  // namespace

extern "C" {

const char* mboit_last_error(void) { return g_err.c_str(); }

mboit_status mboit_split_cells(const float* verts, int64_t n_verts, const int32_t* cells, const int32_t* cell_types,
                               int64_t n_cells, int32_t quantum_log2, int32_t* tets_out, int32_t* neighbors_out,
                               int64_t* cell_of_tet, int64_t max_tets, int64_t* n_tets) {
    g_err.clear();
    if (!verts || !cells || !cell_types || !tets_out || !neighbors_out || !cell_of_tet || !n_tets)
        return fail(MBOIT_ERR_INVALID_ARG, "NULL pointer");
    if (n_verts < 4 || n_verts > INT32_MAX) return fail(MBOIT_ERR_INVALID_ARG, "n_verts must be in [4, 2^31)");
    if (n_cells < 1 || max_tets < 1) return fail(MBOIT_ERR_INVALID_ARG, "n_cells and max_tets must be >= 1");
    if (quantum_log2 < 0 || quantum_log2 > 24) return fail(MBOIT_ERR_INVALID_ARG, "quantum_log2 must be in [0, 24]");
    const int qs = quantum_log2;
    auto q = [&](int32_t v, int c) { return (long long)std::nearbyint(std::ldexp((double)verts[4 * (int64_t)v + c], qs)); };
    int64_t n = 0;
    std::string err;
    // one tet, positively oriented on the snapped vertices (exact: 64-bit
    // differences, 128-bit products)
    auto emit = [&](int32_t a, int32_t b, int32_t c, int32_t d, int64_t cell) {
        int32_t t[4] = {a, b, c, d};
        for (int i = 0; i < 4; ++i)
            if (t[i] < 0 || t[i] >= n_verts) {
                err = "cell " + std::to_string(cell) + ": vertex id out of range";
                return false;
            }
        long long e[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c2 = 0; c2 < 3; ++c2) e[r][c2] = q(t[r + 1], c2) - q(t[0], c2);
        const __int128 det = (__int128)e[0][0] * ((__int128)e[1][1] * e[2][2] - (__int128)e[1][2] * e[2][1]) -
                             (__int128)e[0][1] * ((__int128)e[1][0] * e[2][2] - (__int128)e[1][2] * e[2][0]) +
                             (__int128)e[0][2] * ((__int128)e[1][0] * e[2][1] - (__int128)e[1][1] * e[2][0]);
        if (det == 0) {
            err = "cell " + std::to_string(cell) + " gives a flat tet after snapping";
            return false;
        }
        if (det < 0) std::swap(t[2], t[3]);
        if (n >= max_tets) {
            err = "max_tets too small";
            return false;
        }
        std::memcpy(tets_out + 4 * n, t, sizeof t);
        cell_of_tet[n++] = cell;
        return true;
    };
    for (int64_t i = 0; i < n_cells; ++i) {
        const int32_t* c = cells + 6 * i;
        bool ok = true;
        switch (cell_types[i]) {
            case 4:
                ok = emit(c[0], c[1], c[2], c[3], i);
                break;
            case 5: {
                // base quad c0 c1 c2 c3: cut along the diagonal holding its smallest id
                const int32_t mn = std::min(std::min(c[0], c[1]), std::min(c[2], c[3]));
                const int j = (mn == c[0] || mn == c[2]) ? 0 : 1;
                ok = emit(c[j], c[j + 1], c[j + 2], c[4], i) && emit(c[j], c[j + 2], c[(j + 3) & 3], c[4], i);
                break;
            }
            case 6: {
                // the smallest id becomes local vertex 0: swap the triangles if
                // it is on top, then rotate them; its two quad faces are cut
                // through it, the opposite quad (1 2 5 4) through its smallest
                int im = 0;
                for (int k = 1; k < 6; ++k)
                    if (c[k] < c[im]) im = k;
                const int lo = im < 3 ? 0 : 3, hi = 3 - lo, r = im % 3;
                int32_t v[6];
                for (int k = 0; k < 3; ++k) {
                    v[k] = c[lo + (r + k) % 3];
                    v[k + 3] = c[hi + (r + k) % 3];
                }
                if (std::min(v[1], v[5]) < std::min(v[2], v[4]))
                    ok = emit(v[0], v[1], v[2], v[5], i) && emit(v[0], v[1], v[5], v[4], i);
                else
                    ok = emit(v[0], v[1], v[2], v[4], i) && emit(v[0], v[4], v[2], v[5], i);
                ok = ok && emit(v[0], v[4], v[5], v[3], i);
                break;
            }
            default:
                err = "cell " + std::to_string(i) + ": type must be 4, 5 or 6";
                ok = false;
        }
        if (!ok) return fail(MBOIT_ERR_INVALID_ARG, err);
    }
    // face neighbours: sort the faces by their vertex triple; equal triples pair up
    struct Face {
        int32_t a, b, c, tet, slot;
    };
    std::vector<Face> faces((size_t)n * 4);
    for (int64_t t = 0; t < n; ++t)
        for (int i = 0; i < 4; ++i) {
            int32_t f[3], m = 0;
            for (int k = 0; k < 4; ++k)
                if (k != i) f[m++] = tets_out[4 * t + k];
            std::sort(f, f + 3);
            faces[(size_t)(4 * t + i)] = Face{f[0], f[1], f[2], (int32_t)t, i};
        }
    std::sort(faces.begin(), faces.end(), [](const Face& x, const Face& y) {
        return x.a != y.a ? x.a < y.a : x.b != y.b ? x.b < y.b : x.c < y.c;
    });
    for (int64_t t = 0; t < 4 * n; ++t) neighbors_out[t] = -1;
    for (size_t k = 0; k < faces.size();) {
        size_t e = k + 1;
        while (e < faces.size() && faces[e].a == faces[k].a && faces[e].b == faces[k].b && faces[e].c == faces[k].c) ++e;
        if (e - k > 2) return fail(MBOIT_ERR_INVALID_ARG, "a face is shared by more than two tets");
        if (e - k == 2) {
            neighbors_out[4 * (int64_t)faces[k].tet + faces[k].slot] = faces[k + 1].tet;
            neighbors_out[4 * (int64_t)faces[k + 1].tet + faces[k + 1].slot] = faces[k].tet;
        }
        k = e;
    }
    *n_tets = n;
    return MBOIT_OK;
}

size_t mboit_moment_image_bytes(int32_t width, int32_t height, int32_t moment_set, int32_t storage) {
    if (width < 1 || height < 1) return 0;
    const bool power = (moment_set == MBOIT_POWER4 || moment_set == MBOIT_POWER6 || moment_set == MBOIT_POWER8) &&
                       storage == MBOIT_STORE_F32;
    const bool trig = is_trig(moment_set) && (storage == MBOIT_STORE_F16 || storage == MBOIT_STORE_BF16);
    if (!power && !trig) return 0;
    const size_t P = (((size_t)width * (size_t)height) + 3) / 4 * 4;
    return (size_t)slab_bytes_per_px(moment_set) * P;
}

mboit_status mboit_create_volume(const mboit_volume_desc* d, mboit_volume* out) {
    g_err.clear();
    Range nvtx("mboit_create_volume");
    if (!d || !out) return fail(MBOIT_ERR_INVALID_ARG, "desc and out must be non-NULL");
    if (d->kind != MBOIT_GRID && d->kind != MBOIT_AMR && d->kind != MBOIT_TET)
        return fail(MBOIT_ERR_UNSUPPORTED, "unknown volume kind");
    const bool is_amr = d->kind == MBOIT_AMR;
    const bool is_tet = d->kind == MBOIT_TET;
    if (d->moment_set < MBOIT_POWER4 || d->moment_set > MBOIT_POWER8) return fail(MBOIT_ERR_UNSUPPORTED, "unknown moment set");
    if (!is_trig(d->moment_set) && d->storage != MBOIT_STORE_F32)
        return fail(MBOIT_ERR_UNSUPPORTED, "power moments are stored in float32");
    if (is_trig(d->moment_set) && d->storage != MBOIT_STORE_F16 && d->storage != MBOIT_STORE_BF16)
        return fail(MBOIT_ERR_UNSUPPORTED, "trigonometric moments are stored in float16 or bfloat16");
    if ((d->moment_set == MBOIT_POWER6 || d->moment_set == MBOIT_POWER8) && !(d->moment_bias > 0.0f))
        return fail(MBOIT_ERR_INVALID_ARG, "6 and 8 power moments need moment_bias > 0");
    if (is_trig(d->moment_set) &&
        !(d->moment_bias >= (d->storage == MBOIT_STORE_F16 ? 2e-3f : 2e-2f)))
        return fail(MBOIT_ERR_INVALID_ARG, "trigonometric moments in 16 bits need moment_bias >= 2e-3 (float16) or "
                                           ">= 2e-2 (bfloat16) to keep the stored Toeplitz matrices positive definite");
    if (d->flags & ~(MBOIT_FLAG_RAW_SUM | MBOIT_FLAG_DETERMINISTIC | MBOIT_FLAG_ADAPTIVE_STEP | MBOIT_FLAG_FP64_SETUP))
        return fail(MBOIT_ERR_INVALID_ARG, "unknown flag bits");
    if ((d->flags & MBOIT_FLAG_ADAPTIVE_STEP) && !is_amr)
        return fail(MBOIT_ERR_INVALID_ARG, "MBOIT_FLAG_ADAPTIVE_STEP applies to octrees only");
    if (!is_amr && !is_tet && !d->field) return fail(MBOIT_ERR_INVALID_ARG, "field is NULL");
    if (is_amr) {
        if (!d->leaf_values || !d->leaf_table) return fail(MBOIT_ERR_INVALID_ARG, "leaf_values and leaf_table are required");
        if (d->n_leaves < 1) return fail(MBOIT_ERR_INVALID_ARG, "n_leaves must be >= 1");
        if (d->max_level < 0 || d->max_level > 10) return fail(MBOIT_ERR_INVALID_ARG, "max_level must be in [0, 10]");
        if (d->dims[0] != d->dims[1] || d->dims[0] != d->dims[2])
            return fail(MBOIT_ERR_INVALID_ARG, "octree domains are cubes: dims must be equal");
    }
    if (!is_tet) {
        for (int c = 0; c < 3; ++c)
            if (d->dims[c] < 2 || d->dims[c] > (1 << 20)) return fail(MBOIT_ERR_INVALID_ARG, "dims must be in [2, 2^20]");
        if (d->brick_log2 < 0 || d->brick_log2 > 7) return fail(MBOIT_ERR_INVALID_ARG, "brick_log2 must be in [0, 7]");
    }
    mboit_status cs = check_sampling(d);
    if (cs != MBOIT_OK) return cs;
    std::vector<float4> tf(256);
    cs = convert_tf(d, tf.data());
    if (cs != MBOIT_OK) return cs;
    // octree: leaf table checks and the finest-brick -> leaf map (host)
    std::vector<int32_t> fmap;
    int64_t fdim = 0;
    if (is_amr) {
        const int64_t D = d->dims[0] - 1;
        const int64_t fb = int64_t(1) << d->brick_log2;
        fdim = (D + fb - 1) / fb;
        if (fdim * fdim * fdim > (int64_t(1) << 31)) return fail(MBOIT_ERR_INVALID_ARG, "octree domain too large");
        fmap.assign((size_t)(fdim * fdim * fdim), -1);
        for (int32_t l = 0; l < d->n_leaves; ++l) {
            const int32_t* L = d->leaf_table + 4 * (size_t)l;
            if (L[3] < 0 || L[3] > d->max_level)
                return fail(MBOIT_ERR_INVALID_ARG, "leaf " + std::to_string(l) + ": level out of range");
            const int64_t nb = int64_t(1) << (d->max_level - L[3]);
            int64_t b0[3];
            for (int c = 0; c < 3; ++c) {
                if (L[c] < 0 || (L[c] % fb) != 0)
                    return fail(MBOIT_ERR_INVALID_ARG, "leaf " + std::to_string(l) + ": origin not on the brick lattice");
                b0[c] = L[c] / fb;
                if (b0[c] + nb > fdim) return fail(MBOIT_ERR_INVALID_ARG, "leaf " + std::to_string(l) + " leaves the domain");
            }
            for (int64_t z = b0[2]; z < b0[2] + nb; ++z)
                for (int64_t y = b0[1]; y < b0[1] + nb; ++y)
                    for (int64_t x = b0[0]; x < b0[0] + nb; ++x) {
                        int32_t& m = fmap[(size_t)((z * fdim + y) * fdim + x)];
                        if (m >= 0)
                            return fail(MBOIT_ERR_INVALID_ARG, "leaves " + std::to_string(m) + " and " +
                                                                   std::to_string(l) + " overlap");
                        m = l;
                    }
        }
    }
    TetHost th;
    if (is_tet) {
        const mboit_status ts = prepare_tets(d, th);
        if (ts != MBOIT_OK) return ts;
    }
    int dev = 0;
    MB_CUDA(cudaGetDevice(&dev));
    if (!is_tet) {
        cudaPointerAttributes attr{};
        const void* data_ptr = is_amr ? (const void*)d->leaf_values : (const void*)d->field;
        if (cudaPointerGetAttributes(&attr, data_ptr) != cudaSuccess ||
            (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(MBOIT_ERR_INVALID_ARG,
                        is_amr ? "leaf_values must be a device pointer" : "field must be a device pointer");
        }
        if (attr.device != dev) return fail(MBOIT_ERR_INVALID_ARG, "volume data lives on another device than the current one");
    }

    mboit_volume v = new (std::nothrow) mboit_volume_s();
    if (!v) return fail(MBOIT_ERR_OUT_OF_MEMORY, "host allocation failed");
    v->device = dev;
    v->desc = *d;
    v->desc.tf_rgba = nullptr;
    mb::GridD& g = v->grid;
    fill_grid(d, g);
    fill_trig(g.trig, d->moment_set, d->storage, d->moment_bias);
    v->nbricks = (int64_t)g.nbx * g.nby * g.nbz;
    v->field_bytes = (size_t)g.nx * g.ny * g.nz * sizeof(float);
    v->kind = d->kind;
    // one launch where it measured faster without tuning (grids); the
    // autotuner times both forms for every kind with four power moments
    v->frame_launches = (d->kind == MBOIT_GRID && d->moment_set == MBOIT_POWER4) ? 1 : 2;
    if (d->kind == MBOIT_GRID) v->has_field_map = mb::encode_field_maps(g, v->field_map);
    if (is_amr) {
        g.field = nullptr;
        v->nbricks = d->n_leaves;  // the units of an octree are its leaves
        const int nv = (1 << d->brick_log2) + 1;
        v->field_bytes = (size_t)d->n_leaves * nv * nv * nv * sizeof(float);
        v->leaf_table.assign(d->leaf_table, d->leaf_table + 4 * (size_t)d->n_leaves);
        v->desc.leaf_table = nullptr;
    }
    if (is_tet) {
        g.field = nullptr;
        g.nx = g.ny = g.nz = 0;
        g.nbx = g.nby = g.nbz = 0;
        g.hx = d->tet_box[0];
        g.hy = d->tet_box[1];
        g.hz = d->tet_box[2];
        v->nbricks = d->n_tets;  // the units of a mesh are its tets
        v->field_bytes = (size_t)d->n_verts * sizeof(float);
        v->tet_cells.assign(d->tet_cells, d->tet_cells + 4 * (size_t)d->n_tets);
        v->tet_xyz.resize(3 * (size_t)d->n_verts);
        for (int64_t i = 0; i < d->n_verts; ++i)
            for (int c = 0; c < 3; ++c) v->tet_xyz[3 * i + c] = d->tet_verts[4 * i + c];
        v->desc.tet_verts = nullptr;
        v->desc.tet_cells = nullptr;
        v->desc.tet_neighbors = nullptr;
    }
    v->pob.assign((size_t)v->nbricks, -1);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&v->d_tf, 256 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&v->d_pob, (size_t)v->nbricks * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&v->d_sel, (size_t)v->nbricks);
    if (e == cudaSuccess) e = cudaMalloc(&v->d_ctr, sizeof(mb::Counters));
    if (e == cudaSuccess) e = cudaMemcpy(v->d_tf, tf.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice);
    v->tf_host = tf;
    if (e == cudaSuccess) e = cudaMemset(v->d_pob, 0xff, (size_t)v->nbricks * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(v->d_ctr, 0, sizeof(mb::Counters));
    if (e == cudaSuccess && is_amr) {
        e = cudaMalloc(&v->d_leaves, (size_t)d->n_leaves * sizeof(int4));
        if (e == cudaSuccess) e = cudaMalloc(&v->d_fmap, fmap.size() * sizeof(int32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(v->d_leaves, d->leaf_table, (size_t)d->n_leaves * sizeof(int4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(v->d_fmap, fmap.data(), fmap.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        // per leaf its origin in finest cells and 1 / cell size, as the march reads them
        std::vector<float4> box((size_t)d->n_leaves);
        for (int32_t l = 0; l < d->n_leaves; ++l) {
            const int32_t* L = d->leaf_table + 4 * (size_t)l;
            box[(size_t)l] = make_float4((float)L[0], (float)L[1], (float)L[2], std::ldexp(1.0f, L[3] - d->max_level));
        }
        if (e == cudaSuccess) e = cudaMalloc(&v->d_leaf_box, box.size() * sizeof(float4));
        if (e == cudaSuccess)
            e = cudaMemcpy(v->d_leaf_box, box.data(), box.size() * sizeof(float4), cudaMemcpyHostToDevice);
        v->amr.g = g;
        v->amr.values = d->leaf_values;
        v->amr.leaves = v->d_leaves;
        v->amr.leaf_box = v->d_leaf_box;
        v->amr.fmap = v->d_fmap;
        v->amr.fdim = (int32_t)fdim;
        v->amr.nv = (1 << d->brick_log2) + 1;
        v->amr.max_level = d->max_level;
        v->amr.complete = std::find(fmap.begin(), fmap.end(), -1) == fmap.end() ? 1 : 0;
        v->amr.n_leaves = d->n_leaves;
        v->amr.err = &v->d_ctr->error;
    }
    if (e == cudaSuccess && is_tet) {
        auto up = [&](auto*& dst, const auto& src) {
            using T = typename std::remove_reference<decltype(src)>::type::value_type;
            cudaError_t r = cudaMalloc(&dst, std::max<size_t>(src.size(), 1) * sizeof(T));
            if (r == cudaSuccess && !src.empty())
                r = cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
            return r;
        };
        e = up(v->d_tcorners, th.corners);
        if (e == cudaSuccess) e = up(v->d_tnbrs, th.nbrs);
        if (e == cudaSuccess) e = up(v->d_tcells, th.cells);
        if (e == cudaSuccess) e = up(v->d_bin_start, th.bin_start);
        if (e == cudaSuccess) e = up(v->d_bin_tets, th.bin_tets);
        if (e == cudaSuccess) e = cudaMalloc(&v->d_tvals, v->field_bytes);
        mb::TetD& m = v->tet;
        m.g = g;
        m.corners = v->d_tcorners;
        m.nbrs = v->d_tnbrs;
        m.narrow = th.narrow ? 1 : 0;
        m.n_tets = (int32_t)d->n_tets;
        m.n_bin_tets = (int32_t)th.bin_tets.size();
        m.err = &v->d_ctr->error;
        m.bin_start = v->d_bin_start;
        m.bin_tets = v->d_bin_tets;
        for (int c = 0; c < 3; ++c) m.bdim[c] = th.bdim[c];
        m.bin_shift = th.bin_shift;
        m.qscale = std::ldexp(1.0f, d->quantum_log2);
        // walk steps before the bin search takes over; MBOIT_TET_MAX_WALK
        // overrides it (1: every point is found by the search), to exercise
        // and measure the fallback
        m.max_walk = 64;
        if (const char* w = std::getenv("MBOIT_TET_MAX_WALK")) m.max_walk = std::max(1, std::atoi(w));
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&v->frame_ev[i]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = mb::prepare_kernels();
    if (e != cudaSuccess) {
        const mboit_status s = (e == cudaErrorMemoryAllocation) ? MBOIT_ERR_OUT_OF_MEMORY : MBOIT_ERR_CUDA;
        const std::string msg = std::string("volume set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        mboit_destroy_volume(v);
        return fail(s, msg);
    }
    *out = v;
    return MBOIT_OK;
}

mboit_status mboit_destroy_volume(mboit_volume v) {
    g_err.clear();
    if (!v) return MBOIT_OK;
    {
        DeviceGuard dg(v->device);
        cudaDeviceSynchronize();
        drop_graphs(v);
        if (v->cap_stream) cudaStreamDestroy(v->cap_stream);
        for (cudaEvent_t ev : v->frame_ev)
            if (ev) cudaEventDestroy(ev);
        if (v->done_ev) cudaEventDestroy(v->done_ev);
        cudaFree(v->d_tf);
        cudaFree(v->d_leaves);
        cudaFree(v->d_leaf_box);
        cudaFree(v->d_fmap);
        cudaFree(v->d_tcorners);
        cudaFree(v->d_tnbrs);
        cudaFree(v->d_tcells);
        cudaFree(v->d_tcvals);
        cudaFree(v->d_tile_base);
        cudaFree(v->d_rows);
        cudaFree(v->d_bin_start);
        cudaFree(v->d_bin_tets);
        cudaFree(v->d_tvals);
        cudaFree(v->d_pob);
        cudaFree(v->d_sel);
        cudaFree(v->d_ctr);
        cudaFree(v->sl_counts);
        cudaFree(v->sl_starts);
        cudaFree(v->sl_totals);
        cudaFree(v->sl_base);
        cudaFree(v->sl_bsum);
        cudaFree(v->sl_key);
        cudaFree(v->sl_col);
    }
    delete v;
    return MBOIT_OK;
}

mboit_status mboit_add_piece(mboit_volume v, const int32_t* ids, int64_t n, int32_t ids_on_device,
                             int32_t* piece_id_out) {
    g_err.clear();
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (!ids || n < 1) return fail(MBOIT_ERR_INVALID_ARG, "a piece needs at least one brick id");
    if (n > v->nbricks) return fail(MBOIT_ERR_INVALID_ARG, "more brick ids than bricks");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    std::vector<int32_t> h((size_t)n);
    if (ids_on_device) {
        MB_CUDA(cudaMemcpy(h.data(), ids, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(h.data(), ids, (size_t)n * sizeof(int32_t));
    }
    const int32_t K = (int32_t)v->boxes.size();
    std::vector<uint8_t> seen((size_t)v->nbricks, 0);
    int bmin[3] = {1 << 30, 1 << 30, 1 << 30}, bmax[3] = {-1, -1, -1};
    const mb::GridD& g = v->grid;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t b = h[i];
        if (b < 0 || b >= v->nbricks) return fail(MBOIT_ERR_INVALID_ARG, "brick id " + std::to_string(b) + " out of range");
        if (seen[b]) return fail(MBOIT_ERR_INVALID_ARG, "brick id " + std::to_string(b) + " listed twice");
        if (v->pob[b] >= 0)
            return fail(MBOIT_ERR_INVALID_ARG, "brick " + std::to_string(b) + " already belongs to piece " +
                                                   std::to_string(v->pob[b]) + " (pieces must not overlap)");
        seen[b] = 1;
        if (v->kind != MBOIT_GRID) continue;
        const int bc[3] = {b % g.nbx, (b / g.nbx) % g.nby, b / (g.nbx * g.nby)};
        for (int c = 0; c < 3; ++c) {
            bmin[c] = bc[c] < bmin[c] ? bc[c] : bmin[c];
            bmax[c] = bc[c] > bmax[c] ? bc[c] : bmax[c];
        }
    }
    for (int64_t i = 0; i < n; ++i) v->pob[h[i]] = K;
    cudaError_t e = cudaMemcpy(v->d_pob, v->pob.data(), (size_t)v->nbricks * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        for (int64_t i = 0; i < n; ++i) v->pob[h[i]] = -1;
        return fail(MBOIT_ERR_CUDA, std::string("uploading brick ownership: ") + cudaGetErrorString(e));
    }
    const int B = 1 << g.brick_log2;
    const float hi[3] = {g.hx, g.hy, g.hz};
    mb::PieceBox box;
    if (v->kind == MBOIT_TET) {
        // union of the tets' boxes, padded by one quantum (a sample snaps by up to half of one)
        const float pad = std::ldexp(1.0f, -v->desc.quantum_log2);
        for (int c = 0; c < 3; ++c) {
            box.lo[c] = 3.0e38f;
            box.hi[c] = -3.0e38f;
        }
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 4; ++k) {
                const float* P = &v->tet_xyz[3 * (size_t)v->tet_cells[4 * (size_t)h[i] + k]];
                for (int c = 0; c < 3; ++c) {
                    box.lo[c] = std::min(box.lo[c], P[c]);
                    box.hi[c] = std::max(box.hi[c], P[c]);
                }
            }
        for (int c = 0; c < 3; ++c) {
            box.lo[c] = std::max(box.lo[c] - pad, 0.0f);
            box.hi[c] = std::min(box.hi[c] + pad, hi[c]);
        }
    } else if (v->kind == MBOIT_AMR) {
        // union of the leaves' boxes
        for (int c = 0; c < 3; ++c) {
            box.lo[c] = 3.0e38f;
            box.hi[c] = 0.0f;
        }
        for (int64_t i = 0; i < n; ++i) {
            const int32_t* L = &v->leaf_table[4 * (size_t)h[i]];
            const float size = (float)(B << (v->desc.max_level - L[3]));
            for (int c = 0; c < 3; ++c) {
                box.lo[c] = std::min(box.lo[c], (float)L[c]);
                box.hi[c] = std::max(box.hi[c], std::min((float)L[c] + size, hi[c]));
            }
        }
    } else {
        for (int c = 0; c < 3; ++c) {
            box.lo[c] = (float)(bmin[c] * B);
            const float top = (float)((bmax[c] + 1) * B);
            box.hi[c] = top < hi[c] ? top : hi[c];
        }
    }
    v->boxes.push_back(box);
    v->owned += n;
    v->sel_uploaded = false;
    drop_graphs(v);
    if (piece_id_out) *piece_id_out = K;
    return MBOIT_OK;
}

mboit_status mboit_render_moments(mboit_volume v, const mboit_view* views, int32_t n_views, const int32_t* pieces,
                                  int32_t n_pieces, int32_t mode, void* moments, void* stream) {
    g_err.clear();
    Range nvtx("mboit_render_moments");
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    if (mode != MBOIT_MOMENTS_PER_PIECE && mode != MBOIT_MOMENTS_REDUCED) return fail(MBOIT_ERR_INVALID_ARG, "unknown mode");
    if (!moments) return fail(MBOIT_ERR_INVALID_ARG, "moments is NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    mb::ViewTable vt;
    if ((st = build_views(views, n_views, vt, slab_bytes_per_px(v->desc.moment_set), v->packet)) != MBOIT_OK) return st;
    std::vector<int32_t> list;
    const uint8_t* mask = nullptr;
    if ((st = select_pieces(v, pieces, n_pieces, list, &mask)) != MBOIT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = claim_stream(v, s)) != MBOIT_OK) return st;
    MB_CUDA(cudaMemsetAsync(&v->d_ctr->samples[0], 0, sizeof(unsigned long long), s));
    if (mode == MBOIT_MOMENTS_REDUCED) {
        MB_CUDA(pass1_batched(v, mask, vt, moments, s));
    } else {
        const int32_t slots = (int32_t)list.size();
        MB_CUDA(check_tables(v, s));
        for (int32_t j = 0; j < slots; ++j) {
            const mb::PieceBox& box = v->boxes[list[j]];
            if (v->kind == MBOIT_AMR)
                MB_CUDA(mb::launch_pass1_piece(v->amr, v->d_tf, v->d_pob, list[j], box, vt, j, slots, moments, v->d_ctr, s));
            else if (v->kind == MBOIT_TET)
                MB_CUDA(mb::launch_pass1_piece(v->tet, v->d_tf, v->d_pob, list[j], box, vt, j, slots, moments, v->d_ctr, s));
            else
                MB_CUDA(mb::launch_pass1_piece(v->grid, v->d_tf, v->d_pob, list[j], box, vt, j, slots, moments, v->d_ctr, s));
        }
    }
    release_stream(v, s);
    return MBOIT_OK;
}

mboit_status mboit_reconstruct_blend(mboit_volume v, const mboit_view* views, int32_t n_views, const int32_t* pieces,
                                     int32_t n_pieces, const void* global_moments, int32_t mode, float* color,
                                     void* stream) {
    g_err.clear();
    Range nvtx("mboit_reconstruct_blend");
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    if (mode != MBOIT_COLOR_PER_PIECE && mode != MBOIT_COLOR_REDUCED && mode != MBOIT_COLOR_RESOLVED)
        return fail(MBOIT_ERR_INVALID_ARG, "unknown mode");
    if (!global_moments || !color) return fail(MBOIT_ERR_INVALID_ARG, "global_moments and color must be non-NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    mb::ViewTable vt;
    if ((st = build_views(views, n_views, vt, slab_bytes_per_px(v->desc.moment_set), v->packet)) != MBOIT_OK) return st;
    std::vector<int32_t> list;
    const uint8_t* mask = nullptr;
    if ((st = select_pieces(v, pieces, n_pieces, list, &mask)) != MBOIT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = claim_stream(v, s)) != MBOIT_OK) return st;
    MB_CUDA(cudaMemsetAsync(&v->d_ctr->samples[1], 0, 2 * sizeof(unsigned long long), s));
    MB_CUDA(cudaMemsetAsync(&v->d_ctr->fp64_pixels, 0, sizeof(unsigned long long), s));
    if (mode == MBOIT_COLOR_PER_PIECE) {
        const int32_t slots = (int32_t)list.size();
        MB_CUDA(check_tables(v, s));
        for (int32_t j = 0; j < slots; ++j) {
            const mb::PieceBox& box = v->boxes[list[j]];
            if (v->kind == MBOIT_AMR)
                MB_CUDA(mb::launch_pass2_piece(v->amr, v->d_tf, v->d_pob, list[j], box, vt, j, slots, global_moments,
                                               color, v->d_ctr, s));
            else if (v->kind == MBOIT_TET)
                MB_CUDA(mb::launch_pass2_piece(v->tet, v->d_tf, v->d_pob, list[j], box, vt, j, slots, global_moments,
                                               color, v->d_ctr, s));
            else
                MB_CUDA(mb::launch_pass2_piece(v->grid, v->d_tf, v->d_pob, list[j], box, vt, j, slots, global_moments,
                                               color, v->d_ctr, s));
        }
    } else {
        const int32_t md = mode == MBOIT_COLOR_RESOLVED ? mb::kColorResolved : mb::kColorReduced;
        MB_CUDA(pass2_batched(v, mask, vt, global_moments, color, md, s));
    }
    release_stream(v, s);
    return MBOIT_OK;
}

mboit_status mboit_composite(mboit_volume v, int32_t op, int32_t width, int32_t height, int32_t n_views,
                             int32_t n_inputs, const void* in, void* out, const void* global_moments, const float* bg,
                             void* stream) {
    g_err.clear();
    Range nvtx("mboit_composite");
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (op != MBOIT_OP_MOMENTS_SUM && op != MBOIT_OP_COLOR_SUM_RESOLVE) return fail(MBOIT_ERR_INVALID_ARG, "unknown op");
    if (n_inputs < 1) return fail(MBOIT_ERR_INVALID_ARG, "n_inputs must be >= 1");
    if (!in || !out) return fail(MBOIT_ERR_INVALID_ARG, "in and out must be non-NULL");
    const bool raw = (v->grid.flags & MBOIT_FLAG_RAW_SUM) != 0;
    if (op == MBOIT_OP_COLOR_SUM_RESOLVE && !raw && !global_moments)
        return fail(MBOIT_ERR_INVALID_ARG, "global_moments is needed to renormalise");
    float4 b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (bg) {
        if (!std::isfinite(bg[0]) || !std::isfinite(bg[1]) || !std::isfinite(bg[2]) || !std::isfinite(bg[3]))
            return fail(MBOIT_ERR_INVALID_ARG, "non-finite background");
        b = make_float4(bg[0], bg[1], bg[2], bg[3]);
    }
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    mb::ViewTable vt;
    mboit_status st = build_images(width, height, n_views, vt, slab_bytes_per_px(v->desc.moment_set));
    if (st != MBOIT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (op == MBOIT_OP_MOMENTS_SUM) {
        MB_CUDA(mb::launch_moments_sum(v->grid, vt, n_inputs, in, out, s));
    } else {
        MB_CUDA(mb::launch_color_resolve(vt, n_inputs, static_cast<const float*>(in), static_cast<float*>(out),
                                         global_moments, b, raw ? 1 : 0, s));
    }
    return MBOIT_OK;
}

mboit_status mboit_render_frame(mboit_volume v, const mboit_view* views, int32_t n_views, void* moments_scratch,
                                float* rgba, void* stream) {
    g_err.clear();
    Range nvtx("mboit_render_frame");
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    if (!moments_scratch || !rgba) return fail(MBOIT_ERR_INVALID_ARG, "moments_scratch and rgba must be non-NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    mb::ViewTable vt;
    if ((st = build_views(views, n_views, vt, slab_bytes_per_px(v->desc.moment_set), v->packet)) != MBOIT_OK) return st;
    std::vector<int32_t> list;
    const uint8_t* mask = nullptr;
    if ((st = select_pieces(v, nullptr, 0, list, &mask)) != MBOIT_OK) return st;
    if ((st = claim_stream(v, static_cast<cudaStream_t>(stream))) != MBOIT_OK) return st;
    // graph key: the view table and the output pointers
    std::vector<char> key(sizeof vt + 2 * sizeof(void*));
    std::memcpy(key.data(), &vt, sizeof vt);
    std::memcpy(key.data() + sizeof vt, &moments_scratch, sizeof(void*));
    std::memcpy(key.data() + sizeof vt + sizeof(void*), &rgba, sizeof(void*));
    cudaGraphExec_t exec = nullptr;
    for (auto& ge : v->graphs)
        if (ge.key == key) exec = ge.exec;
    if (!exec) {
        mb::TileCache tc;
        if ((st = tile_cache(v, vt, tc)) != MBOIT_OK) return st;
        int32_t* d_order = nullptr;
        if (v->tile_order && (st = make_tile_order(v, vt, &d_order)) != MBOIT_OK) return st;
        vt.order = d_order;
        cudaStream_t cs = v->cap_stream;
        MB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(&v->d_ctr->samples[0], 0, 3 * sizeof(unsigned long long), cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(&v->d_ctr->fp64_pixels, 0, sizeof(unsigned long long), cs);
        // external record nodes: the events are recorded each time the graph runs
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(v->frame_ev[0], cs, cudaEventRecordExternal);
        if (v->frame_launches == 1) {
            if (e == cudaSuccess) e = frame_batched(v, mask, vt, moments_scratch, rgba, cs, v->tune1, tc);
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(v->frame_ev[1], cs, cudaEventRecordExternal);
        } else {
            if (e == cudaSuccess) e = pass1_batched(v, mask, vt, moments_scratch, cs, tc);
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(v->frame_ev[1], cs, cudaEventRecordExternal);
            if (e == cudaSuccess) e = pass2_batched(v, mask, vt, moments_scratch, rgba, mb::kColorResolved, cs, tc);
        }
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(v->frame_ev[2], cs, cudaEventRecordExternal);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            cudaFree(d_order);
            return fail(MBOIT_ERR_CUDA, std::string("capturing the frame: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaFree(d_order);
            return fail(MBOIT_ERR_CUDA, std::string("instantiating the frame graph: ") + cudaGetErrorString(e));
        }
        if (v->graphs.size() >= 8) drop_graphs(v);
        v->graphs.push_back(GraphEntry{key, exec, d_order});
    }
    MB_CUDA(cudaGraphLaunch(exec, static_cast<cudaStream_t>(stream)));
    v->frame_timed = true;
    release_stream(v, static_cast<cudaStream_t>(stream));
    return MBOIT_OK;
}

mboit_status mboit_render_frame_multi(const mboit_volume* vols, int32_t n_vols, const mboit_view* views,
                                      const int32_t* view_volume, int32_t n_views, void* moments_scratch, float* rgba,
                                      void* stream) {
    g_err.clear();
    Range nvtx("mboit_render_frame_multi");
    if (!vols || !view_volume || !moments_scratch || !rgba)
        return fail(MBOIT_ERR_INVALID_ARG, "vols, view_volume, moments_scratch and rgba must be non-NULL");
    if (n_vols < 1 || n_vols > mb::kMaxVolumes)
        return fail(MBOIT_ERR_INVALID_ARG, "n_vols must be in [1, " + std::to_string(mb::kMaxVolumes) + "]");
    for (int32_t i = 0; i < n_vols; ++i) {
        const mboit_status st = check_volume(vols[i]);
        if (st != MBOIT_OK) return st;
        const mboit_volume v = vols[i];
        const std::string at = "volume " + std::to_string(i) + ": ";
        if ((v->kind != MBOIT_GRID && v->kind != MBOIT_AMR) || v->desc.moment_set != MBOIT_POWER4 ||
            v->desc.storage != MBOIT_STORE_F32 || (v->desc.flags & MBOIT_FLAG_ADAPTIVE_STEP))
            return fail(MBOIT_ERR_UNSUPPORTED, at + "multi-volume frames take grid or octree volumes with four float32 "
                                                    "power moments and the fixed step");
        if (v->kind != vols[0]->kind) return fail(MBOIT_ERR_INVALID_ARG, at + "the volumes of one frame are of one kind");
        if (v->device != vols[0]->device) return fail(MBOIT_ERR_INVALID_ARG, at + "on another device");
        if (v->tf_host.size() != vols[0]->tf_host.size() ||
            std::memcmp(v->tf_host.data(), vols[0]->tf_host.data(), v->tf_host.size() * sizeof(float4)) != 0)
            return fail(MBOIT_ERR_INVALID_ARG, at + "the volumes of one frame share one transfer function and step");
        for (int32_t j = 0; j < i; ++j)
            if (vols[j] == v) return fail(MBOIT_ERR_INVALID_ARG, at + "listed twice");
    }
    for (int32_t i = 0; i < n_views && views; ++i)
        if (view_volume[i] < 0 || view_volume[i] >= n_vols)
            return fail(MBOIT_ERR_INVALID_ARG, "view_volume[" + std::to_string(i) + "] out of range");
    // every volume's lock, in one global (address) order
    std::vector<mboit_volume> order(vols, vols + n_vols);
    std::sort(order.begin(), order.end(), std::less<mboit_volume>());
    std::vector<std::unique_lock<std::mutex>> locks;
    for (mboit_volume v : order) locks.emplace_back(v->mu);
    const mboit_volume v0 = vols[0];
    DeviceGuard dg(v0->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int32_t i = 0; i < n_vols; ++i) {
        const mboit_status cs = claim_stream(vols[i], s);
        if (cs != MBOIT_OK) return cs;
    }
    mb::ViewTable vt;
    mboit_status st = build_views(views, n_views, vt, slab_bytes_per_px(MBOIT_POWER4), v0->packet);
    if (st != MBOIT_OK) return st;
    const bool amr = v0->kind == MBOIT_AMR;
    mb::GridTable gt;
    mb::AmrTable at;
    std::memset(&gt, 0, sizeof gt);
    std::memset(&at, 0, sizeof at);
    bool vec = true, holes = false;
    for (int32_t i = 0; i < n_vols; ++i) {
        gt.g[i] = vols[i]->grid;
        vec = vec && mb::stage_config_eligible(gt.g[i], 3);
        if (amr) {
            at.a[i] = vols[i]->amr;
            holes = holes || !vols[i]->amr.complete;
        }
    }
    for (int32_t i = 0; i < n_views; ++i) vt.s[i].vol = view_volume[i];
    // the sample cache: rows of every volume's views, counted per volume
    cudaStream_t cs = v0->cap_stream;
    if (!v0->d_rows) MB_CUDA(cudaMalloc(&v0->d_rows, sizeof(unsigned long long)));
    MB_CUDA(cudaMemsetAsync(v0->d_rows, 0, sizeof(unsigned long long), cs));
    for (int32_t i = 0; i < n_vols; ++i) {
        std::vector<mboit_view> mine;
        for (int32_t j = 0; j < n_views; ++j)
            if (view_volume[j] == i) mine.push_back(views[j]);
        if (mine.empty()) continue;
        mb::ViewTable sub;
        if ((st = build_views(mine.data(), (int32_t)mine.size(), sub, slab_bytes_per_px(MBOIT_POWER4), v0->packet)) !=
            MBOIT_OK)
            return st;
        MB_CUDA(mb::launch_tile_rows(gt.g[i], sub, v0->d_rows, cs));
    }
    unsigned long long rows = 0;
    MB_CUDA(cudaMemcpyAsync(&rows, v0->d_rows, sizeof rows, cudaMemcpyDeviceToHost, cs));
    MB_CUDA(cudaStreamSynchronize(cs));
    mb::TileCache tc;
    if ((st = cache_buffers(v0, rows, vt.total_tiles, tc)) != MBOIT_OK) return st;
    MB_CUDA(cudaMemsetAsync(&v0->d_ctr->samples[0], 0, 3 * sizeof(unsigned long long), s));
    MB_CUDA(cudaMemsetAsync(&v0->d_ctr->fp64_pixels, 0, sizeof(unsigned long long), s));
    if (amr) {
        // every octree's index tables checked on this stream first (its error word)
        for (int32_t i = 0; i < n_vols; ++i) MB_CUDA(check_tables(vols[i], s));
        MB_CUDA(mb::launch_pass1_multi_amr(at, v0->d_tf, vt, moments_scratch, v0->d_ctr, s, holes, tc));
        MB_CUDA(mb::launch_pass2_multi_amr(at, v0->d_tf, vt, moments_scratch, rgba, v0->d_ctr, s, holes, tc));
    } else {
        MB_CUDA(mb::launch_pass1_multi(gt, v0->d_tf, vt, moments_scratch, v0->d_ctr, s, vec, tc));
        MB_CUDA(mb::launch_pass2_multi(gt, v0->d_tf, vt, moments_scratch, rgba, v0->d_ctr, s, vec, tc));
    }
    v0->frame_timed = false;
    for (int32_t i = 0; i < n_vols; ++i) release_stream(vols[i], s);
    return MBOIT_OK;
}

mboit_status mboit_render_frame_host(mboit_volume v, const float* field_host, const mboit_view* views, int32_t n_views,
                                     void* moments_scratch, float* rgba_device, float* rgba_host, void* stream) {
    g_err.clear();
    Range nvtx("mboit_render_frame_host");
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    if (!field_host || !rgba_host || !rgba_device) return fail(MBOIT_ERR_INVALID_ARG, "NULL buffer");
    mb::ViewTable vt;
    if ((st = build_views(views, n_views, vt, slab_bytes_per_px(v->desc.moment_set), v->packet)) != MBOIT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lk(v->mu);
        if ((st = claim_stream(v, s)) != MBOIT_OK) return st;
    }
    {
        DeviceGuard dg(v->device);
        if (v->kind == MBOIT_TET) {
            // vertex values live in the vertex records: stage, then scatter
            MB_CUDA(cudaMemcpyAsync(v->d_tvals, field_host, v->field_bytes, cudaMemcpyHostToDevice, s));
            MB_CUDA(mb::launch_tet_values(v->d_tcorners, v->d_tcells, v->desc.n_tets, v->d_tvals, s));
        } else {
            float* dst = const_cast<float*>(v->kind == MBOIT_AMR ? v->amr.values : v->grid.field);
            MB_CUDA(cudaMemcpyAsync(dst, field_host, v->field_bytes, cudaMemcpyHostToDevice, s));
        }
    }
    if ((st = mboit_render_frame(v, views, n_views, moments_scratch, rgba_device, stream)) != MBOIT_OK) return st;
    int64_t floats = 0;
    for (int i = 0; i < n_views; ++i) floats += (int64_t)4 * views[i].width * views[i].height;
    DeviceGuard dg(v->device);
    MB_CUDA(cudaMemcpyAsync(rgba_host, rgba_device, (size_t)floats * sizeof(float), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    return MBOIT_OK;
}

mboit_status mboit_synchronize(mboit_volume v, void* stream) {
    g_err.clear();
    Range nvtx("mboit_synchronize");
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    DeviceGuard dg(v->device);
    MB_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int32_t err = 0;
    MB_CUDA(cudaMemcpy(&err, &v->d_ctr->error, sizeof err, cudaMemcpyDeviceToHost));
    if (err == 0) return MBOIT_OK;
    MB_CUDA(cudaMemset(&v->d_ctr->error, 0, sizeof err));   // reported once
    if (err & mb::kErrTmaTimeout)
        return fail(MBOIT_ERR_TIMEOUT, "a TMA window load did not complete within its wait limit (code " +
                                           std::to_string(err) + "); the render stopped early and its images are not valid");
    std::string what;
    if (err & mb::kErrLeafId) what += " an octree finest-brick map entry is not a leaf id;";
    if (err & mb::kErrTetId) what += " a mesh face-neighbour or bin-list entry is not a tet id;";
    if (err & mb::kErrBinRange) what += " a mesh bin's range leaves the bin list;";
    return fail(MBOIT_ERR_DEVICE_ASSERT, "kernel-side checks failed (code " + std::to_string(err) + "):" + what +
                                             " the accesses were skipped; the frame's images are not valid");
}

mboit_status mboit_debug_corrupt(mboit_volume v, int32_t what) {
    g_err.clear();
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    if (what == 1) {
        if (v->kind != MBOIT_AMR) return fail(MBOIT_ERR_INVALID_ARG, "what = 1 needs an octree volume");
        // every finest brick maps to no leaf (a single entry could go unread:
        // a lane inside a leaf's box does not consult the map)
        const int64_t f = v->amr.fdim;
        std::vector<int32_t> bad((size_t)(f * f * f), v->amr.n_leaves + 7);
        MB_CUDA(cudaMemcpy(v->d_fmap, bad.data(), bad.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    } else if (what == 2) {
        if (v->kind != MBOIT_TET) return fail(MBOIT_ERR_INVALID_ARG, "what = 2 needs a mesh volume");
        // every tet's neighbour across face 0 becomes no tet
        std::vector<int4> nb((size_t)v->tet.n_tets);
        MB_CUDA(cudaMemcpy(nb.data(), v->d_tnbrs, nb.size() * sizeof(int4), cudaMemcpyDeviceToHost));
        for (auto& n : nb)
            if (n.x >= 0) n.x = v->tet.n_tets + 7;
        MB_CUDA(cudaMemcpy(v->d_tnbrs, nb.data(), nb.size() * sizeof(int4), cudaMemcpyHostToDevice));
    } else if (what == 3) {
        if (v->kind != MBOIT_GRID) return fail(MBOIT_ERR_INVALID_ARG, "what = 3 needs a grid volume");
        // TMA window loads arm their barrier and issue no copy: every wait runs out
        v->grid.flags |= mb::kFlagDebugNoCopy;
    } else {
        return fail(MBOIT_ERR_INVALID_ARG, "what must be 1 (octree map), 2 (mesh neighbours) or 3 (grid TMA loads)");
    }
    drop_graphs(v);
    return MBOIT_OK;
}

mboit_status mboit_get_stats(mboit_volume v, mboit_stats* out) {
    g_err.clear();
    if (!v || !out) return fail(MBOIT_ERR_INVALID_ARG, "volume and out must be non-NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    MB_CUDA(cudaDeviceSynchronize());
    mb::Counters c;
    MB_CUDA(cudaMemcpy(&c, v->d_ctr, sizeof c, cudaMemcpyDeviceToHost));
    out->samples_pass1 = (int64_t)c.samples[0];
    out->samples_pass2 = (int64_t)c.samples[1];
    out->singular_pixels = (int64_t)c.singular;
    out->n_pieces = (int32_t)v->boxes.size();
    out->device = v->device;
    out->tuning_pass1 = v->tune1;
    out->tuning_pass2 = v->tune2;
    out->sortlast_segments = v->sl_segments;
    out->sortlast_max_segments = c.max_segments;
    out->fp64_pixels = (int32_t)std::min<unsigned long long>(c.fp64_pixels, 0x7fffffffull);
    out->packet = v->packet;
    out->frame_launches = v->frame_launches;
    out->tile_order = v->tile_order;
    out->frame_pass1_ms = out->frame_pass2_ms = -1.0f;
    if (v->frame_timed && (cudaEventElapsedTime(&out->frame_pass1_ms, v->frame_ev[0], v->frame_ev[1]) != cudaSuccess ||
                           cudaEventElapsedTime(&out->frame_pass2_ms, v->frame_ev[1], v->frame_ev[2]) != cudaSuccess)) {
        cudaGetLastError();
        out->frame_pass1_ms = out->frame_pass2_ms = -1.0f;
    }
    return MBOIT_OK;
}

mboit_status mboit_render_sortlast(mboit_volume v, const mboit_view* views, int32_t n_views, float* rgba,
                                   int32_t* segments_per_pixel, void* stream) {
    g_err.clear();
    Range nvtx("mboit_render_sortlast");
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    if (!rgba) return fail(MBOIT_ERR_INVALID_ARG, "rgba is NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    mb::ViewTable vt;
    if ((st = build_views(views, n_views, vt, slab_bytes_per_px(v->desc.moment_set), v->packet)) != MBOIT_OK) return st;
    int64_t total_px = 0;
    for (int i = 0; i < n_views; ++i) total_px += (int64_t)views[i].width * views[i].height;
    const int32_t K = (int32_t)v->boxes.size();
    const size_t slots_px = (size_t)K * (size_t)total_px;
    const size_t nb = (size_t)((total_px + 1023) / 1024);
    MB_CUDA(ensure_capacity(v->sl_counts, v->cap_counts, slots_px));
    MB_CUDA(ensure_capacity(v->sl_starts, v->cap_starts, slots_px));
    MB_CUDA(ensure_capacity(v->sl_totals, v->cap_totals, (size_t)total_px));
    MB_CUDA(ensure_capacity(v->sl_base, v->cap_base, (size_t)total_px + 1));
    MB_CUDA(ensure_capacity(v->sl_bsum, v->cap_bsum, nb));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = claim_stream(v, s)) != MBOIT_OK) return st;
    MB_CUDA(cudaMemsetAsync(&v->d_ctr->segments, 0, sizeof(unsigned long long) + sizeof(int32_t), s));
    MB_CUDA(check_tables(v, s));
    auto march = [&](bool fill, int32_t p) {
        const int64_t* st = fill ? v->sl_starts : nullptr;
        int32_t* key = fill ? v->sl_key : nullptr;
        float4* col = fill ? v->sl_col : nullptr;
        if (v->kind == MBOIT_AMR)
            return mb::launch_sortlast_march(fill, v->amr, v->d_tf, v->d_pob, p, v->boxes[p], vt, p, K, v->sl_counts, st,
                                             key, col, s);
        if (v->kind == MBOIT_TET)
            return mb::launch_sortlast_march(fill, v->tet, v->d_tf, v->d_pob, p, v->boxes[p], vt, p, K, v->sl_counts, st,
                                             key, col, s);
        return mb::launch_sortlast_march(fill, v->grid, v->d_tf, v->d_pob, p, v->boxes[p], vt, p, K, v->sl_counts, st,
                                         key, col, s);
    };
    for (int32_t p = 0; p < K; ++p) MB_CUDA(march(false, p));
    MB_CUDA(mb::launch_sortlast_offsets(vt, K, v->sl_counts, v->sl_totals, v->sl_base, v->sl_bsum, v->sl_starts,
                                        total_px, s));
    int64_t total = 0;
    MB_CUDA(cudaMemcpyAsync(&total, v->sl_base + total_px, sizeof total, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    MB_CUDA(ensure_capacity(v->sl_key, v->cap_seg, (size_t)total));
    MB_CUDA(ensure_capacity(v->sl_col, v->cap_col, (size_t)total));
    for (int32_t p = 0; p < K; ++p) MB_CUDA(march(true, p));
    MB_CUDA(mb::launch_sortlast_blend(v->sl_base, v->sl_key, v->sl_col, rgba, total_px, v->d_ctr, s));
    if (segments_per_pixel)
        MB_CUDA(cudaMemcpyAsync(segments_per_pixel, v->sl_totals, (size_t)total_px * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, s));
    v->sl_segments = total;
    release_stream(v, s);
    return MBOIT_OK;
}

mboit_status mboit_set_tuning(mboit_volume v, int32_t pass1, int32_t pass2) {
    g_err.clear();
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (v->kind != MBOIT_GRID && (pass1 != 0 || pass2 != 0))
        return fail(MBOIT_ERR_INVALID_ARG, "octree and mesh volumes have one configuration (0)");
    if (v->kind == MBOIT_GRID && (!config_usable(v, pass1) || !config_usable(v, pass2)))
        return fail(MBOIT_ERR_INVALID_ARG, "tuning must be in [0, " + std::to_string(mb::kNumStageConfigs - 1) +
                                               "]; 2-6 need dims[0] % 4 == 0 and a 16-byte aligned field, 5 and 6 "
                                               "also the field's tensor maps (TMA)");
    std::lock_guard<std::mutex> lk(v->mu);
    v->tune1 = pass1;
    v->tune2 = pass2;
    drop_graphs(v);
    return MBOIT_OK;
}

mboit_status mboit_set_frame_launches(mboit_volume v, int32_t launches) {
    g_err.clear();
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (launches != 1 && launches != 2) return fail(MBOIT_ERR_INVALID_ARG, "launches must be 1 or 2");
    if (launches == 1 && v->desc.moment_set != MBOIT_POWER4)
        return fail(MBOIT_ERR_UNSUPPORTED, "the one-launch frame covers four power moments");
    std::lock_guard<std::mutex> lk(v->mu);
    v->frame_launches = launches;
    drop_graphs(v);
    return MBOIT_OK;
}

mboit_status mboit_set_tile_order(mboit_volume v, int32_t order) {
    g_err.clear();
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (order != 0 && order != 1) return fail(MBOIT_ERR_INVALID_ARG, "order must be 0 (tile order) or 1 (longest first)");
    std::lock_guard<std::mutex> lk(v->mu);
    v->tile_order = order;
    drop_graphs(v);
    return MBOIT_OK;
}

mboit_status mboit_set_packet(mboit_volume v, int32_t packet) {
    g_err.clear();
    if (!v) return fail(MBOIT_ERR_INVALID_ARG, "volume is NULL");
    if (packet != MBOIT_PACKET_8X4 && packet != MBOIT_PACKET_4X8) return fail(MBOIT_ERR_INVALID_ARG, "unknown packet");
    std::lock_guard<std::mutex> lk(v->mu);
    v->packet = packet;
    drop_graphs(v);
    return MBOIT_OK;
}

}  // extern "C"

namespace {

// The autotuner's choices, kept per process by configuration: the volume's
// kind, shape, sampling and moment format, its piece count, which window
// configurations it can take, the views, and the device's SM count.  The
// field's values are not part of the key (they change the work little).
struct Tuned {
    int32_t tune1, tune2, packet, launches, order;
};
std::mutex g_tuned_mu;
std::map<std::vector<char>, Tuned> g_tuned;

std::vector<char> tuning_key(mboit_volume v, const mboit_view* views, int32_t n_views) {
    std::vector<char> k;
    auto put = [&](const void* p, size_t n) { k.insert(k.end(), (const char*)p, (const char*)p + n); };
    const mboit_volume_desc& d = v->desc;
    const int64_t ints[] = {d.kind, d.dims[0], d.dims[1], d.dims[2], d.brick_log2, d.moment_set, d.storage,
                            (int64_t)d.flags, d.n_leaves, d.max_level, d.n_verts, d.n_tets,
                            (int64_t)v->boxes.size(), n_views};
    put(ints, sizeof ints);
    put(&d.step, sizeof d.step);
    int32_t usable = 0;
    for (int c = 0; c < mb::kNumStageConfigs; ++c)
        if (v->kind == MBOIT_GRID && config_usable(v, c)) usable |= 1 << c;
    put(&usable, sizeof usable);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v->device);
    put(&sms, sizeof sms);
    put(views, sizeof(mboit_view) * (size_t)n_views);
    return k;
}

}  // namespace

extern "C" {

void mboit_clear_tuning_cache(void) {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned.clear();
}

mboit_status mboit_autotune(mboit_volume v, const mboit_view* views, int32_t n_views, void* moments_scratch, float* rgba,
                            void* stream, int32_t* chosen) {
    g_err.clear();
    Range nvtx("mboit_autotune");
    mboit_status st = check_volume(v);
    if (st != MBOIT_OK) return st;
    if (!moments_scratch || !rgba) return fail(MBOIT_ERR_INVALID_ARG, "moments_scratch and rgba must be non-NULL");
    if (!views || n_views < 1 || n_views > mb::kMaxViews)
        return fail(MBOIT_ERR_INVALID_ARG, "n_views must be in [1, " + std::to_string(mb::kMaxViews) + "]");
    std::lock_guard<std::mutex> lk(v->mu);
    DeviceGuard dg(v->device);
    const std::vector<char> key = tuning_key(v, views, n_views);
    {
        std::lock_guard<std::mutex> tl(g_tuned_mu);
        const auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            const Tuned& t = it->second;
            v->tune1 = t.tune1;
            v->tune2 = t.tune2;
            v->packet = t.packet;
            v->frame_launches = t.launches;
            v->tile_order = t.order;
            drop_graphs(v);
            if (chosen) {
                chosen[0] = t.tune1;
                chosen[1] = t.tune2;
                chosen[2] = t.packet;
            }
            return MBOIT_OK;
        }
    }
    std::vector<int32_t> list;
    const uint8_t* mask = nullptr;
    if ((st = select_pieces(v, nullptr, 0, list, &mask)) != MBOIT_OK) return st;
    const bool grid = v->kind == MBOIT_GRID;  // octrees and meshes have one window configuration
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = claim_stream(v, s)) != MBOIT_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MB_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(MBOIT_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
    }
    // times `launch` (one warm-up, then 3 runs) in ms
    auto time3 = [&](auto&& launch, float& ms) {
        ce = launch();
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && ce == cudaSuccess; ++r) ce = launch();
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        ms = 3.0e38f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    };
    // Per packet: the split calls' configurations (pass 1, then pass 2 on the
    // fastest pass 1's moments); with four power moments also the frame's
    // form on that packet (two launches with those configurations against
    // one launch in each eligible configuration, all with the frame's sample
    // cache).  The packet whose frame is fastest wins (without frame forms:
    // whose split calls are).
    float best_total = 3.0e38f;
    int best[3] = {v->tune1, v->tune2, v->packet};
    int launches = v->frame_launches, order = v->tile_order;
    const bool forms = v->desc.moment_set == MBOIT_POWER4;
    for (int packet = MBOIT_PACKET_8X4; packet <= MBOIT_PACKET_4X8 && ce == cudaSuccess; ++packet) {
        mb::ViewTable vt;
        if ((st = build_views(views, n_views, vt, slab_bytes_per_px(v->desc.moment_set), packet)) != MBOIT_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        float best_ms[2] = {3.0e38f, 3.0e38f};
        int pick[2] = {0, 0};
        for (int pass = 0; pass < 2 && ce == cudaSuccess; ++pass) {
            for (int cfg = 0; cfg < mb::kNumStageConfigs && ce == cudaSuccess; ++cfg) {
                if (grid ? !config_usable(v, cfg) : cfg != 0) continue;
                float ms;
                time3([&]() {
                    if (!grid)
                        return pass == 0 ? pass1_batched(v, mask, vt, moments_scratch, s)
                                         : pass2_batched(v, mask, vt, moments_scratch, rgba, mb::kColorResolved, s);
                    return pass == 0 ? mb::launch_pass1_fused(v->grid, v->d_tf, mask, vt, moments_scratch, v->d_ctr, s, cfg,
                                                              mb::TileCache{}, field_map_of(v, cfg))
                                     : mb::launch_pass2_fused(v->grid, v->d_tf, mask, vt, moments_scratch, rgba,
                                                              mb::kColorResolved, v->d_ctr, s, cfg);
                }, ms);
                if (ce == cudaSuccess && ms < best_ms[pass]) {
                    best_ms[pass] = ms;
                    pick[pass] = cfg;
                }
            }
            // pass 2 is timed on the moments of the fastest pass 1
            if (pass == 0 && ce == cudaSuccess)
                ce = grid ? mb::launch_pass1_fused(v->grid, v->d_tf, mask, vt, moments_scratch, v->d_ctr, s, pick[0],
                                                   mb::TileCache{}, field_map_of(v, pick[0]))
                          : pass1_batched(v, mask, vt, moments_scratch, s);
        }
        float total = best_ms[0] + best_ms[1];
        int form_launches = launches, cfg1 = pick[0], form_order = 0;
        if (ce == cudaSuccess && forms) {
            mb::TileCache tc;
            st = tile_cache(v, vt, tc);
            if (st != MBOIT_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            if (tc.vals) {
                // form 0: two launches; form c + 1: one launch in configuration c
                auto frame = [&](int form, const mb::ViewTable& t) {
                    if (form > 0) return frame_batched(v, mask, t, moments_scratch, rgba, s, form - 1, tc);
                    if (!grid) {
                        cudaError_t e = pass1_batched(v, mask, t, moments_scratch, s, tc);
                        return e != cudaSuccess ? e
                                                : pass2_batched(v, mask, t, moments_scratch, rgba, mb::kColorResolved,
                                                                s, tc);
                    }
                    cudaError_t e = mb::launch_pass1_fused(v->grid, v->d_tf, mask, t, moments_scratch, v->d_ctr, s,
                                                           pick[0], tc, field_map_of(v, pick[0]));
                    return e != cudaSuccess ? e
                                            : mb::launch_pass2_fused(v->grid, v->d_tf, mask, t, moments_scratch, rgba,
                                                                     mb::kColorResolved, v->d_ctr, s, pick[1], tc);
                };
                total = 3.0e38f;
                int best_form = 0;
                for (int form = 0; form <= mb::kNumStageConfigs && ce == cudaSuccess; ++form) {
                    if (form > 0 && (grid ? !config_usable(v, form - 1) : form != 1)) continue;
                    float ms;
                    time3([&]() { return frame(form, vt); }, ms);
                    if (ce == cudaSuccess && ms < total) {
                        total = ms;
                        best_form = form;
                        form_launches = form == 0 ? 2 : 1;
                        cfg1 = form == 0 ? pick[0] : form - 1;
                    }
                }
                // the fastest form again with its ray tiles dequeued longest first
                int32_t* d_order = nullptr;
                if (ce == cudaSuccess && (st = make_tile_order(v, vt, &d_order)) != MBOIT_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st;
                }
                if (ce == cudaSuccess) {
                    mb::ViewTable vto = vt;
                    vto.order = d_order;
                    float ms;
                    time3([&]() { return frame(best_form, vto); }, ms);
                    if (ce == cudaSuccess && ms < total) {
                        total = ms;
                        form_order = 1;
                    }
                }
                cudaFree(d_order);
            }
        }
        if (ce == cudaSuccess && total < best_total) {
            best_total = total;
            best[0] = cfg1;
            best[1] = pick[1];
            best[2] = packet;
            launches = form_launches;
            order = form_order;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return fail(MBOIT_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
    v->frame_launches = launches;
    v->tile_order = order;
    v->tune1 = best[0];
    v->tune2 = best[1];
    v->packet = best[2];
    {
        std::lock_guard<std::mutex> tl(g_tuned_mu);
        g_tuned[key] = Tuned{best[0], best[1], best[2], launches, order};
    }
    release_stream(v, s);
    drop_graphs(v);
    if (chosen) {
        chosen[0] = best[0];
        chosen[1] = best[1];
        chosen[2] = best[2];
    }
    return MBOIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Pass 1 with no device allocation: scratch in a fixed device array.

namespace {

constexpr size_t kNoallocMaxBricks = size_t(1) << 20;
constexpr size_t kNoallocTfOff = 256;
constexpr size_t kNoallocSelOff = kNoallocTfOff + 256 * sizeof(float4);
constexpr size_t kNoallocBytes = kNoallocSelOff + kNoallocMaxBricks;
static_assert(sizeof(mb::Counters) <= kNoallocTfOff, "counters must fit their slot");

// Work-queue head, sample counters, transfer function and brick mask of
// mboit_render_moments_noalloc.  Host code must not use its name as an
// address: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The converted transfer function, passed by value: the launch copies it, so
// no host buffer has to outlive the call.
struct NoallocTf {
    float4 e[256];
};
static_assert(sizeof(NoallocTf) <= 4096, "kernel parameters are limited to 4 KB");

// Writes the transfer function into its slot of the scratch array and
// clears the work-queue head and counters (the array keeps the previous
// call's contents).
__global__ void __launch_bounds__(256) k_noalloc_setup(const NoallocTf tf) {
    float4* dst = reinterpret_cast<float4*>(g_noalloc_scratch + kNoallocTfOff);
    for (int i = threadIdx.x; i < 256; i += blockDim.x) dst[i] = tf.e[i];
    uint32_t* ctr = reinterpret_cast<uint32_t*>(g_noalloc_scratch);
    for (int i = threadIdx.x; i < (int)(sizeof(mb::Counters) / sizeof(uint32_t)); i += blockDim.x) ctr[i] = 0u;
}

}  // namespace

extern "C" mboit_status mboit_render_moments_noalloc(const mboit_volume_desc* d, const uint8_t* brick_selected,
                                                     const mboit_view* views, int32_t n_views, void* moments,
                                                     void* stream) {
    g_err.clear();
    if (!d || !moments) return fail(MBOIT_ERR_INVALID_ARG, "desc and moments must be non-NULL");
    if (d->kind != MBOIT_GRID) return fail(MBOIT_ERR_UNSUPPORTED, "only MBOIT_GRID volumes are implemented");
    if (d->moment_set != MBOIT_POWER4 || d->storage != MBOIT_STORE_F32)
        return fail(MBOIT_ERR_UNSUPPORTED, "only float32 power moments are implemented");
    if (d->flags & ~(MBOIT_FLAG_RAW_SUM | MBOIT_FLAG_DETERMINISTIC | MBOIT_FLAG_FP64_SETUP))
        return fail(MBOIT_ERR_INVALID_ARG, "unknown flag bits");
    if (!d->field) return fail(MBOIT_ERR_INVALID_ARG, "field must be non-NULL");
    for (int c = 0; c < 3; ++c)
        if (d->dims[c] < 2 || d->dims[c] > (1 << 20)) return fail(MBOIT_ERR_INVALID_ARG, "dims must be in [2, 2^20]");
    if (d->brick_log2 < 0 || d->brick_log2 > 7) return fail(MBOIT_ERR_INVALID_ARG, "brick_log2 must be in [0, 7]");
    mboit_status st = check_sampling(d);
    if (st != MBOIT_OK) return st;
    const int B = 1 << d->brick_log2;
    const int64_t nbx = (d->dims[0] - 1 + B - 1) / B, nby = (d->dims[1] - 1 + B - 1) / B,
                  nbz = (d->dims[2] - 1 + B - 1) / B;
    const int64_t nbricks = nbx * nby * nbz;
    if (nbricks > (int64_t)kNoallocMaxBricks)
        return fail(MBOIT_ERR_INVALID_ARG, "the volume has " + std::to_string(nbricks) +
                                               " bricks; the allocation-free pass 1 handles at most " +
                                               std::to_string(kNoallocMaxBricks) + " (use a larger brick_log2)");
    NoallocTf tf;
    st = convert_tf(d, tf.e);
    if (st != MBOIT_OK) return st;
    mb::ViewTable vt;
    st = build_views(views, n_views, vt);
    if (st != MBOIT_OK) return st;

    int dev = 0;
    MB_CUDA(cudaGetDevice(&dev));
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, d->field) != cudaSuccess ||
        (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) || attr.device != dev) {
        cudaGetLastError();
        return fail(MBOIT_ERR_INVALID_ARG, "field must be a device pointer on the current device");
    }
    // The array's address in the current device's context, looked up on every
    // call (a lookup, no allocation), so that a context created anew after a
    // cudaDeviceReset is served its own copy.
    void* p = nullptr;
    const cudaError_t ge = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (ge != cudaSuccess || !p)
        return fail(MBOIT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(ge));
    unsigned char* scratch = static_cast<unsigned char*>(p);

    mb::GridD g{};
    fill_grid(d, g);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mb::Counters* ctr = reinterpret_cast<mb::Counters*>(scratch);
    float4* tf_dev = reinterpret_cast<float4*>(scratch + kNoallocTfOff);
    uint8_t* sel_dev = brick_selected ? scratch + kNoallocSelOff : nullptr;
    k_noalloc_setup<<<1, 256, 0, s>>>(tf);
    MB_CUDA(cudaGetLastError());
    if (sel_dev) MB_CUDA(cudaMemcpyAsync(sel_dev, brick_selected, (size_t)nbricks, cudaMemcpyHostToDevice, s));
    MB_CUDA(mb::launch_pass1_fused(g, tf_dev, sel_dev, vt, moments, ctr, s));
    return MBOIT_OK;
}
