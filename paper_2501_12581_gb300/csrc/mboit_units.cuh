// Kernel templates of the octree and tetrahedral-mesh passes and of the plain
// per-piece and sort-last marches of every volume kind (sm_103a), shared by
// mboit_units.cu (launchers; four power and trigonometric moments) and
// mboit_units_power.cu (the 6- and 8-power-moment instantiations, compiled in
// parallel).  Internal: an unnamed namespace per translation unit.
//
// The fused octree / mesh passes are persistent like the grid's (one warp =
// one 8 x 4 ray tile from the work queue); the octree finds each lattice
// point's leaf in a finest-brick map, the mesh walks between face neighbours
// with exact predicates.  The per-piece kernels are the plain form: one
// launch per piece, rays clipped to the piece's box, non-owned units skipped,
// one image per piece.
#pragma once
#include <type_traits>
#include "mboit_common.cuh"

namespace mb {
namespace {

// ------------------------------------------------------------------------
// plain per-piece passes

// Sampling units: the bricks of a grid or the leaves of an octree.  For a
// point inside the domain: its unit (-1: none), the trilinear value there,
// and the unit's box (for skipping units a piece does not own).
__device__ __forceinline__ const GridD& common(const GridD& g) { return g; }
__device__ __forceinline__ const GridD& common(const AmrD& a) { return a.g; }
__device__ __forceinline__ const GridD& common(const TetD& m) { return m.g; }

__device__ __forceinline__ int unit_of(const GridD& g, const float p[3]) {
    const int ix = (int)p[0], iy = (int)p[1], iz = (int)p[2];
    return ((iz >> g.brick_log2) * g.nby + (iy >> g.brick_log2)) * g.nbx + (ix >> g.brick_log2);
}

__device__ __forceinline__ float unit_value(const GridD& g, const float p[3], int) {
    const int ix = (int)p[0], iy = (int)p[1], iz = (int)p[2];
    const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * (size_t)g.ny;
    const float* __restrict__ c = g.field + (size_t)iz * sz + (size_t)iy * sy + (size_t)ix;
    return trilinear8(__ldg(c), __ldg(c + 1), __ldg(c + sy), __ldg(c + sy + 1), __ldg(c + sz), __ldg(c + sz + 1),
                      __ldg(c + sz + sy), __ldg(c + sz + sy + 1), p[0] - (float)ix, p[1] - (float)iy, p[2] - (float)iz);
}

__device__ __forceinline__ void unit_box(const GridD& g, const float p[3], int, float lo[3], float& size) {
    size = (float)(1 << g.brick_log2);
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = floorf(p[c] / size) * size;
}

// The leaf of an in-domain point from the finest-brick map (-1: a hole).
// Every entry was checked to be a leaf id or -1 before the kernel ran (see
// tables_bad).
__device__ __forceinline__ int unit_of(const AmrD& a, const float p[3]) {
    const int bl = a.g.brick_log2;
    const int fx = (int)p[0] >> bl, fy = (int)p[1] >> bl, fz = (int)p[2] >> bl;
    return __ldg(a.fmap + ((size_t)fz * a.fdim + fy) * (size_t)a.fdim + fx);
}

// True when the table checks of this render (k_check_* in mboit_kernels.cu,
// launched before the passes on the same stream) found an entry out of range
// in the volume's tables; every kernel that reads those tables then returns
// at once, so no out-of-range index is ever used.  Grids have no such tables.
__device__ __forceinline__ bool tables_bad(const GridD&) { return false; }
__device__ __forceinline__ bool tables_bad(const AmrD& a) { return *(volatile const int32_t*)a.err != 0; }
__device__ __forceinline__ bool tables_bad(const TetD& m) { return *(volatile const int32_t*)m.err != 0; }

// Trilinear value in leaf `leaf` with origin lo (finest cells) and inverse
// cell size inv_h.  Local coordinates (p - origin) / h are exact in float32
// (h a power of two, |p - origin| below the leaf size), so cells match the
// oracle's.
__device__ __forceinline__ float leaf_value(const AmrD& a, const float p[3], int leaf, const float lo[3], float inv_h) {
    const float qx = (p[0] - lo[0]) * inv_h, qy = (p[1] - lo[1]) * inv_h, qz = (p[2] - lo[2]) * inv_h;
    const int cx = min((int)qx, a.nv - 2), cy = min((int)qy, a.nv - 2), cz = min((int)qz, a.nv - 2);
    const int nv = a.nv;
    const float* __restrict__ c = a.values + (size_t)leaf * nv * nv * nv + (cz * nv + cy) * nv + cx;
    const int sy = nv, sz = nv * nv;
    return trilinear8(__ldg(c), __ldg(c + 1), __ldg(c + sy), __ldg(c + sy + 1), __ldg(c + sz), __ldg(c + sz + 1),
                      __ldg(c + sz + sy), __ldg(c + sz + sy + 1), qx - (float)cx, qy - (float)cy, qz - (float)cz);
}

__device__ __forceinline__ float leaf_inv_h(const AmrD& a, int level) {
    return __int_as_float((127 - (a.max_level - level)) << 23);  // 2^-(max_level - level)
}

__device__ __forceinline__ float unit_value(const AmrD& a, const float p[3], int leaf) {
    const int4 L = __ldg(a.leaves + leaf);
    const float lo[3] = {(float)L.x, (float)L.y, (float)L.z};
    return leaf_value(a, p, leaf, lo, leaf_inv_h(a, L.w));
}

// The leaf of a lane's previous sample: a sample inside its box (half-open,
// in finest cells, like the finest-brick map it stands for) skips the map and
// the leaf table, two dependent loads.  u: the leaf, or -1 where the box
// holds no selected leaf (outside every leaf, or a leaf of a piece left out).
struct LeafCache {
    int u = -1, shift = 0;
    float lo[3] = {0.0f, 0.0f, 0.0f}, size = 0.0f, inv_h = 0.0f;   // size 0: no box
    __device__ __forceinline__ bool holds(const float p[3]) const {
        // p - lo is exact (both below 2^24, p >= lo in the test that matters)
        return p[0] >= lo[0] && p[0] - lo[0] < size && p[1] >= lo[1] && p[1] - lo[1] < size && p[2] >= lo[2] &&
               p[2] - lo[2] < size;
    }
    // Looks p up; returns its selected leaf or -1.
    template <bool kSel>
    __device__ __forceinline__ int find(const AmrD& a, const uint8_t* __restrict__ sel, const float p[3]) {
        if (holds(p)) return u;
        const int v = unit_of(a, p);
        if (v < 0) {
            // no leaf: forget the box, so the next sample looks up again
            u = -1;
            size = 0.0f;
            return -1;
        }
        const int4 L = __ldg(a.leaves + v);
        size = (float)((1 << a.g.brick_log2) << (a.max_level - L.w));
        lo[0] = (float)L.x; lo[1] = (float)L.y; lo[2] = (float)L.z;
        inv_h = leaf_inv_h(a, L.w);
        shift = a.max_level - L.w;
        u = (kSel && sel && !__ldg(sel + v)) ? -1 : v;
        return u;
    }
};

__device__ __forceinline__ void unit_box(const AmrD& a, const float[3], int leaf, float lo[3], float& size) {
    const int4 L = __ldg(a.leaves + leaf);
    size = (float)((1 << a.g.brick_log2) << (a.max_level - L.w));
    lo[0] = (float)L.x;
    lo[1] = (float)L.y;
    lo[2] = (float)L.z;
}

// Next lattice index worth testing after point k fell in a unit the piece
// does not own: the ray's exit from that unit's box, pulled back by a
// padding that covers float32 position rounding, and by one lattice step.
template <class V>
__device__ __forceinline__ int skip_unit(const V& vol, int unit, const float o[3], const float d[3], float t, int k) {
    const GridD& g = common(vol);
    const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
    float lo[3], size;
    unit_box(vol, p, unit, lo, size);
    float t_exit = 3.0e38f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0f) continue;
        const float face = d[c] > 0.0f ? lo[c] + size : lo[c];
        const float inv = 1.0f / d[c];
        const float tc = (face - o[c]) * inv;
        const float pad = (fabsf(o[c]) + fabsf(face) + 1.0f) * 3.814697265625e-06f * fabsf(inv);
        t_exit = fmin_(t_exit, tc - pad);
    }
    const float kn = ceilf(t_exit / g.step - 0.5f) - 1.0f;
    if (!(kn > (float)(k + 1))) return k + 1;
    return kn > 4194303.0f ? 4194304 : (int)kn;
}

// Adaptive dyadic step of octrees: the level shift max_level - L of unit u's
// leaf, whose points count only at multiples of 2^shift (-1: every point
// counts, as on grids or without MBOIT_FLAG_ADAPTIVE_STEP).
__device__ __forceinline__ int step_shift(const GridD&, int) { return -1; }
__device__ __forceinline__ int step_shift(const AmrD& a, int u) {
    return (a.g.flags & kFlagAdaptiveStep) ? a.max_level - __ldg(a.leaves + u).w : -1;
}
// Mantissa bits that carry the level shift of an adaptive-step sample.
__device__ __forceinline__ int shift_tag_mask(const GridD&) { return 0; }
__device__ __forceinline__ int shift_tag_mask(const AmrD& a) { return tag_mask(a.max_level); }

// Next lattice index to test after point k of unit u, which is not on the
// unit's nested lattice of 2^shift steps: its next lattice point, or the
// first index that may lie outside the unit (never beyond k_end).
template <class V>
__device__ __forceinline__ int next_on_lattice(const V& vol, int u, int shift, const float o[3], const float d[3],
                                               float t, int k, int k_end) {
    const int kn = min((k | ((1 << shift) - 1)) + 1, skip_unit(vol, u, o, d, t, k));
    return min(kn, k_end);
}

// Whether pass 2 from the cache must test its rows for unsampled points
// (NaN).  Octrees launch the kSel kernels when a piece is left out or when a
// finest brick has no leaf (holes; sel is then NULL), so an unchecked octree
// kernel sees every in-domain point sampled; meshes are always checked.
template <class V, bool kSel> struct RowsChecked { static constexpr bool value = true; };
template <bool kSel> struct RowsChecked<AmrD, kSel> { static constexpr bool value = kSel; };

// Per-ray state of a sampler: none for grids and octrees (a point's unit is
// a table lookup), the current tet for meshes (the walk starts there).
struct NoWalk {};
struct TetWalk;
template <class V> struct WalkOf { using type = NoWalk; };
template <bool kNarrow> struct WalkOf<TetT<kNarrow>> { using type = TetWalk; };

// One owned sample of `piece` at lattice index k (its table coordinate in
// `val`), or the next index to try.
template <class V>
__device__ __forceinline__ bool piece_sample(const V& vol, const int32_t* __restrict__ pou, int piece, float t,
                                             const float o[3], const float d[3], int k, float& val, int& k_next,
                                             float& ws, NoWalk&) {
    const GridD& g = common(vol);
    k_next = k + 1;
    ws = 1.0f;
    const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
    if (!(p[0] >= 0.0f && p[0] < g.hx && p[1] >= 0.0f && p[1] < g.hy && p[2] >= 0.0f && p[2] < g.hz)) return false;
    const int u = unit_of(vol, p);
    if (u < 0) return false;
    if (__ldg(pou + u) != piece) {
        k_next = skip_unit(vol, u, o, d, t, k);
        return false;
    }
    const int shift = step_shift(vol, u);
    if (shift >= 0) {
        if (k & ((1 << shift) - 1)) {
            k_next = next_on_lattice(vol, u, shift, o, d, t, k, 4194304);
            return false;
        }
        ws = (float)(1 << shift);
        val = tag_shift(tf_x(g, unit_value(vol, p, u)), shift, shift_tag_mask(vol));
        return true;
    }
    val = tf_x(g, unit_value(vol, p, u));
    return true;
}

template <class V, int MS>
__global__ void __launch_bounds__(128) k_pass1_piece(const __grid_constant__ V vol, const float4* __restrict__ tf,
                                                     const int32_t* __restrict__ pob, int piece,
                                                     const __grid_constant__ PieceBox box,
                                                     const __grid_constant__ ViewTable vt, int slot, int n_slots,
                                                     char* __restrict__ moments, Counters* __restrict__ ctr) {
    if (tables_bad(vol)) return;
    const GridD& g = common(vol);
    __shared__ float2 s_sig[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= vt.total_tiles) return;
    const int vi = find_view(vt, tile);
    const ViewSlot& S = vt.s[vi];
    const int lt = tile - S.tile_base;
    int px, py;
    tile_pixel(S, lt, lane, px, py);
    unsigned n = 0;
    if (px < S.v.width && py < S.v.height) {
        auto body = make_moment_body<MS>(s_sig, g, S.v);
        float o[3], d[3];
        make_ray(S.v, px, py, o, d);
        int k0, k1;
        if (lattice_range(o, d, box.lo, box.hi, g.step, &k0, &k1)) {
            typename WalkOf<V>::type walk;
            for (int k = k0; k <= k1;) {
                const float t = lattice_t(k, g.step);
                float val, ws;
                int kn;
                const bool owned = piece_sample(vol, pob, piece, t, o, d, k, val, kn, ws, walk);
                k = kn;
                if (owned) body(t, val, ws);
            }
        }
        n = body.n;
        body.store(g, moments, S, S.moment_off * n_slots + slot * slab_bytes(g, S.plane), py * S.v.width + px);
    }
    warp_add_u64(&ctr->samples[0], n);
}

template <class V, int MS>
__global__ void __launch_bounds__(128) k_pass2_piece(const __grid_constant__ V vol, const float4* __restrict__ tf,
                                                     const int32_t* __restrict__ pob, int piece,
                                                     const __grid_constant__ PieceBox box,
                                                     const __grid_constant__ ViewTable vt, int slot, int n_slots,
                                                     const char* __restrict__ moments, float* __restrict__ color,
                                                     Counters* __restrict__ ctr) {
    if (tables_bad(vol)) return;
    const GridD& g = common(vol);
    __shared__ float4 s_tf[512];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= vt.total_tiles) return;
    const int vi = find_view(vt, tile);
    const ViewSlot& S = vt.s[vi];
    const int lt = tile - S.tile_base;
    int px, py;
    tile_pixel(S, lt, lane, px, py);
    unsigned n = 0;
    if (px < S.v.width && py < S.v.height) {
        const int pix = py * S.v.width + px;
        float4 C = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float o[3], d[3];
        make_ray(S.v, px, py, o, d);
        int k0, k1;
        if (lattice_range(o, d, box.lo, box.hi, g.step, &k0, &k1)) {
            auto body = make_blend_body<MS>(s_tf, g, S, moments, S.moment_off, pix, true);
            typename WalkOf<V>::type walk;
            for (int k = k0; k <= k1;) {
                const float t = lattice_t(k, g.step);
                float val, ws;
                int kn;
                const bool owned = piece_sample(vol, pob, piece, t, o, d, k, val, kn, ws, walk);
                k = kn;
                if (owned) body(t, val, ws);
            }
            C = body.C;
            n = body.n;
        }
        const int64_t img = (int64_t)4 * S.v.width * S.v.height;
        reinterpret_cast<float4*>(color + S.color_off * n_slots + slot * img)[pix] = C;
    }
    warp_add_u64(&ctr->samples[1], n);
}

// ------------------------------------------------------------------------
// tetrahedral meshes: exact point location.  A point snaps to integer
// quanta; D_i(q), six times the signed volume of the tet with corner i
// replaced by q, is n_i . (q - b_i) with n_i the cross product of two edges
// of face i and b_i a corner of it.  All of it is exact in 64-bit integers
// (the volume checks the coordinate range), so the two tets of a face see
// exactly opposite signs; a zero is decided by the symbolic perturbation
// q + (e, e^2, e^3): the sign of n_i.x, then n_i.y, then n_i.z.

__device__ __forceinline__ void snap_point(const TetD& m, const float p[3], int q[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) q[c] = __float2int_rn(fmul(p[c], m.qscale));
}

// Sign of D for face (a, b) around `base` at q, D itself in D.  Narrow:
// edges below 2^15 quanta, so the normal's components fit in 32 bits and D
// is three 32 x 32 -> 64-bit multiply-adds.
template <bool kNarrow>
__device__ __forceinline__ bool face_positive(const int4 a, const int4 b, const int4 base, const int q[3],
                                              long long& D) {
    const int ax = a.x - base.x, ay = a.y - base.y, az = a.z - base.z;
    const int bx = b.x - base.x, by = b.y - base.y, bz = b.z - base.z;
    const int dx = q[0] - base.x, dy = q[1] - base.y, dz = q[2] - base.z;
    long long nx, ny, nz;
    if (kNarrow) {
        const int n0 = ay * bz - az * by, n1 = az * bx - ax * bz, n2 = ax * by - ay * bx;
        D = (long long)n0 * dx + (long long)n1 * dy + (long long)n2 * dz;
        nx = n0;
        ny = n1;
        nz = n2;
    } else {
        nx = (long long)ay * bz - (long long)az * by;
        ny = (long long)az * bx - (long long)ax * bz;
        nz = (long long)ax * by - (long long)ay * bx;
        D = nx * dx + ny * dy + nz * dz;
    }
    if (D != 0) return D > 0;
    if (nx != 0) return nx > 0;
    if (ny != 0) return ny > 0;
    return nz > 0;
}

// D_0..D_3 of q; returns -1 if q is inside, else a face that q lies
// strictly outside of (the first one from `rot`, so that walks do not
// always prefer one face).  Face `skip` (-1: none) is known to pass, its D
// already in D[skip].
template <bool kNarrow>
__device__ __forceinline__ int tet_exit_face(const int4 v[4], const int q[3], long long D[4], int rot, int skip) {
    unsigned out = 0;  // bit i: q is outside face i
    if (skip != 0 && !face_positive<kNarrow>(v[2], v[1], v[3], q, D[0])) out |= 1u;
    if (skip != 1 && !face_positive<kNarrow>(v[2], v[3], v[0], q, D[1])) out |= 2u;
    if (skip != 2 && !face_positive<kNarrow>(v[3], v[1], v[0], q, D[2])) out |= 4u;
    if (skip != 3 && !face_positive<kNarrow>(v[1], v[2], v[0], q, D[3])) out |= 8u;
    if (!out) return -1;
    rot &= 3;
    const unsigned r = ((out >> rot) | (out << (4 - rot))) & 15u;
    return (rot + __ffs(r) - 1) & 3;
}

__device__ __forceinline__ int pick(const int4 a, int i) { return i == 0 ? a.x : i == 1 ? a.y : i == 2 ? a.z : a.w; }

// The range [j0, j1) of bin b's entries in the bin list.
__device__ __forceinline__ void bin_range(const TetD& m, int b, int& j0, int& j1) {
    j0 = __ldg(m.bin_start + b);
    j1 = __ldg(m.bin_start + b + 1);
}

__device__ __forceinline__ int bin_of(const TetD& m, const int q[3]) {
    int b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) b[c] = min(max(q[c] >> m.bin_shift, 0), m.bdim[c] - 1);
    return (b[2] * m.bdim[1] + b[1]) * m.bdim[0] + b[0];
}

// Per-ray walk state: the current tet, its neighbours and its corners
// (snapped x, y, z, value bits).
struct TetWalk {
    int T = -1;
    int4 nb;
    int4 v[4];
};

__device__ __forceinline__ void load_tet(const TetD& m, int T, TetWalk& w) {
    w.T = T;
    w.nb = __ldg(m.nbrs + T);
    const int4* c = m.corners + 4 * (size_t)T;
    w.v[0] = __ldg(c);
    w.v[1] = __ldg(c + 1);
    w.v[2] = __ldg(c + 2);
    w.v[3] = __ldg(c + 3);
}

// Tests the tets listed in q's bin one by one (the walk's fallback); on
// success w holds the owner and D its volumes, else w is unchanged.
template <bool kNarrow>
__device__ __forceinline__ bool tet_search(const TetD& m, TetWalk& w, const int q[3], long long D[4]) {
    int j0, j1;
    bin_range(m, bin_of(m, q), j0, j1);
    for (int j = j0; j < j1; ++j) {
        TetWalk u;
        load_tet(m, __ldg(m.bin_tets + j), u);
        if (tet_exit_face<kNarrow>(u.v, q, D, 0, -1) < 0) {
            w = u;
            return true;
        }
    }
    return false;
}

// Finds the tet owning q.  The walk starts at w.T (the tet of the previous
// sample; -1: the first tet listed in q's bin) and crosses a face that q is
// outside of, at most max_walk times; after a crossing the entry face is
// known to pass (its D is the exact negative of the exit face's).  If the
// walk leaves the mesh or runs long, the tets listed in q's bin are tested
// one by one.  On success w holds the owner and D its four volumes at q; on
// failure (no tet owns q) w still holds one tet near q.
template <bool kNarrow>
__device__ __forceinline__ bool tet_walk(const TetD& m, TetWalk& w, const int q[3], long long D[4]) {
    if (w.T < 0) {
        const int b = bin_of(m, q);
        int j0, j1;
        bin_range(m, b, j0, j1);
        if (j0 == j1) return false;  // no tet comes near q
        load_tet(m, __ldg(m.bin_tets + j0), w);
    }
    int skip = -1;
    for (int step = 0;; ++step) {
        const int f = tet_exit_face<kNarrow>(w.v, q, D, step, skip);
        if (f < 0) return true;
        if (step + 1 >= m.max_walk) break;
        const int nt = pick(w.nb, f);
        if (nt < 0) break;
        const int from = w.T;
        const long long Df = f == 0 ? D[0] : f == 1 ? D[1] : f == 2 ? D[2] : D[3];
        load_tet(m, nt, w);
        skip = w.nb.x == from ? 0 : w.nb.y == from ? 1 : w.nb.z == from ? 2 : 3;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (skip == i) D[i] = -Df;
    }
    return tet_search<kNarrow>(m, w, q, D);
}

// 0 <= x < 2^23 as float, exactly: x is the mantissa of 2^23 + x.
__device__ __forceinline__ float small_to_float(long long x) {
    return __int_as_float(0x4b000000 | (int)x) - 8388608.0f;
}

// Barycentric interpolation of the corner values: lambda_i = D_i / sum D.
// Inside a tet every D_i >= 0; all four are shifted right together until
// the sum fits in 23 bits, so each weight is off by at most 2^-23 and no
// 64-bit conversion (a double-precision-pipe instruction) is needed.
__device__ __forceinline__ float tet_value(const long long D[4], const int4 v[4]) {
    const long long tot = D[0] + D[1] + D[2] + D[3];
    const int sh = max(0, 41 - __clzll(tot));
    const float inv = 1.0f / small_to_float(tot >> sh);
    float s = small_to_float(D[0] >> sh) * __int_as_float(v[0].w);
    s = ffma(small_to_float(D[1] >> sh), __int_as_float(v[1].w), s);
    s = ffma(small_to_float(D[2] >> sh), __int_as_float(v[2].w), s);
    s = ffma(small_to_float(D[3] >> sh), __int_as_float(v[3].w), s);
    return s * inv;
}

template <bool kNarrow>
__device__ __forceinline__ bool piece_sample(const TetT<kNarrow>& m, const int32_t* __restrict__ pou, int piece,
                                             float t, const float o[3], const float d[3], int k, float& val,
                                             int& k_next, float& ws, TetWalk& w) {
    ws = 1.0f;
    const GridD& g = m.g;
    k_next = k + 1;
    const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
    if (!(p[0] >= 0.0f && p[0] < g.hx && p[1] >= 0.0f && p[1] < g.hy && p[2] >= 0.0f && p[2] < g.hz)) return false;
    int q[3];
    snap_point(m, p, q);
    long long D[4];
    if (!tet_walk<kNarrow>(m, w, q, D)) return false;
    if (__ldg(pou + w.T) != piece) return false;
    val = tf_x(g, tet_value(D, w.v));
    return true;
}

// ------------------------------------------------------------------------
// fused, persistent passes over a brick octree or a tetrahedral mesh
// (direct gathers).  Octree: the leaf of each lattice point comes from the
// finest-brick map, its value from the leaf's own vertex block.  Mesh: the
// tet comes from a walk that starts at the previous sample's tet.

// Batched march over a mesh.  One iteration is one tet test for every lane
// of the warp: it either places the current lattice point (the sample is
// taken, the next point comes up) or crosses a face towards it, so the
// lanes stay together in the test and part only for the sample or the
// crossing.  The owners are those of tet_walk: the same walk, the same
// fallback.  `store` gets every lattice point's value (NaN: not sampled).
template <bool kSel, class Body, bool kNarrow, class Store = NoStore>
__device__ __forceinline__ void march_unit(const TetT<kNarrow>& m, const uint8_t* __restrict__ sel, const float o[3],
                                           const float d[3], int k0, int k1, Body& body, Store store = Store{}) {
    const GridD& g = m.g;
    if (k0 > k1) return;
    store.seek(k0);
    const float tz = lattice_t(k1, g.step);
    float t = lattice_t(k0, g.step);
    int q[3];
    {
        const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
        snap_point(m, p, q);
    }
    TetWalk w;
    {
        const int b = bin_of(m, q);
        int j0, j1;
        bin_range(m, b, j0, j1);
        if (j0 < j1) load_tet(m, __ldg(m.bin_tets + j0), w);
    }
    long long D[4];
    int skip = -1, steps = 0;
    while (t <= tz) {
        const int f = w.T >= 0 ? tet_exit_face<kNarrow>(w.v, q, D, steps, skip) : -2;
        if (f >= 0) {
            const int nt = pick(w.nb, f);
            if (nt >= 0 && steps + 1 < m.max_walk) {
                const int from = w.T;
                const long long Df = f == 0 ? D[0] : f == 1 ? D[1] : f == 2 ? D[2] : D[3];
                load_tet(m, nt, w);
                skip = w.nb.x == from ? 0 : w.nb.y == from ? 1 : w.nb.z == from ? 2 : 3;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (skip == i) D[i] = -Df;
                ++steps;
                continue;
            }
        }
        const bool found = f == -1 || tet_search<kNarrow>(m, w, q, D);
        float val = __int_as_float(0x7fc00000);
        if (found && (!kSel || __ldg(sel + w.T))) {
            // the corner values (the .w words) read again here rather than
            // kept live through the walk, which only tests x, y, z: fewer
            // spilled registers in the loop (the same bits, so the same value)
            const int* cw = reinterpret_cast<const int*>(m.corners + 4 * (size_t)w.T);
            const int4 vw[4] = {make_int4(0, 0, 0, __ldg(cw + 3)), make_int4(0, 0, 0, __ldg(cw + 7)),
                                make_int4(0, 0, 0, __ldg(cw + 11)), make_int4(0, 0, 0, __ldg(cw + 15))};
            val = tf_x(g, tet_value(D, vw));
            body(t, val);
        }
        store.put(val);
        t += g.step;
        const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
        snap_point(m, p, q);
        skip = -1;
        steps = 0;
    }
}

// Fixed-step octree march of pass 1 for leaves of NV^3 vertices, in
// lockstep: the warp walks the lattice rows kmin..kmax in windows of
// kDepthRows, each lane sampling the rows of its own [k0, k1], and the depth
// powers of a window's rows are computed once for the warp (DepthRows).  A
// lane keeps its previous sample's leaf: q = (p - lo) / h is exact in float32
// (lo a multiple of ulp(p), h a power of two), p lies in the leaf's half-open
// box iff 0 <= q < NV - 1 per axis (one unsigned compare of the float bits:
// negative values and NaN have the sign bit or a large exponent), and then q
// is also the sample's local coordinate, its cell (int)q <= NV - 2.  Points
// outside every leaf (holes) and in unselected leaves are stored as NaN, as
// in march_unit.  Results equal march_unit's with MomentBody bit for bit.
template <int NV, bool kSel, class Store>
__device__ __forceinline__ void march_amr_rows(const AmrD& a, const uint8_t* __restrict__ sel, const float o[3],
                                               const float d[3], int k0, int k1, MomentBody& body, Store& store,
                                               DepthRows rows) {
    const GridD& g = a.g;
    const unsigned full = 0xffffffffu;
    const bool any = k0 <= k1;
    const int kmin = __reduce_min_sync(full, any ? k0 : 0x7fffffff);
    const int kmax = __reduce_max_sync(full, any ? k1 : -1);
    if (any) store.seek(k0);
    constexpr unsigned kEdge = 0x41000000u;            // bits of 8.0f = NV - 1 for NV = 9
    static_assert(NV == 9, "the box test's bound is NV - 1 = 8");
    const float* blk = nullptr;                         // the cached leaf's vertex block (NULL: none selected)
    float lo0 = __int_as_float(0x7f800000), lo1 = lo0, lo2 = lo0, inv_h = 1.0f;   // no box yet
    // one lattice point: leaf box test (a leaf change where it fails), the
    // trilinear value, the store and the moments; j = the point's row in the window
    auto point = [&](float t, int j) {
        const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
        float q0 = (p0 - lo0) * inv_h, q1 = (p1 - lo1) * inv_h, q2 = (p2 - lo2) * inv_h;
        if (!(__float_as_uint(q0) < kEdge && __float_as_uint(q1) < kEdge && __float_as_uint(q2) < kEdge)) {
            // a new leaf: the finest-brick map, then the leaf's box
            const float p[3] = {p0, p1, p2};
            const int v = unit_of(a, p);
            if (v < 0) {
                lo0 = lo1 = lo2 = __int_as_float(0x7f800000);
                blk = nullptr;
                store.put(__int_as_float(0x7fc00000));
                return;
            }
            const float4 L = __ldg(a.leaf_box + v);
            lo0 = L.x;
            lo1 = L.y;
            lo2 = L.z;
            inv_h = L.w;
            blk = (kSel && sel && !__ldg(sel + v)) ? nullptr : a.values + (size_t)v * (NV * NV * NV);
            q0 = (p0 - lo0) * inv_h;
            q1 = (p1 - lo1) * inv_h;
            q2 = (p2 - lo2) * inv_h;
        }
        if (kSel && !blk) {
            store.put(__int_as_float(0x7fc00000));
            return;
        }
        const int cx = (int)q0, cy = (int)q1, cz = (int)q2;
        const float* __restrict__ c = blk + (cz * NV + cy) * NV + cx;
        const float val = tf_x(g, trilinear8(__ldg(c), __ldg(c + 1), __ldg(c + NV), __ldg(c + NV + 1),
                                             __ldg(c + NV * NV), __ldg(c + NV * NV + 1), __ldg(c + NV * NV + NV),
                                             __ldg(c + NV * NV + NV + 1), q0 - (float)cx, q1 - (float)cy,
                                             q2 - (float)cz));
        store.put(val);
        body.add(val, 1.0f, rows.z[j]);
    };
    // Without holes or a selection (every point has a leaf): the leaf of a
    // point and its local coordinates, after a leaf change where its box test
    // fails.
    auto locate = [&](float t, float& q0, float& q1, float& q2) {
        const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
        q0 = (p0 - lo0) * inv_h;
        q1 = (p1 - lo1) * inv_h;
        q2 = (p2 - lo2) * inv_h;
        if (!(__float_as_uint(q0) < kEdge && __float_as_uint(q1) < kEdge && __float_as_uint(q2) < kEdge)) {
            const float p[3] = {p0, p1, p2};
            const int v = unit_of(a, p);
            const float4 L = __ldg(a.leaf_box + v);
            lo0 = L.x;
            lo1 = L.y;
            lo2 = L.z;
            inv_h = L.w;
            blk = a.values + (size_t)v * (NV * NV * NV);
            q0 = (p0 - lo0) * inv_h;
            q1 = (p1 - lo1) * inv_h;
            q2 = (p2 - lo2) * inv_h;
        }
        return blk;
    };
    auto value = [&](const float* b, float q0, float q1, float q2) {
        const int cx = (int)q0, cy = (int)q1, cz = (int)q2;
        const float* __restrict__ c = b + (cz * NV + cy) * NV + cx;
        return tf_x(g, trilinear8(__ldg(c), __ldg(c + 1), __ldg(c + NV), __ldg(c + NV + 1), __ldg(c + NV * NV),
                                  __ldg(c + NV * NV + 1), __ldg(c + NV * NV + NV), __ldg(c + NV * NV + NV + 1),
                                  q0 - (float)cx, q1 - (float)cy, q2 - (float)cz));
    };
    for (int kw = kmin; kw <= kmax; kw += kDepthRows) {
        rows.fill(kw, g.step, body.wa, body.wb);
        const int ka = max(kw, k0), kz = min(kw + kDepthRows - 1, k1);
        float t = lattice_t(ka, g.step);
        if (ka == kw && kz == kw + kDepthRows - 1) {
            // the lane samples every row of the window: unrolled
            if constexpr (!kSel) {
                // two rows at a time: both leaf tests, then both points'
                // gathers (16 loads in flight together), then the store and
                // the moments in row order
#pragma unroll
                for (int j = 0; j < kDepthRows; j += 2) {
                    const float tb = t + g.step;
                    float qa0, qa1, qa2, qb0, qb1, qb2;
                    const float* ba = locate(t, qa0, qa1, qa2);
                    const float* bb = locate(tb, qb0, qb1, qb2);
                    const float va = value(ba, qa0, qa1, qa2), vb = value(bb, qb0, qb1, qb2);
                    store.put(va);
                    body.add(va, 1.0f, rows.z[j]);
                    store.put(vb);
                    body.add(vb, 1.0f, rows.z[j + 1]);
                    t = tb + g.step;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kDepthRows; ++j, t += g.step) point(t, j);
            }
        } else {
            for (int k = ka; k <= kz; ++k, t += g.step) point(t, k - kw);
        }
    }
}

template <bool kSel, class Body, class Store = NoStore>
__device__ __forceinline__ void march_unit(const AmrD& a, const uint8_t* __restrict__ sel, const float o[3],
                                           const float d[3], int k0, int k1, Body& body, Store store = Store{},
                                           float4* zrows = nullptr) {
    const GridD& g = a.g;
    if (g.flags & kFlagAdaptiveStep) {
        // adaptive dyadic step: a point counts only on its leaf's nested
        // lattice.  The warp walks the lattice indices in lockstep (each lane
        // active inside its own [k0, k1]; all 32 lanes reach the reductions),
        // so lanes in leaves of one level skip the same points together
        // instead of diverging.
        const unsigned full = 0xffffffffu;
        const bool any = k0 <= k1;
        const int kmin = __reduce_min_sync(full, any ? k0 : 0x7fffffff);
        const int kmax = __reduce_max_sync(full, any ? k1 : -1);
        if (any) store.seek(k0);
        LeafCache lc;
        for (int k = kmin; k <= kmax; ++k) {
            if (k < k0 || k > k1) continue;
            const float t = lattice_t(k, g.step);
            const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
            const int u = lc.find<kSel>(a, sel, p);
            if (u < 0) {
                store.put(__int_as_float(0x7fc00000));
                continue;
            }
            const int shift = lc.shift;
            if (k & ((1 << shift) - 1)) {
                store.put(__int_as_float(0x7fc00000));
                continue;
            }
            const float val = tag_shift(tf_x(g, leaf_value(a, p, u, lc.lo, lc.inv_h)), shift, tag_mask(a.max_level));
            store.put(val);
            body(t, val, (float)(1 << shift));
        }
        return;
    }
    if constexpr (std::is_same<Body, MomentBody>::value) {
        if (zrows && a.nv == 9) {
            march_amr_rows<9, kSel>(a, sel, o, d, k0, k1, body, store, DepthRows{zrows});
            return;
        }
    }
    if (k0 > k1) return;
    store.seek(k0);
    const float tz = lattice_t(k1, g.step);
    LeafCache lc;
    for (float t = lattice_t(k0, g.step); t <= tz; t += g.step) {
        const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
        const int u = lc.find<kSel>(a, sel, p);
        if (u < 0) {
            store.put(__int_as_float(0x7fc00000));
            continue;
        }
        const float val = tf_x(g, leaf_value(a, p, u, lc.lo, lc.inv_h));
        store.put(val);
        body(t, val);
    }
}

// Resident 256-thread blocks per SM the unit kernels are compiled for (the
// walks and gathers are latency-bound: more warps hide more of it); the
// trigonometric and 6-/8-power-moment bodies get 2, so that they keep their
// registers.
#ifndef MB_TET_MIN_BLOCKS
#define MB_TET_MIN_BLOCKS 3
#endif
template <class V, int kPass> struct MinBlocks { static constexpr int value = kPass == 2 ? 4 : 1; };
// octrees: 4 for both passes (pass 1 fits 56 registers; at 5 blocks, 48
// registers, its warps share the L1 that serves their gathers and it slows)
template <int kPass> struct MinBlocks<AmrD, kPass> { static constexpr int value = 4; };
template <bool k, int kPass> struct MinBlocks<TetT<k>, kPass> { static constexpr int value = MB_TET_MIN_BLOCKS; };

template <class V, bool kSel, int MS, bool kCache = false>
__global__ void __launch_bounds__(256, MS == 0 ? MinBlocks<V, 1>::value : 2) k_pass1_unit(const __grid_constant__ V a, const float4* __restrict__ tf,
                                                    const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                    char* __restrict__ moments, Counters* __restrict__ ctr,
                                                    const TileCache cache) {
    if (tables_bad(a)) return;
    __shared__ float2 s_sig[256];
    __shared__ float4 s_z[kFusedWarps][kDepthRows];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    __syncthreads();
    const GridD& g = a.g;
    float4* zrows = s_z[threadIdx.x >> 5];
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        auto body = make_moment_body<MS>(s_sig, g, S.v);
        if constexpr (std::is_same<V, AmrD>::value) {
            if constexpr (kCache) {
                RowStore st{tile_rows(cache, ctr, tile, k0, k1)};
                march_unit<kSel>(a, sel, o, d, k0, k1, body, st, zrows);
            } else {
                march_unit<kSel>(a, sel, o, d, k0, k1, body, NoStore{}, zrows);
            }
        } else if constexpr (kCache) {
            RowStore st{tile_rows(cache, ctr, tile, k0, k1)};
            march_unit<kSel>(a, sel, o, d, k0, k1, body, st);
        } else {
            march_unit<kSel>(a, sel, o, d, k0, k1, body);
        }
        if (valid) body.store(g, moments, S, S.moment_off, py * S.v.width + px);
        warp_add_u64(&ctr->samples[0], body.n);
    }
}

template <class V, bool kSel, int MS, bool kCache = false>
__global__ void __launch_bounds__(256, MS == 0 ? MinBlocks<V, 2>::value : 2) k_pass2_unit(const __grid_constant__ V a, const float4* __restrict__ tf,
                                                    const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                    const char* __restrict__ moments, float* __restrict__ color, int mode,
                                                    Counters* __restrict__ ctr, const TileCache cache) {
    if (tables_bad(a)) return;
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_rows[kCache ? kFusedWarps : 1][kCache ? kUnitRowBuf : 4];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    }
    __syncthreads();
    const GridD& g = a.g;
    const bool raw = (g.flags & 1u) != 0;
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[1], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        const int pix = valid ? py * S.v.width + px : 0;
        auto body = make_blend_body<MS>(s_tf, g, S, moments, S.moment_off, pix, valid);
        count_frames(ctr, body, valid);
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const long long tb = kCache ? cache.tile_base[tile] : -1;
        if (kCache && tb >= 0) {
            const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
            float* buf = s_rows[kCache ? threadIdx.x >> 5 : 0];
            bool tagged = false;  // octree samples of the adaptive step carry their weight
            int tmask = 0;
            if constexpr (std::is_same<V, AmrD>::value) {
                tagged = (g.flags & kFlagAdaptiveStep) != 0;
                tmask = tag_mask(a.max_level);
            }
            if (tagged)
                blend_rows<true, true, kUnitRowChunk>(g, cache.vals + tb * 32, kmin, kmax, k0, k1, buf, body, tmask);
            else
                blend_rows<RowsChecked<V, kSel>::value, false, kUnitRowChunk>(g, cache.vals + tb * 32, kmin, kmax, k0,
                                                                               k1, buf, body);
        } else {
            march_unit<kSel>(a, sel, o, d, k0, k1, body);
        }
        if (valid) {
            float4* out = reinterpret_cast<float4*>(color + S.color_off) + pix;
            *out = mode == kColorResolved ? resolve_pixel(body.C, body.b0, make_float4(0.0f, 0.0f, 0.0f, 0.0f), raw)
                                          : body.C;
        }
        warp_add_u64(&ctr->samples[1], body.n);
    }
}

// ------------------------------------------------------------------------
// GPU exact sort-last baseline (the segment-layer compositor of Sec. 5).
// Every piece, like a rank, turns each maximal run of consecutive lattice
// points it owns into one segment (front-to-back "over" inside the run:
// premultiplied colour and opacity, keyed by the run's first lattice index);
// per pixel the segments of all pieces are sorted by that key and blended
// front to back.  Counting and filling are separate marches so the segment
// buffer can be sized exactly.

template <class V, bool kFill>
__global__ void __launch_bounds__(128) k_sortlast_piece(const __grid_constant__ V vol, const float4* __restrict__ tf,
                                                        const int32_t* __restrict__ pob, int piece,
                                                        const __grid_constant__ PieceBox box,
                                                        const __grid_constant__ ViewTable vt, int slot, int n_slots,
                                                        int32_t* __restrict__ counts, const int64_t* __restrict__ starts,
                                                        int32_t* __restrict__ seg_key, float4* __restrict__ seg_col) {
    const bool bad = tables_bad(vol);   // bad tables: count no segments, fill none
    const GridD& g = common(vol);
    __shared__ float4 s_tf[256];
    if (kFill) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_tf[i] = tf[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tile >= vt.total_tiles) return;
    const int vi = find_view(vt, tile);
    const ViewSlot& S = vt.s[vi];
    const int lt = tile - S.tile_base;
    int px, py;
    tile_pixel(S, lt, lane, px, py);
    if (px >= S.v.width || py >= S.v.height) return;
    const int64_t npix = (int64_t)S.v.width * S.v.height;
    const int64_t gpix = S.color_off / 4 + py * S.v.width + px;  // pixel index over all views
    const int64_t cidx = (S.color_off / 4) * n_slots + slot * npix + (py * S.v.width + px);
    float o[3], d[3];
    make_ray(S.v, px, py, o, d);
    int k0, k1;
    int nseg = 0;
    if (!bad && lattice_range(o, d, box.lo, box.hi, g.step, &k0, &k1)) {
        int64_t out = kFill ? starts[cidx] : 0;
        int prev = -2, key = 0;
        float4 cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float tr = 1.0f;
        typename WalkOf<V>::type walk;
        for (int k = k0; k <= k1;) {
            const float t = lattice_t(k, g.step);
            float val, ws;
            int kn;
            if (!piece_sample(vol, pob, piece, t, o, d, k, val, kn, ws, walk)) {
                k = kn;
                continue;
            }
            if (k != prev + 1) {
                if (kFill && nseg > 0) {
                    seg_key[out] = key;
                    seg_col[out] = make_float4(cur.x, cur.y, cur.z, 1.0f - tr);
                    ++out;
                }
                ++nseg;
                key = k;
                cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                tr = 1.0f;
            }
            prev = k;
            k = kn;
            if (kFill) {
                // val is the table coordinate; a tagged one may sit a few ulp above 255
                const int i = min((int)val, 254);
                const float f = fmin_(val - (float)i, 1.0f);
                const float4 e0 = s_tf[i], e1 = s_tf[i + 1];
                const float a = fmin_(ffma(f, e1.w - e0.w, e0.w) * ws, g.absorbance_max);
                const float w = tr * one_minus_exp_neg(a);
                cur.x = ffma(w, ffma(f, e1.x - e0.x, e0.x), cur.x);
                cur.y = ffma(w, ffma(f, e1.y - e0.y, e0.y), cur.y);
                cur.z = ffma(w, ffma(f, e1.z - e0.z, e0.z), cur.z);
                tr *= fexp2(-a * kLog2e);
            }
        }
        if (kFill && nseg > 0) {
            seg_key[out] = key;
            seg_col[out] = make_float4(cur.x, cur.y, cur.z, 1.0f - tr);
        }
    }
    if (!kFill) counts[cidx] = nseg;
    (void)gpix;
}

}  // namespace
}  // namespace mb
