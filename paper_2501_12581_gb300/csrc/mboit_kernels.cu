// CUDA kernels of the MBOIT puzzle-piece render for sm_103a.
//
// Work decomposition.  One thread marches one ray; a warp owns an 8 x 4
// pixel tile, so the 32 rays of a warp are spatial neighbours and their
// trilinear gathers at the same lattice index hit a few adjacent cache lines.
// The fused passes are persistent: grid = SMs x resident CTAs, each warp pops
// tiles from an atomic work-queue head (no waits, no spins), which balances
// long centre rays against short silhouette rays.  The transfer function
// (256 x float4, 4 KB) is staged once per CTA in shared memory.
//
// Pass 1 (Sec. 4.1, Alg. 2) accumulates b_j += a z^j in registers over all
// selected pieces: summing the pieces' moment images (the Allreduce add) is
// done in registers because addition commutes.  Pass 2 (Sec. 4.2, Alg. 1
// loop 2, Alg. 3) builds the per-pixel reconstruction frame from the global
// moments in FP64 once per ray, then adds T * alpha * (r, g, b, 1) per sample
// in FP32; the resolved mode also applies the renormalisation (Sec. 4.3) in
// the epilogue, so the frame needs no separate colour reduction.
//
// The per-piece kernels are the plain form: one launch per piece, the rays
// clipped to the piece's box, non-owned bricks skipped forward, one image per
// piece; the image-space kernels then sum the K images (compensated).
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mboit_internal.h"
#include "mboit_trig.cuh"

namespace mb {

namespace {

__device__ __forceinline__ float one_minus_exp_neg(float a) {
    // 1 - e^-a without cancellation: Taylor series a * sum_{n>=0} (-a)^n / (n+1)!
    // truncated after (-a)^5/6! for a < 1/4 (relative error < 5e-8); the
    // direct form above, where cancellation costs at most a few ulp.
    if (a < 0.25f) {
        float p = ffma(a, -1.0f / 720.0f, 1.0f / 120.0f);
        p = ffma(a, p, -1.0f / 24.0f);
        p = ffma(a, p, 1.0f / 6.0f);
        p = ffma(a, p, -0.5f);
        p = ffma(a, p, 1.0f);
        return a * p;
    }
    return 1.0f - fexp2(-a * kLog2e);
}

// Position of lattice point t on the ray, domain test, optional brick
// selection, trilinear value.  Cells are half-open, so a point inside
// [0, n-1) has all 8 corner vertices in range.
template <bool kSel>
__device__ __forceinline__ bool field_sample(const GridD& g, const uint8_t* __restrict__ sel, float t,
                                             const float o[3], const float d[3], float& val) {
    const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
    if (!(p0 >= 0.0f && p0 < g.hx && p1 >= 0.0f && p1 < g.hy && p2 >= 0.0f && p2 < g.hz)) return false;
    const int ix = (int)p0, iy = (int)p1, iz = (int)p2;
    if (kSel) {
        const int b = ((iz >> g.brick_log2) * g.nby + (iy >> g.brick_log2)) * g.nbx + (ix >> g.brick_log2);
        if (!__ldg(sel + b)) return false;
    }
    const float fx = p0 - (float)ix, fy = p1 - (float)iy, fz = p2 - (float)iz;
    const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * (size_t)g.ny;
    const float* __restrict__ c = g.field + (size_t)iz * sz + (size_t)iy * sy + (size_t)ix;
    const float v000 = __ldg(c), v100 = __ldg(c + 1);
    const float v010 = __ldg(c + sy), v110 = __ldg(c + sy + 1);
    const float v001 = __ldg(c + sz), v101 = __ldg(c + sz + 1);
    const float v011 = __ldg(c + sz + sy), v111 = __ldg(c + sz + sy + 1);
    const float a00 = ffma(fx, v100 - v000, v000), a10 = ffma(fx, v110 - v010, v010);
    const float a01 = ffma(fx, v101 - v001, v001), a11 = ffma(fx, v111 - v011, v011);
    const float b0 = ffma(fy, a10 - a00, a00), b1 = ffma(fy, a11 - a01, a01);
    val = ffma(fz, b1 - b0, b0);
    return true;
}

__device__ __forceinline__ float tf_coord(const GridD& g, float v, int& i) {
    const float xt = fclamp(ffma(v, g.tf_scale, g.tf_bias), 0.0f, 255.0f);
    i = min((int)xt, 254);
    return xt - (float)i;
}

__device__ __forceinline__ int find_view(const ViewTable& vt, int tile) {
    int vi = 0;
    while (vi + 1 < vt.n && tile >= vt.s[vi + 1].tile_base) ++vi;
    return vi;
}

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned n) {
    unsigned long long v = n;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

__device__ __forceinline__ void store_moments(char* base, const ViewSlot& S, int64_t slab_off, int pix,
                                              float m0, float m1, float m2, float m3, float m4) {
    char* slab = base + slab_off;
    reinterpret_cast<float*>(slab)[pix] = m0;
    reinterpret_cast<float4*>(slab + (size_t)4 * S.plane)[pix] = make_float4(m1, m2, m3, m4);
}

__device__ __forceinline__ void load_moments(const char* base, const ViewSlot& S, int64_t slab_off, int pix,
                                             float m[5]) {
    const char* slab = base + slab_off;
    m[0] = __ldg(reinterpret_cast<const float*>(slab) + pix);
    const float4 q = __ldg(reinterpret_cast<const float4*>(slab + (size_t)4 * S.plane) + pix);
    m[1] = q.x; m[2] = q.y; m[3] = q.z; m[4] = q.w;
}

__device__ __forceinline__ float4 resolve_pixel(float4 C, float m0, float4 bg, bool raw) {
    if (raw) return C;
    const float A = -expm1f(-m0);
    const float T = 1.0f - A;
    const float k = C.w > 0.0f ? A / C.w : 0.0f;
    return make_float4(ffma(C.x, k, T * bg.x), ffma(C.y, k, T * bg.y), ffma(C.z, k, T * bg.z), A + T * bg.w);
}

// ------------------------------------------------------------------------
// fused, persistent passes
//
// Warp-cooperative staging.  The 32 rays of a warp advance in lockstep over
// the lattice index k; at one k their sample points lie a few voxels apart.
// For a window of S consecutive indices the warp takes the bounding box of
// the cells its samples can touch (from the exact float32 positions of each
// lane's first and last sample in the window: positions are monotone in t,
// so every sample in between lies inside), and if the box fits a WX x WY x WZ
// block, the warp copies that block of the field into its own shared-memory
// slot once, then reads all trilinear corners from shared memory.  Each field
// row is fetched once per window instead of eight times per lattice step.  A
// box that does not fit (widely spread rays) falls back to direct loads.

template <int S_, int WX_, int WY_, int WZ_, bool kVec_>
struct StageCfg {
    static constexpr int S = S_, WX = WX_, WY = WY_, WZ = WZ_;
    static constexpr bool kVec = kVec_;  // 16-byte loads: x origin rounded down to a multiple of 4
    // scalar windows pad rows to an odd pitch; vector windows keep 16-byte rows
    // and shift each plane by 4 floats, both to spread shared-memory banks
    static constexpr int Pitch = kVec_ ? WX_ : WX_ + 1;
    static constexpr int Plane = kVec_ ? WY_ * WX_ + 4 : WY_ * (WX_ + 1);
    static constexpr int Floats = WZ_ * Plane;
    static constexpr int Elems = WX_ * WY_ * WZ_;
    static_assert(!kVec_ || WX_ % 4 == 0, "vector windows need a multiple of 4 in x");
};
// The configurations the autotuner chooses from (index = tuning id).
using Stage0 = StageCfg<6, 8, 8, 8, false>;
using Stage1 = StageCfg<8, 8, 8, 8, false>;
using Stage2 = StageCfg<6, 12, 8, 8, true>;
using Stage3 = StageCfg<6, 16, 8, 8, true>;
using Stage4 = StageCfg<8, 16, 8, 10, true>;
constexpr int kFusedWarps = 8;  // 256 threads per CTA

__device__ __forceinline__ float trilinear8(float v000, float v100, float v010, float v110, float v001, float v101,
                                            float v011, float v111, float fx, float fy, float fz) {
    const float a00 = ffma(fx, v100 - v000, v000), a10 = ffma(fx, v110 - v010, v010);
    const float a01 = ffma(fx, v101 - v001, v001), a11 = ffma(fx, v111 - v011, v011);
    const float b0 = ffma(fy, a10 - a00, a00), b1 = ffma(fy, a11 - a01, a01);
    return ffma(fz, b1 - b0, b0);
}

// Bounding box of the cells that lane samples in [ka, kz] can touch, reduced
// over the warp; true if it fits the window.
template <class Cfg>
__device__ __forceinline__ bool window_box(const GridD& g, const float o[3], const float d[3], int ka, int kz,
                                           int LO[3]) {
    const unsigned full = 0xffffffffu;
    const int nmax[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-1, -1, -1};
    if (ka <= kz) {
        const float ta = lattice_t(ka, g.step), tz = lattice_t(kz, g.step);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float pa = ffma(ta, d[c], o[c]), pz = ffma(tz, d[c], o[c]);
            lo[c] = max((int)floorf(fmin_(pa, pz)), 0);
            hi[c] = min((int)floorf(fmax_(pa, pz)) + 1, nmax[c]);
        }
    }
    bool fits = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        LO[c] = __reduce_min_sync(full, lo[c]);
        const int HI = __reduce_max_sync(full, hi[c]);
        if (c == 0 && Cfg::kVec) LO[0] &= ~3;
        const int ext = c == 0 ? Cfg::WX : (c == 1 ? Cfg::WY : Cfg::WZ);
        fits = fits && HI >= LO[c] && HI - LO[c] < ext;
    }
    return fits;
}

// Marches the lattice indices [k0, k1] of this lane's ray (exactly the
// in-domain points; k0 > k1: none), calling body(t, value) for every owned
// sample in depth order.  All 32 lanes of the warp call it together.
// Where a march puts every lattice point's value: nowhere, or a tile-cache
// row (the lane's slot of row k; NaN for a point no selected piece owns).
struct NoStore {
    __device__ __forceinline__ void seek(int) {}
    __device__ __forceinline__ void put(float) {}
};
struct RowStore {
    float* base;  // slot of row 0: vals + (tile_base - kmin) * 32 + lane; NULL: off
    float* at = nullptr;
    __device__ __forceinline__ void seek(int k) { at = base + (int64_t)k * 32; }
    __device__ __forceinline__ void put(float v) {
        if (base) __stcs(at, v);  // streaming store: read once by pass 2, keep the field in L2
        at += 32;
    }
};

template <class Cfg, bool kSel, class Body, class Store = NoStore>
__device__ __forceinline__ void march_fused(const GridD& g, const uint8_t* __restrict__ sel, float* __restrict__ win,
                                            const float o[3], const float d[3], int k0, int k1, Body& body,
                                            Store store = Store{}) {
    const unsigned full = 0xffffffffu;
    const int kmin = __reduce_min_sync(full, k0);
    const int kmax = __reduce_max_sync(full, k1);
    const int nmax[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    for (int kb = kmin; kb <= kmax;) {
        // the longest window (2S, then S steps) whose box fits
        int LO[3];
        int ke = min(kb + 2 * Cfg::S - 1, kmax);
        bool fits = window_box<Cfg>(g, o, d, max(kb, k0), min(ke, k1), LO);
        if (!fits && ke > kb + Cfg::S - 1) {
            ke = kb + Cfg::S - 1;
            fits = window_box<Cfg>(g, o, d, max(kb, k0), min(ke, k1), LO);
        }
        const int ka = max(kb, k0), kz = min(ke, k1);
        if (fits) {
            __syncwarp();
            const int lane = threadIdx.x & 31;
            if (Cfg::kVec) {
                // nx % 4 == 0 and a 16-byte aligned field (checked by the launcher):
                // every chunk start gx is a multiple of 4 and gx + 3 < nx
                constexpr int QX = Cfg::WX / 4;
                if (QX * Cfg::WY == 32) {
                    // one plane per warp-wide step: lane -> fixed (xq, y), z = step
                    const int xq = lane % QX, y = lane / QX;
                    const int gx = min(LO[0] + 4 * xq, g.nx - 4), gy = min(LO[1] + y, nmax[1]);
                    const float* src = g.field + (size_t)gy * g.nx + gx;
                    float* dst = win + y * Cfg::Pitch + 4 * xq;
                    const size_t zs = (size_t)g.nx * g.ny;
#pragma unroll
                    for (int z = 0; z < Cfg::WZ; ++z) {
                        const int gz = min(LO[2] + z, nmax[2]);
                        *reinterpret_cast<float4*>(dst + z * Cfg::Plane) =
                            __ldg(reinterpret_cast<const float4*>(src + gz * zs));
                    }
                } else {
#pragma unroll 2
                    for (int e = lane; e < QX * Cfg::WY * Cfg::WZ; e += 32) {
                        const int xq = e % QX, y = (e / QX) % Cfg::WY, z = e / (QX * Cfg::WY);
                        const int gx = min(LO[0] + 4 * xq, g.nx - 4), gy = min(LO[1] + y, nmax[1]),
                                  gz = min(LO[2] + z, nmax[2]);
                        *reinterpret_cast<float4*>(win + z * Cfg::Plane + y * Cfg::Pitch + 4 * xq) = __ldg(
                            reinterpret_cast<const float4*>(g.field + ((size_t)gz * g.ny + gy) * (size_t)g.nx + gx));
                    }
                }
            } else {
#pragma unroll 4
                for (int e = lane; e < Cfg::Elems; e += 32) {
                    const int x = e % Cfg::WX, y = (e / Cfg::WX) % Cfg::WY, z = e / (Cfg::WX * Cfg::WY);
                    const int gx = min(LO[0] + x, nmax[0]), gy = min(LO[1] + y, nmax[1]), gz = min(LO[2] + z, nmax[2]);
                    win[z * Cfg::Plane + y * Cfg::Pitch + x] =
                        __ldg(g.field + ((size_t)gz * g.ny + gy) * (size_t)g.nx + gx);
                }
            }
            __syncwarp();
            const float* wbase = win - LO[2] * Cfg::Plane - LO[1] * Cfg::Pitch - LO[0];
            // t_{k+1} = t_k + step exactly (odd multiples of step/2 below 2^24), so the
            // loop runs on t itself
            const float tz = lattice_t(kz, g.step);
            store.seek(ka);
            for (float t = lattice_t(ka, g.step); t <= tz; t += g.step) {
                const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
                const int ix = (int)p0, iy = (int)p1, iz = (int)p2;
                if (kSel) {
                    const int b = ((iz >> g.brick_log2) * g.nby + (iy >> g.brick_log2)) * g.nbx + (ix >> g.brick_log2);
                    if (!__ldg(sel + b)) {
                        store.put(__int_as_float(0x7fc00000));
                        continue;
                    }
                }
                const float* c = wbase + iz * Cfg::Plane + iy * Cfg::Pitch + ix;
                const float val = trilinear8(c[0], c[1], c[Cfg::Pitch], c[Cfg::Pitch + 1], c[Cfg::Plane],
                                             c[Cfg::Plane + 1], c[Cfg::Plane + Cfg::Pitch],
                                             c[Cfg::Plane + Cfg::Pitch + 1], p0 - (float)ix, p1 - (float)iy,
                                             p2 - (float)iz);
                store.put(val);
                body(t, val);
            }
        } else {
            const float tz = lattice_t(kz, g.step);
            store.seek(ka);
            for (float t = lattice_t(ka, g.step); t <= tz; t += g.step) {
                float val;
                if (!field_sample<kSel>(g, sel, t, o, d, val)) {
                    store.put(__int_as_float(0x7fc00000));
                    continue;
                }
                store.put(val);
                body(t, val);
            }
        }
        kb = ke + 1;
    }
}

// Alg. 2 per sample: absorbance a = min(sigma*step, A_max), b_j += a z^j.
struct MomentBody {
    const float2* s_sig;  // (sigma*step of entry i, of entry i+1 minus entry i)
    float tf_scale, tf_bias, amax, wa, wb;
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, m3 = 0.0f, m4 = 0.0f;
    unsigned n = 0;
    __device__ __forceinline__ void operator()(float t, float val) {
        // entry 255 has a zero delta, so xt = 255 needs no special index
        const float xt = fclamp(ffma(val, tf_scale, tf_bias), 0.0f, 255.0f);
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float2 s = s_sig[i];
        const float a = fmin_(ffma(f, s.y, s.x), amax);
        const float z = warp_depth(t, wa, wb);
        m0 += a;
        m1 = ffma(a, z, m1);
        const float az = a * z;
        m2 = ffma(az, z, m2);
        const float az2 = az * z;
        m3 = ffma(az2, z, m3);
        m4 = ffma(az2 * z, z, m4);
        ++n;
    }
    __device__ __forceinline__ void store(const GridD&, char* base, const ViewSlot& S, int64_t off, int pix) {
        store_moments(base, S, off, pix, m0, m1, m2, m3, m4);
    }
};

// Alg. 1 loop 2 per sample: colour += T(z) * alpha * (r, g, b, 1).
struct BlendBody {
    const float4* s_tf;   // [2*i] = entry i (r, g, b, sigma*step), [2*i+1] = entry i+1 minus entry i
    Frame F;
    float tf_scale, tf_bias, amax, wa, wb, w0;
    float b0;
    float4 C = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    unsigned n = 0;
    __device__ __forceinline__ void operator()(float t, float val) {
        const float xt = fclamp(ffma(val, tf_scale, tf_bias), 0.0f, 255.0f);
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float4 e0 = s_tf[2 * i], de = s_tf[2 * i + 1];
        const float a = fmin_(ffma(f, de.w, e0.w), amax);
        const float alpha = one_minus_exp_neg(a);
        const float z = warp_depth(t, wa, wb);
        const float wgt = transmittance(F, z, w0) * alpha;
        C.x = ffma(wgt, ffma(f, de.x, e0.x), C.x);
        C.y = ffma(wgt, ffma(f, de.y, e0.y), C.y);
        C.z = ffma(wgt, ffma(f, de.z, e0.z), C.z);
        C.w += wgt;
        ++n;
    }
    __device__ __forceinline__ bool singular() const { return F.kind == kFrameOneAtom || F.kind == kFrameTwoAtoms; }
};

// Bytes of one moment slab of P pixels in the volume's format.
__device__ __forceinline__ int64_t slab_bytes(const GridD& g, int plane) {
    return g.trig.n ? (int64_t)(4 + 4 * g.trig.n) * plane : (int64_t)20 * plane;
}

__device__ __forceinline__ uint32_t pack16(const GridD& g, float x, float y) {
    if (g.trig.storage == 2) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ cf unpack16(const GridD& g, uint32_t bits) {
    if (g.trig.storage == 2) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&bits);
        return {__low2float(h), __high2float(h)};
    }
    const __half2 h = *reinterpret_cast<const __half2*>(&bits);
    return {__low2float(h), __high2float(h)};
}

// Trigonometric moment slab: b0 plane (float), then plane j of tau_j = t_j / b0
// as a 16-bit pair.
__device__ __forceinline__ void store_trig(const GridD& g, char* base, const ViewSlot& S, int64_t slab_off, int pix,
                                           float m0, const cf* t, int n) {
    char* slab = base + slab_off;
    reinterpret_cast<float*>(slab)[pix] = m0;
    const float inv = m0 > 0.0f ? 1.0f / m0 : 0.0f;
    for (int j = 0; j < n; ++j)
        reinterpret_cast<uint32_t*>(slab + (size_t)4 * S.plane * (1 + j))[pix] = pack16(g, t[j].x * inv, t[j].y * inv);
}

__device__ __forceinline__ float load_trig(const GridD& g, const char* base, const ViewSlot& S, int64_t slab_off,
                                           int pix, cf* tau, int n) {
    const char* slab = base + slab_off;
    for (int j = 0; j < n; ++j)
        tau[j] = unpack16(g, __ldg(reinterpret_cast<const uint32_t*>(slab + (size_t)4 * S.plane * (1 + j)) + pix));
    return __ldg(reinterpret_cast<const float*>(slab) + pix);
}

// Pass 1 with trigonometric moments: b0 += a, t_j += a e^{i j phi}.
template <int N>
struct TrigMomentBody {
    const float2* s_sig;
    float tf_scale, tf_bias, amax, wa, wb, zs;
    float m0 = 0.0f;
    cf t[N];
    unsigned n = 0;
    __device__ __forceinline__ void operator()(float tt, float val) {
        const float xt = fclamp(ffma(val, tf_scale, tf_bias), 0.0f, 255.0f);
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float2 s = s_sig[i];
        const float a = fmin_(ffma(f, s.y, s.x), amax);
        const float phi = warp_depth(tt, wa, wb) * zs;
        float sn, cs;
        __sincosf(phi, &sn, &cs);
        const cf u = {cs, sn};
        cf p = u;
        m0 += a;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j > 0) p = cmul(p, u);
            t[j].x = ffma(a, p.x, t[j].x);
            t[j].y = ffma(a, p.y, t[j].y);
        }
        ++n;
    }
    __device__ __forceinline__ void store(const GridD& g, char* base, const ViewSlot& S, int64_t off, int pix) {
        store_trig(g, base, S, off, pix, m0, t, N);
    }
};

// Pass 2 with trigonometric moments.
template <int N>
struct TrigBlendBody {
    const float4* s_tf;
    const TrigTables* T;
    TrigFrame F;
    float tf_scale, tf_bias, amax, wa, wb, w0;
    float b0;
    float4 C = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    unsigned n = 0;
    __device__ __forceinline__ void operator()(float t, float val) {
        const float xt = fclamp(ffma(val, tf_scale, tf_bias), 0.0f, 255.0f);
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float4 e0 = s_tf[2 * i], de = s_tf[2 * i + 1];
        const float a = fmin_(ffma(f, de.w, e0.w), amax);
        const float alpha = one_minus_exp_neg(a);
        const float z = warp_depth(t, wa, wb);
        const float A = trig_fraction<N>(F, *T, z, w0);
        const float wgt = fclamp(fexp2(-F.m0_log2e * A), 0.0f, 1.0f) * alpha;
        C.x = ffma(wgt, ffma(f, de.x, e0.x), C.x);
        C.y = ffma(wgt, ffma(f, de.y, e0.y), C.y);
        C.z = ffma(wgt, ffma(f, de.z, e0.z), C.z);
        C.w += wgt;
        ++n;
    }
    __device__ __forceinline__ bool singular() const { return b0 > 0.0f && F.n == 0; }
};

template <int MS> struct Bodies;
template <> struct Bodies<0> {
    using Moment = MomentBody;
    using Blend = BlendBody;
};
template <> struct Bodies<3> {
    using Moment = TrigMomentBody<3>;
    using Blend = TrigBlendBody<3>;
};
template <> struct Bodies<4> {
    using Moment = TrigMomentBody<4>;
    using Blend = TrigBlendBody<4>;
};

template <int MS>
__device__ __forceinline__ typename Bodies<MS>::Moment make_moment_body(const float2* s_sig, const GridD& g,
                                                                        const ViewD& v) {
    typename Bodies<MS>::Moment b;
    b.s_sig = s_sig;
    b.tf_scale = g.tf_scale;
    b.tf_bias = g.tf_bias;
    b.amax = g.absorbance_max;
    b.wa = v.warp_a;
    b.wb = v.warp_b;
    if constexpr (MS != 0) {
        b.zs = g.trig.zone_scale;
        for (int j = 0; j < MS; ++j) b.t[j] = {0.0f, 0.0f};
    }
    return b;
}

// Loads the pixel's global moments (if `valid`) and builds the reconstruction.
template <int MS>
__device__ __forceinline__ typename Bodies<MS>::Blend make_blend_body(const float4* s_tf, const GridD& g, const ViewSlot& S,
                                                                      const char* moments, int64_t off, int pix,
                                                                      bool valid) {
    typename Bodies<MS>::Blend b;
    b.s_tf = s_tf;
    b.tf_scale = g.tf_scale;
    b.tf_bias = g.tf_bias;
    b.amax = g.absorbance_max;
    b.wa = S.v.warp_a;
    b.wb = S.v.warp_b;
    b.w0 = g.overestimation;
    if constexpr (MS == 0) {
        float m[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (valid) load_moments(moments, S, off, pix, m);
        b.F = make_frame(m, g.moment_bias, g.bias_vector);
        b.b0 = m[0];
    } else {
        cf tau[MS];
        for (int j = 0; j < MS; ++j) tau[j] = {0.0f, 0.0f};
        b.b0 = valid ? load_trig(g, moments, S, off, pix, tau, MS) : 0.0f;
        b.T = &g.trig;
        b.F = make_trig_frame(b.b0, tau, MS, g.trig.beta);
    }
    return b;
}


// Pops the next 8x4 ray tile of the work queue; returns false when empty.
__device__ __forceinline__ bool next_tile(const ViewTable& vt, int32_t* head, int& vi, int& px, int& py, int& tile) {
    const int lane = threadIdx.x & 31;
    tile = 0;
    if (lane == 0) tile = atomicAdd(head, 1);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= vt.total_tiles) return false;
    vi = find_view(vt, tile);
    const ViewSlot& S = vt.s[vi];
    const int lt = tile - S.tile_base;
    px = (lt % S.ntx) * kTileW + (lane & 7);
    py = (lt / S.ntx) * kTileH + (lane >> 3);
    return true;
}

__device__ __forceinline__ bool inside_domain(const GridD& g, const float o[3], const float d[3], int k) {
    const float t = lattice_t(k, g.step);
    const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
    return p0 >= 0.0f && p0 < g.hx && p1 >= 0.0f && p1 < g.hy && p2 >= 0.0f && p2 < g.hz;
}

// Ray of pixel (px, py) and the exact interval [k0, k1] of lattice indices
// whose float32 positions lie inside the domain (k0 > k1 if none).  Each
// coordinate of fma(t, d, o) is monotone in t, so the inside set of a box is
// one interval: it is found by shrinking the conservative range.
__device__ __forceinline__ void ray_range(const GridD& g, const ViewD& V, bool valid, int px, int py, float o[3],
                                          float d[3], int& k0, int& k1) {
    k0 = 0x7fffffff;
    k1 = -1;
    o[0] = o[1] = o[2] = 0.0f;
    d[0] = d[1] = d[2] = 0.0f;
    if (!valid) return;
    make_ray(V, px, py, o, d);
    const float lo[3] = {0.0f, 0.0f, 0.0f};
    const float hi[3] = {g.hx, g.hy, g.hz};
    int a, b;
    if (!lattice_range(o, d, lo, hi, g.step, &a, &b)) return;
    while (a <= b && !inside_domain(g, o, d, a)) ++a;
    while (b >= a && !inside_domain(g, o, d, b)) --b;
    if (a <= b) {
        k0 = a;
        k1 = b;
    }
}

// Asynchronous 16-byte global -> shared copies (no register staging).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kRowChunk = 8;                    // cache rows per prefetch
constexpr int kRowBuf = 2 * kRowChunk * 32;     // floats of a warp's double buffer

// Pass 2 of the batched frame from the tile cache.  The tile's rows are
// contiguous (rows[r * 32 + lane], r = k - kmin), so the warp copies them
// into its shared-memory buffer 8 rows (1 KiB) at a time, one chunk ahead of
// the one it blends, and every lane takes its own column over its own
// [k0, k1].  buf: 16-byte aligned, kRowBuf floats, this warp's only.
template <bool kSel, class Body>
__device__ __forceinline__ void march_rows(const GridD& g, const float* __restrict__ rows, int kmin, int kmax, int k0,
                                           int k1, float* __restrict__ buf, Body& body) {
    if (kmin > kmax) return;
    const int lane = threadIdx.x & 31;
    const int nrows = kmax - kmin + 1;
    const int nchunks = (nrows + kRowChunk - 1) / kRowChunk;
    auto fetch = [&](int c) {
        float* dst = buf + (c & 1) * kRowChunk * 32;
#pragma unroll
        for (int h = 0; h < kRowChunk / 4; ++h) {       // 16-byte pieces: 8 per row
            const int piece = lane + 32 * h, r = piece >> 3, q = (piece & 7) * 4;
            if (c * kRowChunk + r < nrows)
                cp_async16(dst + r * 32 + q, rows + (int64_t)(c * kRowChunk + r) * 32 + q);
        }
        cp_async_commit();
    };
    fetch(0);
    float t = lattice_t(kmin, g.step);
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks) {
            fetch(c + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const float* src = buf + (c & 1) * kRowChunk * 32 + lane;
        const int kc = kmin + c * kRowChunk;
        const int n = min(kRowChunk, kmax - kc + 1);
        for (int i = 0; i < n; ++i, t += g.step) {
            const int k = kc + i;
            if (k < k0 || k > k1) continue;
            const float val = src[i * 32];
            if (!kSel || val == val) body(t, val);  // every in-domain point is owned when no piece is left out
        }
        __syncwarp();  // every lane is done with the chunk before it is refilled
    }
}

// Pass 1: the tile's rows of the cache (lane 0 takes them, all lanes get the
// base; a tile that does not fit gets -1 and is marched again in pass 2).
__device__ __forceinline__ float* tile_rows(const TileCache& c, Counters* ctr, int tile, int k0, int k1) {
    const unsigned full = 0xffffffffu;
    const int kmin = __reduce_min_sync(full, k0), kmax = __reduce_max_sync(full, k1);
    long long base = -1;
    if ((threadIdx.x & 31) == 0) {
        if (kmax >= kmin) {
            const long long rows = (long long)kmax - kmin + 1;
            const long long r = (long long)atomicAdd(&ctr->cache_rows, (unsigned long long)rows);
            if (r + rows <= c.rows_cap) base = r;
        }
        c.tile_base[tile] = base;
    }
    base = __shfl_sync(full, base, 0);
    return base >= 0 ? c.vals + (base - kmin) * 32 + (threadIdx.x & 31) : nullptr;
}

template <bool kSel, class Cfg, int MS, bool kCache = false>
__global__ void __launch_bounds__(256) k_pass1_fused(const __grid_constant__ GridD g, const float4* __restrict__ tf,
                                                     const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                     char* __restrict__ moments, Counters* __restrict__ ctr,
                                                     const TileCache cache) {
    __shared__ float2 s_sig[256];
    __shared__ __align__(16) float s_win[kFusedWarps][Cfg::Floats];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    __syncthreads();
    float* win = s_win[threadIdx.x >> 5];
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        auto body = make_moment_body<MS>(s_sig, g, S.v);
        if constexpr (kCache) {
            RowStore st{tile_rows(cache, ctr, tile, k0, k1)};
            march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body, st);
        } else {
            march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body);
        }
        if (valid) body.store(g, moments, S, S.moment_off, py * S.v.width + px);
        warp_add_u64(&ctr->samples[0], body.n);
    }
}

template <bool kSel, class Cfg, int MS, bool kCache = false>
__global__ void __launch_bounds__(256) k_pass2_fused(const __grid_constant__ GridD g, const float4* __restrict__ tf,
                                                     const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                     const char* __restrict__ moments, float* __restrict__ color,
                                                     int mode, Counters* __restrict__ ctr, const TileCache cache) {
    static_assert(Cfg::Floats >= kRowBuf && Cfg::Floats % 4 == 0, "the window slot doubles as the row buffer");
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_win[kFusedWarps][Cfg::Floats];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    }
    __syncthreads();
    float* win = s_win[threadIdx.x >> 5];
    const bool raw = (g.flags & 1u) != 0;
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[1], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        const int pix = valid ? py * S.v.width + px : 0;
        auto body = make_blend_body<MS>(s_tf, g, S, moments, S.moment_off, pix, valid);
        if (valid && body.singular()) atomicAdd(&ctr->singular, 1ull);
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const long long tb = kCache ? cache.tile_base[tile] : -1;
        if (kCache && tb >= 0) {
            const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
            march_rows<kSel>(g, cache.vals + tb * 32, kmin, kmax, k0, k1, win, body);
        } else {
            march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body);
        }
        if (valid) {
            float4* out = reinterpret_cast<float4*>(color + S.color_off) + pix;
            if (mode == kColorResolved)
                *out = resolve_pixel(body.C, body.b0, make_float4(0.0f, 0.0f, 0.0f, 0.0f), raw);
            else
                *out = body.C;
        }
        warp_add_u64(&ctr->samples[1], body.n);
    }
}

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

__device__ __forceinline__ int unit_of(const AmrD& a, const float p[3]) {
    const int bl = a.g.brick_log2;
    const int fx = (int)p[0] >> bl, fy = (int)p[1] >> bl, fz = (int)p[2] >> bl;
    return __ldg(a.fmap + ((size_t)fz * a.fdim + fy) * (size_t)a.fdim + fx);
}

// Local coordinates (p - origin) / h are exact in float32 (h a power of two,
// |p - origin| below the leaf size), so cells match the oracle's.
__device__ __forceinline__ float unit_value(const AmrD& a, const float p[3], int leaf) {
    const int4 L = __ldg(a.leaves + leaf);
    const float inv_h = __int_as_float((127 - (a.max_level - L.w)) << 23);  // 2^-(max_level - level)
    const float qx = (p[0] - (float)L.x) * inv_h, qy = (p[1] - (float)L.y) * inv_h, qz = (p[2] - (float)L.z) * inv_h;
    const int cx = min((int)qx, a.nv - 2), cy = min((int)qy, a.nv - 2), cz = min((int)qz, a.nv - 2);
    const int nv = a.nv;
    const float* __restrict__ c = a.values + (size_t)leaf * nv * nv * nv + (cz * nv + cy) * nv + cx;
    const int sy = nv, sz = nv * nv;
    return trilinear8(__ldg(c), __ldg(c + 1), __ldg(c + sy), __ldg(c + sy + 1), __ldg(c + sz), __ldg(c + sz + 1),
                      __ldg(c + sz + sy), __ldg(c + sz + sy + 1), qx - (float)cx, qy - (float)cy, qz - (float)cz);
}

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

// Per-ray state of a sampler: none for grids and octrees (a point's unit is
// a table lookup), the current tet for meshes (the walk starts there).
struct NoWalk {};
struct TetWalk;
template <class V> struct WalkOf { using type = NoWalk; };
template <bool kNarrow> struct WalkOf<TetT<kNarrow>> { using type = TetWalk; };

// One owned sample of `piece` at lattice index k, or the next index to try.
template <class V>
__device__ __forceinline__ bool piece_sample(const V& vol, const int32_t* __restrict__ pou, int piece, float t,
                                             const float o[3], const float d[3], int k, float& val, int& k_next,
                                             NoWalk&) {
    const GridD& g = common(vol);
    k_next = k + 1;
    const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
    if (!(p[0] >= 0.0f && p[0] < g.hx && p[1] >= 0.0f && p[1] < g.hy && p[2] >= 0.0f && p[2] < g.hz)) return false;
    const int u = unit_of(vol, p);
    if (u < 0) return false;
    if (__ldg(pou + u) != piece) {
        k_next = skip_unit(vol, u, o, d, t, k);
        return false;
    }
    val = unit_value(vol, p, u);
    return true;
}

template <class V, int MS>
__global__ void __launch_bounds__(128) k_pass1_piece(const __grid_constant__ V vol, const float4* __restrict__ tf,
                                                     const int32_t* __restrict__ pob, int piece,
                                                     const __grid_constant__ PieceBox box,
                                                     const __grid_constant__ ViewTable vt, int slot, int n_slots,
                                                     char* __restrict__ moments, Counters* __restrict__ ctr) {
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
    const int px = (lt % S.ntx) * kTileW + (lane & 7);
    const int py = (lt / S.ntx) * kTileH + (lane >> 3);
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
                float val;
                int kn;
                const bool owned = piece_sample(vol, pob, piece, t, o, d, k, val, kn, walk);
                k = kn;
                if (owned) body(t, val);
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
    const int px = (lt % S.ntx) * kTileW + (lane & 7);
    const int py = (lt / S.ntx) * kTileH + (lane >> 3);
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
                float val;
                int kn;
                const bool owned = piece_sample(vol, pob, piece, t, o, d, k, val, kn, walk);
                k = kn;
                if (owned) body(t, val);
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
    const int b = bin_of(m, q);
    const int j1 = __ldg(m.bin_start + b + 1);
    for (int j = __ldg(m.bin_start + b); j < j1; ++j) {
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
        const int j0 = __ldg(m.bin_start + b);
        if (j0 == __ldg(m.bin_start + b + 1)) return false;  // no tet comes near q
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
                                             int& k_next, TetWalk& w) {
    const GridD& g = m.g;
    k_next = k + 1;
    const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
    if (!(p[0] >= 0.0f && p[0] < g.hx && p[1] >= 0.0f && p[1] < g.hy && p[2] >= 0.0f && p[2] < g.hz)) return false;
    int q[3];
    snap_point(m, p, q);
    long long D[4];
    if (!tet_walk<kNarrow>(m, w, q, D)) return false;
    if (__ldg(pou + w.T) != piece) return false;
    val = tet_value(D, w.v);
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
        const int j0 = __ldg(m.bin_start + b);
        if (j0 < __ldg(m.bin_start + b + 1)) load_tet(m, __ldg(m.bin_tets + j0), w);
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
            val = tet_value(D, w.v);
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

template <bool kSel, class Body, class Store = NoStore>
__device__ __forceinline__ void march_unit(const AmrD& a, const uint8_t* __restrict__ sel, const float o[3],
                                           const float d[3], int k0, int k1, Body& body, Store store = Store{}) {
    const GridD& g = a.g;
    if (k0 > k1) return;
    store.seek(k0);
    const float tz = lattice_t(k1, g.step);
    for (float t = lattice_t(k0, g.step); t <= tz; t += g.step) {
        const float p[3] = {ffma(t, d[0], o[0]), ffma(t, d[1], o[1]), ffma(t, d[2], o[2])};
        const int u = unit_of(a, p);
        if (u < 0 || (kSel && !__ldg(sel + u))) {
            store.put(__int_as_float(0x7fc00000));
            continue;
        }
        const float val = unit_value(a, p, u);
        store.put(val);
        body(t, val);
    }
}

// Resident 256-thread blocks per SM the unit kernels are compiled for (the
// mesh walk is latency-bound: more warps hide more of it).
#ifndef MB_TET_MIN_BLOCKS
#define MB_TET_MIN_BLOCKS 3
#endif
template <class V> struct MinBlocks { static constexpr int value = 1; };
template <bool k> struct MinBlocks<TetT<k>> { static constexpr int value = MB_TET_MIN_BLOCKS; };

template <class V, bool kSel, int MS, bool kCache = false>
__global__ void __launch_bounds__(256, MinBlocks<V>::value) k_pass1_unit(const __grid_constant__ V a, const float4* __restrict__ tf,
                                                    const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                    char* __restrict__ moments, Counters* __restrict__ ctr,
                                                    const TileCache cache) {
    __shared__ float2 s_sig[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    __syncthreads();
    const GridD& g = a.g;
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        auto body = make_moment_body<MS>(s_sig, g, S.v);
        if constexpr (kCache) {
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
__global__ void __launch_bounds__(256, MinBlocks<V>::value) k_pass2_unit(const __grid_constant__ V a, const float4* __restrict__ tf,
                                                    const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                    const char* __restrict__ moments, float* __restrict__ color, int mode,
                                                    Counters* __restrict__ ctr, const TileCache cache) {
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_rows[kCache ? kFusedWarps : 1][kCache ? kRowBuf : 4];
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
        if (valid && body.singular()) atomicAdd(&ctr->singular, 1ull);
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const long long tb = kCache ? cache.tile_base[tile] : -1;
        if (kCache && tb >= 0) {
            const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
            march_rows<true>(g, cache.vals + tb * 32, kmin, kmax, k0, k1, s_rows[kCache ? threadIdx.x >> 5 : 0], body);
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
    const int px = (lt % S.ntx) * kTileW + (lane & 7);
    const int py = (lt / S.ntx) * kTileH + (lane >> 3);
    if (px >= S.v.width || py >= S.v.height) return;
    const int64_t npix = (int64_t)S.v.width * S.v.height;
    const int64_t gpix = S.color_off / 4 + py * S.v.width + px;  // pixel index over all views
    const int64_t cidx = (S.color_off / 4) * n_slots + slot * npix + (py * S.v.width + px);
    float o[3], d[3];
    make_ray(S.v, px, py, o, d);
    int k0, k1;
    int nseg = 0;
    if (lattice_range(o, d, box.lo, box.hi, g.step, &k0, &k1)) {
        int64_t out = kFill ? starts[cidx] : 0;
        int prev = -2, key = 0;
        float4 cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float tr = 1.0f;
        typename WalkOf<V>::type walk;
        for (int k = k0; k <= k1;) {
            const float t = lattice_t(k, g.step);
            float val;
            int kn;
            if (!piece_sample(vol, pob, piece, t, o, d, k, val, kn, walk)) {
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
                int i;
                const float f = tf_coord(g, val, i);
                const float4 e0 = s_tf[i], e1 = s_tf[i + 1];
                const float a = fmin_(ffma(f, e1.w - e0.w, e0.w), g.absorbance_max);
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

// Per pixel: total segments over the pieces, and each (piece, pixel) run of
// counts turned into start offsets in place (given the pixel's base offset).
__global__ void k_sortlast_totals(const ViewTable vt, int n_slots, const int32_t* __restrict__ counts,
                                  int32_t* __restrict__ totals, int64_t total_px) {
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_px;
         gp += (int64_t)gridDim.x * blockDim.x) {
        int vi = 0;
        while (vi + 1 < vt.n && gp >= vt.s[vi + 1].color_off / 4) ++vi;
        const ViewSlot& S = vt.s[vi];
        const int64_t npix = (int64_t)S.v.width * S.v.height, local = gp - S.color_off / 4;
        const int32_t* c = counts + (S.color_off / 4) * n_slots + local;
        int32_t sum = 0;
        for (int j = 0; j < n_slots; ++j) sum += c[j * npix];
        totals[gp] = sum;
    }
}

__global__ void k_sortlast_starts(const ViewTable vt, int n_slots, const int32_t* __restrict__ counts,
                                  const int64_t* __restrict__ base, int64_t* __restrict__ starts, int64_t total_px) {
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_px;
         gp += (int64_t)gridDim.x * blockDim.x) {
        int vi = 0;
        while (vi + 1 < vt.n && gp >= vt.s[vi + 1].color_off / 4) ++vi;
        const ViewSlot& S = vt.s[vi];
        const int64_t npix = (int64_t)S.v.width * S.v.height, local = gp - S.color_off / 4;
        const int64_t off = (S.color_off / 4) * n_slots + local;
        int64_t run = base[gp];
        for (int j = 0; j < n_slots; ++j) {
            starts[off + j * npix] = run;
            run += counts[off + j * npix];
        }
    }
}

// Exclusive scan of int32 counts into int64 offsets, out[n] = total
// (three phases: 1024-element blocks, block sums, block offsets).
__global__ void __launch_bounds__(1024) k_scan_blocks(const int32_t* __restrict__ in, int64_t* __restrict__ out,
                                                      int64_t* __restrict__ bsum, int64_t n) {
    __shared__ int64_t wtot[32];
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t x = i < n ? in[i] : 0;
    int64_t v = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    if (lane == 31) wtot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = wtot[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        wtot[lane] = w;
    }
    __syncthreads();
    const int64_t incl = v + (warp > 0 ? wtot[warp - 1] : 0);
    if (i < n) out[i] = incl - x;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* __restrict__ bsum, int64_t nb, int64_t* __restrict__ total) {
    __shared__ int64_t wtot[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t x = i < nb ? bsum[i] : 0;
        int64_t v = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane == 31) wtot[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = wtot[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            wtot[lane] = w;
        }
        __syncthreads();
        const int64_t incl = v + (warp > 0 ? wtot[warp - 1] : 0) + carry;
        if (i < nb) bsum[i] = incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ bsum, int64_t n) {
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

// Per pixel: sort its segments by first lattice index (insertion sort; up to
// 64 in registers-backed local arrays, longer lists in place in global
// memory) and composite them front to back.
__global__ void k_sortlast_blend(const int64_t* __restrict__ base, int32_t* __restrict__ seg_key,
                                 float4* __restrict__ seg_col, float* __restrict__ rgba, int64_t total_px,
                                 Counters* __restrict__ ctr) {
    constexpr int kLocal = 64;
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_px;
         gp += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = base[gp], n = base[gp + 1] - b;
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float tr = 1.0f;
        if (n <= kLocal) {
            int key[kLocal];
            int idx[kLocal];
            for (int j = 0; j < n; ++j) {
                const int kj = seg_key[b + j];
                int m = j;
                while (m > 0 && key[m - 1] > kj) {
                    key[m] = key[m - 1];
                    idx[m] = idx[m - 1];
                    --m;
                }
                key[m] = kj;
                idx[m] = j;
            }
            for (int j = 0; j < n; ++j) {
                const float4 c = seg_col[b + idx[j]];
                acc.x = ffma(tr, c.x, acc.x);
                acc.y = ffma(tr, c.y, acc.y);
                acc.z = ffma(tr, c.z, acc.z);
                tr *= 1.0f - c.w;
            }
        } else {
            for (int64_t j = 1; j < n; ++j) {
                const int kj = seg_key[b + j];
                const float4 cj = seg_col[b + j];
                int64_t m = j;
                while (m > 0 && seg_key[b + m - 1] > kj) {
                    seg_key[b + m] = seg_key[b + m - 1];
                    seg_col[b + m] = seg_col[b + m - 1];
                    --m;
                }
                seg_key[b + m] = kj;
                seg_col[b + m] = cj;
            }
            for (int64_t j = 0; j < n; ++j) {
                const float4 c = seg_col[b + j];
                acc.x = ffma(tr, c.x, acc.x);
                acc.y = ffma(tr, c.y, acc.y);
                acc.z = ffma(tr, c.z, acc.z);
                tr *= 1.0f - c.w;
            }
        }
        reinterpret_cast<float4*>(rgba)[gp] = make_float4(acc.x, acc.y, acc.z, 1.0f - tr);
        if (n > 0) atomicMax(&ctr->max_segments, (int)n);
    }
}

// ------------------------------------------------------------------------
// image-space reductions (compensated, fixed input order)

struct Neumaier {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ float get() const { return s + c; }
};

__global__ void k_moments_sum(const float4* __restrict__ in, float4* __restrict__ out, int64_t n4, int n_inputs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        Neumaier x, y, z, w;
        for (int j = 0; j < n_inputs; ++j) {
            const float4 v = __ldg(in + (int64_t)j * n4 + i);
            x.add(v.x);
            y.add(v.y);
            z.add(v.z);
            w.add(v.w);
        }
        out[i] = make_float4(x.get(), y.get(), z.get(), w.get());
    }
}

// Trigonometric slabs: per pixel sum b0 and b0 * tau_j over the inputs
// (compensated), then renormalise and round to the storage format again.
template <int N>
__global__ void k_moments_sum_trig(const __grid_constant__ GridD g, const char* __restrict__ in, char* __restrict__ out,
                                   int64_t plane, int64_t npix, int n_inputs) {
    const int64_t slab = (int64_t)(4 + 4 * N) * plane;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
        Neumaier b0;
        Neumaier tr[N], ti[N];
        for (int j = 0; j < n_inputs; ++j) {
            const char* sl = in + j * slab;
            const float m0 = __ldg(reinterpret_cast<const float*>(sl) + i);
            b0.add(m0);
            for (int k = 0; k < N; ++k) {
                const cf t = unpack16(g, __ldg(reinterpret_cast<const uint32_t*>(sl + 4 * plane * (1 + k)) + i));
                tr[k].add(t.x * m0);
                ti[k].add(t.y * m0);
            }
        }
        const float m0 = b0.get();
        const float inv = m0 > 0.0f ? 1.0f / m0 : 0.0f;
        reinterpret_cast<float*>(out)[i] = m0;
        for (int k = 0; k < N; ++k)
            reinterpret_cast<uint32_t*>(out + 4 * plane * (1 + k))[i] = pack16(g, tr[k].get() * inv, ti[k].get() * inv);
    }
}

__global__ void k_color_resolve(const float4* __restrict__ in, float4* __restrict__ out, const float* __restrict__ b0,
                                int64_t npix, int n_inputs, float4 bg, int raw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
        Neumaier x, y, z, w;
        for (int j = 0; j < n_inputs; ++j) {
            const float4 v = __ldg(in + (int64_t)j * npix + i);
            x.add(v.x);
            y.add(v.y);
            z.add(v.z);
            w.add(v.w);
        }
        const float4 C = make_float4(x.get(), y.get(), z.get(), w.get());
        out[i] = resolve_pixel(C, raw ? 0.0f : __ldg(b0 + i), bg, raw != 0);
    }
}

// Resident CTAs per SM x SMs for a persistent kernel, cached per function.
int persistent_blocks(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, fn});
    if (it != cache.end()) return it->second;
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    const int nb = sms * (occ > 0 ? occ : 1);
    cache[{dev, fn}] = nb;
    return nb;
}

template <int MS, bool kC>
const void* pass1_fn_ms(int cfg, bool sel) {
    if (sel) return (const void*)k_pass1_fused<true, Stage0, MS, kC>;
    if constexpr (MS != 0) return cfg == 3 ? (const void*)k_pass1_fused<false, Stage3, MS, kC>
                                           : (const void*)k_pass1_fused<false, Stage0, MS, kC>;
    switch (cfg) {
        case 1: return (const void*)k_pass1_fused<false, Stage1, MS, kC>;
        case 2: return (const void*)k_pass1_fused<false, Stage2, MS, kC>;
        case 3: return (const void*)k_pass1_fused<false, Stage3, MS, kC>;
        case 4: return (const void*)k_pass1_fused<false, Stage4, MS, kC>;
        default: return (const void*)k_pass1_fused<false, Stage0, MS, kC>;
    }
}

template <int MS, bool kC>
const void* pass2_fn_ms(int cfg, bool sel) {
    if (sel) return (const void*)k_pass2_fused<true, Stage0, MS, kC>;
    if constexpr (MS != 0) return cfg == 3 ? (const void*)k_pass2_fused<false, Stage3, MS, kC>
                                           : (const void*)k_pass2_fused<false, Stage0, MS, kC>;
    switch (cfg) {
        case 1: return (const void*)k_pass2_fused<false, Stage1, MS, kC>;
        case 2: return (const void*)k_pass2_fused<false, Stage2, MS, kC>;
        case 3: return (const void*)k_pass2_fused<false, Stage3, MS, kC>;
        case 4: return (const void*)k_pass2_fused<false, Stage4, MS, kC>;
        default: return (const void*)k_pass2_fused<false, Stage0, MS, kC>;
    }
}

template <bool kC = false>
const void* pass1_fn(int cfg, bool sel, int ms) {
    return ms == 3 ? pass1_fn_ms<3, kC>(cfg, sel) : ms == 4 ? pass1_fn_ms<4, kC>(cfg, sel) : pass1_fn_ms<0, kC>(cfg, sel);
}
template <bool kC = false>
const void* pass2_fn(int cfg, bool sel, int ms) {
    return ms == 3 ? pass2_fn_ms<3, kC>(cfg, sel) : ms == 4 ? pass2_fn_ms<4, kC>(cfg, sel) : pass2_fn_ms<0, kC>(cfg, sel);
}

// One warp per ray tile: adds the tile's cache rows (kmax - kmin + 1 over its
// rays' exact in-domain intervals, as pass 1 will take them) to *rows.
__global__ void __launch_bounds__(256) k_tile_rows(const __grid_constant__ GridD g, const __grid_constant__ ViewTable vt,
                                                   unsigned long long* __restrict__ rows) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    unsigned long long mine = 0;
    for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < vt.total_tiles; tile += warps) {
        const int vi = find_view(vt, tile);
        const ViewSlot& S = vt.s[vi];
        const int lt = tile - S.tile_base;
        const int px = (lt % S.ntx) * kTileW + (lane & 7);
        const int py = (lt / S.ntx) * kTileH + (lane >> 3);
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
        if (kmax >= kmin) mine += (unsigned long long)(kmax - kmin + 1);
    }
    if (lane == 0 && mine) atomicAdd(rows, mine);
}
template <class V, bool kC = false>
const void* unit1_fn(bool sel, int ms) {
    if (ms == 3) return sel ? (const void*)k_pass1_unit<V, true, 3, kC> : (const void*)k_pass1_unit<V, false, 3, kC>;
    if (ms == 4) return sel ? (const void*)k_pass1_unit<V, true, 4, kC> : (const void*)k_pass1_unit<V, false, 4, kC>;
    return sel ? (const void*)k_pass1_unit<V, true, 0, kC> : (const void*)k_pass1_unit<V, false, 0, kC>;
}
template <class V, bool kC = false>
const void* unit2_fn(bool sel, int ms) {
    if (ms == 3) return sel ? (const void*)k_pass2_unit<V, true, 3, kC> : (const void*)k_pass2_unit<V, false, 3, kC>;
    if (ms == 4) return sel ? (const void*)k_pass2_unit<V, true, 4, kC> : (const void*)k_pass2_unit<V, false, 4, kC>;
    return sel ? (const void*)k_pass2_unit<V, true, 0, kC> : (const void*)k_pass2_unit<V, false, 0, kC>;
}

__global__ void k_tet_values(int4* __restrict__ corners, const int4* __restrict__ cells, int64_t n_tets,
                             const float* __restrict__ values) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets; t += (int64_t)gridDim.x * blockDim.x) {
        const int4 c = cells[t];
        corners[4 * t].w = __float_as_int(values[c.x]);
        corners[4 * t + 1].w = __float_as_int(values[c.y]);
        corners[4 * t + 2].w = __float_as_int(values[c.z]);
        corners[4 * t + 3].w = __float_as_int(values[c.w]);
    }
}

bool vec_config(int cfg) { return cfg == 2 || cfg == 3 || cfg == 4; }

}  // namespace

bool stage_config_eligible(const GridD& g, int cfg) {
    if (cfg < 0 || cfg >= kNumStageConfigs) return false;
    if (g.trig.n != 0 && cfg != 0 && cfg != 3) return false;
    if (!vec_config(cfg)) return true;
    return g.nx % 4 == 0 && g.nx >= 4 && (reinterpret_cast<uintptr_t>(g.field) & 15u) == 0;
}

cudaError_t prepare_kernels() {
    // Loads every kernel and fills the occupancy cache, so that no module
    // loading happens later inside a stream capture.
    const void* fns[] = {(const void*)k_pass1_piece<GridD, 0>, (const void*)k_pass2_piece<GridD, 0>,
                         (const void*)k_pass1_piece<GridD, 3>, (const void*)k_pass2_piece<GridD, 3>,
                         (const void*)k_pass1_piece<GridD, 4>, (const void*)k_pass2_piece<GridD, 4>,
                         (const void*)k_pass1_piece<AmrD, 0>, (const void*)k_pass2_piece<AmrD, 0>,
                         (const void*)k_pass1_piece<AmrD, 3>, (const void*)k_pass2_piece<AmrD, 3>,
                         (const void*)k_pass1_piece<AmrD, 4>, (const void*)k_pass2_piece<AmrD, 4>,
                         (const void*)k_moments_sum_trig<3>, (const void*)k_moments_sum_trig<4>,
                         (const void*)k_moments_sum,        (const void*)k_color_resolve,
                         (const void*)k_sortlast_piece<GridD, true>, (const void*)k_sortlast_piece<GridD, false>,
                         (const void*)k_sortlast_piece<AmrD, true>, (const void*)k_sortlast_piece<AmrD, false>,
                         (const void*)k_pass1_piece<TetT<true>, 0>, (const void*)k_pass2_piece<TetT<true>, 0>,
                         (const void*)k_pass1_piece<TetT<true>, 3>, (const void*)k_pass2_piece<TetT<true>, 3>,
                         (const void*)k_pass1_piece<TetT<true>, 4>, (const void*)k_pass2_piece<TetT<true>, 4>,
                         (const void*)k_sortlast_piece<TetT<true>, true>, (const void*)k_sortlast_piece<TetT<true>, false>,
                         (const void*)k_pass1_piece<TetT<false>, 0>, (const void*)k_pass2_piece<TetT<false>, 0>,
                         (const void*)k_pass1_piece<TetT<false>, 3>, (const void*)k_pass2_piece<TetT<false>, 3>,
                         (const void*)k_pass1_piece<TetT<false>, 4>, (const void*)k_pass2_piece<TetT<false>, 4>,
                         (const void*)k_sortlast_piece<TetT<false>, true>, (const void*)k_sortlast_piece<TetT<false>, false>,
                         (const void*)k_tet_values,         (const void*)k_tile_rows,
                         (const void*)k_sortlast_totals,    (const void*)k_sortlast_starts,
                         (const void*)k_scan_blocks,        (const void*)k_scan_sums,
                         (const void*)k_scan_add,           (const void*)k_sortlast_blend};
    for (const void* f : fns) {
        cudaFuncAttributes a;
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    const int sets[3] = {0, 3, 4};
    for (int ms : sets)
        for (int cfg = 0; cfg < kNumStageConfigs; ++cfg)
            for (int sel = 0; sel < 2; ++sel) {
                const void* fs[4] = {pass1_fn(cfg, sel, ms), pass2_fn(cfg, sel, ms), pass1_fn<true>(cfg, sel, ms),
                                     pass2_fn<true>(cfg, sel, ms)};
                for (const void* f : fs) {
                    cudaFuncAttributes a;
                    const cudaError_t e = cudaFuncGetAttributes(&a, f);
                    if (e != cudaSuccess) return e;
                    persistent_blocks(f, 256, 0);
                }
            }
    for (int ms : sets)
        for (int sel = 0; sel < 2; ++sel) {
            persistent_blocks(unit1_fn<AmrD>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<AmrD>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<AmrD, true>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<AmrD, true>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<true>>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<true>>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<false>>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<false>>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<true>, true>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<true>, true>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<false>, true>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<false>, true>(sel, ms), 256, 0);
        }
    return cudaGetLastError();
}

cudaError_t launch_pass1_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               void* moments, Counters* ctr, cudaStream_t s, int cfg, TileCache cache) {
    if (!stage_config_eligible(g, cfg)) cfg = 0;
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = brick_sel != nullptr;
    const void* fn = cache.vals ? pass1_fn<true>(cfg, sel, g.trig.n) : pass1_fn(cfg, sel, g.trig.n);
    char* m = static_cast<char*>(moments);
    void* args[] = {(void*)&g, (void*)&tf, (void*)&brick_sel, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass2_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                               int cfg, TileCache cache) {
    if (!stage_config_eligible(g, cfg)) cfg = 0;
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const bool sel = brick_sel != nullptr;
    const void* fn = cache.vals ? pass2_fn<true>(cfg, sel, g.trig.n) : pass2_fn(cfg, sel, g.trig.n);
    const char* m = static_cast<const char*>(moments);
    int md = mode;
    void* args[] = {(void*)&g, (void*)&tf, (void*)&brick_sel, (void*)&vt, (void*)&m, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_tile_rows(const GridD& g, const ViewTable& vt, unsigned long long* rows, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 7) / 8;
    k_tile_rows<<<blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096, 256, 0, s>>>(g, vt, rows);
    return cudaGetLastError();
}

cudaError_t launch_pass1_piece(const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               void* moments, Counters* ctr, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    char* m = static_cast<char*>(moments);
    if (g.trig.n == 3) k_pass1_piece<GridD, 3><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, m, ctr);
    else if (g.trig.n == 4) k_pass1_piece<GridD, 4><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, m, ctr);
    else k_pass1_piece<GridD, 0><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, m, ctr);
    return cudaGetLastError();
}

cudaError_t launch_pass2_piece(const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               const void* moments, float* color, Counters* ctr, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    const char* m = static_cast<const char*>(moments);
    if (g.trig.n == 3) k_pass2_piece<GridD, 3><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, m, color, ctr);
    else if (g.trig.n == 4) k_pass2_piece<GridD, 4><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, m, color, ctr);
    else k_pass2_piece<GridD, 0><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, m, color, ctr);
    return cudaGetLastError();
}

cudaError_t launch_moments_sum(const GridD& g, const ViewTable& vt, int32_t n_inputs, const void* in, void* out,
                               cudaStream_t s) {
    for (int v = 0; v < vt.n; ++v) {
        const ViewSlot& S = vt.s[v];
        if (g.trig.n) {
            const int64_t npix = (int64_t)S.v.width * S.v.height;
            const char* src = static_cast<const char*>(in) + S.moment_off * n_inputs;
            char* dst = static_cast<char*>(out) + S.moment_off;
            const int blocks = (int)((npix + 255) / 256 < 4096 ? (npix + 255) / 256 : 4096);
            if (g.trig.n == 3)
                k_moments_sum_trig<3><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g, src, dst, S.plane, npix, n_inputs);
            else
                k_moments_sum_trig<4><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g, src, dst, S.plane, npix, n_inputs);
            continue;
        }
        const int64_t n4 = (int64_t)5 * S.plane / 4;
        const float4* src = reinterpret_cast<const float4*>(static_cast<const char*>(in) + S.moment_off * n_inputs);
        float4* dst = reinterpret_cast<float4*>(static_cast<char*>(out) + S.moment_off);
        const int blocks = (int)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
        k_moments_sum<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(src, dst, n4, n_inputs);
    }
    return cudaGetLastError();
}

cudaError_t launch_color_resolve(const ViewTable& vt, int32_t n_inputs, const float* in, float* out,
                                 const void* moments, float4 bg, int32_t raw_sum, cudaStream_t s) {
    for (int v = 0; v < vt.n; ++v) {
        const ViewSlot& S = vt.s[v];
        const int64_t npix = (int64_t)S.v.width * S.v.height;
        const float4* src = reinterpret_cast<const float4*>(in + S.color_off * n_inputs);
        float4* dst = reinterpret_cast<float4*>(out + S.color_off);
        const float* b0 = moments ? reinterpret_cast<const float*>(static_cast<const char*>(moments) + S.moment_off)
                                  : nullptr;
        const int blocks = (int)((npix + 255) / 256 < 4096 ? (npix + 255) / 256 : 4096);
        k_color_resolve<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(src, dst, b0, npix, n_inputs, bg, raw_sum);
    }
    return cudaGetLastError();
}

cudaError_t launch_sortlast_march(bool fill, const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    if (fill)
        k_sortlast_piece<GridD, true><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, counts, starts, seg_key,
                                                      seg_col);
    else
        k_sortlast_piece<GridD, false><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, counts, starts,
                                                       seg_key, seg_col);
    return cudaGetLastError();
}

cudaError_t launch_sortlast_offsets(const ViewTable& vt, int32_t n_slots, const int32_t* counts, int32_t* totals,
                                   int64_t* base, int64_t* bsum, int64_t* starts, int64_t total_px, cudaStream_t s) {
    const int grid = (int)((total_px + 255) / 256 < 8192 ? (total_px + 255) / 256 : 8192);
    k_sortlast_totals<<<grid, 256, 0, s>>>(vt, n_slots, counts, totals, total_px);
    const int64_t nb = (total_px + 1023) / 1024;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, s>>>(totals, base, bsum, total_px);
    k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, base + total_px);
    k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(base, bsum, total_px);
    k_sortlast_starts<<<grid, 256, 0, s>>>(vt, n_slots, counts, base, starts, total_px);
    return cudaGetLastError();
}

cudaError_t launch_sortlast_blend(const int64_t* base, int32_t* seg_key, float4* seg_col, float* rgba, int64_t total_px,
                                  Counters* ctr, cudaStream_t s) {
    const int grid = (int)((total_px + 127) / 128 < 16384 ? (total_px + 127) / 128 : 16384);
    k_sortlast_blend<<<grid, 128, 0, s>>>(base, seg_key, seg_col, rgba, total_px, ctr);
    return cudaGetLastError();
}

cudaError_t launch_pass1_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, Counters* ctr, cudaStream_t s, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr;
    const void* fn = cache.vals ? unit1_fn<AmrD, true>(sel, a.g.trig.n) : unit1_fn<AmrD>(sel, a.g.trig.n);
    char* m = static_cast<char*>(moments);
    void* args[] = {(void*)&a, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass2_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr;
    const void* fn = cache.vals ? unit2_fn<AmrD, true>(sel, a.g.trig.n) : unit2_fn<AmrD>(sel, a.g.trig.n);
    const char* m = static_cast<const char*>(moments);
    int md = mode;
    void* args[] = {(void*)&a, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&m, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass1_piece(const AmrD& a, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, void* moments, Counters* ctr,
                               cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    char* m = static_cast<char*>(moments);
    if (a.g.trig.n == 3) k_pass1_piece<AmrD, 3><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, m, ctr);
    else if (a.g.trig.n == 4) k_pass1_piece<AmrD, 4><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, m, ctr);
    else k_pass1_piece<AmrD, 0><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, m, ctr);
    return cudaGetLastError();
}

cudaError_t launch_pass2_piece(const AmrD& a, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, const void* moments, float* color,
                               Counters* ctr, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    const char* m = static_cast<const char*>(moments);
    if (a.g.trig.n == 3) k_pass2_piece<AmrD, 3><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, m, color, ctr);
    else if (a.g.trig.n == 4) k_pass2_piece<AmrD, 4><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, m, color, ctr);
    else k_pass2_piece<AmrD, 0><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, m, color, ctr);
    return cudaGetLastError();
}

cudaError_t launch_sortlast_march(bool fill, const AmrD& a, const float4* tf, const int32_t* pou, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    if (fill)
        k_sortlast_piece<AmrD, true><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                            seg_key, seg_col);
    else
        k_sortlast_piece<AmrD, false><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                             seg_key, seg_col);
    return cudaGetLastError();
}

namespace {

template <bool kN>
TetT<kN> as_tet(const TetD& m) {
    TetT<kN> t;
    static_cast<TetD&>(t) = m;
    return t;
}

template <class V>
cudaError_t launch_unit1(const V& vol, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt, void* moments,
                         Counters* ctr, cudaStream_t s, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr;
    const void* fn = cache.vals ? unit1_fn<V, true>(sel, vol.g.trig.n) : unit1_fn<V>(sel, vol.g.trig.n);
    char* mo = static_cast<char*>(moments);
    void* args[] = {(void*)&vol, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&mo, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

template <class V>
cudaError_t launch_unit2(const V& vol, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                         const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                         TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr;
    const void* fn = cache.vals ? unit2_fn<V, true>(sel, vol.g.trig.n) : unit2_fn<V>(sel, vol.g.trig.n);
    const char* mo = static_cast<const char*>(moments);
    int md = mode;
    void* args[] = {(void*)&vol, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&mo, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

template <class V>
cudaError_t launch_piece1(const V& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                          const ViewTable& vt, int32_t slot, int32_t n_slots, void* moments, Counters* ctr,
                          cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    char* mo = static_cast<char*>(moments);
    if (m.g.trig.n == 3) k_pass1_piece<V, 3><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, mo, ctr);
    else if (m.g.trig.n == 4) k_pass1_piece<V, 4><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, mo, ctr);
    else k_pass1_piece<V, 0><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, mo, ctr);
    return cudaGetLastError();
}

template <class V>
cudaError_t launch_piece2(const V& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                          const ViewTable& vt, int32_t slot, int32_t n_slots, const void* moments, float* color,
                          Counters* ctr, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    const char* mo = static_cast<const char*>(moments);
    if (m.g.trig.n == 3) k_pass2_piece<V, 3><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, mo, color, ctr);
    else if (m.g.trig.n == 4) k_pass2_piece<V, 4><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, mo, color, ctr);
    else k_pass2_piece<V, 0><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, mo, color, ctr);
    return cudaGetLastError();
}

template <class V>
cudaError_t launch_sortlast(bool fill, const V& m, const float4* tf, const int32_t* pou, int32_t piece,
                            const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots, int32_t* counts,
                            const int64_t* starts, int32_t* seg_key, float4* seg_col, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    if (fill)
        k_sortlast_piece<V, true><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                         seg_key, seg_col);
    else
        k_sortlast_piece<V, false><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                          seg_key, seg_col);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass1_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, Counters* ctr, cudaStream_t s, TileCache cache) {
    return m.narrow ? launch_unit1(as_tet<true>(m), tf, unit_sel, vt, moments, ctr, s, cache)
                    : launch_unit1(as_tet<false>(m), tf, unit_sel, vt, moments, ctr, s, cache);
}

cudaError_t launch_pass2_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache) {
    return m.narrow ? launch_unit2(as_tet<true>(m), tf, unit_sel, vt, moments, color, mode, ctr, s, cache)
                    : launch_unit2(as_tet<false>(m), tf, unit_sel, vt, moments, color, mode, ctr, s, cache);
}

cudaError_t launch_pass1_piece(const TetD& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, void* moments, Counters* ctr,
                               cudaStream_t s) {
    return m.narrow ? launch_piece1(as_tet<true>(m), tf, pou, piece, box, vt, slot, n_slots, moments, ctr, s)
                    : launch_piece1(as_tet<false>(m), tf, pou, piece, box, vt, slot, n_slots, moments, ctr, s);
}

cudaError_t launch_pass2_piece(const TetD& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, const void* moments, float* color,
                               Counters* ctr, cudaStream_t s) {
    return m.narrow ? launch_piece2(as_tet<true>(m), tf, pou, piece, box, vt, slot, n_slots, moments, color, ctr, s)
                    : launch_piece2(as_tet<false>(m), tf, pou, piece, box, vt, slot, n_slots, moments, color, ctr, s);
}

cudaError_t launch_sortlast_march(bool fill, const TetD& m, const float4* tf, const int32_t* pou, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s) {
    return m.narrow ? launch_sortlast(fill, as_tet<true>(m), tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                      seg_key, seg_col, s)
                    : launch_sortlast(fill, as_tet<false>(m), tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                      seg_key, seg_col, s);
}

cudaError_t launch_tet_values(int4* corners, const int4* cells, int64_t n_tets, const float* values, cudaStream_t s) {
    const int64_t nb = (n_tets + 255) / 256;
    k_tet_values<<<(unsigned)(nb < 4096 ? (nb > 0 ? nb : 1) : 4096), 256, 0, s>>>(corners, cells, n_tets, values);
    return cudaGetLastError();
}

}  // namespace mb
