// Device code shared by the kernel translation units of the MBOIT
// puzzle-piece render (sm_103a): transfer-function and moment-image helpers,
// the per-sample bodies of pass 1 (Alg. 2) and pass 2 (Alg. 1 loop 2, Alg. 3),
// the work queue of 8 x 4 ray tiles, exact in-domain ray intervals, and the
// frame's tile-row sample cache (pass 1 stores, pass 2 prefetches and reads).
// Everything here is internal (an unnamed namespace per translation unit).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mboit_internal.h"
#include "mboit_power.cuh"
#include "mboit_trig.cuh"

namespace mb {

// Resident CTAs per SM x SMs for a persistent kernel, cached per function.
int persistent_blocks(const void* fn, int threads, size_t smem);

namespace {

constexpr int kFusedWarps = 8;  // 256 threads per CTA

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

// Transfer-function table coordinate of sample value v (O5): the value
// normalised to [0, 1] by the table's range, times 255, clamped.  The
// marches hand this to the per-sample bodies, and the frame's sample cache
// stores it, so pass 2 repeats none of it.
__device__ __forceinline__ float tf_x(const GridD& g, float v) {
    return fclamp(ffma(v, g.tf_scale, g.tf_bias), 0.0f, 255.0f);
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

// a - b per component, one rounding each (fma(b, -1, a)), as one packed
// FP32x2 instruction.
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// Trilinear interpolation: x lerps of the four edges, y lerps of the two
// faces, z lerp.  The z = 0 and z = 1 halves go through the packed FP32x2
// pipe together (two IEEE operations per instruction), so every value is
// rounded exactly as in the scalar form a = fma(fx, v1 - v0, v0).
__device__ __forceinline__ float trilinear8(float v000, float v100, float v010, float v110, float v001, float v101,
                                            float v011, float v111, float fx, float fy, float fz) {
    const float2 fx2 = make_float2(fx, fx);
    const float2 lo0 = make_float2(v000, v001), lo1 = make_float2(v010, v011);
    const float2 a0 = __ffma2_rn(fx2, fsub2(make_float2(v100, v101), lo0), lo0);  // (a00, a01)
    const float2 a1 = __ffma2_rn(fx2, fsub2(make_float2(v110, v111), lo1), lo1);  // (a10, a11)
    const float2 b = __ffma2_rn(make_float2(fy, fy), fsub2(a1, a0), a0);          // (b0, b1)
    return ffma(fz, b.y - b.x, b.x);
}

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

// Depth terms of lattice depth t for four power moments: the warped depth z
// (Alg. 2) and its powers z^2 = z z, z^3 = z^2 z, z^4 = z^3 z.  They depend on
// t only, so a warp whose lanes sit at the same lattice index can compute
// them once per row (DepthRows) and share them.
__device__ __forceinline__ float4 depth_powers(float t, float wa, float wb) {
    const float z = warp_depth(t, wa, wb);
    const float z2 = z * z, z3 = z2 * z;
    return make_float4(z, z2, z3, z3 * z);
}

// The pixel's reconstruction frame: float-float FP32 set-up with FP64 for
// near-singular Hankel matrices, or FP64 for every pixel (kFlagFp64Setup).
__device__ __forceinline__ Frame pixel_frame(const GridD& g, const float m[5], bool* fp64) {
    if (g.flags & kFlagFp64Setup) {
        *fp64 = m[0] > 0.0f;
        return make_frame(m, g.moment_bias, g.bias_vector);
    }
    return make_frame_ff(m, g.moment_bias, g.bias_vector, fp64);
}

struct MomentBody {
    const float2* s_sig;  // (sigma*step of entry i, of entry i+1 minus entry i)
    float tf_scale, tf_bias, amax, wa, wb;
    float m0 = 0.0f;
    float2 m12 = make_float2(0.0f, 0.0f), m34 = make_float2(0.0f, 0.0f);   // (b1, b2), (b3, b4)
    unsigned n = 0;
    // b_j += a z^j from the sample's table coordinate xt (tf_x) and the depth
    // powers zp of its lattice point; entry 255 has a zero delta, so xt = 255
    // needs no special index
    __device__ __forceinline__ void add(float xt, float ws, float4 zp) {
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float2 s = s_sig[i];
        const float a = fmin_(ffma(f, s.y, s.x) * ws, amax);
        m0 += a;
        // b_j += a z^j for j = 1, 2 and j = 3, 4 as two packed FP32x2 fmas
        // (each half rounded as a scalar fma)
        const float2 aa = make_float2(a, a);
        m12 = __ffma2_rn(aa, make_float2(zp.x, zp.y), m12);
        m34 = __ffma2_rn(aa, make_float2(zp.z, zp.w), m34);
        ++n;
    }
    __device__ __forceinline__ void operator()(float t, float xt, float ws = 1.0f) {
        add(xt, ws, depth_powers(t, wa, wb));
    }
    __device__ __forceinline__ void store(const GridD&, char* base, const ViewSlot& S, int64_t off, int pix) {
        store_moments(base, S, off, pix, m0, m12.x, m12.y, m34.x, m34.y);
    }
};

// A warp's shared depth terms of kDepthRows consecutive lattice rows (one
// float4 per row in the warp's shared memory): lanes 0..kDepthRows-1 compute
// one row each, every lane reads the rows it samples.
constexpr int kDepthRows = 8;
struct DepthRows {
    float4* z;   // this warp's kDepthRows slots
    __device__ __forceinline__ void fill(int kw, float step, float wa, float wb) {
        const int lane = threadIdx.x & 31;
        __syncwarp();   // every lane is done with the previous rows
        if (lane < kDepthRows) z[lane] = depth_powers(lattice_t(kw + lane, step), wa, wb);
        __syncwarp();
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
    bool fp64 = false;    // the frame was set up in FP64 (near-singular Hankel matrix)
    // kGeneric: the frame is known to be generic (no test of its kind)
    template <bool kGeneric = false>
    __device__ __forceinline__ void sample(float t, float xt, float ws) {
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float4 e0 = s_tf[2 * i], de = s_tf[2 * i + 1];
        const float a = fmin_(ffma(f, de.w, e0.w) * ws, amax);
        const float alpha = one_minus_exp_neg(a);
        const float z = warp_depth(t, wa, wb);
        const float wgt = (kGeneric ? transmittance_generic(F, z, w0) : transmittance(F, z, w0)) * alpha;
        C.x = ffma(wgt, ffma(f, de.x, e0.x), C.x);
        C.y = ffma(wgt, ffma(f, de.y, e0.y), C.y);
        C.z = ffma(wgt, ffma(f, de.z, e0.z), C.z);
        C.w += wgt;
        ++n;
    }
    __device__ __forceinline__ void operator()(float t, float xt, float ws = 1.0f) { sample<false>(t, xt, ws); }
    __device__ __forceinline__ bool singular() const { return F.kind == kFrameOneAtom || F.kind == kFrameTwoAtoms; }

    // Two consecutive lattice points (warped depths z.x, z.y; weight 1, the
    // fixed step) of a generic frame: the arithmetic of sample<true> on both,
    // each operation in one
    // packed FP32x2 instruction with the scalar form's rounding, and the
    // colour sums taken for a, then b.  The result equals two sample<true>
    // calls bit for bit.  A point with ok = false adds nothing: its table
    // coordinate is replaced by 0 (no NaN enters) and its weight by 0, and
    // fma(0, c, C) = C.
    __device__ __forceinline__ float depth(float t) const { return warp_depth(t, wa, wb); }
    __device__ __forceinline__ void pair_generic(float2 z, float xa, float xb, bool oka, bool okb, unsigned act) {
        xa = oka ? xa : 0.0f;
        xb = okb ? xb : 0.0f;
        const int ia = (int)xa, ib = (int)xb;
        const float fa = xa - (float)ia, fb = xb - (float)ib;
        const float4 ea = s_tf[2 * ia], da = s_tf[2 * ia + 1], eb = s_tf[2 * ib], db = s_tf[2 * ib + 1];
        // the table lerps as pairs: (r, g) and (b, absorbance) of each point
        const float2 rga = __ffma2_rn(make_float2(fa, fa), make_float2(da.x, da.y), make_float2(ea.x, ea.y));
        const float2 bwa = __ffma2_rn(make_float2(fa, fa), make_float2(da.z, da.w), make_float2(ea.z, ea.w));
        const float2 rgb = __ffma2_rn(make_float2(fb, fb), make_float2(db.x, db.y), make_float2(eb.x, eb.y));
        const float2 bwb = __ffma2_rn(make_float2(fb, fb), make_float2(db.z, db.w), make_float2(eb.z, eb.w));
        const float2 a = make_float2(fmin_(bwa.y, amax), fmin_(bwb.y, amax));
        // opacity 1 - e^-a: the series, and the direct form only when a lane of
        // the branch has an absorbance at or above 1/4 (one_minus_exp_neg)
        float2 p = __ffma2_rn(a, make_float2(-1.0f / 720.0f, -1.0f / 720.0f), make_float2(1.0f / 120.0f, 1.0f / 120.0f));
        p = __ffma2_rn(a, p, make_float2(-1.0f / 24.0f, -1.0f / 24.0f));
        p = __ffma2_rn(a, p, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
        p = __ffma2_rn(a, p, make_float2(-0.5f, -0.5f));
        p = __ffma2_rn(a, p, make_float2(1.0f, 1.0f));
        float2 alpha = __fmul2_rn(a, p);
        if (__any_sync(act, a.x >= 0.25f || a.y >= 0.25f)) {
            const float2 ng = __fmul2_rn(a, make_float2(-kLog2e, -kLog2e));
            const float2 dir = __ffma2_rn(make_float2(fexp2(ng.x), fexp2(ng.y)), make_float2(-1.0f, -1.0f),
                                          make_float2(1.0f, 1.0f));
            alpha = make_float2(a.x < 0.25f ? alpha.x : dir.x, a.y < 0.25f ? alpha.y : dir.y);
        }
        const float2 A = bound_generic2(F, z, w0, act);
        const float2 ex = __fmul2_rn(make_float2(-F.m0_log2e, -F.m0_log2e), A);
        float2 wgt = __fmul2_rn(make_float2(fexp2(ex.x), fexp2(ex.y)), alpha);
        wgt.x = oka ? wgt.x : 0.0f;
        wgt.y = okb ? wgt.y : 0.0f;
        // colour sums as pairs: (r, g) and (b, alpha); C.w + w = fma(w, 1, C.w)
        float2 cxy = __ffma2_rn(make_float2(wgt.x, wgt.x), rga, make_float2(C.x, C.y));
        float2 czw = __ffma2_rn(make_float2(wgt.x, wgt.x), make_float2(bwa.x, 1.0f), make_float2(C.z, C.w));
        cxy = __ffma2_rn(make_float2(wgt.y, wgt.y), rgb, cxy);
        czw = __ffma2_rn(make_float2(wgt.y, wgt.y), make_float2(bwb.x, 1.0f), czw);
        C = make_float4(cxy.x, cxy.y, czw.x, czw.y);
        n += (unsigned)oka + (unsigned)okb;
    }
};

// The pass-2 body for a warp whose lanes with samples all have a generic
// frame: the same operations without the per-sample test of the frame's kind.
struct GenericBlend {
    BlendBody& b;
    __device__ __forceinline__ void operator()(float t, float xt, float ws = 1.0f) { b.sample<true>(t, xt, ws); }
    __device__ __forceinline__ float depth(float t) const { return b.depth(t); }
    __device__ __forceinline__ void pair(float2 z, float xa, float xb, bool oka, bool okb, unsigned act) {
        b.pair_generic(z, xa, xb, oka, okb, act);
    }
};
// Bodies that take two lattice points at once (pair(...), equal to two calls).
template <class B> struct HasPair : std::false_type {};
template <> struct HasPair<GenericBlend> : std::true_type {};
// Bodies whose per-sample code is short enough to copy into a fully
// unrolled chunk loop (the four-power-moment blends).  The bodies of 6 and 8
// power moments and of trigonometric moments (root solves, series) take the
// loop rolled: 8 or 16 inlined copies of them overflow the instruction cache
// (octree frame with 8 power moments: 103 ms unrolled by 8, 219 ms by 16).
template <class B> struct RowUnroll : std::integral_constant<bool, HasPair<B>::value> {};
template <> struct RowUnroll<BlendBody> : std::true_type {};

// Bytes of one moment slab of P pixels in the volume's format.
__device__ __forceinline__ int64_t slab_bytes(const GridD& g, int plane) {
    return g.trig.n ? (int64_t)(4 + 4 * g.trig.n) * plane : (int64_t)(4 + 4 * (g.trig.sel ? g.trig.sel : 4)) * plane;
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
    __device__ __forceinline__ void operator()(float tt, float xt, float ws = 1.0f) {
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float2 s = s_sig[i];
        const float a = fmin_(ffma(f, s.y, s.x) * ws, amax);
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
    __device__ __forceinline__ void operator()(float t, float xt, float ws = 1.0f) {
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float4 e0 = s_tf[2 * i], de = s_tf[2 * i + 1];
        const float a = fmin_(ffma(f, de.w, e0.w) * ws, amax);
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

// Slab of 2N power moments: b0 plane (float), the float4 plane of b1..b4,
// then b5, b6 (float2 plane, N = 3) or b5..b8 (float4 plane, N = 4).
template <int N>
__device__ __forceinline__ void store_power(char* base, const ViewSlot& S, int64_t slab_off, int pix, const float* m) {
    char* slab = base + slab_off;
    reinterpret_cast<float*>(slab)[pix] = m[0];
    reinterpret_cast<float4*>(slab + (size_t)4 * S.plane)[pix] = make_float4(m[1], m[2], m[3], m[4]);
    if constexpr (N == 3)
        reinterpret_cast<float2*>(slab + (size_t)20 * S.plane)[pix] = make_float2(m[5], m[6]);
    else
        reinterpret_cast<float4*>(slab + (size_t)20 * S.plane)[pix] = make_float4(m[5], m[6], m[7], m[8]);
}

template <int N>
__device__ __forceinline__ void load_power(const char* base, const ViewSlot& S, int64_t slab_off, int pix, float* m) {
    const char* slab = base + slab_off;
    m[0] = __ldg(reinterpret_cast<const float*>(slab) + pix);
    const float4 q = __ldg(reinterpret_cast<const float4*>(slab + (size_t)4 * S.plane) + pix);
    m[1] = q.x; m[2] = q.y; m[3] = q.z; m[4] = q.w;
    if constexpr (N == 3) {
        const float2 r = __ldg(reinterpret_cast<const float2*>(slab + (size_t)20 * S.plane) + pix);
        m[5] = r.x; m[6] = r.y;
    } else {
        const float4 r = __ldg(reinterpret_cast<const float4*>(slab + (size_t)20 * S.plane) + pix);
        m[5] = r.x; m[6] = r.y; m[7] = r.z; m[8] = r.w;
    }
}

// Pass 1 with 2N power moments: b_j += a z^j, j = 0..2N (Alg. 2).
template <int N>
struct PowerMomentBody {
    const float2* s_sig;
    float tf_scale, tf_bias, amax, wa, wb;
    float m[2 * N + 1];
    unsigned n = 0;
    __device__ __forceinline__ void operator()(float t, float xt, float ws = 1.0f) {
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float2 s = s_sig[i];
        const float a = fmin_(ffma(f, s.y, s.x) * ws, amax);
        const float z = warp_depth(t, wa, wb);
        m[0] += a;
        float p = a;
#pragma unroll
        for (int j = 1; j <= 2 * N; ++j) {
            m[j] = ffma(p, z, m[j]);
            if (j < 2 * N) p *= z;
        }
        ++n;
    }
    __device__ __forceinline__ void store(const GridD&, char* base, const ViewSlot& S, int64_t off, int pix) {
        store_power<N>(base, S, off, pix, m);
    }
};

// Pass 2 with 2N power moments.
template <int N>
struct PowerBlendBody {
    const float4* s_tf;
    PowerFrame<N> F;
    float tf_scale, tf_bias, amax, wa, wb, w0;
    float b0;
    float4 C = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    unsigned n = 0;
    __device__ __forceinline__ void operator()(float t, float xt, float ws = 1.0f) {
        const int i = (int)xt;
        const float f = xt - (float)i;
        const float4 e0 = s_tf[2 * i], de = s_tf[2 * i + 1];
        const float a = fmin_(ffma(f, de.w, e0.w) * ws, amax);
        const float alpha = one_minus_exp_neg(a);
        const float z = warp_depth(t, wa, wb);
        const float A = power_fraction<N>(F, z, w0);
        const float wgt = fclamp(fexp2(-F.m0_log2e * A), 0.0f, 1.0f) * alpha;
        C.x = ffma(wgt, ffma(f, de.x, e0.x), C.x);
        C.y = ffma(wgt, ffma(f, de.y, e0.y), C.y);
        C.z = ffma(wgt, ffma(f, de.z, e0.z), C.z);
        C.w += wgt;
        ++n;
    }
    __device__ __forceinline__ bool singular() const { return F.kind == kFrameFourMoments; }
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
template <> struct Bodies<6> {
    using Moment = PowerMomentBody<3>;
    using Blend = PowerBlendBody<3>;
};
template <> struct Bodies<8> {
    using Moment = PowerMomentBody<4>;
    using Blend = PowerBlendBody<4>;
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
    if constexpr (MS == 3 || MS == 4) {
        b.zs = g.trig.zone_scale;
        for (int j = 0; j < MS; ++j) b.t[j] = {0.0f, 0.0f};
    }
    if constexpr (MS == 6 || MS == 8)
        for (int j = 0; j <= MS; ++j) b.m[j] = 0.0f;
    return b;
}

// Pass-2 body of a pixel from the float32 moments pass 1 left in registers.
__device__ __forceinline__ BlendBody blend_body_of(const float4* s_tf, const GridD& g, const ViewSlot& S,
                                                   const MomentBody& mb, bool valid) {
    BlendBody b;
    b.s_tf = s_tf;
    b.tf_scale = g.tf_scale;
    b.tf_bias = g.tf_bias;
    b.amax = g.absorbance_max;
    b.wa = S.v.warp_a;
    b.wb = S.v.warp_b;
    b.w0 = g.overestimation;
    const float m[5] = {valid ? mb.m0 : 0.0f, valid ? mb.m12.x : 0.0f, valid ? mb.m12.y : 0.0f,
                        valid ? mb.m34.x : 0.0f, valid ? mb.m34.y : 0.0f};
    b.F = pixel_frame(g, m, &b.fp64);
    b.b0 = m[0];
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
        b.F = pixel_frame(g, m, &b.fp64);
        b.b0 = m[0];
    } else if constexpr (MS == 6 || MS == 8) {
        float m[MS + 1];
        for (int j = 0; j <= MS; ++j) m[j] = 0.0f;
        if (valid) load_power<MS / 2>(moments, S, off, pix, m);
        b.F = make_power_frame<MS / 2>(m, g.moment_bias);
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


// Per-pixel statistics of pass 2: pixels on a one- or two-atom branch, and
// pixels whose frame was set up in FP64.  Called by all 32 lanes together.
template <class Body>
__device__ __forceinline__ void count_frames(Counters* ctr, const Body& body, bool valid) {
    const unsigned full = 0xffffffffu;
    const unsigned sing = __ballot_sync(full, valid && body.singular());
    bool f64 = false;
    if constexpr (std::is_same<Body, BlendBody>::value) f64 = body.fp64;
    const unsigned dp = __ballot_sync(full, valid && f64);
    if ((threadIdx.x & 31) == 0) {
        if (sing) atomicAdd(&ctr->singular, (unsigned long long)__popc(sing));
        if (dp) atomicAdd(&ctr->fp64_pixels, (unsigned long long)__popc(dp));
    }
}

// Pops the next 8x4 ray tile of the work queue; returns false when empty.
__device__ __forceinline__ bool next_tile(const ViewTable& vt, int32_t* head, int& vi, int& px, int& py, int& tile) {
    const int lane = threadIdx.x & 31;
    tile = 0;
    if (lane == 0) {
        tile = atomicAdd(head, 1);
        if (vt.order && tile < vt.total_tiles) tile = __ldg(vt.order + tile);
    }
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= vt.total_tiles) return false;
    vi = find_view(vt, tile);
    const ViewSlot& S = vt.s[vi];
    const int lt = tile - S.tile_base;
    tile_pixel(S, lt, lane, px, py);
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

// A warp's buffer for chunks of `chunk` cache rows: a double buffer of rows
// (2 chunk 32 floats) followed by the warped depths of a chunk's rows.
constexpr int row_buf_floats(int chunk) { return 2 * chunk * 32 + chunk; }
constexpr int kRowChunk = 8;                    // cache rows per prefetch (grids: the window slot is the buffer)
constexpr int kRowBuf = row_buf_floats(kRowChunk);
constexpr int kUnitRowChunk = 16;               // octrees and meshes: their own buffer, longer chunks
constexpr int kUnitRowBuf = row_buf_floats(kUnitRowChunk);

// Pass 2 of the batched frame from the tile cache.  The tile's rows are
// contiguous (rows[r * 32 + lane], r = k - kmin), so the warp copies them
// into its shared-memory buffer 8 rows (1 KiB) at a time, one chunk ahead of
// the one it blends, and every lane takes its own column over its own
// [k0, k1].  buf: 16-byte aligned, kRowBuf floats, this warp's only.  For a
// body that takes two points at once, lanes 0..7 also compute the warped
// depths of the chunk's 8 rows into buf[kRowZ..], which every lane reads.
// Octree adaptive step: a sample's table coordinate carries its leaf's level
// shift in its low mantissa bits, as few as max_level needs (2 for max_level
// 2 or 3: the coordinate moves by at most 3 ulp, the same in both passes, the
// split calls and the per-piece path), so that pass 2 can weigh cached
// samples.
__device__ __forceinline__ int tag_mask(int max_level) { return (1 << (32 - __clz(max_level))) - 1; }
__device__ __forceinline__ float tag_shift(float v, int shift, int mask) {
    return __int_as_float((__float_as_int(v) & ~mask) | shift);
}
__device__ __forceinline__ float tagged_weight(float v, int mask) {
    return __int_as_float((127 + (__float_as_int(v) & mask)) << 23);  // 2^shift
}

template <bool kSel, class Body, bool kTagged = false, int kRowChunk = mb::kRowChunk>
__device__ __forceinline__ void march_rows(const GridD& g, const float* __restrict__ rows, int kmin, int kmax, int k0,
                                           int k1, float* __restrict__ buf, Body& body, int tmask = 0) {
    constexpr int kRowZ = 2 * kRowChunk * 32;
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
        const int kc = kmin + c * kRowChunk;
        if constexpr (HasPair<Body>::value && !kTagged) {
            if (lane < kRowChunk) buf[kRowZ + lane] = body.depth(lattice_t(kc + lane, g.step));
        }
        __syncwarp();
        const float* src = buf + (c & 1) * kRowChunk * 32 + lane;
        const int n = min(kRowChunk, kmax - kc + 1);
        if (kc >= k0 && kc + kRowChunk - 1 <= k1) {
            // the whole chunk lies in this lane's interval (and, without a
            // selection, every point of it is owned)
            if constexpr (HasPair<Body>::value && !kTagged) {
                // two lattice points per call (packed FP32x2 arithmetic); with a
                // selection, a pair no lane of this branch samples is skipped.
                // (The adaptive step leaves most points unsampled, lane-coherently:
                // there the single-point loop below skips more.)
                const unsigned act = __activemask();
                const float2* zr = reinterpret_cast<const float2*>(buf + kRowZ);
#pragma unroll
                for (int i = 0; i < kRowChunk; i += 2) {
                    const float va = src[i * 32], vb = src[(i + 1) * 32];
                    const bool oka = !kSel || va == va, okb = !kSel || vb == vb;
                    if (kSel && !__any_sync(act, oka || okb)) continue;
                    body.pair(zr[i / 2], va, vb, oka, okb, act);
                }
                t += kRowChunk * g.step;
            } else if constexpr (RowUnroll<Body>::value) {
#pragma unroll
                for (int i = 0; i < kRowChunk; ++i, t += g.step) {
                    const float val = src[i * 32];
                    if (!kSel || val == val) body(t, val, kTagged ? tagged_weight(val, tmask) : 1.0f);
                }
            } else {
#pragma unroll 1
                for (int i = 0; i < kRowChunk; ++i, t += g.step) {
                    const float val = src[i * 32];
                    if (!kSel || val == val) body(t, val, kTagged ? tagged_weight(val, tmask) : 1.0f);
                }
            }
        } else {
            // the chunk's points of this lane's interval; every in-domain
            // point is owned when no piece is left out
            auto point = [&](int i) {
                const int k = kc + i;
                const float val = src[i * 32];
                if (k >= k0 && k <= k1 && (!kSel || val == val))
                    body(t, val, kTagged ? tagged_weight(val, tmask) : 1.0f);
            };
            if constexpr (RowUnroll<Body>::value) {
                for (int i = 0; i < n; ++i, t += g.step) point(i);
            } else {
#pragma unroll 1
                for (int i = 0; i < n; ++i, t += g.step) point(i);
            }
        }
        __syncwarp();  // every lane is done with the chunk before it is refilled
    }
}

// Pass 2 from the tile's cache rows.  With four power moments, a warp whose
// lanes with samples all have a generic frame (lanes without samples never
// call the body) takes the loop without the per-sample test of the frame's
// kind; the arithmetic, and so the result, is the same.
template <bool kSel, bool kTagged = false, int kChunk = kRowChunk, class Body>
__device__ __forceinline__ void blend_rows(const GridD& g, const float* __restrict__ rows, int kmin, int kmax, int k0,
                                           int k1, float* __restrict__ buf, Body& body, int tmask = 0) {
    if constexpr (std::is_same<Body, BlendBody>::value) {
        if (__all_sync(0xffffffffu, k0 > k1 || body.F.kind == kFrameGeneric)) {
            GenericBlend gb{body};
            march_rows<kSel, GenericBlend, kTagged, kChunk>(g, rows, kmin, kmax, k0, k1, buf, gb, tmask);
            return;
        }
    }
    march_rows<kSel, Body, kTagged, kChunk>(g, rows, kmin, kmax, k0, k1, buf, body, tmask);
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


}  // namespace
}  // namespace mb
