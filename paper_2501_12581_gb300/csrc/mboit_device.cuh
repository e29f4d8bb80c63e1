// Device-side arithmetic of the MBOIT puzzle-piece render (sm_103a).
//
// Everything a kernel does per ray and per sample lives here as inline
// functions: ray set-up, sample lattice, brick ownership, trilinear sample,
// transfer-function lookup, the log-depth warp (Alg. 2), and the moment-bound
// transmittance (Alg. 3).
//
// Moment bound, as computed here.  Alg. 3 solves B q = (1, z0, z0^2) with the
// 3x3 Hankel matrix B of the biased normalised moments, takes the roots of q
// as the two other support points of the canonical representation through
// z0, and sums the representation's weights with w = (overestimation,
// [z1 < z0], [z2 < z0]).  We compute the same representation in the frame
// where the biased measure has mean 0 and variance 1 (an affine change of
// depth, which preserves the order of support points and the weights):
//   x = (z - mu) / s,  Hankel [[1,0,1],[0,1,g],[1,g,k]] = L diag(1,1,d) L^T,
//   g = skewness, d = kurtosis - 1 - g^2 > 0.
// With y(x) = (1, x, x^2 - g x - 1) the kernel K(x, x') = v(x)^T B^-1 v(x') is
//   K(x, x') = 1 + x x' + y3(x) y3(x') / d.
// The support points other than x0 are the roots of K(., x0); every support
// point x_i carries the Christoffel weight rho_i = 1 / K(x_i, x_i), a sum of
// positive terms (no cancellation).  With x1 < x2:
//   K(., x0) opens downward (y3(x0) < 0)  <=>  x1 < x0 < x2:  A = w0 rho0 + rho1
//   otherwise x0 < x1 (A = w0 rho0) or x0 > x2 (A = w0 rho0 + 1 - rho0).
// The per-pixel frame (mu, s, g, d) is built once per ray from the FP32
// moments in float-float FP32 (make_frame_ff), in FP64 only for a
// near-singular Hankel matrix (make_frame); per sample only FP32 arithmetic
// remains.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define MB_HD __host__ __device__ __forceinline__
#else
#include <math.h>
#define MB_HD static inline
#endif

namespace mb {

// ---------------------------------------------------------------------------
// correctly rounded float ops that the compiler may not contract or reorder
MB_HD float fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
MB_HD float fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
MB_HD float fdiv(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdiv_rn(a, b);
#else
    return a / b;
#endif
}
MB_HD float fsqrt(float a) {
#if defined(__CUDA_ARCH__)
    return __fsqrt_rn(a);
#else
    return sqrtf(a);
#endif
}
MB_HD float ffma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
// fast transcendental approximations (accuracy ~2 ulp, ample for 2e-4 images)
MB_HD float flog2(float x) {
#if defined(__CUDA_ARCH__)
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));  // one MUFU op; lattice depths are never denormal
    return y;
#else
    return log2f(x);
#endif
}
MB_HD float fexp2(float x) {
#if defined(__CUDA_ARCH__)
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));  // one MUFU op, ~2 ulp
    return y;
#else
    return exp2f(x);
#endif
}
// square root for values that only steer a continuous result (not correctly rounded)
MB_HD float fsqrt_fast(float x) {
#if defined(__CUDA_ARCH__)
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
#else
    return sqrtf(x);
#endif
}
MB_HD float frsqrt_fast(float x) {
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);  // one MUFU op
#else
    return 1.0f / sqrtf(x);
#endif
}
MB_HD float fdiv_fast(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdividef(a, b);  // 2 ulp for |b| < 2^126; every divisor here is far below
#else
    return a / b;
#endif
}
MB_HD float frcp(float x) { return fdiv_fast(1.0f, x); }
MB_HD float fmin_(float a, float b) { return a < b ? a : b; }
MB_HD float fmax_(float a, float b) { return a > b ? a : b; }
MB_HD float fclamp(float x, float lo, float hi) { return fmin_(fmax_(x, lo), hi); }

constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------------------
// views and volumes as the kernels see them

struct ViewD {
    float eye[3], u[3], v[3], w[3];
    int32_t width, height, projection, pad0;
    float scale_u, scale_v;
    float warp_a, warp_b;  // warped depth z = clamp(warp_a * log2(t) + warp_b, -1, 1)
};

// Trigonometric moments: coefficients of s^m in (s + i)^k (s - i)^(n-k)
// (k, m = 0..n, filled on the host) and the angle mapping.
struct TrigTables {
    float er[5][5], ei[5][5];
    float zone_scale;     // phi = z * zone_scale = z (1 - zeta) pi
    float beta;
    int32_t n;            // 3 or 4 complex moments (0: power moments)
    int32_t storage;      // 1 float16, 2 bfloat16
    int32_t sel;          // kernel variant: 0 four power moments, 3 / 4 trigonometric, 6 / 8 power moments
    int32_t pad;
};

// GridD::flags bits (the descriptor's MBOIT_FLAG_* values)
constexpr uint32_t kFlagRawSum = 0x1u;
constexpr uint32_t kFlagAdaptiveStep = 0x4u;
constexpr uint32_t kFlagFp64Setup = 0x8u;   // every pixel's frame set up in FP64
// Test hook of the TMA wait limit (set by mboit_debug_corrupt, never by a
// descriptor): window loads arm their barrier but issue no copy.
constexpr uint32_t kFlagDebugNoCopy = 0x80000000u;

struct GridD {
    const float* field;           // [nz][ny][nx]
    int32_t nx, ny, nz;
    int32_t brick_log2, nbx, nby, nbz;
    float hx, hy, hz;             // nx-1, ny-1, nz-1
    float step;
    float tf_scale, tf_bias;      // table coordinate = clamp(v * tf_scale + tf_bias, 0, 255)
    float absorbance_max;
    float moment_bias, overestimation;
    float bias_vector[4];
    uint32_t flags;
    TrigTables trig;
};

// ---------------------------------------------------------------------------
// rays: float32, correctly rounded, fixed order (the same bits as the oracle)

MB_HD void make_ray(const ViewD& V, int px, int py, float o[3], float d[3]) {
    float fx = fadd((float)px, 0.5f);
    float fy = fadd((float)py, 0.5f);
    if (V.projection == 0) {
        float sx = fmul(fadd(fdiv(fx, (float)V.width), -0.5f), V.scale_u);
        float sy = fmul(fadd(fdiv(fy, (float)V.height), -0.5f), V.scale_v);
        for (int c = 0; c < 3; ++c) {
            o[c] = fadd(fadd(V.eye[c], fmul(sx, V.u[c])), fmul(sy, V.v[c]));
            d[c] = V.w[c];
        }
    } else {
        float sx = fmul(fadd(fdiv(fmul(2.0f, fx), (float)V.width), -1.0f), V.scale_u);
        float sy = fmul(fadd(fdiv(fmul(2.0f, fy), (float)V.height), -1.0f), V.scale_v);
        float dir[3];
        for (int c = 0; c < 3; ++c) dir[c] = fadd(fadd(V.w[c], fmul(sx, V.u[c])), fmul(sy, V.v[c]));
        float len = fsqrt(fadd(fadd(fmul(dir[0], dir[0]), fmul(dir[1], dir[1])), fmul(dir[2], dir[2])));
        for (int c = 0; c < 3; ++c) {
            o[c] = V.eye[c];
            d[c] = fdiv(dir[c], len);
        }
    }
}

// Lattice indices [k0, k1] that surely contain every lattice point whose
// float32 position lies in the box [lo, hi) (padding covers the rounding of
// positions and of this computation; the per-sample position test decides).
MB_HD bool lattice_range(const float o[3], const float d[3], const float lo[3], const float hi[3], float step,
                         int* k0, int* k1) {
    float t0 = 0.0f, t1 = 3.0e38f;
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0f) {
            if (!(o[c] >= lo[c] && o[c] < hi[c])) return false;
            continue;
        }
        float inv = 1.0f / d[c];
        float a = (lo[c] - o[c]) * inv, b = (hi[c] - o[c]) * inv;
        if (a > b) { float s = a; a = b; b = s; }
        float pad = (fabsf(o[c]) + fabsf(lo[c]) + fabsf(hi[c]) + 1.0f) * 3.814697265625e-06f * fabsf(inv);
        t0 = fmax_(t0, a - pad);
        t1 = fmin_(t1, b + pad);
    }
    if (!(t1 >= t0)) return false;
    float inv_step = 1.0f / step;
    float klo = ceilf(t0 * inv_step - 0.5f) - 2.0f;
    float khi = floorf(t1 * inv_step - 0.5f) + 2.0f;
    if (klo < 0.0f) klo = 0.0f;
    // t_k = (k + 1/2) step is exact in float32, and t_{k+1} = t_k + step
    // exactly, for k < 2^22: farther lattice points are not sampled
    if (khi > 4194303.0f) khi = 4194303.0f;
    if (khi < klo) return false;
    *k0 = (int)klo;
    *k1 = (int)khi;
    return true;
}

// Lattice parameter of point k: exact in float32 for k < 2^22 and a power-of-two step.
MB_HD float lattice_t(int k, float step) { return fmul(fadd((float)k, 0.5f), step); }

MB_HD float warp_depth(float t, float wa, float wb) { return fclamp(ffma(flog2(t), wa, wb), -1.0f, 1.0f); }

// ---------------------------------------------------------------------------
// per-pixel reconstruction frame (FP64 set-up, Alg. 3 "mix" + "SolveMat")

enum : int32_t { kFrameEmpty = 0, kFrameGeneric = 1, kFrameOneAtom = 2, kFrameTwoAtoms = 3 };

struct Frame {
    int32_t kind;
    float m0_log2e;          // b0 * log2(e): T = exp2(-m0_log2e * A)
    // generic: x = z * inv_s + nmu; skew g; inv_d = 1/d
    // one atom: atom at p0;  two atoms: atoms p0 < p1 with weights p2, p3
    float p0, p1, p2, p3;
};

MB_HD Frame make_frame(const float m_in[5], float moment_bias, const float bias_vector[4]) {
    Frame F;
    F.kind = kFrameEmpty;
    F.m0_log2e = 0.0f;
    F.p0 = F.p1 = F.p2 = F.p3 = 0.0f;
    double m0 = (double)m_in[0];
    if (!(m0 > 0.0)) return F;
    double beta = (double)moment_bias;
    double b[5];
    b[0] = 1.0;
    for (int j = 1; j <= 4; ++j) b[j] = (1.0 - beta) * ((double)m_in[j] / m0) + beta * (double)bias_vector[j - 1];
    F.m0_log2e = (float)(m0 * 1.4426950408889634);
    double mu = b[1];
    double var = b[2] - mu * mu;
    // Singular Hankel matrices.  The moments were stored in float32, so a
    // one- or two-atom measure shows up with rounding noise of ~1e-7 relative
    // to b2 (variance) or b4 (Schur complement D33).  Thresholds of 1e-6
    // relative catch that noise; with any bias >= 5e-5 the mixed-in bias
    // measure keeps var/b2 >= 6.8e-5 and D33/b4 >= 1.7e-5, far above them.
    const double rel = 1e-6;
    if (var <= rel * b[2]) {
        F.kind = kFrameOneAtom;
        F.p0 = (float)mu;
        return F;
    }
    double k3 = b[3] - 3.0 * mu * b[2] + 2.0 * mu * mu * mu;
    double k4 = b[4] - 4.0 * mu * b[3] + 6.0 * mu * mu * b[2] - 3.0 * mu * mu * mu * mu;
    double D33 = k4 - var * var - k3 * k3 / var;  // Schur complement of the raw Hankel matrix
    if (D33 <= rel * b[4]) {
        // two atoms about the mean: roots of x^2 - (k3/var) x - var (centred),
        // weights from the first moment
        double gk = k3 / var;
        double disc = gk * gk + 4.0 * var;
        double sq = sqrt(disc > 0.0 ? disc : 0.0);
        double q = 0.5 * (gk + (gk >= 0.0 ? sq : -sq));
        double r1 = q, r2 = (q != 0.0) ? -var / q : q;
        if (r1 > r2) { double s = r1; r1 = r2; r2 = s; }
        double w2 = (r2 != r1) ? (0.0 - r1) / (r2 - r1) : 0.0;
        F.kind = kFrameTwoAtoms;
        F.p0 = (float)(r1 + mu);
        F.p1 = (float)(r2 + mu);
        F.p2 = (float)(1.0 - w2);
        F.p3 = (float)w2;
        return F;
    }
    double s = sqrt(var);
    double g = k3 / (var * s);
    double dd = D33 / (var * var);
    F.kind = kFrameGeneric;
    F.p0 = (float)(1.0 / s);
    F.p1 = (float)(-mu / s);
    F.p2 = (float)g;
    F.p3 = (float)(1.0 / dd);
    return F;
}

// ---------------------------------------------------------------------------
// float-float arithmetic (an unevaluated sum hi + lo of two floats, ~48
// significant bits) from error-free transformations: Knuth's TwoSum and the
// fma-based TwoProduct, with Dekker's normalisation.  The per-pixel frame is
// set up with it in FP32, so that only near-singular pixels need FP64.

struct ff {
    float hi, lo;
};
// s + e = a + b exactly (Knuth's TwoSum)
MB_HD ff ff_two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fadd(s, -a);
    return {s, fadd(fadd(a, -fadd(s, -bb)), fadd(b, -bb))};
}
// s + e = a + b exactly, for |a| >= |b| or a = 0 (Dekker's FastTwoSum)
MB_HD ff ff_fast_sum(float a, float b) {
    const float s = fadd(a, b);
    return {s, fadd(b, -fadd(s, -a))};
}
// p + e = a b exactly (the fma returns the product's rounding error)
MB_HD ff ff_two_prod(float a, float b) {
    const float p = fmul(a, b);
    return {p, ffma(a, b, -p)};
}
MB_HD ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s = ff_fast_sum(s.hi, fadd(s.lo, t.hi));
    return ff_fast_sum(s.hi, fadd(s.lo, t.lo));
}
MB_HD ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
MB_HD ff ff_mul(ff a, ff b) {
    const ff p = ff_two_prod(a.hi, b.hi);
    return ff_fast_sum(p.hi, ffma(a.hi, b.lo, ffma(a.lo, b.hi, p.lo)));
}
MB_HD ff ff_mulf(ff a, float b) {
    const ff p = ff_two_prod(a.hi, b);
    return ff_fast_sum(p.hi, ffma(a.lo, b, p.lo));
}
// a / b for floats: the quotient's rounding error from the exact remainder
// a - q b (an fma), divided once more
MB_HD ff ff_divf(float a, float b) {
    const float q = fdiv(a, b);
    return ff_fast_sum(q, fdiv(ffma(-q, b, a), b));
}
MB_HD ff ff_div(ff a, ff b) {
    const float q1 = fdiv(a.hi, b.hi);
    const ff r = ff_add(a, ff_neg(ff_mulf(b, q1)));
    return ff_fast_sum(q1, fdiv(r.hi, b.hi));
}

// Frame of a pixel (as make_frame) with the set-up in float-float: the
// cancellations in the central moments (variance b2 - b1^2, third and fourth
// central moments, Schur complement D33) keep ~48 bits, so a generic frame
// comes out as FP64 would give it, to a few float32 ulp in the outputs.  A
// pixel whose variance or Schur complement is within 1e-4 of b2 or b4 (near
// the 1e-6 thresholds of the one- and two-atom branches) is near-singular:
// it is set up by make_frame in FP64, and *fp64 is set.
MB_HD Frame make_frame_ff(const float m_in[5], float moment_bias, const float bias_vector[4], bool* fp64) {
    *fp64 = false;
    const float m0 = m_in[0];
    if (!(m0 > 0.0f)) {
        Frame F;
        F.kind = kFrameEmpty;
        F.m0_log2e = 0.0f;
        F.p0 = F.p1 = F.p2 = F.p3 = 0.0f;
        return F;
    }
    // b_j = (1 - beta) m_j / m0 + beta bv_j = n_j - beta (n_j - bv_j)
    const float beta = moment_bias;
    ff b[5];
    for (int j = 1; j <= 4; ++j) {
        const ff n = ff_divf(m_in[j], m0);
        const ff dv = ff_add(n, {-bias_vector[j - 1], 0.0f});
        b[j] = ff_add(n, ff_neg(ff_mulf(dv, beta)));
    }
    const ff mu = b[1];
    const ff mu2 = ff_mul(mu, mu);
    const ff var = ff_add(b[2], ff_neg(mu2));
    // k3 = b3 - 3 mu b2 + 2 mu^3,  k4 = b4 - 4 mu b3 + 6 mu^2 b2 - 3 mu^4
    const ff mub2 = ff_mul(mu, b[2]);
    const ff mu3 = ff_mul(mu2, mu);
    const ff k3 = ff_add(ff_add(b[3], ff_mulf(mub2, -3.0f)), ff_mulf(mu3, 2.0f));
    const ff k4 = ff_add(ff_add(ff_add(b[4], ff_mulf(ff_mul(mu, b[3]), -4.0f)), ff_mulf(ff_mul(mu2, b[2]), 6.0f)),
                         ff_mulf(ff_mul(mu2, mu2), -3.0f));
    const bool near_one = !(var.hi > 1e-4f * b[2].hi);
    ff D33 = {0.0f, 0.0f};
    if (!near_one) D33 = ff_add(ff_add(k4, ff_neg(ff_mul(var, var))), ff_neg(ff_div(ff_mul(k3, k3), var)));
    if (near_one || !(D33.hi > 1e-4f * b[4].hi)) {
        *fp64 = true;
        return make_frame(m_in, moment_bias, bias_vector);
    }
    Frame F;
    F.kind = kFrameGeneric;
    F.m0_log2e = fmul(m0, kLog2e);
    const float s = fsqrt(var.hi);
    F.p0 = fdiv(1.0f, s);
    F.p1 = fdiv(-mu.hi, s);
    F.p2 = fdiv(k3.hi, fmul(var.hi, s));
    F.p3 = fdiv(fmul(var.hi, var.hi), D33.hi);
    return F;
}

MB_HD float step_weight(float x, float z0, float w0) { return x < z0 ? 1.0f : (x == z0 ? w0 : 0.0f); }

// Alg. 3 for a generic frame (three support points): fraction A(z0) of the
// optical depth in front of warped depth z0.
MB_HD float bound_generic(const Frame& F, float z0, float w0) {
    const float inv_s = F.p0, nmu = F.p1, g = F.p2, inv_d = F.p3;
    float x0 = ffma(z0, inv_s, nmu);
    float y3 = ffma(x0, x0 - g, -1.0f);
    float e = y3 * inv_d;                         // leading coefficient of K(., x0)
    float rho0 = frcp(ffma(y3, e, ffma(x0, x0, 1.0f)));
    // x0 outside [x1, x2] (y3 >= 0): left of both iff K'(x0) < 0, and
    // K'(x0) = x0 (1 + 2e) - g e has the sign of x0 there (y3 >= 0 puts x0 at
    // or beyond a root of x^2 - g x - 1, whose roots r- < 0 < r+ satisfy r- <= g
    // for g < 0 and r+ >= g for g > 0), so the sign of x0 decides
    float A_out = x0 < 0.0f ? w0 * rho0 : ffma(w0 - 1.0f, rho0, 1.0f);
    // x1 < x0 < x2 (y3 < 0, so e < 0): the weight rho1 of the smaller root
    // from the representation's moments of order 0 and 1 (rho0 + rho1 +
    // rho2 = 1, rho0 x0 + rho1 x1 + rho2 x2 = 0) and the roots' sum and
    // spread (-c1/e, sqrt(c1^2 - 4 e c0)/|e|):
    //   rho1 = R/2 + (R c1/2 - rho0 x0 e) / sqrt(c1^2 - 4 e c0),  R = 1 - rho0
    float c1 = ffma(-g, e, x0);
    float c0 = 1.0f - e;
    float disc = fmax_(ffma(c1, c1, -4.0f * e * c0), 1e-30f);
    float R = 1.0f - rho0;
    float rho1 = ffma(ffma(0.5f * R, c1, -rho0 * x0 * e), frsqrt_fast(disc), 0.5f * R);
    rho1 = fclamp(rho1, 0.0f, R);
    return y3 < 0.0f ? ffma(w0, rho0, rho1) : A_out;
}

// Alg. 3: fraction A(z0) of the optical depth in front of warped depth z0.
MB_HD float bound_fraction(const Frame& F, float z0, float w0) {
    if (F.kind == kFrameGeneric) return bound_generic(F, z0, w0);
    if (F.kind == kFrameOneAtom) return step_weight(F.p0, z0, w0);
    if (F.kind == kFrameTwoAtoms) return F.p2 * step_weight(F.p0, z0, w0) + F.p3 * step_weight(F.p1, z0, w0);
    return 0.0f;
}

#if defined(__CUDACC__)
// bound_generic for two depths at once: every operation of the scalar form
// on both, as one packed FP32x2 instruction (each half rounded exactly as the
// scalar instruction), the MUFU reciprocal / square root per half.  Equal to
// (bound_generic(F, z0.x, w0), bound_generic(F, z0.y, w0)) bit for bit.
// `act`: the lanes calling together; the branch between the roots (y3 < 0)
// runs only when one of them needs it.
__device__ __forceinline__ float2 bound_generic2(const Frame& F, float2 z0, float w0, unsigned act) {
    const float2 one = make_float2(1.0f, 1.0f), mone = make_float2(-1.0f, -1.0f);
    const float2 ng = make_float2(-F.p2, -F.p2), inv_d = make_float2(F.p3, F.p3);
    const float2 x0 = __ffma2_rn(z0, make_float2(F.p0, F.p0), make_float2(F.p1, F.p1));
    const float2 y3 = __ffma2_rn(x0, __fadd2_rn(x0, ng), mone);
    const float2 e = __fmul2_rn(y3, inv_d);
    const float2 K = __ffma2_rn(y3, e, __ffma2_rn(x0, x0, one));
    const float2 rho0 = make_float2(frcp(K.x), frcp(K.y));
    const float2 lo = __fmul2_rn(make_float2(w0, w0), rho0);
    const float2 hi = __ffma2_rn(make_float2(w0 - 1.0f, w0 - 1.0f), rho0, one);
    float2 A = make_float2(x0.x < 0.0f ? lo.x : hi.x, x0.y < 0.0f ? lo.y : hi.y);
    if (__any_sync(act, y3.x < 0.0f || y3.y < 0.0f)) {
        const float2 c1 = __ffma2_rn(ng, e, x0);
        const float2 c0 = __ffma2_rn(e, mone, one);
        const float2 dq = __ffma2_rn(c1, c1, __fmul2_rn(__fmul2_rn(make_float2(-4.0f, -4.0f), e), c0));
        const float2 R = __ffma2_rn(rho0, mone, one);
        const float2 hR = __fmul2_rn(make_float2(0.5f, 0.5f), R);
        // -rho0 * x0 * e = ((-rho0) x0) e, with the sign moved onto x0 (exact)
        const float2 q = __fmul2_rn(__fmul2_rn(rho0, __fmul2_rn(x0, mone)), e);
        const float2 in = __ffma2_rn(hR, c1, q);
        float2 rho1 =
            __ffma2_rn(in, make_float2(frsqrt_fast(fmax_(dq.x, 1e-30f)), frsqrt_fast(fmax_(dq.y, 1e-30f))), hR);
        rho1 = make_float2(fclamp(rho1.x, 0.0f, R.x), fclamp(rho1.y, 0.0f, R.y));
        const float2 Ain = __ffma2_rn(make_float2(w0, w0), rho0, rho1);
        A = make_float2(y3.x < 0.0f ? Ain.x : A.x, y3.y < 0.0f ? Ain.y : A.y);
    }
    return A;
}
#endif

// T = exp(-b0 A(z0)), A from the frame's representation; A lies in [0, 1]
// for the one- and two-atom frames, and in [0, 1] up to rounding for a
// generic frame (below), so T needs no clamp.
MB_HD float transmittance(const Frame& F, float z0, float w0) {
    float A = bound_fraction(F, z0, w0);
    return fexp2(-F.m0_log2e * A);
}
// For a generic frame A >= 0 up to rounding (w0 rho0 >= 0, 1 - (1 - w0) rho0 >=
// w0 since rho0 = 1 / K(x0, x0) <= 1, rho1 clamped to [0, 1 - rho0]), so T
// exceeds 1 by at most a rounding error and needs no clamp.
MB_HD float transmittance_generic(const Frame& F, float z0, float w0) {
    float A = bound_generic(F, z0, w0);
    return fexp2(-F.m0_log2e * A);
}

}  // namespace mb
