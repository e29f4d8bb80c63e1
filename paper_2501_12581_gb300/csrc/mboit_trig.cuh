// Trigonometric-moment variant of the moment bound (n = 3 or 4 complex
// moments, the "6 / 8 trigonometric moments" of Sec. 4.3 and Fig. 3).
//
// Depth z maps to the angle phi = z (1 - zeta) pi, leaving a wrapping zone of
// width 2 zeta pi between the farthest and the nearest depth.  Pass 1 sums
// b0 = sum a and t_j = sum a e^{i j phi}; the stored moments are
// tau_j = t_j / b0 (float16 / bfloat16).  The bias mixes them with the
// uniform measure on the circle: tau'_j = (1 - beta) tau_j, which keeps the
// Toeplitz matrix G[k][l] = tau'_{l-k} positive definite.
//
// Bound at u0 = e^{i phi0}: the canonical (Szego) representation through u0
// has its other nodes at the roots of K(u, u0) = v(u)^T G^-1 conj(v(u0))
// (v(u) = (1, u, .., u^n)) and every node u_i carries the Christoffel weight
// 1 / K(u_i, u_i).  Substituting u = u0 (s + i) / (s - i), which sends u0 to
// s = infinity, turns K(., u0) into a real polynomial in s of degree n whose
// leading coefficient is K(u0, u0) > 0, so after division it is monic and
// real; its n real roots come from closed forms (Viete for the cubic, Ferrari
// for the quartic) polished by Newton steps.  A node lies in front of u0
// (angle in (-pi, phi0)) exactly when s < tan(phi0 / 2).  The result is
// A = w0 rho0 + the weights of the nodes in front.
//
// The per-pixel factorisation G = L D L^H runs in FP64; per sample all
// arithmetic is FP32.  The conditioning of G is bounded by the bias (about
// 1 / beta); the 16-bit storages need beta >= 2e-3, where FP32 suffices.
#pragma once
#include "mboit_device.cuh"

namespace mb {

MB_HD float fcos(float x) {
#if defined(__CUDA_ARCH__)
    return __cosf(x);
#else
    return cosf(x);
#endif
}

struct cf {
    float x, y;
};
MB_HD cf cmul(cf a, cf b) { return {ffma(a.x, b.x, -a.y * b.y), ffma(a.x, b.y, a.y * b.x)}; }
MB_HD cf cconj(cf a) { return {a.x, -a.y}; }
MB_HD cf csub(cf a, cf b) { return {a.x - b.x, a.y - b.y}; }
MB_HD cf cscale(cf a, float s) { return {a.x * s, a.y * s}; }
// a - b * c
MB_HD cf cfms(cf a, cf b, cf c) { return {ffma(-b.x, c.x, ffma(b.y, c.y, a.x)), ffma(-b.x, c.y, ffma(-b.y, c.x, a.y))}; }
// a - conj(b) * c
MB_HD cf cfms_conj(cf a, cf b, cf c) { return {ffma(-b.x, c.x, ffma(-b.y, c.y, a.x)), ffma(-b.x, c.y, ffma(b.y, c.x, a.y))}; }

struct TrigFrame {
    int32_t n;            // 0: no absorber, or G not positive definite (then A = 0)
    float m0_log2e;
    cf L[10];             // strictly lower part of L, row i at i (i - 1) / 2
    float invD[5];
};

// FP64 factorisation of the biased Toeplitz matrix of one pixel.
MB_HD TrigFrame make_trig_frame(float b0, const cf* tau, int n, float beta) {
    TrigFrame F;
    F.n = 0;
    F.m0_log2e = 0.0f;
    for (int i = 0; i < 10; ++i) F.L[i] = {0.0f, 0.0f};
    for (int i = 0; i < 5; ++i) F.invD[i] = 0.0f;
    if (!(b0 > 0.0f)) return F;
    const int n1 = n + 1;
    double tr[5], ti[5];
    tr[0] = 1.0;
    ti[0] = 0.0;
    for (int j = 1; j <= n; ++j) {
        tr[j] = (1.0 - (double)beta) * (double)tau[j - 1].x;
        ti[j] = (1.0 - (double)beta) * (double)tau[j - 1].y;
    }
    double Lr[5][5], Li[5][5], D[5];
    for (int j = 0; j < n1; ++j) {
        // G[j][j] = 1
        double s = 1.0;
        for (int k = 0; k < j; ++k) s -= (Lr[j][k] * Lr[j][k] + Li[j][k] * Li[j][k]) * D[k];
        if (!(s > 0.0)) return F;
        D[j] = s;
        for (int i = j + 1; i < n1; ++i) {
            // G[i][j] = conj(tau'[i - j])
            double xr = tr[i - j], xi = -ti[i - j];
            for (int k = 0; k < j; ++k) {
                // L[i][k] conj(L[j][k]) D[k]
                const double pr = Lr[i][k] * Lr[j][k] + Li[i][k] * Li[j][k];
                const double pi = Li[i][k] * Lr[j][k] - Lr[i][k] * Li[j][k];
                xr -= pr * D[k];
                xi -= pi * D[k];
            }
            Lr[i][j] = xr / D[j];
            Li[i][j] = xi / D[j];
        }
    }
    for (int i = 1; i < n1; ++i)
        for (int j = 0; j < i; ++j) F.L[i * (i - 1) / 2 + j] = {(float)Lr[i][j], (float)Li[i][j]};
    for (int i = 0; i < n1; ++i) F.invD[i] = (float)(1.0 / D[i]);
    F.n = n;
    F.m0_log2e = (float)((double)b0 * 1.4426950408889634);
    return F;
}

// Real roots of the monic cubic s^3 + a s^2 + b s + c whose roots are all
// real (Viete's trigonometric form), then one Newton step each.
MB_HD void cubic3(float a, float b, float c, float r[3]) {
    const float a3 = a * (1.0f / 3.0f);
    const float p = ffma(-a, a3, b);
    const float q = ffma(ffma(2.0f * a3, a3, -b), a3, c);  // 2 a3^3 - b a3 + c
    const float pm = fmin_(p, -1e-30f);
    const float m = 2.0f * fsqrt_fast(-pm * (1.0f / 3.0f));
    const float arg = fclamp(fdiv_fast(3.0f * q, pm * m), -1.0f, 1.0f);
    const float th = acosf(arg) * (1.0f / 3.0f);  // th in [0, pi/3]: the fast cosine is accurate on this range
    const float k2 = 2.0943951023931957f;  // 2 pi / 3
    r[0] = ffma(m, fcos(th), -a3);
    r[1] = ffma(m, fcos(th - k2), -a3);
    r[2] = ffma(m, fcos(th + k2), -a3);
    for (int i = 0; i < 3; ++i) {
        const float s = r[i];
        const float f = ffma(ffma(s + a, s, b), s, c);
        const float df = ffma(ffma(3.0f, s, 2.0f * a), s, b);
        if (df != 0.0f) r[i] = s - fdiv_fast(f, df);   // Newton corrects the 2-ulp quotient
    }
}

// The largest real root of the monic cubic s^3 + a s^2 + b s + c whose roots
// are all real: Viete's root of the largest cosine (th in [0, pi/3]), then one
// Newton step.
MB_HD float cubic3_max(float a, float b, float c) {
    const float a3 = a * (1.0f / 3.0f);
    const float p = ffma(-a, a3, b);
    const float q = ffma(ffma(2.0f * a3, a3, -b), a3, c);
    const float pm = fmin_(p, -1e-30f);
    const float m = 2.0f * fsqrt_fast(-pm * (1.0f / 3.0f));
    const float arg = fclamp(fdiv_fast(3.0f * q, pm * m), -1.0f, 1.0f);
    const float s = ffma(m, fcos(acosf(arg) * (1.0f / 3.0f)), -a3);
    const float f = ffma(ffma(s + a, s, b), s, c);
    const float df = ffma(ffma(3.0f, s, 2.0f * a), s, b);
    return df != 0.0f ? s - fdiv_fast(f, df) : s;
}

// Real roots of the monic quartic s^4 + a s^3 + b s^2 + c s + d whose roots
// are all real (Ferrari: resolvent cubic, two quadratics), then Newton steps.
MB_HD void quartic4(float a, float b, float c, float d, float r[4]) {
    const float a4 = 0.25f * a;
    const float a42 = a4 * a4;
    const float p = ffma(-6.0f, a42, b);
    const float q = ffma(ffma(8.0f, a42, -2.0f * b), a4, c);              // c - 2 b a4 + 8 a4^3
    const float rr = ffma(ffma(ffma(-3.0f, a42, b), a4, -c), a4, d);      // d - c a4 + b a4^2 - 3 a4^4
    float y[4];
    const float scale = fmax_(fabsf(p), fmax_(fsqrt_fast(fabsf(rr)), 1e-30f));
    if (fabsf(q) <= 1e-6f * scale * fsqrt_fast(scale)) {
        // biquadratic: y^2 = (-p +- sqrt(p^2 - 4 r)) / 2
        const float disc = fsqrt_fast(fmax_(ffma(p, p, -4.0f * rr), 0.0f));
        const float y1 = fsqrt_fast(fmax_(0.5f * (-p + disc), 0.0f));
        const float y2 = fsqrt_fast(fmax_(0.5f * (-p - disc), 0.0f));
        y[0] = -y1; y[1] = -y2; y[2] = y2; y[3] = y1;
    } else {
        // m^3 + p m^2 + (p^2/4 - r) m - q^2/8 = 0, largest root (positive)
        const float m = fmax_(cubic3_max(p, ffma(0.25f * p, p, -rr), -0.125f * q * q), 1e-30f);
        const float sq = fsqrt_fast(2.0f * m);
        const float h = 0.5f * p + m, g = fdiv_fast(q, 2.0f * sq);
        // y^2 - sq y + (h + g) = 0 and y^2 + sq y + (h - g) = 0
        const float d1 = fsqrt_fast(fmax_(ffma(sq, sq, -4.0f * (h + g)), 0.0f));
        const float d2 = fsqrt_fast(fmax_(ffma(sq, sq, -4.0f * (h - g)), 0.0f));
        y[0] = 0.5f * (sq - d1); y[1] = 0.5f * (sq + d1);
        y[2] = 0.5f * (-sq - d2); y[3] = 0.5f * (-sq + d2);
    }
    for (int i = 0; i < 4; ++i) {
        float s = y[i] - a4;
        for (int it = 0; it < 1; ++it) {
            const float f = ffma(ffma(ffma(s + a, s, b), s, c), s, d);
            const float df = ffma(ffma(ffma(4.0f, s, 3.0f * a), s, 2.0f * b), s, c);
            if (df != 0.0f) s = s - fdiv_fast(f, df);
        }
        r[i] = s;
    }
}

// K(u, u) = sum_k |x_k|^2 / D_k with L x = conj(v(u)).
template <int N>
MB_HD float trig_kernel_diag(const TrigFrame& F, cf u) {
    cf x[N + 1];
    cf ub = cconj(u), p = {1.0f, 0.0f};
    float K = 0.0f;
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        cf xi = p;
#pragma unroll
        for (int k = 0; k < i; ++k) xi = cfms(xi, F.L[i * (i - 1) / 2 + k], x[k]);
        x[i] = xi;
        K = ffma(ffma(xi.x, xi.x, xi.y * xi.y), F.invD[i], K);
        p = cmul(p, ub);
    }
    return K;
}

// Alg. 3 for trigonometric moments: fraction A of the optical depth in front
// of warped depth z0.
template <int N>
MB_HD float trig_fraction(const TrigFrame& F, const TrigTables& T, float z0, float w0) {
    if (F.n == 0) return 0.0f;
    const float phi = z0 * T.zone_scale;
#if defined(__CUDA_ARCH__)
    float sn, cs;
    __sincosf(phi, &sn, &cs);
#else
    const float sn = sinf(phi), cs = cosf(phi);
#endif
    const cf u0 = {cs, sn};
    // y = G^-1 w, w = conj(v(u0)) = (1, conj(u0), conj(u0)^2, ..)
    cf w[N + 1], y[N + 1];
    w[0] = {1.0f, 0.0f};
#pragma unroll
    for (int k = 1; k <= N; ++k) w[k] = cmul(w[k - 1], cconj(u0));
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        cf t = w[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t = cfms(t, F.L[i * (i - 1) / 2 + k], y[k]);
        y[i] = t;
    }
#pragma unroll
    for (int i = 0; i <= N; ++i) y[i] = cscale(y[i], F.invD[i]);
#pragma unroll
    for (int i = N; i >= 0; --i) {
        cf t = y[i];
#pragma unroll
        for (int k = i + 1; k <= N; ++k) t = cfms_conj(t, F.L[k * (k - 1) / 2 + i], y[k]);
        y[i] = t;
    }
    // z_k = y_k u0^k; K(u0, u0) = Re sum z_k; real polynomial coefficients
    float zr[N + 1], zi[N + 1], K00 = 0.0f;
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        const cf z = cmul(y[k], cconj(w[k]));
        zr[k] = z.x;
        zi[k] = z.y;
        K00 += z.x;
    }
    const float invK = frcp(K00);
    float coef[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k <= N; ++k) acc = ffma(zr[k], T.er[k][m], ffma(-zi[k], T.ei[k][m], acc));
        coef[m] = acc * invK;
    }
    float rts[N];
    if (N == 3)
        cubic3(coef[2], coef[1], coef[0], rts);
    else
        quartic4(coef[3], coef[2], coef[1], coef[0], rts);
    const float sp = sn / (1.0f + cs);  // tan(phi0 / 2); |phi0| < pi by the wrapping zone
    float A = w0 * invK;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float s = rts[i];
        if (!(s < sp)) continue;
        const float inv = frcp(ffma(s, s, 1.0f));
        const cf e = {(s * s - 1.0f) * inv, 2.0f * s * inv};  // (s + i) / (s - i)
        A += frcp(trig_kernel_diag<N>(F, cmul(u0, e)));
    }
    return A;
}

}  // namespace mb
