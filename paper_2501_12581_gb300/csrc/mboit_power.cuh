// Moment bound with 2n power moments, n = 3 or 4 (the 6- and 8-moment
// variants of Sec. 4.3 / Fig. 3; Alg. 3 at order n).
//
// Alg. 3 at order n solves B q = (1, z0, .., z0^n) with the (n+1) x (n+1)
// Hankel matrix B of the biased normalised moments, takes the n roots of
// sum q_j x^j as the other support points of the canonical representation
// through z0 and sums its weights with w = (overestimation, [z_i < z0]).
// As for four moments we compute that representation in the standardised
// frame x = (z - mu) / s of the biased measure (mean 0, variance 1; an affine
// map keeps the order of the support points and their weights):
//   per pixel, FP64: b' = (1 - beta) b / b0 + beta c (c: moments of the
//     arcsine law on [-1, 1], b'_2k = C(2k, k) / 4^k), the standardised
//     moments h_j = E'[x^j] and H[i][j] = h_{i+j} = L D L^T;
//   per sample, FP32: y = L^-1 v(x0), K(x0, x0) = sum y_k^2 / D_k,
//     q = L^-T D^-1 y (the kernel polynomial K(., x0) = sum q_j x^j), its n
//     real roots in the variable s = 1 / (x - x0) from closed forms (Viete,
//     Ferrari) polished by Newton steps, and the Christoffel weight
//     1 / K(x_i, x_i) of every root in front:
//     A = w0 / K(x0, x0) + sum_{x_i < x0} 1 / K(x_i, x_i).
// Every weight is a sum of positive terms, so no cancellation enters A.  A
// pixel whose Hankel matrix is numerically singular (a pivot below 1e-12 of
// its diagonal entry: no bias and at most n absorbers) falls back to the
// four-moment frame, which handles one- and two-atom measures exactly.
#pragma once
#include "mboit_trig.cuh"

namespace mb {

// A pixel set up with the four-moment frame (numerically singular Hankel matrix).
constexpr int32_t kFrameFourMoments = 4;

// b'_2k of the arcsine law, k = 1..4: C(2k, k) / 4^k.
MB_HD double arcsine_moment(int j) {
    return (j & 1) ? 0.0 : j == 2 ? 0.5 : j == 4 ? 0.375 : j == 6 ? 0.3125 : j == 8 ? 0.2734375 : 1.0;
}

template <int N>
struct PowerFrame {
    int32_t kind;             // kFrameEmpty, kFrameGeneric or kFrameFourMoments (then F4)
    float m0_log2e;           // b0 log2(e)
    float inv_s, nmu;         // x = z inv_s + nmu
    float L[N * (N + 1) / 2]; // strictly lower part of L, row i at i (i - 1) / 2
    float invD[N + 1];
    Frame F4;
};

// FP64 set-up of one pixel from its 2N + 1 float moments.
template <int N>
MB_HD PowerFrame<N> make_power_frame(const float* m_in, float moment_bias) {
    PowerFrame<N> P;
    P.kind = kFrameEmpty;
    P.m0_log2e = 0.0f;
    P.inv_s = 1.0f;
    P.nmu = 0.0f;
    for (int i = 0; i < N * (N + 1) / 2; ++i) P.L[i] = 0.0f;
    for (int i = 0; i <= N; ++i) P.invD[i] = 0.0f;
    P.F4.kind = kFrameEmpty;
    P.F4.m0_log2e = 0.0f;
    P.F4.p0 = P.F4.p1 = P.F4.p2 = P.F4.p3 = 0.0f;
    const double m0 = (double)m_in[0];
    if (!(m0 > 0.0)) return P;
    const double beta = (double)moment_bias;
    double b[2 * N + 1];
    b[0] = 1.0;
    for (int j = 1; j <= 2 * N; ++j) b[j] = (1.0 - beta) * ((double)m_in[j] / m0) + beta * arcsine_moment(j);
    P.m0_log2e = (float)(m0 * 1.4426950408889634);
    const double mu = b[1];
    const double var = b[2] - mu * mu;
    bool ok = var > 1e-12 * b[2];
    double L[N + 1][N + 1], D[N + 1];
    if (ok) {
        // standardised moments h_j = sum_i C(j, i) b_i (-mu)^(j-i) / s^j
        const double s = sqrt(var), inv_s = 1.0 / s;
        double h[2 * N + 1];
        double sj = 1.0;
        for (int j = 0; j <= 2 * N; ++j) {
            double acc = 0.0, c = 1.0, pw = 1.0;  // c = C(j, i), pw = (-mu)^(j-i) from i = j down
            for (int i = j; i >= 0; --i) {
                acc += c * b[i] * pw;
                c = c * (double)i / (double)(j - i + 1);
                pw *= -mu;
            }
            h[j] = acc * sj;
            sj *= inv_s;
        }
        h[0] = 1.0;
        h[1] = 0.0;
        h[2] = 1.0;
        for (int j = 0; j <= N && ok; ++j) {
            double d = h[2 * j];
            for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k] * D[k];
            if (!(d > 1e-12 * fabs(h[2 * j]))) {
                ok = false;
                break;
            }
            D[j] = d;
            for (int i = j + 1; i <= N; ++i) {
                double t = h[i + j];
                for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k] * D[k];
                L[i][j] = t / d;
            }
        }
        if (ok) {
            P.kind = kFrameGeneric;
            P.inv_s = (float)inv_s;
            P.nmu = (float)(-mu * inv_s);
            for (int i = 1; i <= N; ++i)
                for (int k = 0; k < i; ++k) P.L[i * (i - 1) / 2 + k] = (float)L[i][k];
            for (int i = 0; i <= N; ++i) P.invD[i] = (float)(1.0 / D[i]);
            return P;
        }
    }
    // numerically singular: the four-moment frame of b0..b4 (exact for one
    // or two atoms)
    const float bv4[4] = {0.0f, 0.5f, 0.0f, 0.375f};
    P.F4 = make_frame(m_in, moment_bias, bv4);
    P.kind = P.F4.kind == kFrameEmpty ? kFrameEmpty : kFrameFourMoments;
    return P;
}

// K(x, x) = sum_k (L^-1 v(x))_k^2 / D_k.
template <int N>
MB_HD float power_kernel_diag(const PowerFrame<N>& P, float x) {
    float y[N + 1], v = 1.0f, K = 0.0f;
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        float t = v;
#pragma unroll
        for (int k = 0; k < i; ++k) t = ffma(-P.L[i * (i - 1) / 2 + k], y[k], t);
        y[i] = t;
        K = ffma(t * t, P.invD[i], K);
        v *= x;
    }
    return K;
}

// Alg. 3 at order N: fraction A of the optical depth in front of warped
// depth z0.
template <int N>
MB_HD float power_fraction(const PowerFrame<N>& P, float z0, float w0) {
    if (P.kind != kFrameGeneric) return P.kind == kFrameEmpty ? 0.0f : bound_fraction(P.F4, z0, w0);
    const float x0 = ffma(z0, P.inv_s, P.nmu);
    float u[N + 1], y[N + 1], v = 1.0f, K00 = 0.0f;
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        float t = v;
#pragma unroll
        for (int k = 0; k < i; ++k) t = ffma(-P.L[i * (i - 1) / 2 + k], u[k], t);
        u[i] = t;
        y[i] = t * P.invD[i];
        K00 = ffma(t, y[i], K00);
        v *= x0;
    }
    // q = L^-T D^-1 y: coefficients of K(., x0) in the standardised frame
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        float t = y[i];
#pragma unroll
        for (int k = i + 1; k <= N; ++k) t = ffma(-P.L[k * (k - 1) / 2 + i], y[k], t);
        y[i] = t;
    }
    // Substituting x = x0 + 1/s sends x0 to s = infinity: s^N K(x0 + 1/s, x0)
    // = sum_k r_k s^(N-k) with r_k the Taylor coefficients of K(., x0) at x0
    // (a Taylor shift by repeated synthetic division), and r_0 = K(x0, x0) > 0
    // leads.  A support point that escapes to infinity (x0 near a zero of the
    // degree-N orthogonal polynomial) sits near s = 0, where it is harmless,
    // and x_i < x0 exactly when s_i < 0.
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int i = N - 1; i >= k; --i) y[i] = ffma(x0, y[i + 1], y[i]);
    const float iK = frcp(K00);
    float rts[N];
    if (N == 3)
        cubic3(y[1] * iK, y[2] * iK, y[3] * iK, rts);
    else
        quartic4(y[1] * iK, y[2] * iK, y[3] * iK, y[4] * iK, rts);
    float A = w0 * iK;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        // |s| < 1e-4: a point beyond |x - x0| = 1e4, weight below 1e-30
        if (!(rts[i] < -1e-4f)) continue;
        A += frcp(power_kernel_diag<N>(P, x0 + frcp(rts[i])));
    }
    return fclamp(A, 0.0f, 1.0f);
}

}  // namespace mb
