/*
 * FP64 CPU oracle of the two-pass MBOIT puzzle-piece render.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU baseline; the product library never links or calls it.
 * Single-threaded, plain loops, one pixel at a time, in the order of the
 * paper:
 *   Alg. 1 (RenderMBOIT): loop 1 accumulates moments, loop 2 adds
 *          getTransmittance(b, depth) * colour;
 *   Alg. 2 (GeneratePowerMoments): warp depth, absorbance = -log(transmittance)
 *          clamped, b_i += depth^i * absorbance;
 *   Alg. 3 (getTransmittance): warp, mix with the bias vector, Cholesky of the
 *          Hankel matrix, roots, weights (overestimation, indicators),
 *          interpolating polynomial, absorbance = p . (1, b), exp;
 *   Sec. 4.1: per-piece ("per-rank") moment images, summed (Allreduce add);
 *   Sec. 4.2: per-piece colour images from the global moments, summed
 *          (Reduce add).
 * Readings where the paper is silent:
 *   - sample lattice t_k = (k + 1/2) * step from the eye; rays and sample
 *     positions are specified in float32 (correctly rounded ops in a fixed
 *     order, positions by fmaf); everything after the position is FP64;
 *   - a lattice point belongs to the piece owning the brick of its cell
 *     (half-open cells; pieces never overlap, Sec. 6);
 *   - transfer-function alpha is the opacity of one voxel of material,
 *     sigma = -ln(1 - alpha); (r, g, b, sigma) interpolate linearly;
 *     absorbance a = min(sigma * step, ABSORBANCE_MAX), opacity 1 - e^-a;
 *   - the resolve renormalises: alpha = 1 - e^-b0 (zeroth moment), colour =
 *     (sum T a c) / (sum T a) * alpha (the renormalisation of Sec. 4.3);
 *   - singular Hankel matrices (one or two absorbers, zero bias) take the
 *     one- or two-atom canonical measure;
 *   - the exact reference blends the same samples front to back; the
 *     sort-last route turns each contiguous per-piece run into a segment.
 * Build: cc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction
 * so the float32 ray set-up rounds exactly as written).
 */
#include "mboit_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>

#define ORC_PI 3.14159265358979323846
#include <string.h>

#define ORC_TAU 1e-12

/* ------------------------------------------------------------------------ */
/* depth warp (Alg. 2, Alg. 3: "rescale logged depth value to [-1, 1]")     */

double orc_log_warp(double t, double znear, double zfar)
{
    double z = 2.0 * (log(t) - log(znear)) / (log(zfar) - log(znear)) - 1.0;
    if (z < -1.0) z = -1.0;
    if (z > 1.0) z = 1.0;
    return z;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3                                                                    */

/* Real roots of a*x^2 + b*x + c with the cancellation-free formula; the
 * discriminant is clamped at zero.  Returns the number of finite roots. */
static int quadratic_roots(double a, double b, double c, double* r1, double* r2)
{
    if (a == 0.0) {
        if (b == 0.0) return 0;
        *r1 = -c / b;
        return 1;
    }
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) disc = 0.0;
    double q = -0.5 * (b + copysign(sqrt(disc), b));
    double x1 = q / a;
    double x2 = (q != 0.0) ? c / q : x1;
    if (x1 > x2) { double s = x1; x1 = x2; x2 = s; }
    *r1 = x1;
    *r2 = x2;
    return 2;
}

static double step_weight(double x, double z0, double w0)
{
    if (x < z0) return 1.0;
    if (x == z0) return w0;
    return 0.0;
}

double orc_mboit_bound(const double m[5], double z0, double moment_bias,
                       const double bias_vector[4], double overestimation, int* flags)
{
    if (flags) *flags = 0;
    if (!(m[0] > 0.0)) return 0.0;

    /* b_tmp = (b1..b4) / b0, then mix with the bias vector */
    double b[5];
    b[0] = 1.0;
    for (int j = 1; j <= 4; ++j) {
        double bj = m[j] / m[0];
        b[j] = (1.0 - moment_bias) * bj + moment_bias * bias_vector[j - 1];
    }

    /* SolveMat: Hankel matrix B[i][j] = b[i+j] (i, j = 0..2) as L D L^T */
    double D22 = b[2] - b[1] * b[1];
    if (D22 <= ORC_TAU) {
        /* single atom at b1 */
        if (flags) *flags = 1;
        return step_weight(b[1], z0, overestimation);
    }
    double L32 = (b[3] - b[1] * b[2]) / D22;
    double D33 = b[4] - b[2] * b[2] - L32 * L32 * D22;
    double scale = fabs(b[4]) > 1.0 ? fabs(b[4]) : 1.0;
    if (D33 <= ORC_TAU * scale) {
        /* two atoms: roots of x^2 + e1 x + e0 with
         * [[1, b1], [b1, b2]] (e0, e1)^T = -(b2, b3)^T */
        double det = b[2] - b[1] * b[1];
        double e0 = (-b[2] * b[2] + b[1] * b[3]) / det;
        double e1 = (-b[3] + b[1] * b[2]) / det;
        double x1, x2;
        if (quadratic_roots(1.0, e1, e0, &x1, &x2) != 2) return step_weight(b[1], z0, overestimation);
        double rho2 = (x2 != x1) ? (b[1] - x1) / (x2 - x1) : 0.0;
        double rho1 = 1.0 - rho2;
        if (flags) *flags = 2;
        return rho1 * step_weight(x1, z0, overestimation) + rho2 * step_weight(x2, z0, overestimation);
    }

    /* solve B q = (1, z0, z0^2): forward, diagonal, backward */
    double y1 = 1.0;
    double y2 = z0 - b[1] * y1;
    double y3 = z0 * z0 - b[2] * y1 - L32 * y2;
    y2 /= D22;
    y3 /= D33;
    double q2 = y3;
    double q1 = y2 - L32 * q2;
    double q0 = y1 - b[1] * q1 - b[2] * q2;

    /* SolvePowerEquation: the other two support points, roots of
     * q2 x^2 + q1 x + q0 */
    double z[3];
    z[0] = z0;
    z[1] = z[2] = z0;
    int nroot = quadratic_roots(q2, q1, q0, &z[1], &z[2]);
    if (nroot == 0) return overestimation;  /* constant kernel polynomial: all mass at z0 */

    /* weights: overestimation at z0, indicator z_i < z0 elsewhere */
    double w[3];
    w[0] = overestimation;
    w[1] = (z[1] < z0) ? 1.0 : 0.0;
    w[2] = (nroot == 2 && z[2] < z0) ? 1.0 : 0.0;

    /* solvePolynomial: Newton interpolation of the weights at the nodes,
     * p(x) = w0 + f01 (x - z0) + f012 (x - z0)(x - z1), expanded */
    double p0, p1, p2;
    if (z[1] == z0) return w[0];  /* measure-zero: z0 is a support point */
    double f01 = (w[1] - w[0]) / (z[1] - z0);
    if (nroot == 2 && z[2] != z[1] && z[2] != z0) {
        double f12 = (w[2] - w[1]) / (z[2] - z[1]);
        double f012 = (f12 - f01) / (z[2] - z0);
        p2 = f012;
        p1 = f01 - f012 * (z0 + z[1]);
        p0 = w[0] - f01 * z0 + f012 * z0 * z[1];
    } else {
        p2 = 0.0;
        p1 = f01;
        p0 = w[0] - f01 * z0;
    }
    /* absorbance = p . (1, b_tmp) */
    return p0 + p1 * b[1] + p2 * b[2];
}

/* ------------------------------------------------------------------------ */
/* the volume being rendered: a regular grid or a brick octree               */

typedef struct {
    int kind;                      /* 0 grid, 1 brick octree, 2 tetrahedral mesh */
    const orc_grid* g;
    const orc_amr* a;
    int32_t* fmap;                 /* octree: finest brick -> leaf (-1 none) */
    int64_t fdim;                  /* finest bricks per axis */
    const orc_tet* m;
    int64_t* vq;                   /* tets: snapped vertex coordinates [n_verts][3] */
    int32_t *bin_start, *bin_tets; /* tets: unit bins -> tets whose box meets the bin */
    int64_t bdim[3];
    int overlap;                   /* tets: set when two tets claim one point */
    double hi[3];                  /* the domain is [0, hi) per axis */
    int n_pieces;
    const uint8_t* piece_selected;
    const float* tf;
    double vmin, vmax, step, moment_bias, overestimation, absorbance_max;
    const double* bias_vector;
    int n_trig;                    /* 0: power moments; 3 or 4 complex trigonometric moments */
    int n_power;                   /* 2n power moments b0..b_2n: n = 2, 3 or 4 (0 with trig moments) */
    double power_bias[8];          /* bias measure of the 6- and 8-moment sets */
    int storage;                   /* 0, 1 float16, 2 bfloat16 (normalised trig moments) */
    double trig_zone;
    const double* given_moments;   /* NULL, or per listed pixel the global moments stage two uses */
} vol_t;

#define ORC_MAX_NM 9

static int n_moments(const vol_t* g) { return g->n_trig ? 1 + 2 * g->n_trig : 1 + 2 * g->n_power; }

/* moment_set 0 / 6 / 8: 4 / 6 / 8 power moments (FP64, no storage rounding);
 * 3 / 4: complex trigonometric moments, optionally rounded to 16 bits. */
static int set_moments(vol_t* v, int32_t moment_set, int32_t storage, double trig_zone)
{
    int trig = moment_set == 3 || moment_set == 4;
    if (!trig && moment_set != 0 && moment_set != 6 && moment_set != 8) return -1;
    if (storage < 0 || storage > 2 || (storage && !trig)) return -1;
    v->n_trig = trig ? moment_set : 0;
    v->n_power = trig ? 0 : moment_set == 0 ? 2 : moment_set / 2;
    if (v->n_power > 2) orc_power_bias(v->n_power, v->power_bias);
    v->storage = storage;
    v->trig_zone = trig_zone;
    return 0;
}

/* round-to-nearest-even float -> float16 -> float (finite inputs) */
static float round_f16(float x)
{
    union { float f; uint32_t u; } v = {x};
    uint32_t sign = v.u & 0x80000000u, ax = v.u & 0x7fffffffu;
    float a = fabsf(x);
    if (a >= 65520.0f) return sign ? -INFINITY : INFINITY;
    if (a < 6.103515625e-05f) {                       /* subnormal half: quantum 2^-24 */
        float q = nearbyintf(a * 16777216.0f) / 16777216.0f;
        return sign ? -q : q;
    }
    uint32_t lsb = (ax >> 13) & 1u;
    ax += 0x0fffu + lsb;                               /* RNE on the 13 dropped bits */
    ax &= 0xffffe000u;
    v.u = sign | ax;
    return v.f;
}

/* round-to-nearest-even float -> bfloat16 -> float (finite inputs) */
static float round_bf16(float x)
{
    union { float f; uint32_t u; } v = {x};
    uint32_t lsb = (v.u >> 16) & 1u;
    v.u += 0x7fffu + lsb;
    v.u &= 0xffff0000u;
    return v.f;
}

double orc_store_round(double x, int storage)
{
    float f = (float)x;
    return storage == 1 ? (double)round_f16(f) : storage == 2 ? (double)round_bf16(f) : (double)f;
}

/* The moments as the renderer stores them: trigonometric moments normalised
 * by b0 in float32, then rounded to the 16-bit format. */
static void store_moments(const vol_t* g, double* m)
{
    if (!g->n_trig || !g->storage || !(m[0] > 0.0)) return;
    for (int j = 1; j <= 2 * g->n_trig; ++j) {
        float t = (float)(m[j] / m[0]);
        t = (g->storage == 1) ? round_f16(t) : round_bf16(t);
        m[j] = (double)t * m[0];
    }
}

/* ------------------------------------------------------------------------ */
/* trigonometric moments                                                     */

/* Hermitian Toeplitz G[k][l] = tau[l - k] (tau[-j] = conj tau[j]) as
 * L D L^H; returns -1 unless every pivot is positive. */
static int toeplitz_ldl(int n1, const double complex* tau, double complex L[5][5], double D[5])
{
    double complex G[5][5];
    for (int k = 0; k < n1; ++k)
        for (int l = 0; l < n1; ++l) G[k][l] = (l >= k) ? tau[l - k] : conj(tau[k - l]);
    for (int j = 0; j < n1; ++j) {
        double complex s = G[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * conj(L[j][k]) * D[k];
        D[j] = creal(s);
        if (!(D[j] > 0.0)) return -1;
        L[j][j] = 1.0;
        for (int i = j + 1; i < n1; ++i) {
            double complex t = G[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * conj(L[j][k]) * D[k];
            L[i][j] = t / D[j];
        }
    }
    return 0;
}

/* x = G^-1 b with G = L D L^H */
static void toeplitz_solve(int n1, double complex L[5][5], const double D[5], const double complex* b,
                           double complex* x)
{
    double complex y[5];
    for (int i = 0; i < n1; ++i) {
        y[i] = b[i];
        for (int k = 0; k < i; ++k) y[i] -= L[i][k] * y[k];
    }
    for (int i = 0; i < n1; ++i) y[i] /= D[i];
    for (int i = n1 - 1; i >= 0; --i) {
        x[i] = y[i];
        for (int k = i + 1; k < n1; ++k) x[i] -= conj(L[k][i]) * x[k];
    }
}

/* Reproducing kernel K(u, u) = v(u)^T G^-1 conj(v(u)), v(u) = (1, u, .., u^n) */
static double kernel_diag(int n1, double complex L[5][5], const double D[5], double complex u)
{
    double complex w[5], x[5];
    double complex p = 1.0;
    for (int k = 0; k < n1; ++k) {
        w[k] = conj(p);
        p *= u;
    }
    toeplitz_solve(n1, L, D, w, x);
    double complex s = 0.0;
    p = 1.0;
    for (int k = 0; k < n1; ++k) {
        s += p * x[k];
        p *= u;
    }
    return creal(s);
}

/* Roots of c[0] + c[1] u + ... + c[n] u^n by the Aberth-Ehrlich iteration. */
static int poly_roots(int n, const double complex* c, double complex* r)
{
    for (int i = 0; i < n; ++i) r[i] = 0.9 * cexp(I * (2.0 * ORC_PI * i / n + 0.4));
    double last = INFINITY;
    for (int it = 0; it < 500; ++it) {
        double change = 0.0;
        for (int i = 0; i < n; ++i) {
            double complex pv = c[n], dv = 0.0;
            for (int k = n - 1; k >= 0; --k) {
                dv = dv * r[i] + pv;
                pv = pv * r[i] + c[k];
            }
            if (pv == 0.0) continue;
            double complex ratio = pv / dv;
            double complex sum = 0.0;
            for (int j = 0; j < n; ++j)
                if (j != i) sum += 1.0 / (r[i] - r[j]);
            double complex step = ratio / (1.0 - ratio * sum);
            r[i] -= step;
            double a = cabs(step);
            if (a > change) change = a;
        }
        if (change < 4e-15) return 0;
        last = change;
    }
    return last < 1e-10 ? 0 : -2;
}

static double trig_bound_impl(const double* m, int n, double phi0, double moment_bias, double overestimation,
                              int* status, double* weights_sum, double* nodes, double* weights);

double orc_trig_bound(const double* m, int n, double phi0, double moment_bias, double overestimation,
                      int* status, double* weights_sum)
{
    return trig_bound_impl(m, n, phi0, moment_bias, overestimation, status, weights_sum, NULL, NULL);
}

int orc_trig_nodes(const double* m, int n, double phi0, double moment_bias, double* nodes, double* weights)
{
    int st = 0;
    trig_bound_impl(m, n, phi0, moment_bias, 0.0, &st, NULL, nodes, weights);
    return st;
}

static double trig_bound_impl(const double* m, int n, double phi0, double moment_bias, double overestimation,
                              int* status, double* weights_sum, double* nodes, double* weights)
{
    if (status) *status = 0;
    if (weights_sum) *weights_sum = 0.0;
    if (!(m[0] > 0.0)) return 0.0;
    int n1 = n + 1;
    double complex tau[5];
    tau[0] = 1.0;
    for (int j = 1; j <= n; ++j) tau[j] = (1.0 - moment_bias) * (m[2 * j - 1] + I * m[2 * j]) / m[0];
    double complex L[5][5];
    double D[5] = {0, 0, 0, 0, 0};
    if (toeplitz_ldl(n1, tau, L, D) != 0) {
        if (status) *status = -1;
        return 0.0;
    }
    /* kernel polynomial through u0: coefficients y = G^-1 conj(v(u0)) */
    double complex u0 = cexp(I * phi0), w[5], y[5], p = 1.0;
    for (int k = 0; k < n1; ++k) {
        w[k] = conj(p);
        p *= u0;
    }
    toeplitz_solve(n1, L, D, w, y);
    double k00 = 0.0;
    p = 1.0;
    for (int k = 0; k < n1; ++k) {
        k00 += creal(p * y[k]);
        p *= u0;
    }
    double rho0 = 1.0 / k00;
    double complex roots[4];
    if (poly_roots(n, y, roots) != 0 && status) *status = -2;
    double A = overestimation * rho0, sum = rho0;
    if (nodes) {
        nodes[0] = creal(u0);
        nodes[1] = cimag(u0);
        weights[0] = rho0;
    }
    for (int i = 0; i < n; ++i) {
        double complex ui = roots[i] / cabs(roots[i]);  /* the nodes lie on the unit circle */
        double rho = 1.0 / kernel_diag(n1, L, D, ui);
        sum += rho;
        if (carg(ui) < phi0) A += rho;
        if (nodes) {
            nodes[2 * i + 2] = creal(ui);
            nodes[2 * i + 3] = cimag(ui);
            weights[i + 1] = rho;
        }
    }
    if (weights_sum) *weights_sum = sum;
    return A;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 with 2n power moments (n = 2, 3, 4)                                */

void orc_power_bias(int n, double* bias)
{
    double c = 1.0;  /* C(2k, k) / 4^k = prod_{i <= k} (2i - 1) / (2i) */
    for (int j = 1; j <= 2 * n; ++j) {
        if (j % 2) {
            bias[j - 1] = 0.0;
            continue;
        }
        c *= (double)(j - 1) / (double)j;
        bias[j - 1] = c;
    }
}

/* x = B^-1 r for the leading n1 x n1 block of B = L D L^T */
static void hankel_solve(int n1, double L[5][5], const double D[5], const double* r, double* x)
{
    double y[5];
    for (int i = 0; i < n1; ++i) {
        y[i] = r[i];
        for (int k = 0; k < i; ++k) y[i] -= L[i][k] * y[k];
    }
    for (int i = 0; i < n1; ++i) y[i] /= D[i];
    for (int i = n1 - 1; i >= 0; --i) {
        x[i] = y[i];
        for (int k = i + 1; k < n1; ++k) x[i] -= L[k][i] * x[k];
    }
}

/* Real parts of the roots of c[0] + c[1] x + .. + c[deg] x^deg, ascending
 * (the roots are real here: zeros of a kernel or orthogonal polynomial).
 * Returns their number (the degree after dropping zero leading terms). */
static int real_roots(int deg, const double* c, double* r)
{
    while (deg > 0 && c[deg] == 0.0) --deg;
    if (deg <= 0) return 0;
    double complex cc[5], rc[4];
    for (int k = 0; k <= deg; ++k) cc[k] = c[k];
    poly_roots(deg, cc, rc);
    for (int k = 0; k < deg; ++k) r[k] = creal(rc[k]);
    for (int a = 1; a < deg; ++a)
        for (int b = a; b > 0 && r[b - 1] > r[b]; --b) {
            double t = r[b];
            r[b] = r[b - 1];
            r[b - 1] = t;
        }
    return deg;
}

double orc_power_bound(const double* m, int n, double z0, double moment_bias, const double* bias,
                       double overestimation, int* flags, double* nodes)
{
    if (flags) *flags = 0;
    if (!(m[0] > 0.0) || n < 1 || n > 4) return 0.0;
    const int n1 = n + 1;

    /* b_tmp = (b1..b2n) / b0, mixed with the bias measure */
    double b[9];
    b[0] = 1.0;
    for (int j = 1; j <= 2 * n; ++j) b[j] = (1.0 - moment_bias) * (m[j] / m[0]) + moment_bias * bias[j - 1];

    /* Hankel matrix B[i][j] = b[i + j] as L D L^T, column by column; the
     * first pivot that is not positive ends it: k atoms */
    double L[5][5], D[5];
    int k = n1;
    for (int j = 0; j < n1; ++j) {
        double s = b[2 * j];
        for (int l = 0; l < j; ++l) s -= L[j][l] * L[j][l] * D[l];
        double scale = fabs(b[2 * j]) > 1.0 ? fabs(b[2 * j]) : 1.0;
        if (s <= ORC_TAU * scale) {
            k = j;
            break;
        }
        D[j] = s;
        L[j][j] = 1.0;
        for (int i = j + 1; i < n1; ++i) {
            double t = b[i + j];
            for (int l = 0; l < j; ++l) t -= L[i][l] * L[j][l] * D[l];
            L[i][j] = t / D[j];
        }
    }

    if (k < n1) {
        /* a measure of k atoms: the roots of x^k + sum_{j<k} e_j x^j with
         * H_k e = -(b_k, .., b_2k-1), H_k the leading k x k block */
        double r[4], e[5], x[4];
        for (int i = 0; i < k; ++i) r[i] = -b[i + k];
        hankel_solve(k, L, D, r, e);
        e[k] = 1.0;
        int na = real_roots(k, e, x);
        /* weight of atom i: the integral of its Lagrange basis polynomial */
        double A = 0.0;
        for (int i = 0; i < na; ++i) {
            double c[5] = {1.0, 0.0, 0.0, 0.0, 0.0}, den = 1.0;
            int deg = 0;
            for (int o = 0; o < na; ++o) {
                if (o == i) continue;
                c[deg + 1] = c[deg];
                for (int t = deg; t >= 1; --t) c[t] = c[t - 1] - x[o] * c[t];
                c[0] = -x[o] * c[0];
                ++deg;
                den *= x[i] - x[o];
            }
            double rho = 0.0;
            for (int t = 0; t <= deg; ++t) rho += c[t] * b[t];
            A += rho / den * step_weight(x[i], z0, overestimation);
            if (nodes) nodes[i] = x[i];
        }
        if (flags) *flags = k;
        return A;
    }

    /* SolveMat: q = B^-1 (1, z0, .., z0^n) */
    double v[5], q[5];
    v[0] = 1.0;
    for (int i = 1; i < n1; ++i) v[i] = v[i - 1] * z0;
    hankel_solve(n1, L, D, v, q);

    /* SolvePowerEquation: the other n support points are the roots of
     * sum_j q_j x^j */
    double z[5];
    z[0] = z0;
    int nr = real_roots(n, q, z + 1);
    if (nodes)
        for (int i = 0; i <= n; ++i) nodes[i] = i <= nr ? z[i] : NAN;

    /* weights: overestimation at z0, indicator z_i < z0 elsewhere; Newton
     * divided differences over the distinct support points */
    double X[5], F[5];
    int nd = 0;
    for (int i = 0; i <= nr; ++i) {
        int dup = 0;
        for (int l = 0; l < nd; ++l) dup |= X[l] == z[i];
        if (dup) continue;
        X[nd] = z[i];
        F[nd] = (i == 0) ? overestimation : (z[i] < z0 ? 1.0 : 0.0);
        ++nd;
    }
    for (int j = 1; j < nd; ++j)
        for (int i = nd - 1; i >= j; --i) F[i] = (F[i] - F[i - 1]) / (X[i] - X[i - j]);

    /* solvePolynomial: p(x) = sum_j F[j] prod_{l<j} (x - X[l]) expanded */
    double p[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int deg = 0;
    p[0] = F[nd - 1];
    for (int j = nd - 2; j >= 0; --j) {
        p[deg + 1] = p[deg];
        for (int t = deg; t >= 1; --t) p[t] = p[t - 1] - X[j] * p[t];
        p[0] = F[j] - X[j] * p[0];
        ++deg;
    }

    /* absorbance = p . (1, b_tmp) */
    double A = 0.0;
    for (int t = 0; t <= deg; ++t) A += p[t] * b[t];
    return A;
}

static double transmittance(const double* m, double z0, const vol_t* g)
{
    double A;
    if (g->n_trig)
        A = orc_trig_bound(m, g->n_trig, z0 * (1.0 - g->trig_zone) * ORC_PI, g->moment_bias, g->overestimation,
                           NULL, NULL);
    else if (g->n_power > 2)
        A = orc_power_bound(m, g->n_power, z0, g->moment_bias, g->power_bias, g->overestimation, NULL, NULL);
    else
        A = orc_mboit_bound(m, z0, g->moment_bias, g->bias_vector, g->overestimation, NULL);
    double T = exp(-m[0] * A);
    if (T < 0.0) T = 0.0;
    if (T > 1.0) T = 1.0;
    return T;
}

/* ------------------------------------------------------------------------ */
/* rays: float32, correctly rounded, in this exact order                     */

static void make_ray(const orc_view* V, int64_t px, int64_t py, float o[3], float d[3])
{
    float fx = (float)px + 0.5f;
    float fy = (float)py + 0.5f;
    if (V->projection == 0) {
        float sx = (fx / (float)V->width - 0.5f) * V->scale_u;
        float sy = (fy / (float)V->height - 0.5f) * V->scale_v;
        for (int c = 0; c < 3; ++c) {
            o[c] = (V->eye[c] + sx * V->u[c]) + sy * V->v[c];
            d[c] = V->w[c];
        }
    } else {
        float sx = ((2.0f * fx) / (float)V->width - 1.0f) * V->scale_u;
        float sy = ((2.0f * fy) / (float)V->height - 1.0f) * V->scale_v;
        float dir[3];
        for (int c = 0; c < 3; ++c) dir[c] = (V->w[c] + sx * V->u[c]) + sy * V->v[c];
        float len = sqrtf((dir[0] * dir[0] + dir[1] * dir[1]) + dir[2] * dir[2]);
        for (int c = 0; c < 3; ++c) {
            o[c] = V->eye[c];
            d[c] = dir[c] / len;
        }
    }
}

/* Lattice index range [k_lo, k_hi] that surely contains every lattice point
 * whose float32 position is inside the domain (the position test decides). */
static int lattice_range(const vol_t* g, const float o[3], const float d[3], int64_t* k_lo, int64_t* k_hi)
{
    const double* hi = g->hi;
    double t0 = 0.0, t1 = INFINITY;
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0f) {
            if (!(o[c] >= 0.0f && o[c] < (float)hi[c])) return 0;
            continue;
        }
        double a = (0.0 - o[c]) / d[c], b = (hi[c] - o[c]) / d[c];
        if (a > b) { double s = a; a = b; b = s; }
        double pad = ldexp(fabs((double)o[c]) + hi[c] + 1.0, -20) / fabs((double)d[c]);
        a -= pad;
        b += pad;
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
    }
    if (!(t1 >= t0)) return 0;
    double lo = ceil(t0 / g->step - 0.5) - 2.0, up = floor(t1 / g->step - 0.5) + 2.0;
    if (lo < 0.0) lo = 0.0;
    if (up < lo) return 0;
    *k_lo = (int64_t)lo;
    *k_hi = (int64_t)up;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* one sample                                                                */

typedef struct {
    int64_t k;
    int32_t piece;
    double t, z, a, alpha, rgb[3];
} sample_t;

/* Grid: the piece owning the brick of the point's cell, and the trilinear
 * value of the cell's 8 vertices; -1 if the brick belongs to no piece. */
static int locate_grid(const orc_grid* g, const float p[3], double* val)
{
    int cell[3];
    for (int c = 0; c < 3; ++c) cell[c] = (int)floorf(p[c]);
    int B = 1 << g->brick_log2;
    int nbx = (g->nx - 1 + B - 1) / B, nby = (g->ny - 1 + B - 1) / B;
    int brick = ((cell[2] >> g->brick_log2) * nby + (cell[1] >> g->brick_log2)) * nbx + (cell[0] >> g->brick_log2);
    int piece = g->piece_of_brick[brick];
    if (piece < 0) return -1;
    double fx = (double)p[0] - cell[0], fy = (double)p[1] - cell[1], fz = (double)p[2] - cell[2];
    double v = 0.0;
    for (int dz = 0; dz <= 1; ++dz)
        for (int dy = 0; dy <= 1; ++dy)
            for (int dx = 0; dx <= 1; ++dx) {
                double wgt = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
                int64_t idx = ((int64_t)(cell[2] + dz) * g->ny + (cell[1] + dy)) * g->nx + (cell[0] + dx);
                v += wgt * (double)g->field[idx];
            }
    *val = v;
    return piece;
}

/* Octree: the leaf whose half-open box holds the point; local coordinates in
 * the leaf's cells; trilinear value of that cell's 8 vertices. */
static int locate_amr(const vol_t* vol, const float p[3], double* val, int* shift)
{
    const orc_amr* a = vol->a;
    int64_t fb[3];
    for (int c = 0; c < 3; ++c) fb[c] = (int64_t)floorf(p[c]) >> a->brick_log2;
    int32_t leaf = vol->fmap[(fb[2] * vol->fdim + fb[1]) * vol->fdim + fb[0]];
    if (leaf < 0) return -1;
    int piece = a->piece_of_leaf[leaf];
    if (piece < 0) return -1;
    const int32_t* L = a->leaves + 4 * (int64_t)leaf;
    double h = ldexp(1.0, a->max_level - L[3]);    /* finest cells per leaf cell */
    *shift = a->max_level - L[3];
    int n = 1 << a->brick_log2, nv = n + 1;
    int cell[3];
    double f[3];
    for (int c = 0; c < 3; ++c) {
        double q = ((double)p[c] - L[c]) / h;
        int ci = (int)floor(q);
        if (ci < 0) ci = 0;
        if (ci > n - 1) ci = n - 1;
        cell[c] = ci;
        f[c] = q - ci;
    }
    const float* vals = a->values + (int64_t)leaf * nv * nv * nv;
    double v = 0.0;
    for (int dz = 0; dz <= 1; ++dz)
        for (int dy = 0; dy <= 1; ++dy)
            for (int dx = 0; dx <= 1; ++dx) {
                double wgt = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                v += wgt * (double)vals[((cell[2] + dz) * nv + (cell[1] + dy)) * nv + (cell[0] + dx)];
            }
    *val = v;
    return piece;
}

/* ------------------------------------------------------------------------ */
/* tetrahedral mesh: exact point location                                    */

__extension__ typedef __int128 i128;

/* Snap one coordinate to the lattice 2^-s (nearest-even). */
static int64_t snap(double x, int s) { return (int64_t)nearbyint(ldexp(x, s)); }

/* det[P1 - P0, P2 - P0, P3 - P0]: six times the signed volume of P0..P3. */
static i128 orient4(const int64_t P[4][3])
{
    i128 a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = P[1][k] - P[0][k];
        b[k] = P[2][k] - P[0][k];
        c[k] = P[3][k] - P[0][k];
    }
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

static void tet_corners(const vol_t* v, int64_t t, int64_t P[4][3])
{
    const int32_t* T = v->m->tets + 4 * t;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) P[i][k] = v->vq[3 * (int64_t)T[i] + k];
}

/* D_i(q): the orientation with corner i replaced by q (q's barycentric
 * coordinate times six volumes).  Returns 1 if q + (e, e^2, e^3) is strictly
 * on the inner side of every face, and D_0..D_3 at q itself in D. */
static int tet_contains(const vol_t* v, int64_t t, const int64_t q[3], i128 D[4])
{
    int64_t P[4][3];
    tet_corners(v, t, P);
    int inside = 1;
    for (int i = 0; i < 4; ++i) {
        int64_t R[4][3];
        memcpy(R, P, sizeof R);
        for (int k = 0; k < 3; ++k) R[i][k] = q[k];
        D[i] = orient4(R);
        /* D_i is affine in q: its partial derivatives are exact differences */
        i128 sgn = D[i];
        for (int k = 0; k < 3 && sgn == 0; ++k) {
            R[i][k] = q[k] + 1;
            sgn = orient4(R) - D[i];
            R[i][k] = q[k];
        }
        if (sgn <= 0) inside = 0;
    }
    return inside;
}

static double tet_value(const vol_t* v, int64_t t, const i128 D[4])
{
    const int32_t* T = v->m->tets + 4 * t;
    double tot = (double)(D[0] + D[1] + D[2] + D[3]), val = 0.0;
    for (int i = 0; i < 4; ++i) val += (double)D[i] / tot * (double)v->m->verts[4 * (int64_t)T[i] + 3];
    return val;
}

/* The owning tet of the snapped point q (-1 if none); *n_pass = how many
 * tets passed (more than one only for an overlapping mesh). */
static int64_t tet_find(const vol_t* v, const int64_t q[3], int brute, int* n_pass, double* val)
{
    int64_t owner = -1, lo = 0, hi = v->m->n_tets;
    const int32_t* list = NULL;
    if (!brute) {
        int64_t b[3];
        for (int k = 0; k < 3; ++k) {
            b[k] = q[k] >> v->m->quantum_log2;
            if (b[k] < 0) b[k] = 0;
            if (b[k] > v->bdim[k] - 1) b[k] = v->bdim[k] - 1;
        }
        int64_t bin = (b[2] * v->bdim[1] + b[1]) * v->bdim[0] + b[0];
        lo = v->bin_start[bin];
        hi = v->bin_start[bin + 1];
        list = v->bin_tets;
    }
    *n_pass = 0;
    for (int64_t j = lo; j < hi; ++j) {
        int64_t t = list ? list[j] : j;
        i128 D[4];
        if (tet_contains(v, t, q, D)) {
            if (*n_pass == 0) {
                owner = t;
                if (val) *val = tet_value(v, t, D);
            }
            ++*n_pass;
        }
    }
    return owner;
}

static int locate_tet_piece(const vol_t* vol, const float p[3], double* val)
{
    int64_t q[3];
    for (int k = 0; k < 3; ++k) q[k] = snap((double)p[k], vol->m->quantum_log2);
    int n_pass;
    int64_t t = tet_find(vol, q, 0, &n_pass, val);
    if (n_pass > 1) ((vol_t*)vol)->overlap = 1;
    if (t < 0) return -1;
    return vol->m->piece_of_tet[t];
}

static void tet_free(vol_t* v)
{
    free(v->vq);
    free(v->bin_start);
    free(v->bin_tets);
}

/* Snaps the vertices, checks boxes and orientation, bins the tets by their
 * snapped bounding boxes (bins of one unit). */
static int tet_vol(const orc_tet* m, vol_t* v)
{
    memset(v, 0, sizeof *v);
    if (!m || !m->verts || !m->tets || !m->piece_of_tet || !m->tf || m->n_tets <= 0 || m->n_verts <= 0 ||
        m->n_pieces <= 0 || m->quantum_log2 < 0 || m->quantum_log2 > 24)
        return -1;
    if (set_moments(v, m->moment_set, m->storage, m->trig_zone) != 0)
        return -1;
    const int s = m->quantum_log2;
    v->kind = 2;
    v->m = m;
    v->vq = (int64_t*)malloc((size_t)m->n_verts * 3 * sizeof(int64_t));
    for (int k = 0; k < 3; ++k) v->bdim[k] = (snap(m->box[k], s) >> s) + 1;
    int64_t nbins = v->bdim[0] * v->bdim[1] * v->bdim[2];
    v->bin_start = (int32_t*)calloc((size_t)nbins + 1, sizeof(int32_t));
    if (!v->vq || !v->bin_start) { tet_free(v); return -1; }
    for (int64_t i = 0; i < m->n_verts; ++i)
        for (int k = 0; k < 3; ++k) {
            double x = m->verts[4 * i + k];
            if (!(x >= 0.0 && x <= m->box[k])) { tet_free(v); return -1; }
            v->vq[3 * i + k] = snap(x, s);
        }
    /* two sweeps over the tets: count bin entries, then fill them */
    for (int sweep = 0; sweep < 2; ++sweep) {
        if (sweep == 1) {
            for (int64_t b = 0; b < nbins; ++b) v->bin_start[b + 1] += v->bin_start[b];
            v->bin_tets = (int32_t*)malloc((size_t)(v->bin_start[nbins] > 0 ? v->bin_start[nbins] : 1) * sizeof(int32_t));
            if (!v->bin_tets) { tet_free(v); return -1; }
        }
        int64_t* fill = NULL;
        if (sweep == 1) {
            fill = (int64_t*)malloc((size_t)nbins * sizeof(int64_t));
            if (!fill) { tet_free(v); return -1; }
            for (int64_t b = 0; b < nbins; ++b) fill[b] = v->bin_start[b];
        }
        for (int64_t t = 0; t < m->n_tets; ++t) {
            int64_t P[4][3], lo[3], hi[3];
            for (int i = 0; i < 4; ++i)
                if (m->tets[4 * t + i] < 0 || m->tets[4 * t + i] >= m->n_verts) { free(fill); tet_free(v); return -1; }
            tet_corners(v, t, P);
            if (sweep == 0 && orient4(P) <= 0) { tet_free(v); return -1; }
            for (int k = 0; k < 3; ++k) {
                lo[k] = hi[k] = P[0][k];
                for (int i = 1; i < 4; ++i) {
                    if (P[i][k] < lo[k]) lo[k] = P[i][k];
                    if (P[i][k] > hi[k]) hi[k] = P[i][k];
                }
                lo[k] >>= s;
                hi[k] >>= s;
                if (hi[k] > v->bdim[k] - 1) hi[k] = v->bdim[k] - 1;
            }
            for (int64_t z = lo[2]; z <= hi[2]; ++z)
                for (int64_t y = lo[1]; y <= hi[1]; ++y)
                    for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                        int64_t b = (z * v->bdim[1] + y) * v->bdim[0] + x;
                        if (sweep == 0) ++v->bin_start[b + 1];
                        else v->bin_tets[fill[b]++] = (int32_t)t;
                    }
        }
        free(fill);
    }
    v->hi[0] = m->box[0];
    v->hi[1] = m->box[1];
    v->hi[2] = m->box[2];
    v->n_pieces = m->n_pieces;
    v->piece_selected = m->piece_selected;
    v->tf = m->tf;
    v->vmin = m->vmin;
    v->vmax = m->vmax;
    v->step = m->step;
    v->moment_bias = m->moment_bias;
    v->overestimation = m->overestimation;
    v->absorbance_max = m->absorbance_max;
    v->bias_vector = m->bias_vector;
    return 0;
}

/* Classifies lattice point k; returns 1 and fills s if it is inside the
 * domain and owned by a selected piece. */
static int take_sample(const vol_t* g, const orc_view* V, const float o[3], const float d[3],
                       int64_t k, const double* sig_tab, sample_t* s)
{
    float t = ((float)k + 0.5f) * (float)g->step;
    float p[3];
    for (int c = 0; c < 3; ++c) p[c] = fmaf(t, d[c], o[c]);
    for (int c = 0; c < 3; ++c)
        if (!(p[c] >= 0.0f && p[c] < (float)g->hi[c])) return 0;
    double val;
    int shift = 0;
    int piece = (g->kind == 0) ? locate_grid(g->g, p, &val) : (g->kind == 1) ? locate_amr(g, p, &val, &shift)
                                                                             : locate_tet_piece(g, p, &val);
    if (piece < 0) return 0;
    if (g->piece_selected && !g->piece_selected[piece]) return 0;
    /* adaptive dyadic step (octrees): a leaf of level L samples the nested
     * lattice of spacing 2^(max_level - L) steps, each sample standing for
     * that longer interval */
    double step_len = g->step;
    if (g->kind == 1 && g->a->adaptive_step) {
        int64_t stride = (int64_t)1 << shift;
        if (((k % stride) + stride) % stride != 0) return 0;
        step_len = g->step * (double)stride;
    }

    /* transfer function: normalise, 256-entry linear lookup of (r, g, b, sigma) */
    double x = (val - g->vmin) / (g->vmax - g->vmin);
    if (x < 0.0) x = 0.0;
    if (x > 1.0) x = 1.0;
    x *= 255.0;
    int i = (int)floor(x);
    if (i > 254) i = 254;
    double f = x - i;
    for (int c = 0; c < 3; ++c) s->rgb[c] = (1.0 - f) * g->tf[4 * i + c] + f * g->tf[4 * (i + 1) + c];
    double sigma = (1.0 - f) * sig_tab[i] + f * sig_tab[i + 1];

    /* Alg. 2: absorbance = -log(transmittance of the sample), clamped */
    double a = sigma * step_len;
    if (a > g->absorbance_max) a = g->absorbance_max;
    s->k = k;
    s->piece = piece;
    s->t = (double)t;
    s->z = orc_log_warp((double)t, V->znear, V->zfar);
    s->a = a;
    s->alpha = 1.0 - exp(-a);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* one pixel                                                                 */

static int render_impl(const vol_t* g, const orc_view* V,
                       const int64_t* pixels, int64_t n_pixels,
                       double* moments, double* piece_moments, double* piece_color,
                       double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                       double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments);

static int grid_vol(const orc_grid* g, vol_t* v)
{
    if (!g || !g->field || !g->piece_of_brick || !g->tf || g->n_pieces <= 0) return -1;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return -1;
    memset(v, 0, sizeof *v);
    v->kind = 0;
    v->g = g;
    v->hi[0] = g->nx - 1.0;
    v->hi[1] = g->ny - 1.0;
    v->hi[2] = g->nz - 1.0;
    v->n_pieces = g->n_pieces;
    v->piece_selected = g->piece_selected;
    v->tf = g->tf;
    v->vmin = g->vmin;
    v->vmax = g->vmax;
    v->step = g->step;
    v->moment_bias = g->moment_bias;
    v->overestimation = g->overestimation;
    v->absorbance_max = g->absorbance_max;
    v->bias_vector = g->bias_vector;
    if (set_moments(v, g->moment_set, g->storage, g->trig_zone) != 0) return -1;
    return 0;
}

static int render_grid_impl(const orc_grid* g, const orc_view* V,
                            const int64_t* pixels, int64_t n_pixels,
                            double* moments, double* piece_moments, double* piece_color,
                            double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                            double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments)
{
    vol_t v;
    if (grid_vol(g, &v) != 0) return -1;
    return render_impl(&v, V, pixels, n_pixels, moments, piece_moments, piece_color, mboit_rgba, raw_rgba,
                       exact_rgba, sortlast_rgba, nsamples, nsegments);
}

int orc_render_amr(const orc_amr* a, const orc_view* V,
                   const int64_t* pixels, int64_t n_pixels,
                   double* moments, double* piece_moments, double* piece_color,
                   double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                   double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments)
{
    if (!a || !a->values || !a->leaves || !a->piece_of_leaf || !a->tf || a->n_pieces <= 0 || a->n_leaves <= 0)
        return -1;
    if (a->brick_log2 < 0 || a->brick_log2 > 7 || a->max_level < 0 || a->finest_cells < 1) return -1;
    int64_t fdim = ((int64_t)a->finest_cells + (1 << a->brick_log2) - 1) >> a->brick_log2;
    int32_t* fmap = (int32_t*)malloc((size_t)(fdim * fdim * fdim) * sizeof(int32_t));
    if (!fmap) return -1;
    for (int64_t i = 0; i < fdim * fdim * fdim; ++i) fmap[i] = -1;
    for (int32_t l = 0; l < a->n_leaves; ++l) {
        const int32_t* L = a->leaves + 4 * (int64_t)l;
        if (L[3] < 0 || L[3] > a->max_level) { free(fmap); return -1; }
        int64_t nb = (int64_t)1 << (a->max_level - L[3]);      /* finest bricks per side */
        int64_t b0[3];
        for (int c = 0; c < 3; ++c) {
            if (L[c] < 0 || (L[c] & ((1 << a->brick_log2) - 1))) { free(fmap); return -1; }
            b0[c] = L[c] >> a->brick_log2;
            if (b0[c] + nb > fdim) { free(fmap); return -1; }
        }
        for (int64_t z = b0[2]; z < b0[2] + nb; ++z)
            for (int64_t y = b0[1]; y < b0[1] + nb; ++y)
                for (int64_t x = b0[0]; x < b0[0] + nb; ++x) {
                    int32_t* m = fmap + (z * fdim + y) * fdim + x;
                    if (*m >= 0) { free(fmap); return -1; }   /* overlapping leaves */
                    *m = l;
                }
    }
    vol_t v;
    memset(&v, 0, sizeof v);
    v.kind = 1;
    v.a = a;
    v.fmap = fmap;
    v.fdim = fdim;
    v.hi[0] = v.hi[1] = v.hi[2] = (double)a->finest_cells;
    v.n_pieces = a->n_pieces;
    v.piece_selected = a->piece_selected;
    v.tf = a->tf;
    v.vmin = a->vmin;
    v.vmax = a->vmax;
    v.step = a->step;
    v.moment_bias = a->moment_bias;
    v.overestimation = a->overestimation;
    v.absorbance_max = a->absorbance_max;
    v.bias_vector = a->bias_vector;
    if (set_moments(&v, a->moment_set, a->storage, a->trig_zone) != 0) {
        free(fmap);
        return -1;
    }
    int rc = render_impl(&v, V, pixels, n_pixels, moments, piece_moments, piece_color, mboit_rgba, raw_rgba,
                         exact_rgba, sortlast_rgba, nsamples, nsegments);
    free(fmap);
    return rc;
}

int orc_render_grid(const orc_grid* g, const orc_view* V,
                    const int64_t* pixels, int64_t n_pixels,
                    double* moments, double* piece_moments, double* piece_color,
                    double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                    double* sortlast_rgba, int64_t* nsamples)
{
    return render_grid_impl(g, V, pixels, n_pixels, moments, piece_moments, piece_color, mboit_rgba, raw_rgba,
                            exact_rgba, sortlast_rgba, nsamples, NULL);
}

/* Stage two (Alg. 1 loop 2, Sec. 4.2) of the listed pixels from given global
 * moments instead of the ones stage one finds: given_moments holds per pixel
 * the moments in the order of `moments` (b0, then b1.. for power moments, or
 * b0, Re t1, Im t1, .. for trigonometric moments, t_j un-normalised).  The
 * samples, their colours and the blend are the oracle's own. */
int orc_render_grid_given(const orc_grid* g, const orc_view* V, const int64_t* pixels, int64_t n_pixels,
                          const double* given_moments, double* mboit_rgba, double* raw_rgba)
{
    vol_t v;
    if (!given_moments || grid_vol(g, &v) != 0) return -1;
    v.given_moments = given_moments;
    return render_impl(&v, V, pixels, n_pixels, NULL, NULL, NULL, mboit_rgba, raw_rgba, NULL, NULL, NULL, NULL);
}

int orc_render_grid_segments(const orc_grid* g, const orc_view* V,
                             const int64_t* pixels, int64_t n_pixels,
                             double* sortlast_rgba, int64_t* nsegments)
{
    double* tmp = NULL;
    if (!sortlast_rgba) {
        tmp = (double*)malloc((size_t)(n_pixels > 0 ? n_pixels : 1) * 4 * sizeof(double));
        if (!tmp) return -1;
    }
    int rc = render_grid_impl(g, V, pixels, n_pixels, NULL, NULL, NULL, NULL, NULL, NULL,
                              sortlast_rgba ? sortlast_rgba : tmp, NULL, nsegments);
    free(tmp);
    return rc;
}

static int render_impl(const vol_t* g, const orc_view* V,
                       const int64_t* pixels, int64_t n_pixels,
                       double* moments, double* piece_moments, double* piece_color,
                       double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                       double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments)
{
    if (!V || !(g->step > 0.0) || !(g->vmax > g->vmin)) return -1;
    const int K = g->n_pieces;

    double sig_tab[256];
    for (int j = 0; j < 256; ++j) sig_tab[j] = -log(1.0 - (double)g->tf[4 * j + 3]);

    size_t cap = 1024;
    sample_t* S = (sample_t*)malloc(cap * sizeof(sample_t));
    const int NM = n_moments(g);
    double* mP = (double*)malloc((size_t)K * NM * sizeof(double));
    double* cP = (double*)malloc((size_t)K * 4 * sizeof(double));
    if (!S || !mP || !cP) { free(S); free(mP); free(cP); return -1; }

    for (int64_t n = 0; n < n_pixels; ++n) {
        int64_t pix = pixels[n];
        if (pix < 0 || pix >= (int64_t)V->width * V->height) { free(S); free(mP); free(cP); return -1; }
        float o[3], d[3];
        make_ray(V, pix % V->width, pix / V->width, o, d);

        /* gather this ray's owned samples in lattice order */
        size_t ns = 0;
        int64_t k_lo, k_hi;
        if (lattice_range(g, o, d, &k_lo, &k_hi)) {
            for (int64_t k = k_lo; k <= k_hi; ++k) {
                if (ns == cap) {
                    cap *= 2;
                    sample_t* S2 = (sample_t*)realloc(S, cap * sizeof(sample_t));
                    if (!S2) { free(S); free(mP); free(cP); return -1; }
                    S = S2;
                }
                if (take_sample(g, V, o, d, k, sig_tab, &S[ns])) ++ns;
            }
        }

        /* stage one (Sec. 4.1): local moment image of each piece ... */
        memset(mP, 0, (size_t)K * NM * sizeof(double));
        for (size_t i = 0; i < ns; ++i) {
            double* mp = mP + (size_t)NM * S[i].piece;
            if (g->n_trig) {
                /* b0 += a, t_j += a e^{i j phi} */
                double phi = S[i].z * (1.0 - g->trig_zone) * ORC_PI;
                mp[0] += S[i].a;
                for (int j = 1; j <= g->n_trig; ++j) {
                    mp[2 * j - 1] += S[i].a * cos(j * phi);
                    mp[2 * j] += S[i].a * sin(j * phi);
                }
            } else {
                double zp = 1.0;
                for (int j = 0; j <= 2 * g->n_power; ++j) {
                    mp[j] += zp * S[i].a;
                    zp *= S[i].z;
                }
            }
        }
        /* ... summed over pieces (the Allreduce add) */
        double m[ORC_MAX_NM] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int P = 0; P < K; ++P)
            for (int j = 0; j < NM; ++j) m[j] += mP[(size_t)NM * P + j];
        double ms[ORC_MAX_NM];
        memcpy(ms, m, sizeof m);
        store_moments(g, ms);
        /* stage two from given global moments (as stored by another renderer) */
        if (g->given_moments) memcpy(ms, g->given_moments + (size_t)NM * n, (size_t)NM * sizeof(double));

        /* stage two (Sec. 4.2): each piece blends its own samples with the
         * transmittance reconstructed from the (stored) global moments */
        memset(cP, 0, (size_t)K * 4 * sizeof(double));
        for (size_t i = 0; i < ns; ++i) {
            double T = transmittance(ms, S[i].z, g);
            double* cp = cP + 4 * S[i].piece;
            for (int c = 0; c < 3; ++c) cp[c] += T * S[i].alpha * S[i].rgb[c];
            cp[3] += T * S[i].alpha;
        }
        /* final image: sum of the partial images (the Reduce add) */
        double C[4] = {0, 0, 0, 0};
        for (int P = 0; P < K; ++P)
            for (int c = 0; c < 4; ++c) C[c] += cP[4 * P + c];

        if (moments) memcpy(moments + (size_t)NM * n, m, (size_t)NM * sizeof(double));
        if (piece_moments) memcpy(piece_moments + (size_t)n * K * NM, mP, (size_t)K * NM * sizeof(double));
        if (piece_color) memcpy(piece_color + (size_t)n * K * 4, cP, (size_t)K * 4 * sizeof(double));
        if (raw_rgba) memcpy(raw_rgba + 4 * n, C, sizeof C);
        if (mboit_rgba) {
            /* renormalisation: total opacity from the zeroth moment */
            double A = 1.0 - exp(-m[0]);
            double* out = mboit_rgba + 4 * n;
            for (int c = 0; c < 3; ++c) out[c] = (C[3] > 0.0) ? C[c] * A / C[3] : 0.0;
            out[3] = A;
        }
        if (exact_rgba) {
            /* front-to-back over all samples in depth order */
            double acc[3] = {0, 0, 0}, tau = 0.0;
            for (size_t i = 0; i < ns; ++i) {
                double T = exp(-tau);
                for (int c = 0; c < 3; ++c) acc[c] += T * S[i].alpha * S[i].rgb[c];
                tau += S[i].a;
            }
            double* out = exact_rgba + 4 * n;
            for (int c = 0; c < 3; ++c) out[c] = acc[c];
            out[3] = 1.0 - exp(-tau);
        }
        if (sortlast_rgba) {
            /* each maximal run of consecutive lattice points of one piece is a
             * segment, composited in front-to-back order inside itself; the
             * segments are then sorted by their first lattice index (runs
             * are disjoint) and composited with "over" */
            size_t nseg = 0;
            double* seg = (double*)malloc((ns + 1) * 5 * sizeof(double)); /* k_first, r, g, b, alpha */
            if (!seg) { free(S); free(mP); free(cP); return -1; }
            for (int P = 0; P < K; ++P) {
                /* piece P's own samples, as its rank would produce them */
                int64_t prev_k = -2;
                double* sg = NULL;
                double tr = 1.0;
                for (size_t i = 0; i < ns; ++i) {
                    if (S[i].piece != P) continue;
                    if (S[i].k != prev_k + 1) {
                        if (sg) sg[4] = 1.0 - tr;
                        sg = seg + 5 * nseg++;
                        sg[0] = (double)S[i].k;
                        sg[1] = sg[2] = sg[3] = 0.0;
                        tr = 1.0;
                    }
                    for (int c = 0; c < 3; ++c) sg[1 + c] += tr * S[i].alpha * S[i].rgb[c];
                    tr *= 1.0 - S[i].alpha;
                    prev_k = S[i].k;
                }
                if (sg) sg[4] = 1.0 - tr;
            }
            /* insertion sort of all pieces' segments on k_first */
            for (size_t a = 1; a < nseg; ++a)
                for (size_t b = a; b > 0 && seg[5 * (b - 1)] > seg[5 * b]; --b)
                    for (int c = 0; c < 5; ++c) {
                        double s = seg[5 * b + c];
                        seg[5 * b + c] = seg[5 * (b - 1) + c];
                        seg[5 * (b - 1) + c] = s;
                    }
            double acc[3] = {0, 0, 0}, tr = 1.0;
            for (size_t a = 0; a < nseg; ++a) {
                for (int c = 0; c < 3; ++c) acc[c] += tr * seg[5 * a + 1 + c];
                tr *= 1.0 - seg[5 * a + 4];
            }
            double* out = sortlast_rgba + 4 * n;
            for (int c = 0; c < 3; ++c) out[c] = acc[c];
            out[3] = 1.0 - tr;
            if (nsegments) nsegments[n] = (int64_t)nseg;
            free(seg);
        }
        if (nsamples) nsamples[n] = (int64_t)ns;
    }
    free(S);
    free(mP);
    free(cP);
    return 0;
}

int orc_render_tet(const orc_tet* m, const orc_view* V,
                   const int64_t* pixels, int64_t n_pixels,
                   double* moments, double* piece_moments, double* piece_color,
                   double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                   double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments)
{
    vol_t v;
    if (tet_vol(m, &v) != 0) return -1;
    int rc = render_impl(&v, V, pixels, n_pixels, moments, piece_moments, piece_color, mboit_rgba, raw_rgba,
                         exact_rgba, sortlast_rgba, nsamples, nsegments);
    if (v.overlap) rc = -1;
    tet_free(&v);
    return rc;
}

int orc_tet_locate(const orc_tet* m, const float* points, int64_t n, int32_t* tet_out, int32_t* n_pass_out,
                   double* value_out, int32_t brute_force)
{
    vol_t v;
    if (!points || n < 0 || tet_vol(m, &v) != 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t q[3];
        for (int k = 0; k < 3; ++k) q[k] = snap((double)points[3 * i + k], m->quantum_log2);
        int n_pass;
        double val = NAN;
        int64_t t = tet_find(&v, q, brute_force, &n_pass, &val);
        if (tet_out) tet_out[i] = (int32_t)t;
        if (n_pass_out) n_pass_out[i] = n_pass;
        if (value_out) value_out[i] = t >= 0 ? val : NAN;
    }
    tet_free(&v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* mixed cells -> tetrahedra                                                 */

static int emit_tet(const float* verts, int64_t n_verts, int s, int32_t a, int32_t b, int32_t c, int32_t d,
                    int64_t cell, int32_t* out, int64_t* cot, int64_t max_tets, int64_t* n)
{
    int32_t v[4] = {a, b, c, d};
    int64_t P[4][3];
    for (int i = 0; i < 4; ++i) {
        if (v[i] < 0 || v[i] >= n_verts) return -1;
        for (int k = 0; k < 3; ++k) P[i][k] = snap((double)verts[4 * (int64_t)v[i] + k], s);
    }
    i128 o = orient4(P);
    if (o == 0) return -1;
    if (o < 0) {
        int32_t t = v[2];
        v[2] = v[3];
        v[3] = t;
    }
    if (*n >= max_tets) return -1;
    memcpy(out + 4 * *n, v, sizeof v);
    cot[*n] = cell;
    ++*n;
    return 0;
}

int orc_split_cells(const float* verts, int64_t n_verts, const int32_t* cells, const int32_t* types, int64_t n_cells,
                    int32_t quantum_log2, int32_t* tets_out, int64_t* cell_of_tet, int64_t max_tets, int64_t* n_tets)
{
    if (!verts || !cells || !types || !tets_out || !cell_of_tet || !n_tets || quantum_log2 < 0 || quantum_log2 > 24)
        return -1;
    int64_t n = 0;
    const int s = quantum_log2;
    for (int64_t i = 0; i < n_cells; ++i) {
        const int32_t* c = cells + 6 * i;
        int rc = 0;
        if (types[i] == 4) {
            rc = emit_tet(verts, n_verts, s, c[0], c[1], c[2], c[3], i, tets_out, cell_of_tet, max_tets, &n);
        } else if (types[i] == 5) {
            /* the base quad's diagonal through its smallest id */
            int32_t m = c[0];
            for (int k = 1; k < 4; ++k) m = c[k] < m ? c[k] : m;
            int j = (m == c[0] || m == c[2]) ? 0 : 1;
            rc = emit_tet(verts, n_verts, s, c[j], c[j + 1], c[(j + 2) % 4], c[4], i, tets_out, cell_of_tet, max_tets, &n);
            if (!rc)
                rc = emit_tet(verts, n_verts, s, c[j], c[(j + 2) % 4], c[(j + 3) % 4], c[4], i, tets_out, cell_of_tet,
                              max_tets, &n);
        } else if (types[i] == 6) {
            /* relabel (triangle rotations, bottom/top flip) so that local
             * vertex 0 has the smallest id; its two quad faces are cut
             * through it, the opposite quad (1, 2, 5, 4) by its own smallest */
            int best = -1, L[6] = {0, 0, 0, 0, 0, 0};
            for (int r = 0; r < 3; ++r)
                for (int f = 0; f < 2; ++f) {
                    int p[6];
                    for (int k = 0; k < 3; ++k) {
                        p[k] = (k + r) % 3 + 3 * f;
                        p[k + 3] = (k + r) % 3 + 3 * (1 - f);
                    }
                    if (best < 0 || c[p[0]] < c[L[0]]) {
                        best = 1;
                        memcpy(L, p, sizeof p);
                    }
                }
            int32_t v[6];
            for (int k = 0; k < 6; ++k) v[k] = c[L[k]];
            int32_t m15 = v[1] < v[5] ? v[1] : v[5], m24 = v[2] < v[4] ? v[2] : v[4];
            if (m15 < m24) {
                rc = emit_tet(verts, n_verts, s, v[0], v[1], v[2], v[5], i, tets_out, cell_of_tet, max_tets, &n);
                if (!rc) rc = emit_tet(verts, n_verts, s, v[0], v[1], v[5], v[4], i, tets_out, cell_of_tet, max_tets, &n);
            } else {
                rc = emit_tet(verts, n_verts, s, v[0], v[1], v[2], v[4], i, tets_out, cell_of_tet, max_tets, &n);
                if (!rc) rc = emit_tet(verts, n_verts, s, v[0], v[4], v[2], v[5], i, tets_out, cell_of_tet, max_tets, &n);
            }
            if (!rc) rc = emit_tet(verts, n_verts, s, v[0], v[4], v[5], v[3], i, tets_out, cell_of_tet, max_tets, &n);
        } else {
            return -1;
        }
        if (rc) return -1;
    }
    *n_tets = n;
    return 0;
}
