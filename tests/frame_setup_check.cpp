// Host check of the pixel frame set-up: make_frame_ff (float-float FP32,
// FP64 only for near-singular pixels) against make_frame (FP64) on random
// absorber sets, compiled with the host compiler from the library's device
// header.  Prints: pixels set up in FP32, in FP64, kind mismatches, and the
// largest differences of the four frame parameters in float32 ulps.
#include <cmath>
#include <cstdio>
#include <random>

#include "mboit_device.cuh"

static double ulps(float a, float b) {
    return std::fabs((double)a - (double)b) / std::fmax(std::fabs((double)b) * 5.9604644775390625e-08, 1e-45);
}

int main() {
    std::mt19937_64 rng(11);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    const float bv[4] = {0.0f, 0.375f, 0.0f, 0.375f};
    double worst[4] = {0, 0, 0, 0};
    long n32 = 0, n64 = 0, kind = 0;
    for (int it = 0; it < 400000; ++it) {
        const int n = 1 + (int)(U(rng) * (it % 3 == 0 ? 3 : 60));
        const double c = U(rng) * 2 - 1, w = std::pow(10.0, -3.0 * U(rng));
        double m[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            const float z = (float)std::fmin(1.0, std::fmax(-1.0, c + w * (U(rng) * 2 - 1)));
            const double a = std::pow(10.0, -4.0 * U(rng)) * (U(rng) < 0.5 ? 1.0 : 3.0);
            double zp = 1;
            for (int j = 0; j < 5; ++j) {
                m[j] += a * zp;
                zp *= z;
            }
        }
        float mf[5];
        for (int j = 0; j < 5; ++j) mf[j] = (float)m[j];
        const float beta = (it % 5 == 0) ? 0.0f : 5e-5f;
        bool f64 = false;
        const mb::Frame A = mb::make_frame_ff(mf, beta, bv, &f64);
        const mb::Frame B = mb::make_frame(mf, beta, bv);
        if (f64) {
            ++n64;
            continue;
        }
        ++n32;
        if (A.kind != B.kind) {
            ++kind;
            continue;
        }
        const float a[4] = {A.p0, A.p1, A.p2, A.p3}, b[4] = {B.p0, B.p1, B.p2, B.p3};
        for (int k = 0; k < 4; ++k) {
            // the skewness may be near 0: compare it to the largest parameter
            const double u = k == 2 ? std::fabs((double)a[k] - (double)b[k]) / 5.96e-8 / std::fmax(1.0, std::fabs(b[k]))
                                    : ulps(a[k], b[k]);
            worst[k] = std::fmax(worst[k], u);
        }
    }
    std::printf("%ld %ld %ld %.2f %.2f %.2f %.2f\n", n32, n64, kind, worst[0], worst[1], worst[2], worst[3]);
    return 0;
}
