// Host check of the Fourier-slice projector's spreading-kernel numbers
// (sw_slice_plan.h) against independent FP64 references, for the kernel
// shapes beta = 0.97 pi (1 - 1/(2 sigma)) W of the oversampling factors
// sigma = N / L the library uses (1.5 to 3):
//   1. the tap-weight polynomials (FP32 coefficients, evaluated in FP32 by
//      the kernels' own slice_tap_weights) against psi(u) = exp(beta (sqrt(1
//      - (2u/W)^2) - 1)) at u = x + W/2 - a (W/2 = 4) over offsets x in
//      [-1/2, 1/2], and every row of the coefficient table (the mirrored taps
//      included) by Horner against that evaluation;
//   2. the kernel's Fourier transform Psi(k) against a midpoint rule in u;
//   3. a one-dimensional type-2 NUFFT made of exactly these parts (divide by
//      Psi, N-point DFT, W taps of the polynomial weights) against the direct
//      sum sum_c x_c e^{-2 pi i c y / N} at targets |y| <= N/2: its relative
//      l2 error is the accuracy the slice projector's design rests on.
// Prints "ok" and the measured errors, or the first failure (exit status 1).
// Host code only: no device is used.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "sw_slice_plan.h"

using namespace swk;
using cd = std::complex<double>;

static double psi(double u, double beta)
{
    const double z = 2.0 * u / kSliceW, a = 1.0 - z * z;
    return a >= 0.0 ? std::exp(beta * (std::sqrt(a) - 1.0)) : 0.0;
}

static double beta_of(double sigma) { return 0.97 * M_PI * (1.0 - 0.5 / sigma) * kSliceW; }

// Tap a's weight as the kernels evaluate it (slice_tap_weights: FP32, the
// mirrored taps from the even and odd parts in x^2)
static float weight_fp32(const SliceCoef &cf, int a, float x)
{
    float w[kSliceW];
    slice_tap_weights(cf, x, w);
    return w[a];
}

// FP32 Horner in x of tap a's row of the coefficient table
static float horner_fp32(const SliceCoef &cf, int a, float x)
{
    float p = cf.c[a][kSliceDeg];
    for (int d = kSliceDeg - 1; d >= 0; --d) p = std::fmaf(p, x, cf.c[a][d]);
    return p;
}

int main()
{
    const int W = kSliceW;
    // 1. tap weights, and the table rows (mirrored taps included) against
    //    the evaluation the kernels use
    double worst_w = 0.0, worst_rows = 0.0;
    for (double sigma : {1.5, 1.6, 2.0, 3.0}) {
        const double beta = beta_of(sigma);
        SliceCoef cf;
        slice_fit_weights(beta, cf);
        for (int a = 0; a < W; ++a)
            for (int i = 0; i <= 4000; ++i) {
                const float x = (float)(-0.5 + i / 4000.0);
                const double err = std::fabs((double)weight_fp32(cf, a, x) - psi((double)x + W / 2 - a, beta));
                worst_w = std::fmax(worst_w, err);
                worst_rows = std::fmax(worst_rows, std::fabs((double)horner_fp32(cf, a, x) -
                                                             (double)weight_fp32(cf, a, x)));
            }
    }
    if (!(worst_rows < 2e-7)) {
        std::printf("FAIL coefficient rows: max |Horner(row a) - tap a| = %.3e\n", worst_rows);
        return 1;
    }
    // psi peaks at 1; FP32 evaluation of a degree-8 polynomial with
    // coefficients of a few units leaves a few 1e-7
    if (!(worst_w < 5e-7)) {
        std::printf("FAIL tap weights: max |poly - psi| = %.3e\n", worst_w);
        return 1;
    }
    // 2. Fourier transform of the kernel
    double worst_ft = 0.0;
    for (double sigma : {1.5, 2.0, 3.0}) {
        const int N = 192;
        const double beta = beta_of(sigma);
        const int m = 200000;
        const double h = (double)W / m;
        double psi0 = 0.0;
        for (int k = 0; k <= (int)(N / sigma) / 2; ++k) {
            double ref = 0.0;
            for (int i = 0; i < m; ++i) {
                const double u = -0.5 * W + (i + 0.5) * h;
                ref += psi(u, beta) * std::cos(2.0 * M_PI * k * u / N);
            }
            ref *= h;
            if (k == 0) psi0 = ref;
            worst_ft = std::fmax(worst_ft, std::fabs(slice_kernel_ft(k, N, W, beta) - ref) / psi0);
        }
    }
    if (!(worst_ft < 1e-9)) {
        std::printf("FAIL kernel transform: max |Psi - quadrature| / Psi(0) = %.3e\n", worst_ft);
        return 1;
    }
    // 3. one-dimensional type-2 NUFFT from these parts
    std::mt19937_64 rng(20250317);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    double worst_nufft = 0.0;
    struct Case {
        int L, N;
    };
    for (Case cs : {Case{128, 192}, Case{64, 96}, Case{256, 384}, Case{100, 160}, Case{128, 256}}) {
        const int L = cs.L, N = cs.N;
        const double beta = beta_of((double)N / L);
        SliceCoef cf;
        slice_fit_weights(beta, cf);
        // samples x_c >= 0 (projections of non-negative images), c = -L/2 .. L/2 - 1
        std::vector<double> xs(L);
        for (double &v : xs) v = 0.5 * (U(rng) + 1.0);
        // grid G_m = sum_c x_c / Psi(c) e^{-2 pi i c m / N}
        std::vector<cd> G(N);
        for (int mm = 0; mm < N; ++mm) {
            cd acc = 0.0;
            for (int i = 0; i < L; ++i) {
                const int c = i - L / 2;
                acc += xs[i] / slice_kernel_ft(c, N, W, beta) *
                       std::exp(cd(0.0, -2.0 * M_PI * (double)c * mm / N));
            }
            G[mm] = acc;
        }
        double num = 0.0, num64 = 0.0, den = 0.0;
        for (int t = 0; t < 600; ++t) {
            const float y = (float)(0.5 * N * U(rng));
            cd exact = 0.0;
            for (int i = 0; i < L; ++i) {
                const int c = i - L / 2;
                exact += xs[i] * std::exp(cd(0.0, -2.0 * M_PI * (double)c * y / N));
            }
            // first tap f = ceil(y - W/2), offset x = y - f - W/2 (integer W/2) in (-1/2, 1/2]
            const float f = std::ceil(y - 0.5f * (float)W);
            const float x = (y - f) - (float)(W / 2);
            cd approx = 0.0, approx64 = 0.0;
            for (int a = 0; a < W; ++a) {
                const int g = (((int)f + a) % N + N) % N;
                approx += (double)weight_fp32(cf, a, x) * G[g];
                approx64 += psi((double)x + W / 2 - a, beta) * G[g];
            }
            num += std::norm(approx - exact);
            num64 += std::norm(approx64 - exact);
            den += std::norm(exact);
        }
        const double rel = std::sqrt(num / den), rel64 = std::sqrt(num64 / den);
        std::printf("L=%d N=%d sigma=%.3f: NUFFT relative l2 error %.3e (exact psi in FP64: %.3e)\n", L, N,
                    (double)N / L, rel, rel64);
        worst_nufft = std::fmax(worst_nufft, rel);
    }
    // at sigma = 1.5 the kernel's aliasing leaves 3-4e-7 (the FP32 weights
    // add nothing measurable; 1.2e-7 at sigma = 2).  The bound fails a shape
    // without the 0.97 factor (7-9e-7), a shape for another sigma (2e-5) and a
    // deapodisation on the wrong frequency scale (order 1).
    if (!(worst_nufft < 5.5e-7)) {
        std::printf("FAIL NUFFT: relative l2 error %.3e\n", worst_nufft);
        return 1;
    }
    std::printf("tap weights %.3e (table rows %.3e), kernel transform %.3e, NUFFT %.3e\nok\n", worst_w,
                worst_rows, worst_ft, worst_nufft);
    return 0;
}
