// sw_internal.cuh -- device helpers and launcher declarations shared by the
// kernels of the sliced-2-Wasserstein alignment library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace swk {

constexpr int kMaxStages = 12;

// Radix plan of an FFT of length n: n = prod(radix[0..nst)), radices in
// {2, 3, 4, 5, 8}.  Built on the host with, per stage, the span
// Ns of the sub-transforms already done (product of earlier radices), a
// multiply-high reciprocal of Ns (exact for dividends < 2^16) and the
// twiddle index step n / (Ns r).
struct FftPlan {
    int n;
    int nst;
    int radix[kMaxStages];
    int ns[kMaxStages];
    unsigned ns_rcp[kMaxStages];  // ceil(2^32 / Ns)
    int tstep[kMaxStages];
};

// ------------------------------------------------------------------------
// Double-float ("hi + lo") helpers for the compensated CDF.  TwoSum is exact
// for any two floats (Knuth); the sums below keep |lo| <= ulp(hi)/2.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    float s = a + b;
    float v = s - a;
    float e = (a - (s - v)) + (b - v);
    return {s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = df_two_sum(a.hi, b.hi);
    float e = s.lo + (a.lo + b.lo);
    return df_two_sum(s.hi, e);
}

// a >= b for normalised double-floats.
__device__ __forceinline__ bool df_ge(DF a, DF b)
{
    return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo);
}

// z * T with the product error captured by an FMA.
__device__ __forceinline__ DF df_mul_f(DF t, float z)
{
    float p = z * t.hi;
    float e = fmaf(z, t.hi, -p);
    return df_two_sum(p, fmaf(z, t.lo, e));
}

// k * t / d for small integers k, d (exact floats), inv_d ~ 1/d: the product
// is formed error-free; the quotient estimate q carries its exact FMA
// remainder, so the result is accurate whatever the rounding of q.
__device__ __forceinline__ DF df_scale_ratio(DF t, float k, float d, float inv_d)
{
    float p = t.hi * k;
    float e = fmaf(t.hi, k, -p);
    DF num = df_two_sum(p, fmaf(t.lo, k, e));
    float q = num.hi * inv_d;
    float r = fmaf(-q, d, num.hi);
    return df_two_sum(q, (r + num.lo) * inv_d);
}

// ------------------------------------------------------------------------
// Complex helpers.
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// 5-bit bit reversal (lane order of the warp FFTs' outputs)
__device__ __forceinline__ int brev5(int x) { return (int)(__brev((unsigned)x) >> 27); }
// multiply by -i (forward) or +i (inverse):  dir = -1 gives -i*a, +1 gives i*a
__device__ __forceinline__ float2 cmul_i(float2 a, int dir)
{
    return dir < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ------------------------------------------------------------------------
// The 32-point part of a warp-held inverse transform of length N = 32 M:
// five radix-2 decimation-in-frequency stages over the lanes, applied alike
// to the M values of every lane (outputs in bit-reversed lane order).  The
// upper lane of a butterfly keeps (partner - mine) e^{+2 pi i (lane mod h) /
// (2h)}, the lower one mine + partner; tw[q] = e^{-2 pi i q / N}.  Real and
// imaginary parts go through as packed pairs over k1 = 2q, 2q + 1, so that
// each two-wide FP32 operation of Blackwell serves two transforms (an odd M
// leaves its last value to the scalar form).
template <int M>
__device__ __forceinline__ void warp_lane_stages(float2 (&a)[M], const float2 *__restrict__ tw,
                                                 int lane)
{
    constexpr int N = 32 * M, P = M / 2;
    float2 re[P > 0 ? P : 1], im[P > 0 ? P : 1];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        re[q] = make_float2(a[2 * q].x, a[2 * q + 1].x);
        im[q] = make_float2(a[2 * q].y, a[2 * q + 1].y);
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
        const float sg = up ? -1.f : 1.f;
        const float2 SG = make_float2(sg, sg);
        const float2 w = (h > 1 && up) ? cconj(tw[(lane & (h - 1)) * (N / (2 * h))])
                                       : make_float2(1.f, 0.f);
        const float2 WX = make_float2(w.x, w.x), WY = make_float2(w.y, w.y);
        const float2 NWY = make_float2(-w.y, -w.y);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const float2 pr = make_float2(__shfl_xor_sync(0xffffffffu, re[q].x, h),
                                          __shfl_xor_sync(0xffffffffu, re[q].y, h));
            const float2 pi = make_float2(__shfl_xor_sync(0xffffffffu, im[q].x, h),
                                          __shfl_xor_sync(0xffffffffu, im[q].y, h));
            const float2 dr = __ffma2_rn(SG, re[q], pr);
            const float2 di = __ffma2_rn(SG, im[q], pi);
            if (h > 1) {
                re[q] = __ffma2_rn(NWY, di, __fmul2_rn(WX, dr));  // dr wx - di wy
                im[q] = __ffma2_rn(WY, dr, __fmul2_rn(WX, di));   // di wx + dr wy
            } else {
                re[q] = dr;
                im[q] = di;
            }
        }
        if (M % 2) {
            float2 &y = a[M - 1];
            const float px = __shfl_xor_sync(0xffffffffu, y.x, h);
            const float py = __shfl_xor_sync(0xffffffffu, y.y, h);
            const float2 d = make_float2(fmaf(sg, y.x, px), fmaf(sg, y.y, py));
            y = h > 1 ? cmul(d, w) : d;
        }
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
        a[2 * q] = make_float2(re[q].x, im[q].x);
        a[2 * q + 1] = make_float2(re[q].y, im[q].y);
    }
}

// ------------------------------------------------------------------------
// In-lane inverse DFT of length M in registers, y[k] = sum_n v[n] w^{n k}
// with w = e^{+2 pi i / M} = conj(tw[TS]) (tw[q] = e^{-2 pi i q / N}, N = TS M):
// mixed-radix decimation in time with compile-time indices.  M = R Q with R
// in {4, 2, 3, 5}: the R interleaved subsequences v[R m + r] are transformed
// (length Q), twiddled by w^{r k'} and combined by R-point butterflies:
// y[k' + Q s] = sum_r (w^{r k'} Y_r[k']) e^{+2 pi i r s / R}.
template <int M, int TS>
__device__ __forceinline__ void lane_dft(float2 (&v)[M], const float2 *__restrict__ tw)
{
    if constexpr (M > 1) {
        constexpr int R = M % 4 == 0 ? 4 : (M % 2 == 0 ? 2 : (M % 3 == 0 ? 3 : 5));
        constexpr int Q = M / R;
        static_assert(R * Q == M && (M % 5 != 0 || R == 5 || M % 2 == 0 || M % 3 == 0),
                      "M must factor into 2, 3, 4 and 5");
        float2 sub[R][Q];
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int m = 0; m < Q; ++m) sub[r][m] = v[R * m + r];
            lane_dft<Q, TS * R>(sub[r], tw);
        }
#pragma unroll
        for (int kq = 0; kq < Q; ++kq) {
            float2 a[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                a[r] = (r == 0 || kq == 0) ? sub[r][kq] : cmul(sub[r][kq], cconj(tw[TS * r * kq]));
            if constexpr (R == 2) {
                v[kq] = cadd(a[0], a[1]);
                v[kq + Q] = csub(a[0], a[1]);
            } else if constexpr (R == 4) {
                const float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
                const float2 s13 = cadd(a[1], a[3]), d13 = cmul_i(csub(a[1], a[3]), +1);
                v[kq] = cadd(s02, s13);
                v[kq + Q] = cadd(d02, d13);
                v[kq + 2 * Q] = csub(s02, s13);
                v[kq + 3 * Q] = csub(d02, d13);
            } else if constexpr (R == 3) {
                // e^{+2 pi i / 3} = -1/2 + i sqrt(3)/2
                const float s3 = 0.86602540378443864676f;
                const float2 t1 = cadd(a[1], a[2]);
                const float2 t2 = make_float2(a[0].x - 0.5f * t1.x, a[0].y - 0.5f * t1.y);
                float2 t3 = cmul_i(csub(a[1], a[2]), +1);
                t3.x *= s3;
                t3.y *= s3;
                v[kq] = cadd(a[0], t1);
                v[kq + Q] = cadd(t2, t3);
                v[kq + 2 * Q] = csub(t2, t3);
            } else {  // R == 5
                const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
                const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
                const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
                const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
                const float2 a1 = cadd(a[1], a[4]), b1 = csub(a[1], a[4]);
                const float2 a2 = cadd(a[2], a[3]), b2 = csub(a[2], a[3]);
                const float2 r1 = make_float2(a[0].x + c1 * a1.x + c2 * a2.x,
                                              a[0].y + c1 * a1.y + c2 * a2.y);
                const float2 r2 = make_float2(a[0].x + c2 * a1.x + c1 * a2.x,
                                              a[0].y + c2 * a1.y + c1 * a2.y);
                const float2 i1 = cmul_i(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y), +1);
                const float2 i2 = cmul_i(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y), +1);
                v[kq] = make_float2(a[0].x + a1.x + a2.x, a[0].y + a1.y + a2.y);
                v[kq + Q] = cadd(r1, i1);
                v[kq + 4 * Q] = csub(r1, i1);
                v[kq + 2 * Q] = cadd(r2, i2);
                v[kq + 3 * Q] = csub(r2, i2);
            }
        }
    }
}

// ------------------------------------------------------------------------
// Batched complex FFT of length n over NSIG signals held in shared memory
// as buf[k * NSIG + s] (signal s, element k), Stockham self-sorting, mixed
// radix 2/3/4/5/8.  DIR = -1: X(q) = sum_k x(k) e^{-2 pi i k q / n};
// DIR = +1: the unnormalised inverse.  tw[m] = e^{-2 pi i m / n} (shared
// memory).  Each stage reads one buffer and writes the other; returns the
// buffer that holds the result.  Must be called by every thread of the block;
// ends with a __syncthreads().

// One stage of radix R: item t = (j, s) takes x[j + i n/R] (i < R), twiddled
// by w^{i k}, k = j mod Ns, and writes its R outputs at stride Ns from
// (j div Ns) Ns R + k.
template <int R, int NSIG, int DIR>
__device__ __forceinline__ void fft_stage(const float2 *__restrict__ a, float2 *__restrict__ b,
                                          int n, int Ns, unsigned rcp, int tstep,
                                          const float2 *__restrict__ tw)
{
    const int nr = n / R;
    const int total = nr * NSIG;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int s = t % NSIG;
        const int j = t / NSIG;
        const int jq = Ns == 1 ? j : (int)__umulhi((unsigned)j, rcp);  // j / Ns
        const int k = j - jq * Ns;
        float2 v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            float2 x = a[(j + i * nr) * NSIG + s];
            if (i > 0 && k > 0) {
                float2 w = tw[i * k * tstep];  // i k < R Ns, so the index is < n
                if (DIR > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[i] = x;
        }
        float2 V[R];
        if (R == 2) {
            V[0] = cadd(v[0], v[1]);
            V[1] = csub(v[0], v[1]);
        } else if (R == 4) {
            float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
            float2 s13 = cadd(v[1], v[3]), d13 = cmul_i(csub(v[1], v[3]), DIR);
            V[0] = cadd(s02, s13);
            V[2] = csub(s02, s13);
            V[1] = cadd(d02, d13);
            V[3] = csub(d02, d13);
        } else if (R == 3) {
            // w3 = e^{DIR 2 pi i / 3} = -1/2 + DIR i sqrt(3)/2
            const float c3 = -0.5f, s3 = 0.86602540378443864676f;
            float2 t1 = cadd(v[1], v[2]);
            float2 t2 = make_float2(v[0].x + c3 * t1.x, v[0].y + c3 * t1.y);
            float2 t3 = cmul_i(csub(v[1], v[2]), DIR);
            t3.x *= s3;
            t3.y *= s3;
            V[0] = cadd(v[0], t1);
            V[1] = cadd(t2, t3);
            V[2] = csub(t2, t3);
        } else if (R == 8) {
            // two radix-4 butterflies over the even and the odd inputs, then
            // V[m] = E[m] + w8^m O[m], V[m+4] = E[m] - w8^m O[m], with
            // w8 = e^{DIR 2 pi i / 8} = (1 + DIR i) / sqrt(2)
            const float r2 = 0.70710678118654752440f;
            float2 E[4], O[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 e0 = cadd(v[h], v[h + 4]), e1 = csub(v[h], v[h + 4]);
                float2 e2 = cadd(v[h + 2], v[h + 6]);
                float2 e3 = cmul_i(csub(v[h + 2], v[h + 6]), DIR);
                float2 *X = h == 0 ? E : O;
                X[0] = cadd(e0, e2);
                X[2] = csub(e0, e2);
                X[1] = cadd(e1, e3);
                X[3] = csub(e1, e3);
            }
            O[1] = make_float2(r2 * (O[1].x - DIR * O[1].y), r2 * (O[1].y + DIR * O[1].x));
            O[2] = cmul_i(O[2], DIR);
            O[3] = make_float2(r2 * (-O[3].x - DIR * O[3].y), r2 * (-O[3].y + DIR * O[3].x));
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                V[m] = cadd(E[m], O[m]);
                V[m + 4] = csub(E[m], O[m]);
            }
        } else {  // R == 5
            const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
            const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
            const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
            const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
            float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
            float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
            float2 r1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
            float2 r2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
            // i1 = DIR*i*(s1 b1 + s2 b2), i2 = DIR*i*(s2 b1 - s1 b2)
            float2 i1 = cmul_i(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y), DIR);
            float2 i2 = cmul_i(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y), DIR);
            V[0] = make_float2(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
            V[1] = cadd(r1, i1);
            V[4] = csub(r1, i1);
            V[2] = cadd(r2, i2);
            V[3] = csub(r2, i2);
        }
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int i = 0; i < R; ++i) b[(base + i * Ns) * NSIG + s] = V[i];
    }
}

template <int NSIG, int DIR>
__device__ __forceinline__ float2 *fft_smem(float2 *a, float2 *b, const FftPlan &plan,
                                            const float2 *tw)
{
    const int n = plan.n;
    for (int st = 0; st < plan.nst; ++st) {
        const int Ns = plan.ns[st];
        const unsigned rcp = plan.ns_rcp[st];
        const int tstep = plan.tstep[st];
        switch (plan.radix[st]) {
        case 4: fft_stage<4, NSIG, DIR>(a, b, n, Ns, rcp, tstep, tw); break;
        case 8: fft_stage<8, NSIG, DIR>(a, b, n, Ns, rcp, tstep, tw); break;
        case 2: fft_stage<2, NSIG, DIR>(a, b, n, Ns, rcp, tstep, tw); break;
        case 3: fft_stage<3, NSIG, DIR>(a, b, n, Ns, rcp, tstep, tw); break;
        default: fft_stage<5, NSIG, DIR>(a, b, n, Ns, rcp, tstep, tw); break;
        }
        __syncthreads();
        float2 *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

// ------------------------------------------------------------------------
// Launchers.  All return the launch status (cudaGetLastError).

// Projection of nb images (sw_project / first stage of the alignment).
// img: [nb][srcL][srcL]; srcL == L, or srcL == L/2 (2x2 upsampling on load).
// out: full_n ? [nb][2*nh][B] (angles k and k+nh, the latter mirrored)
//             : [nb][nh][B] (angles k < nh only).
// cs: [nh] (cos, sin) of theta_k.  status: [nb], 1 for an unusable image.
// With img2: images [0, nb_first) come from img and [nb_first, nb) from img2
// (two batches in one launch).
// scale[i] = 1 / sum max(img_i, 0) in FP64 (NaN for an image without positive
// mass or with a non-finite pixel); img [nb][L][L].
cudaError_t launch_image_scale(const float *img, int nb, int L, double *scale, cudaStream_t st);

cudaError_t launch_project(const float *img, int nb, int L, int srcL, int nh, int B,
                           const float2 *cs, float *out, int full_n, int32_t *status,
                           cudaStream_t st, int want_ctas = 0, const float *img2 = nullptr,
                           int nb_first = -1);

// The slice projector's spreading kernel width (taps per axis) and the
// degree of the polynomial that gives each tap's weight from the target's
// offset x in (-1/2, 1/2] from its grid cell: c[a] holds psi(x + W/2 - a)
// as sum_d c[a][d] x^d.
constexpr int kSliceW = 9;
constexpr int kSliceDeg = 8;
struct SliceCoef {
    float c[kSliceW][kSliceDeg + 1];
};
// "#pragma unroll" in the device pass only (host compilers do not know it).
#ifdef __CUDA_ARCH__
#define SW_DEVICE_UNROLL _Pragma("unroll")
#else
#define SW_DEVICE_UNROLL
#endif
// The W tap weights at offset x: w[a] = sum_d c[a][d] x^d.  psi is even, so
// tap W-1-a at x is tap a at -x (c[W-1-a][d] = (-1)^d c[a][d]); a mirrored
// pair shares the even and odd parts of the polynomial in x^2,
// w = E(x^2) +- x O(x^2), and the middle tap is E alone: 41 FMAs per axis
// instead of 72 for nine Horner chains in x.  Reads rows 0..W/2 only.
__host__ __device__ __forceinline__ void slice_tap_weights(const SliceCoef &cf, float x,
                                                           float (&w)[kSliceW])
{
    static_assert(kSliceW % 2 == 1 && kSliceDeg % 2 == 0, "odd tap count, even degree");
    constexpr int H = kSliceW / 2;
    const float s = x * x;
SW_DEVICE_UNROLL
    for (int a = 0; a <= H; ++a) {
        float e = cf.c[a][kSliceDeg];
SW_DEVICE_UNROLL
        for (int d = kSliceDeg - 2; d >= 0; d -= 2) e = fmaf(e, s, cf.c[a][d]);
        if (a == H) {
            w[a] = e;
        } else {
            float o = cf.c[a][kSliceDeg - 1];
SW_DEVICE_UNROLL
            for (int d = kSliceDeg - 3; d >= 1; d -= 2) o = fmaf(o, s, cf.c[a][d]);
            w[a] = fmaf(x, o, e);
            w[kSliceW - 1 - a] = fmaf(-x, o, e);
        }
    }
}
// Angles per batch of the slice projector's interpolation (two per warp in
// the inverse FFTs).
constexpr int kSliceBatch = 64;
// Flag of a target-table entry (L <= 128) that stands for the ray-adjacent
// pair (j, j + 1), interpolated together from their union footprint.
constexpr unsigned kSlicePairBit = 0x4000u;
// Grid geometry of the slice projector for an N-point oversampled grid (see
// sw_slice.cu): lowest tap index, kept rows, left and right column counts
// and the row stride (complex elements).
__host__ __device__ inline int slice_lo(int N) { return -N / 2 - kSliceW / 2; }
__host__ __device__ inline int slice_rows(int N) { return N / 2 + kSliceW; }
__host__ __device__ inline int slice_left(int N) { return kSliceW - slice_lo(N); }
__host__ __device__ inline int slice_right(int N) { return N / 2 + kSliceW / 2; }
__host__ __device__ inline int slice_stride(int N)
{
    const int S = slice_left(N) + slice_right(N);
    return S + (17 - S % 16) % 16;
}
// Stored row and column of the first tap of target (j, theta) with e =
// (cos, sin) of theta in FP32 on the grid N = B, exactly as the kernel forms
// them; *left tells the half (taps at increasing columns when set, at
// decreasing ones otherwise).
__host__ __device__ inline void slice_tap_rc(int j, float ex, float ey, int N, int *row, int *col,
                                             bool *left)
{
    const float jf = (float)j, hN = 0.5f * (float)N;
    const float y1 = fminf(fmaxf(-(jf * ex), -hN), hN);
    const float y2 = fminf(fmaxf(-(jf * ey), -hN), 0.f);
    const int i1 = (int)ceilf(y1 - 0.5f * (float)kSliceW);
    *row = (int)ceilf(y2 - 0.5f * (float)kSliceW) - slice_lo(N);
    *left = i1 <= 0;
    *col = *left ? i1 - slice_lo(N) : slice_left(N) + slice_right(N) - i1;
}
// First grid address of the taps of target (j, theta) (see slice_tap_rc).
__host__ __device__ inline int slice_tap_base(int j, float ex, float ey, int N, bool *left)
{
    int row, col;
    slice_tap_rc(j, ex, ey, N, &row, &col, left);
    return row * slice_stride(N) + col;
}
// Images of side L/2 seen as L x L images of 2 x 2 blocks (each pixel split
// into four cells of a quarter of its value): with c' = 2 c'' + u, u in {0, 1},
//   T_L(t) = (1 + e^{-2 pi i t_1}) (1 + e^{-2 pi i t_2}) / 4 * T_{L/2}(2 t),
// and T_{L/2} is 1-periodic, so the L/2 image's own grid of N = B/2 points
// serves the rows of B bins: target (j, theta), j <= B/2 = N, sits at
// y = -j e on that grid.  First tap (i1, i2) and offsets (x1, x2) of the
// target on the stored half grid: y1 wrapped by N into the columns the
// grid keeps; a row footprint below the kept rows wraps into the upper half
// plane, where the target is folded through T(-s) = conj T(s) (*conj set:
// taps reflected, i -> -i - (W - 1), offsets negated).  Integer wrapping
// and folding keep host and kernel in step (both take the same FP32 steps
// up to the cell).
__host__ __device__ inline void slice_up_tap(int j, float ex, float ey, int N, int *i1, int *i2,
                                             float *x1, float *x2, bool *conj)
{
    const float jf = (float)j, Nf = (float)N;
    const float y1 = fminf(fmaxf(-(jf * ex), -Nf), Nf);
    const float y2 = fminf(fmaxf(-(jf * ey), -Nf), 0.f);
    const float f1 = ceilf(y1 - 0.5f * (float)kSliceW);
    const float f2 = ceilf(y2 - 0.5f * (float)kSliceW);
    *x1 = (y1 - f1) - (float)(kSliceW / 2);
    *x2 = (y2 - f2) - (float)(kSliceW / 2);
    int a = (int)f1, b = (int)f2;
    const int lo = slice_lo(N), hi = N / 2 - kSliceW / 2;
    if (a > hi) a -= N;
    else if (a < lo) a += N;
    *conj = b < lo;
    if (*conj) {
        b = -(b + N) - (kSliceW - 1);
        a = -a - (kSliceW - 1);
        *x1 = -*x1;
        *x2 = -*x2;
    }
    *i1 = a;
    *i2 = b;
}
// Stored row, column and half of the first tap of an upsampled-image target
// (see slice_up_tap), as slice_tap_rc gives them for plain targets.
__host__ __device__ inline void slice_up_rc(int j, float ex, float ey, int N, int *row, int *col,
                                            bool *left)
{
    int i1, i2;
    float x1, x2;
    bool conj;
    slice_up_tap(j, ex, ey, N, &i1, &i2, &x1, &x2, &conj);
    *row = i2 - slice_lo(N);
    *left = i1 <= 0;
    *col = *left ? i1 - slice_lo(N) : slice_left(N) + slice_right(N) - i1;
}
// Tiles of the stored half grid for 128 < L: a target belongs to the tile
// holding the top-left cell of its W x W footprint; a tile's shared-memory
// copy is kSliceTileSpan square (the tile and a halo of W - 1), rows
// kSliceTileRS apart (odd: the bank of a cell is (row + col) mod 16).
constexpr int kSliceTile = 56;
constexpr int kSliceTileSpan = kSliceTile + kSliceW - 1;  // 64
constexpr int kSliceTileRS = kSliceTileSpan + 1;          // 65
__host__ __device__ inline int slice_tiles_y(int N)
{
    return (slice_rows(N) - kSliceW) / kSliceTile + 1;
}
__host__ __device__ inline int slice_tiles_x(int N)
{
    return (slice_left(N) + slice_right(N) - kSliceW) / kSliceTile + 1;
}

// Band-limited projection through the Fourier slice theorem (see
// sw_slice.cu): same input, output and status conventions as
// launch_project.  B = 32 M bins with B >= 1.5 L (M <= 6 for L <= 128;
// M = 8, 10 or 12 for 128 < L <= 256), also the oversampled grid length; psi_inv [L] = 1 / Psi(c - floor(L/2)) with Psi
// the Fourier transform of the spreading kernel; tw [B] = e^{-2 pi i q / B}.
// clip = 1 writes max(row, 0).  For L <= 128, one CTA of 1024 threads per
// image with slice_smem_bytes(B) of dynamic shared memory; above, three
// launches per chunk of images with the grids and slice samples in scratch.
// fac: [nh][B/2 + 1] sinc(pi t_1) sinc(pi t_2) (-1)^j e^{i pi j (1 - 2 delta (cos + sin)) / B}
// with t = (j / B)(cos theta_k, sin theta_k), delta = 1/2 for even L, else 0.
// gtab/goff: the targets (kk, j) of angle batch b (angles b batch + kk)
// in half-warp groups of 16 lanes, entries kk * 256 + j (j <= B/2 <= 96),
// with kSlicePairBit set for the pair (j, j + 1) of one half of the grid
// whose footprints start at most one row and column apart, or 0xFFFF
// (idle); pair groups come first and hold only pairs,
// groups goff[b] .. goff[b+1]; every target of the batch appears once.  The
// grouping only orders the work: each group's targets have distinct tap
// addresses mod 16 (or equal ones), so its loads cost one pass.
// L <= 128: the grid in shared memory (one CTA per image, kSliceBatch-angle
// batches, targets grouped by bank).  128 < L <= 256: the grids of chunks of
// kSliceChunk images in the caller's scratch (slice_scratch_bytes), then one
// CTA per (tile, image) with the tile in shared memory writing the slice
// samples to the scratch, then one CTA per (32-angle batch, image) for the
// rows.  ttab/toff: the targets of tile t (slice_tiles_y x slice_tiles_x,
// row-major) in half-warp groups toff[t] .. toff[t+1] of 16 entries
// k << 16 | j or 0xFFFFFFFF, grouped by the bank of the first tap in the
// tile's copy as above (left and right halves apart).
constexpr int kSliceChunk = 1024;
constexpr size_t kSliceSmemMax = 227 * 1024 - 64;  // opt-in dynamic shared memory of a CTA
// 32 ceil(max(min_bins, 1.5 L) / 32), rounded up to 256, 320 or 384 above 192
int slice_default_bins(int L, int min_bins);
bool slice_bins_supported(int L, int B);
size_t slice_smem_bytes(int B);
int slice_batch_of(int L);
// the grids and the slice samples of one chunk (nh angles): 0 for L <= 128
size_t slice_scratch_bytes(int L, int B, int nb, int nh);

// Images of side L/2 upsampled 2 x 2 for 128 < L (see slice_up_tap): one CTA
// of 1024 threads per image holds the L/2 image's grid of N = B/2 points
// (the L <= 128 layout) and writes rows of B bins, kUpBatch angles per
// batch.  Tables (device memory, built with the L x L problem's angles):
//   psi_inv [L/2]  1 / Psi(c - L/4) on the N-point grid (same kernel shape:
//                  the oversampling N / (L/2) = B / L is unchanged);
//   fac [nh][N + 1] the L x L problem's fac times
//                  (1 + e^{-2 pi i t_1}) (1 + e^{-2 pi i t_2}) / 4;
//   gtab/goff      targets (kk, j), j <= N, per kUpBatch-angle batch as for
//                  L <= 128 (pairs by slice_up_rc);
//   tw [N]         e^{-2 pi i q / N} (the grid's FFTs).
// tw_rows [B] e^{-2 pi i q / B} (the rows' inverse FFTs).  img: [nb][L/2][L/2].
constexpr int kUpBatch = 32;
struct SliceUpTables {
    const float *psi_inv;
    const float2 *fac;
    const uint16_t *gtab;
    const int *goff;
    const float2 *tw;
};
// L even, 128 < L, B/2 a supported L/2 grid, shared memory within a CTA's
size_t slice_up_smem_bytes(int B);
bool slice_up_supported(int L, int B);
cudaError_t launch_project_slice_up(const float *img, int nb, int L, int nh, int B,
                                    const float2 *cs, const SliceUpTables &up,
                                    const SliceCoef &coef, const float2 *tw_rows, int clip,
                                    float *out, int full_n, int32_t *status, cudaStream_t st,
                                    const float *img2 = nullptr, int nb_first = -1);
cudaError_t launch_project_slice(const float *img, int nb, int L, int srcL, int nh, int B,
                                 const float2 *cs, const float *psi_inv, const float2 *fac,
                                 const uint16_t *gtab, const int *goff, const uint32_t *ttab,
                                 const int *toff, const SliceCoef &coef, const float2 *tw,
                                 float2 *scratch, int clip, float *out, int full_n,
                                 int32_t *status, cudaStream_t st, const float *img2 = nullptr,
                                 int nb_first = -1);

// Quantiles.  proj: half ? [nb][nh][B] (angle k >= nh read mirrored)
//                        : [nb][2nh][B].
// q: [nb][n][M].  status[r >> status_shift] is OR-ed with 1 when a
// projection of row r has no mass (status_shift 1: two rows per image).
cudaError_t launch_quantiles(const float *proj, int nb, int n, int B, int M, float h,
                             int level_rule, int half, float *q, int32_t *status,
                             cudaStream_t st, int status_shift = 0);

// Ramp filter and split of the projections (ramp-filtered sliced W2):
// proj [nb][nh][B] -> parts [nb][2][nh][B] (positive part, absolute negative
// part) of the rows filtered circularly by |xi| on the bin grid.  plan and
// tw are the FFT plan and twiddles of length B (2/3/5-smooth).
cudaError_t launch_ramp(const float *proj, int nb, int nh, int B, const FftPlan &plan,
                        const float2 *tw, float *parts, cudaStream_t st);

// Centring vector and centred norm of quantiles (public sw_quantiles):
// a = (2/n) sum_k ubar_k theta_k, norm = sum (q - <a, theta_k>)^2.
cudaError_t launch_center_norm(const float *q, int nb, int n, int M, const double2 *cs64,
                               double *center, double *norm, cudaStream_t st);

// Angle spectra of nb images.  For k' = 1..n/2, spec32[(k'-1)*fstride + img*2M + p]
// = Re Qhat(k', p) and [.. + M + p] = Im, where Qhat is the DFT over angle of
// the quantiles centred by a.  prof[img][p] = mean_k q[k][p] (k' = 0 / n).
// norm32[img] = sum over k' != 0 of |Qhat|^2 / n (the centred, mean-free norm);
// lp_kind 1/2 also writes bf16/fp16 copies in rows of ldk = tc_ldk(M)
// elements, zero padded after 2M: queries (img < Nq) to
// lp_q[(k'-1)*lpq_fstride + img*ldk] = [re | im | 0], templates to the doubled
// layout lp_t[(k'-1)*lpt_fstride + (2j)*ldk] = [re | im | 0] and
// [(2j+1)*ldk] = [-im | re | 0], and norm16 from the rounded values.
// lp_kind 3 writes the FP16 split x = hi + lo in rows of 2 ldk elements,
// [hi | lo] (of the same [re|im|0] and [-im|re|0] rows): the correlation
// runs one GEMM over K = 3 ldk, reading the segments (hi, hi), (hi, lo),
// (lo, hi) of the two operands, so that it sums hi*hi + hi*lo + lo*hi.
// With lp_kind != 0, spec32 is not written (may be NULL).
// parts = 2 (ramp-filtered distance): M counts the levels of both parts,
// q is [nb][2][n][M/2], each part is centred by its own vector and center
// is [nb][2][2]; the norms are the sums over both parts.
cudaError_t launch_spectrum(const float *q, int nb, int n, int M, const FftPlan &plan,
                            const float2 *tw, float *spec32, size_t fstride, int lp_kind,
                            void *lp_q, size_t lpq_fstride, void *lp_t, size_t lpt_fstride,
                            int Nq, float *prof, double *center, double *norm32,
                            double *norm16, cudaStream_t st, int nsig = 0, int parts = 1);

// FP32 SIMT correlation: for f < nf, i < Nq, j < Nt
// C[(f*Nq + i)*Nt + j] = sum_p Qhat_i(f,p) conj(Qhat_j(f,p)) as (re, im).
// X rows: X + f*xf + i*2M ([re | im]); Y rows: Y + f*yf + j*2M.
cudaError_t launch_corr_simt(const float *X, size_t xf, const float *Y, size_t yf, int Nq,
                             int Nt, int M, int nf, float2 *C, cudaStream_t st);

// Tensor-core correlation (tcgen05): the same product as launch_corr_simt for
// BF16 (kind 1) or FP16 (kind 2) spectra in the padded K-major layout of
// launch_spectrum: Xq [nf][Nq][ldk], Yt [nf][2Nt][ldk] (doubled template rows).
// *err is set to 1 if a bounded wait gave up.  wait_cycles: limit of each
// wait of one pipeline role on another, in SM clock cycles (0 = ~2 s).
// stall (a test hook): the producer issues no copies, so the MMA role's
// first wait runs out at the limit and *err is set.  tile_n: output tile
// width (columns of D = 2 x templates), 256 or 128.
int tc_ldk(int M);  // K row length: 2M rounded up to 64
int lp_row_len(int M, int lp_kind);  // low-precision row length: ldk, or 2 ldk ([hi | lo]) for the split
cudaError_t launch_corr_tc(const void *Xq, const void *Yt, int Nq, int Nt, int M, int nf,
                           int kind, float2 *C, int *err, int num_sms, cudaStream_t st,
                           long long wait_cycles = 0, int stall = 0, int tile_n = 256);
// kind: 1 bf16, 2 fp16, 3 fp16 split (rows of lp_row_len(M, 3) elements)

// Inverse angle FFT of the correlation spectra, argmin over the rotation
// grid and the FP64 distance at the optimum.  See sw_decide.cu.
struct DecideArgs {
    const float2 *C;      // [nf][Nq][Nt]
    int Nq, Nt, n, M;
    const float *prof_q;  // [Nq][M]
    const float *prof_t;  // [Nt][M]
    const double *ctr_q;  // [Nq][2]
    const double *ctr_t;  // [Nt][2]
    const double *norm_q; // [Nq]
    const double *norm_t; // [Nt]
    const int32_t *st_q;  // [Nq]
    const int32_t *st_t;  // [Nt]
    const double2 *cs64;  // [n] (cos, sin) of alpha_l
    int translation;
    const int *dev_err;   // nonzero: the correlation gave up (status 3), or NULL
    void *out;            // sw_result [Nq][Nt]
    double *curve;        // [n] or NULL (pair 0,0 only)
    double *shifts;       // [n][2] or NULL
    // 1: sliced W2 (ctr [N][2]); 2: ramp-filtered sliced W2, M counts the
    // levels of both parts and ctr is [N][2][2] (a+, a-); the distance adds
    // |d_i - R d_j|^2 / 4, d = a+ - a-, and the rotation-only term is
    // |abar_i - R abar_j|^2 with abar = (a+ + a-)/2 (derivation in the oracle)
    int parts = 1;
    // translation restricted to the grid (i, j) * grid_step, |i|, |j| <= grid_k
    // (grid_k > 0 with translation): the shift is the grid point nearest the
    // closed-form optimum and the distance adds rho |s - c|^2
    int grid_k = 0;
    double grid_step = 0.0;
    // filled by launch_decide: 1/n, 1/(nM), 2 pi/n (no FP64 divisions on the device)
    double inv_n, inv_nM, dalpha;
    // FP32 constants of the argmin keys (filled by launch_decide; GB300 runs
    // FP64 at a small fraction of FP32, so no key work is done in FP64):
    // hnm = (1/2 or 1) n M', qnm = n M' / 4 with M' the levels per part,
    // gstep, 1 / gstep (0 without a grid) and grid_k
    float hnm, qnm, gstep, ginv, gk;
};
// nsig: 0 = default form, 1 = register form (n = 64, 128, 256, 512), 4, 8
// or 16 = shared-memory form with that many signals per CTA.
cudaError_t launch_decide(const DecideArgs &a, const FftPlan &plan, const float2 *tw,
                          cudaStream_t st, int nsig = 0);
// n for which the register form of the decision exists (its default there)
bool decide_reg_ok(int n);

// Max-sliced W2 over rotations: q [Nq][n][M], t [Nt][n][M] uncentred
// quantiles; with translation the columns are centred by ctr ([N][2]).
// curve: scratch [Nq][Nt][n] floats (M times the curve); out: sw_result
// [Nq][Nt]; full / shifts: the curve and shifts of pair (0, 0) or NULL.
struct MswArgs {
    const float *q, *t;
    int Nq, Nt, n, M;
    const double *ctr_q, *ctr_t;
    const int32_t *st_q, *st_t;
    const double2 *cs64;
    int translation;
    float *curve;
    void *out;
    double *full, *shifts;
    double dalpha;  // filled by the launcher
};
cudaError_t launch_msw(const MswArgs &a, cudaStream_t st);

// Best template per query from the [Nq][Nt] results.
cudaError_t launch_best_template(const void *all, int Nq, int Nt, void *out, cudaStream_t st);

}  // namespace swk
