// sw_slice.cu -- band-limited Radon projection through the Fourier slice
// theorem (Sec. 2.1 Eq. 1d_ift; Sec. 2.3 "Computation", which obtains the
// central slices with a NUFFT; Theorem proj_nufft in App. A).
//
// The image is the cell density f_L (mass a[r][c] spread over its cell).
// For every angle theta_k (k < n/2) and slice frequency
// omega_j = 2 pi j / (B h), j = 0..B/2, the slice sample is
//   f_L^(omega_j e_k) = sinc(pi t_1) sinc(pi t_2) e^{-2 pi i delta (t_1 + t_2)} T(t),
//   T(t) = sum_{r', c'} a[r][c] e^{-2 pi i (t_1 c' + t_2 r')},   t = (j / B) e_k,
// with c' = c - floor(L/2), r' likewise, and delta = 1/2 for even L, 0 for
// odd (cell centre x_c = (c' + delta) h).  T is evaluated by a type-2 NUFFT,
// and the row U[k][b] = h g~(s_b) of the band-limited projection is the
// length-B inverse DFT of X_j = f_L^(omega_j e_k) (-1)^j e^{i pi j / B}
// extended Hermitian (X_{-j} = conj X_j), scaled by 1/B.  Angles theta + pi
// are the mirror rows.
//
// Design (GB300): one CTA per image runs the whole transform in shared
// memory, in four phases separated by barriers.
//  A. a[r][c] / (Psi(r') Psi(c')) (Psi: Fourier transform of the spreading
//     kernel, host table), two image columns packed per complex signal,
//     N-point FFTs along r' (N >= 1.5 L, zero padded), unpacked into the
//     grid rows l2 in [-N/2 - W/2, W/2) that the interpolation reads: the
//     targets t_2 = (j/B) sin theta >= 0 lie in one half plane, so half the
//     oversampled grid (plus the kernel's reach) is all that is stored.
//  B. N-point FFTs along c' of every kept row, written so that no tap wraps:
//     the columns l1 <= W - 1 in increasing order ("left", read by targets
//     whose first tap is at l1 <= 0, i.e. theta <= pi/2), then the columns
//     l1 >= 1 in decreasing order ("right", theta > pi/2).  With a row stride
//     of 1 mod 16 (complex elements) the bank of a tap moves by
//     -(|cos theta| + sin theta) in [-sqrt 2, -1] from one target of a ray to
//     the next in both halves, so the 16 lanes of a 64-bit access stay within
//     two passes; one increasing layout for both halves puts every lane of a
//     ray near theta = 3 pi / 4 on one bank.
//  C. per target, W x W taps of the "exponential of semicircle" kernel
//     psi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)); the W weights along each
//     axis are degree-8 polynomials in the target's offset from its grid
//     cell (fitted on the host in FP64 within 1e-8 of psi; coefficients in
//     the kernel parameters), and the cell's sinc factors and the phase come
//     from a host table per (angle, frequency).
//  D. two angles per complex signal (X_a + i X_b, both Hermitian; paired
//     through shared memory, one target per thread in C), B-point inverse FFT; the real and imaginary parts are the two rows, staged
//     through shared memory so that the row stores coalesce.
// With W = 9 and N / L = 1.5 the rows are within ~3e-7 (relative l2) of the
// exact band-limited projection, at the level of FP32 rounding.
#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int kSliceThreads = 1024;
constexpr int kSig = 16;       // signals per batched FFT
constexpr int kPad = 2 * kSig; // extra complex elements per FFT buffer (staging)
static_assert(2 * kSig == kSliceBatch, "two angles per signal of an inverse-FFT batch");

// Items of one column-pair batch per thread in phase A (N kSig <= 4 x 1024).
constexpr int kAItems = 4;

// x mod N for the small excursions of the grid indices (|x| < 2N in practice).
__device__ __forceinline__ int wrap_n(int x, int N)
{
    while (x < 0) x += N;
    while (x >= N) x -= N;
    return x;
}

// Grid layout (sw_internal.cuh): rows l2 = lo + i; left columns l1 in
// [lo, W - 1], then right columns l1 in [1, N/2 + W/2] reversed; row stride
// 1 mod 16 complex elements, so that 16 lanes reading one column of 16 rows
// hit 16 distinct bank pairs.

struct SliceArgs {
    const float *img;   // images [0, nb1)
    const float *img2;  // images [nb1, nb) (may equal img)
    int nb1;
    int L, srcL, nh, B, N;
    int clip, full_n;
    const float2 *cs;       // [nh] (cos, sin) of theta_k
    const float *psi_inv;   // [L] 1 / Psi(c - floor(L/2))
    const float2 *fac;      // [nh][B/2 + 1] sinc factors times phase
    const uint16_t *gtab;   // target groups per angle batch (see launch_project_slice)
    const int *goff;
    const float2 *twN, *twB;
    float *out;
    int32_t *status;
    SliceCoef coef;         // tap weight polynomials (kernel parameter bank)
};

__global__ void __launch_bounds__(kSliceThreads, 1)
k_project_slice(SliceArgs A, FftPlan planN, FftPlan planB)
{
    extern __shared__ float2 sms[];
    const int L = A.L, N = A.N, B = A.B, nh = A.nh;
    const int rows = slice_rows(N), S = slice_stride(N), lo = slice_lo(N);
    const int nleft = slice_left(N), nright = slice_right(N);
    const int Fmax = N > B ? N : B;
    const int fbuf = Fmax * kSig + kPad;
    float2 *G = sms;           // [rows][S] grid
    float2 *b0 = G + rows * S; // FFT buffers [Fmax][kSig] (+ kPad)
    float2 *b1 = b0 + fbuf;
    float2 *twn = b1 + fbuf;   // [N]
    float2 *twb = twn + N;     // [B]
    __shared__ int s_bad, s_mass;

    const int imgi = blockIdx.x;
    const float *src = imgi < A.nb1 ? A.img + (size_t)imgi * A.srcL * A.srcL
                                    : A.img2 + (size_t)(imgi - A.nb1) * A.srcL * A.srcL;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_mass = 0;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) twn[i] = A.twN[i];
    for (int i = threadIdx.x; i < B; i += blockDim.x) twb[i] = A.twB[i];
    __syncthreads();
    const int half = L / 2;
    int bad = 0, mass = 0;

    // ---- A: FFTs along r' of column pairs, kept rows l2 = lo + i.  The
    // pixels of the next batch are loaded into registers before the FFT of
    // the current one, so that their global-memory latency overlaps it.
    float2 pre[kAItems];
    auto load_batch = [&](int c0) {
#pragma unroll
        for (int m = 0; m < kAItems; ++m) {
            const int t = threadIdx.x + m * blockDim.x;
            float2 v = make_float2(0.f, 0.f);
            const int kpos = t / kSig, s = t % kSig;
            const int r = (kpos < N / 2 ? kpos : kpos - N) + half;
            const int c = c0 + 2 * s;
            if (t < N * kSig && r >= 0 && r < L && c < L) {
                float p[2] = {0.f, 0.f};
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int cc = c + h2;
                    if (cc >= L) continue;
                    float x = A.srcL == L ? __ldg(src + (size_t)r * L + cc)
                                          : 0.25f * __ldg(src + (size_t)(r >> 1) * A.srcL + (cc >> 1));
                    if (!isfinite(x)) {
                        bad = 1;
                        x = 0.f;
                    }
                    x = fmaxf(x, 0.f);
                    mass |= x > 0.f;
                    p[h2] = x * __ldg(A.psi_inv + cc);
                }
                const float pr = __ldg(A.psi_inv + r);
                v = make_float2(p[0] * pr, p[1] * pr);
            }
            pre[m] = v;
        }
    };
    load_batch(0);
    for (int c0 = 0; c0 < L; c0 += 2 * kSig) {
#pragma unroll
        for (int m = 0; m < kAItems; ++m) {
            const int t = threadIdx.x + m * blockDim.x;
            if (t < N * kSig) b0[t] = pre[m];
        }
        if (c0 + 2 * kSig < L) load_batch(c0 + 2 * kSig);
        __syncthreads();
        const float2 *R = fft_smem<kSig, 1>(b0, b1, planN, twn);
        for (int t = threadIdx.x; t < rows * kSig; t += blockDim.x) {
            const int i = t / kSig, s = t % kSig;
            const int m = wrap_n(lo + i, N);  // l2 mod N (small grids wrap more than once)
            const int mm = m == 0 ? 0 : N - m;
            const float2 Z = R[m * kSig + s];
            const float2 Zc = cconj(R[mm * kSig + s]);
            // column c: (Z + conj Z(-l2)) / 2; column c + 1: (Z - conj Z(-l2)) / (2i)
            const float2 d = make_float2(0.5f * (Z.x - Zc.x), 0.5f * (Z.y - Zc.y));
            const int c = c0 + 2 * s;
            if (c < L) G[i * S + c] = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
            if (c + 1 < L) G[i * S + c + 1] = make_float2(d.y, -d.x);
        }
        __syncthreads();
    }
    if (bad) atomicOr(&s_bad, 1);
    if (mass) atomicOr(&s_mass, 1);

    // ---- B: FFTs along c' of every kept row, columns l1 = lo + q
    for (int i0 = 0; i0 < rows; i0 += kSig) {
        for (int t = threadIdx.x; t < N * kSig; t += blockDim.x) {
            const int kpos = t / kSig, s = t % kSig;
            const int i = i0 + s;
            const int c = (kpos < N / 2 ? kpos : kpos - N) + half;
            b0[t] = (i < rows && c >= 0 && c < L) ? G[i * S + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const float2 *R = fft_smem<kSig, 1>(b0, b1, planN, twn);
        for (int t = threadIdx.x; t < (nleft + nright) * kSig; t += blockDim.x) {
            const int q = t / kSig, s = t % kSig;
            const int i = i0 + s;
            if (i >= rows) continue;
            // left: l1 = lo + q;  right (reversed): l1 = N/2 + W/2 - (q - nleft)
            const int m = wrap_n(q < nleft ? lo + q : nright - (q - nleft), N);
            G[i * S + q] = R[m * kSig + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) A.status[imgi] = (s_bad || !s_mass) ? 1 : 0;

    // ---- C + D: slice samples of 2 kSig angles, inverse FFTs, rows out
    const int nj = B / 2 + 1;
    const float rNB = (float)N / (float)B, hN = 0.5f * (float)N, invB = 1.f / (float)B;
    const int nrow = A.full_n ? 2 * nh : nh;
    float *outi = A.out + (size_t)imgi * nrow * B;
    for (int k0 = 0; k0 < nh; k0 += 2 * kSig) {
        // slice samples X[kk][j] of the angles k0 + kk, one target per thread,
        // in the host's half-warp groups; staged in b1 (free until the FFT)
        float2 *Xs = b1;
        // rows of angles beyond nh (last batch) read as zero
        for (int it = threadIdx.x + (nh - k0) * nj; it < 2 * kSig * nj; it += blockDim.x)
            Xs[it] = make_float2(0.f, 0.f);
        const int bi = k0 / (2 * kSig);
        const int g0 = __ldg(A.goff + bi), ng = __ldg(A.goff + bi + 1) - g0;
        for (int slot = threadIdx.x; slot < ng * 16; slot += blockDim.x) {
            const unsigned ent = __ldg(A.gtab + (size_t)(g0 + (slot >> 4)) * 16 + (slot & 15));
            if (ent == 0xFFFFu) continue;
            const int kk = (int)(ent >> 11), j = (int)(ent & 2047u);
            const int k = k0 + kk;
            float2 X;
            {
                const float jf = (float)j;
                const float2 e = __ldg(A.cs + k);
                // target y = -t N on the grid (t = (j/B) e), kept inside the
                // stored half plane whatever the rounding
                const float y1 = fminf(fmaxf(-(jf * e.x) * rNB, -hN), hN);
                const float y2 = fminf(fmaxf(-(jf * e.y) * rNB, -hN), 0.f);
                const float f1 = ceilf(y1 - 0.5f * (float)kSliceW);
                const float f2 = ceilf(y2 - 0.5f * (float)kSliceW);
                // offsets from the cell, exact: y - f is in (W/2 - 1, W/2]
                const float x1 = (y1 - f1) - (float)(kSliceW / 2);
                const float x2 = (y2 - f2) - (float)(kSliceW / 2);
                float wx[kSliceW], wy[kSliceW];
#pragma unroll
                for (int a = 0; a < kSliceW; ++a) {
                    float px = A.coef.c[a][kSliceDeg], py = A.coef.c[a][kSliceDeg];
#pragma unroll
                    for (int d = kSliceDeg - 1; d >= 0; --d) {
                        px = fmaf(px, x1, A.coef.c[a][d]);
                        py = fmaf(py, x2, A.coef.c[a][d]);
                    }
                    wx[a] = px;
                    wy[a] = py;
                }
                const int i1 = (int)f1, i2 = (int)f2 - lo;
                // left half: taps at increasing addresses; right half reversed
                const bool left = i1 <= 0;
                const float2 *g = G + i2 * S + (left ? i1 - lo : nleft + nright - i1);
                const int da = left ? 1 : -1;
                float tr = 0.f, ti = 0.f;
#pragma unroll
                for (int b = 0; b < kSliceW; ++b) {
                    float rr = 0.f, ri = 0.f;
#pragma unroll
                    for (int a = 0; a < kSliceW; ++a) {
                        const float2 v = g[b * S + a * da];
                        rr = fmaf(wx[a], v.x, rr);
                        ri = fmaf(wx[a], v.y, ri);
                    }
                    tr = fmaf(wy[b], rr, tr);
                    ti = fmaf(wy[b], ri, ti);
                }
                // cell sinc factors and phase (host table, FP64)
                const float2 fc = __ldg(A.fac + (size_t)k * nj + j);
                X = make_float2(fc.x * tr - fc.y * ti, fc.x * ti + fc.y * tr);
            }
            Xs[kk * nj + j] = X;
        }
        __syncthreads();
        // two angles per complex signal: Y_j = X_a + i X_b and
        // Y_{B-j} = conj X_a + i conj X_b (Y_0, Y_{B/2}: real parts)
        for (int t = threadIdx.x; t < kSig * nj; t += blockDim.x) {
            const int s = t % kSig, j = t / kSig;
            const float2 Xa = Xs[(2 * s) * nj + j], Xb = Xs[(2 * s + 1) * nj + j];
            if (j == 0 || 2 * j == B) {
                b0[j * kSig + s] = make_float2(Xa.x, Xb.x);
            } else {
                b0[j * kSig + s] = make_float2(Xa.x - Xb.y, Xa.y + Xb.x);
                b0[(B - j) * kSig + s] = make_float2(Xa.x + Xb.y, Xb.x - Xa.y);
            }
        }
        __syncthreads();
        const float2 *R = fft_smem<kSig, 1>(b0, b1, planB, twb);
        // stage rows [2 kSig][B + 1] in the free buffer: reads of R run along
        // the signals (conflict-free), the padded rows spread the writes over
        // distinct banks, and the stores below run along b
        float *stg = reinterpret_cast<float *>(R == b0 ? b1 : b0);
        for (int t = threadIdx.x; t < kSig * B; t += blockDim.x) {
            const int s = t % kSig, b = t / kSig;
            const float2 y = R[b * kSig + s];
            stg[(2 * s) * (B + 1) + b] = y.x * invB;
            stg[(2 * s + 1) * (B + 1) + b] = y.y * invB;
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int row = warp; row < 2 * kSig; row += blockDim.x >> 5) {
            const int k = k0 + row;
            if (k >= nh) continue;
            float *o = outi + (size_t)k * B;
            float *om = outi + (size_t)(nh + k) * B + (B - 1);
            for (int b = lane; b < B; b += 32) {
                float v = stg[row * (B + 1) + b];
                if (A.clip) v = fmaxf(v, 0.f);
                o[b] = v;
                if (A.full_n) om[-b] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int slice_grid_n(int L)
{
    int N = (3 * L + 1) / 2;  // ceil(1.5 L)
    for (;; ++N) {
        int m = N;
        for (int q : {2, 3, 5})
            while (m % q == 0) m /= q;
        if (m == 1 && (N & 1) == 0) return N;
    }
}

size_t slice_smem_bytes(int N, int B)
{
    const int Fmax = N > B ? N : B;
    return sizeof(float2) * ((size_t)slice_rows(N) * slice_stride(N) +
                             2 * ((size_t)Fmax * kSig + kPad) + (size_t)N + (size_t)B);
}

cudaError_t launch_project_slice(const float *img, int nb, int L, int srcL, int nh, int B,
                                 const float2 *cs, const float *psi_inv, const float2 *fac,
                                 const uint16_t *gtab, const int *goff,
                                 const SliceCoef &coef, int N, const FftPlan &planN,
                                 const float2 *twN, const FftPlan &planB, const float2 *twB,
                                 int clip, float *out, int full_n, int32_t *status,
                                 cudaStream_t st, const float *img2, int nb_first)
{
    if (nb <= 0) return cudaSuccess;
    SliceArgs a;
    a.img = img;
    a.img2 = img2 ? img2 : img;
    a.nb1 = (img2 && nb_first >= 0) ? nb_first : nb;
    a.L = L;
    a.srcL = srcL;
    a.nh = nh;
    a.B = B;
    a.N = N;
    a.coef = coef;
    a.fac = fac;
    a.gtab = gtab;
    a.goff = goff;
    a.clip = clip;
    a.full_n = full_n;
    a.cs = cs;
    a.psi_inv = psi_inv;
    a.twN = twN;
    a.twB = twB;
    a.out = out;
    a.status = status;
    const size_t smem = slice_smem_bytes(N, B);
    cudaError_t e = cudaFuncSetAttribute(k_project_slice,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_project_slice<<<nb, kSliceThreads, smem, st>>>(a, planN, planB);
    return cudaGetLastError();
}

}  // namespace swk
