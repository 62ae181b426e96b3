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
// odd (cell centre x_c = (c' + delta) h).  T is evaluated by a type-2 NUFFT
// on an N = B point oversampled grid (B >= 1.5 L), and the row
// U[k][b] = h g~(s_b) of the band-limited projection is the length-B inverse
// DFT of X_j = f_L^(omega_j e_k) (-1)^j e^{i pi j / B} extended Hermitian
// (X_{-j} = conj X_j), scaled by 1/B.  Angles theta + pi are the mirror rows.
//
// Design (GB300): every FFT is a warp's own: B = 32 M points held M per
// lane, an M-point DFT in registers, the twiddles, then five radix-2 stages
// across the lanes by shuffles (outputs in bit-reversed lane order), so no
// transform waits on a block barrier.  Four phases:
//  A. a[r][c] / (Psi(r') Psi(c')) (Psi: Fourier transform of the spreading
//     kernel, host table), two image columns packed per complex signal,
//     one warp per column pair: N-point FFT along r' (zero padded), unpacked
//     into the grid rows l2 in [-N/2 - W/2, W/2) that the interpolation
//     reads: the targets t_2 = (j/B) sin theta >= 0 lie in one half plane, so
//     half the oversampled grid (plus the kernel's reach) is all that is
//     stored.
//  B. one warp per kept row: N-point FFT along c', written so that no tap
//     wraps: the columns l1 <= W - 1 in increasing order ("left", read by
//     targets whose first tap is at l1 <= 0, i.e. theta <= pi/2), then the
//     columns l1 >= 1 in decreasing order ("right", theta > pi/2).  With a
//     row stride of 1 mod 16 (complex elements) the bank of a tap moves by
//     -(|cos theta| + sin theta) in [-sqrt 2, -1] along a ray in both halves.
//  C. per target, W x W taps of the "exponential of semicircle" kernel
//     psi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)); the W weights along each
//     axis are degree-8 polynomials in the target's offset from its grid
//     cell (fitted on the host in FP64 within 1e-8 of psi; coefficients in
//     the kernel parameters; psi is even, so the mirrored taps a and W-1-a
//     share the even and odd parts of one polynomial in the offset squared),
//     and the cell's sinc factors and the phase come
//     from a host table per (angle, frequency).  The targets of an angle batch
//     run in host-ordered half-warp groups.
//  D. one warp per pair of angles (X_a + i X_b, both Hermitian): B-point
//     inverse FFT; the real and imaginary parts are the two rows, staged in
//     the warp's own slice-sample rows so that the row stores coalesce.
// Two arrangements:
//  - L <= 128 (k_project_slice): one CTA of 32 warps per image with the whole
//    grid in shared memory (175 KB at L = 128); 64-angle batches; the
//    targets grouped so that each tap load of a half-warp hits 16 distinct
//    banks (one pass).
//  - 128 < L <= 256 (k_slice_grid, k_slice_tile, k_slice_rows): the grid of
//    a chunk of images is built in a global scratch buffer (one CTA of 16
//    warps per image, phases A and B, the image staged in 32-column bands);
//    phase C runs one CTA per (56 x 56 tile of the stored grid, image) with
//    the tile and its halo in shared memory, the targets whose footprint
//    starts in the tile grouped by bank, into a global sample buffer; phase D
//    runs one CTA per (image, 32-angle batch).
// With W = 9 and N / L >= 1.5 the rows are within ~3e-7 (relative l2) of the
// exact band-limited projection, at the level of FP32 rounding.
#include <algorithm>

#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int kSliceThreads = 1024;  // shared-memory grid: 32 warps
constexpr int kBigThreads = 512;     // global grid: 16 warps (more registers per lane)
constexpr int kBigBatch = 32;        // angles per CTA of k_slice_rows
static_assert(2 * (kSliceThreads / 32) == kSliceBatch, "one warp per angle pair of a batch");
static_assert(2 * (kBigThreads / 32) == kBigBatch, "one warp per angle pair of a batch");

// x mod N for the small excursions of the grid indices (|x| < 2N).
__device__ __forceinline__ int wrap_n(int x, int N)
{
    while (x < 0) x += N;
    while (x >= N) x -= N;
    return x;
}

// Unnormalised inverse DFT of length N = 32 M held by one warp:
//   X[k] = sum_n x[n] e^{+2 pi i n k / N}.
// In: v[n1] = x[32 n1 + lane].  Out: v[k1] = X[k1 + M brev5(lane)].
// tw[q] = e^{-2 pi i q / N} in shared memory.  Four-step: an M-point DFT
// over n1 (lane_dft), the twiddles e^{+2 pi i lane k1 / N}, and a 32-point
// transform over the lanes in five radix-2 decimation-in-frequency stages.
template <int M>
__device__ __forceinline__ void warp_ifft(float2 (&v)[M], const float2 *__restrict__ tw, int lane)
{
    lane_dft<M, 32>(v, tw);
#pragma unroll
    for (int k1 = 1; k1 < M; ++k1) v[k1] = cmul(v[k1], cconj(tw[lane * k1]));  // lane k1 < N
    warp_lane_stages<M>(v, tw, lane);
}

struct SliceArgs {
    const float *img;   // images [0, nb1)
    const float *img2;  // images [nb1, nb) (may equal img)
    int nb1;
    int img_off;        // global index of this launch's image 0
    int L, srcL, nh;
    int clip, full_n;
    const float2 *cs;       // [nh] (cos, sin) of theta_k
    const float *psi_inv;   // [L] 1 / Psi(c - floor(L/2))
    const float2 *fac;      // [nh][B/2 + 1] sinc factors times phase
    const uint16_t *gtab;   // target groups per angle batch (see launch_project_slice)
    const int *goff;
    const float2 *tw;       // [B] e^{-2 pi i q / B} (upsampled path: [N], the grid's)
    const float2 *tw2;      // upsampled path: [2 N] e^{-2 pi i q / (2 N)} (the rows')
    float2 *grid;           // global grids [chunk][rows][S] (128 < L only)
    float2 *xs;             // global slice samples [chunk][nh][B/2 + 1] (128 < L only)
    const uint32_t *ttab;   // target groups per tile (128 < L only)
    const int *toff;
    float *out;
    int32_t *status;
    SliceCoef coef;         // tap weight polynomials (kernel parameter bank)
    int pf_ahead;           // k_project_slice: CTA b prefetches image b + pf_ahead into L2
};

// Bulk prefetch of [p, p + bytes) into L2 (the 16-byte-aligned part), in
// 32 KB requests.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes)
{
    size_t a = __cvta_generic_to_global(p);
    size_t e = a + bytes;
    a = (a + 15) & ~(size_t)15;
    e &= ~(size_t)15;
    while (a < e) {
        const unsigned chunk = (unsigned)(e - a < 32768 ? e - a : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(chunk) : "memory");
        a += chunk;
    }
}

__device__ __forceinline__ const float *image_of(const SliceArgs &A, int gi)
{
    const size_t sz = (size_t)A.srcL * A.srcL;
    return gi < A.nb1 ? A.img + (size_t)gi * sz : A.img2 + (size_t)(gi - A.nb1) * sz;
}

// Phases A and B for one image into the grid G (shared or global memory),
// by nw warps; returns the image's bad/mass flags of this thread.
__device__ __forceinline__ void cp_async4z(float *dst, const float *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
                 : "memory");
}

// Phases A and B for one image into the grid G (shared or global memory),
// by nw warps; returns the image's bad/mass flags of this thread.  stage
// (shared memory, two bands of L x 33 floats, or null): with 16 warps and no
// upsampling the image passes through it in 32-column bands by cp.async,
// band b + 1 in flight while the warps transform band b (one column pair
// each); otherwise each lane loads its pixels directly.
template <int M>
__device__ __forceinline__ void slice_grid(const SliceArgs &A, const float *__restrict__ src,
                                           float2 *G, const float2 *tw, int warp, int nw,
                                           int lane, int &bad, int &mass, float *stage = nullptr)
{
    constexpr int N = 32 * M;
    const int L = A.L, half = L / 2;
    const int rows = slice_rows(N), S = slice_stride(N), lo = slice_lo(N);
    const int nleft = slice_left(N), nright = slice_right(N);
    // ---- A: one warp per column pair (c, c+1): FFT along r', kept rows.
    // fetch(r) gives the pixels (r, c) and (r, c + 1).
    auto column_pair = [&](int c, auto fetch) {
        float2 v[M];
        const float pc0 = __ldg(A.psi_inv + c), pc1 = c + 1 < L ? __ldg(A.psi_inv + c + 1) : 0.f;
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const int n = 32 * n1 + lane;
            const int r = (n < N / 2 ? n : n - N) + half;
            v[n1] = make_float2(0.f, 0.f);
            if (r >= 0 && r < L) {
                float2 x = fetch(r);
                if (!isfinite(x.x)) {
                    bad = 1;
                    x.x = 0.f;
                }
                if (!isfinite(x.y)) {
                    bad = 1;
                    x.y = 0.f;
                }
                x.x = fmaxf(x.x, 0.f);
                x.y = fmaxf(x.y, 0.f);
                mass |= (x.x > 0.f) | (x.y > 0.f);
                const float pr = __ldg(A.psi_inv + r);
                v[n1] = make_float2(x.x * pc0 * pr, x.y * pc1 * pr);
            }
        }
        warp_ifft<M>(v, tw, lane);
        // Z[kout] = v[k1], kout = k1 + M brev5(lane); Z[-kout] sits on lane
        // brev5(32 - brev5(lane)) slot 0 (k1 = 0), else lane 31 - lane slot M - k1
        const int kb = M * brev5(lane);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            const int sl = k1 == 0 ? 0 : M - k1;
            const int srcl = k1 == 0 ? brev5((32 - brev5(lane)) & 31) : 31 - lane;
            const float2 Z = v[k1];
            const float2 Zc = make_float2(__shfl_sync(0xffffffffu, v[sl].x, srcl),
                                          -__shfl_sync(0xffffffffu, v[sl].y, srcl));
            const int i = wrap_n(k1 + kb - lo, N);  // kept row of l2 = kout (mod N)
            if (i < rows) {
                // column c: (Z + conj Z(-l2)) / 2; column c + 1: (Z - conj Z(-l2)) / (2i)
                G[i * S + c] = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
                if (c + 1 < L)
                    G[i * S + c + 1] = make_float2(0.5f * (Z.y - Zc.y), -0.5f * (Z.x - Zc.x));
            }
        }
    };
    constexpr int BW = 32, RSB = BW + 1;  // band width; staged row stride (odd: rows on distinct banks)
    if (stage != nullptr && A.srcL == L && 2 * nw == BW) {
        const int nbands = (L + BW - 1) / BW;
        auto issue = [&](int b, float *buf) {
            const int cb = b * BW, w = min(BW, L - cb);
            for (int idx = threadIdx.x; idx < L * BW; idx += blockDim.x) {
                const int r = idx / BW, cc = idx % BW;
                const bool ok = cc < w;
                cp_async4z(buf + r * RSB + cc, ok ? src + (size_t)r * L + cb + cc : src, ok ? 4 : 0);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        issue(0, stage);
        for (int b = 0; b < nbands; ++b) {
            if (b + 1 < nbands) issue(b + 1, stage + ((b + 1) & 1) * L * RSB);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncthreads();
            const float *buf = stage + (b & 1) * L * RSB;
            const int c = b * BW + 2 * warp;
            if (c < L)
                column_pair(c, [&](int r) {
                    const float *row = buf + r * RSB + (c - b * BW);
                    return make_float2(row[0], c + 1 < L ? row[1] : 0.f);
                });
            __syncthreads();  // the band's buffer is refilled two bands on
        }
    } else {
        // 8-byte pixel pairs: L even (every row starts 8-byte aligned, c is
        // even) and the image itself 8-byte aligned
        const bool pair8 = (L & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 7) == 0;
        for (int c = 2 * warp; c < L; c += 2 * nw)
            column_pair(c, [&](int r) {
                if (A.srcL == L && pair8) {
                    // (c, c + 1) in one 8-byte load: each lane reads another
                    // row, so every load instruction costs one L1 line request
                    // per lane, and this halves them
                    return __ldg(reinterpret_cast<const float2 *>(src + (size_t)r * L + c));
                } else if (A.srcL == L) {
                    return make_float2(__ldg(src + (size_t)r * L + c),
                                       c + 1 < L ? __ldg(src + (size_t)r * L + c + 1) : 0.f);
                }
                // 2 x 2 upsampling: columns c, c+1 share a source pixel (c even)
                const float x0 = 0.25f * __ldg(src + (size_t)(r >> 1) * A.srcL + (c >> 1));
                return make_float2(x0, c + 1 < L ? x0 : 0.f);
            });
    }
    __syncthreads();
    // ---- B: one warp per kept row: FFT along c', left and right columns
    for (int i = warp; i < rows; i += nw) {
        float2 v[M];
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const int n = 32 * n1 + lane;
            const int c = (n < N / 2 ? n : n - N) + half;
            v[n1] = (c >= 0 && c < L) ? G[i * S + c] : make_float2(0.f, 0.f);
        }
        __syncwarp();
        warp_ifft<M>(v, tw, lane);
        const int kb = M * brev5(lane);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            const int kout = k1 + kb;
            const int q = wrap_n(kout - lo, N);  // left column with l1 = kout (mod N)
            if (q < nleft) G[i * S + q] = v[k1];
            if (kout >= 1 && kout <= nright) G[i * S + nleft + nright - kout] = v[k1];
        }
    }
}

// Tap weights along each axis from the target's offsets (x1, x2) from its
// cell: the degree-8 polynomials of the kernel parameters, evaluated per
// mirrored pair of taps (slice_tap_weights).
__device__ __forceinline__ void slice_weights(const SliceArgs &A, float x1, float x2,
                                              float (&wx)[kSliceW], float (&wy)[kSliceW])
{
    slice_tap_weights(A.coef, x1, wx);
    slice_tap_weights(A.coef, x2, wy);
}

// The same weights by one Horner chain in x per tap, from every row of the
// (mirror-symmetric) coefficient table: 72 FMAs per axis, but fewer values
// live at once, which the upsampled-image kernel needs to stay within its
// registers.
__device__ __forceinline__ void slice_weights_horner(const SliceArgs &A, float x1, float x2,
                                                     float (&wx)[kSliceW], float (&wy)[kSliceW])
{
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
}

// Weights, first tap and value of slice sample (k, j): the W x W taps of the
// exponential-of-semicircle kernel around y = -(j / B) e_k N on the grid,
// times the cell factor fac[k][j].  tap(row, col) returns the grid cell at a
// stored row and column; the footprint is rows row0..row0+W-1 and columns
// col0, col0 + da, ... (da = +1 on the left half, -1 on the right).
template <int M>
__device__ __forceinline__ void slice_target(const SliceArgs &A, int k, int j, int &row0,
                                             int &col0, bool &left, float (&wx)[kSliceW],
                                             float (&wy)[kSliceW])
{
    constexpr int N = 32 * M;
    const float hN = 0.5f * (float)N;
    const float jf = (float)j;
    const float2 e = __ldg(A.cs + k);
    // target y = -t N on the grid (t = (j/B) e, N = B), kept inside the
    // stored half plane whatever the rounding
    const float y1 = fminf(fmaxf(-(jf * e.x), -hN), hN);
    const float y2 = fminf(fmaxf(-(jf * e.y), -hN), 0.f);
    const float f1 = ceilf(y1 - 0.5f * (float)kSliceW);
    const float f2 = ceilf(y2 - 0.5f * (float)kSliceW);
    // offsets from the cell, exact: y - f is in (W/2 - 1, W/2]
    const float x1 = (y1 - f1) - (float)(kSliceW / 2);
    const float x2 = (y2 - f2) - (float)(kSliceW / 2);
    slice_weights(A, x1, x2, wx, wy);
    const int i1 = (int)f1;
    row0 = (int)f2 - slice_lo(N);
    // left half: taps at increasing addresses; right half reversed
    left = i1 <= 0;
    col0 = left ? i1 - slice_lo(N) : slice_left(N) + slice_right(N) - i1;
}

// The same for a target of an image of side L/2 seen as L x L (grid of the
// L/2 image, N = 32 M points; j <= N): the first tap wrapped and folded by
// slice_up_tap; conj tells that the taps give conj T.
template <int M>
__device__ __forceinline__ void slice_target_up(const SliceArgs &A, int k, int j, int &row0,
                                                int &col0, bool &left, bool &conj,
                                                float (&wx)[kSliceW], float (&wy)[kSliceW])
{
    constexpr int N = 32 * M;
    const float2 e = __ldg(A.cs + k);
    int i1, i2;
    float x1, x2;
    slice_up_tap(j, e.x, e.y, N, &i1, &i2, &x1, &x2, &conj);
    slice_weights_horner(A, x1, x2, wx, wy);
    row0 = i2 - slice_lo(N);
    left = i1 <= 0;
    col0 = left ? i1 - slice_lo(N) : slice_left(N) + slice_right(N) - i1;
}

// Plain or upsampled-image target (see slice_target, slice_target_up).
template <int M, bool UP>
__device__ __forceinline__ void slice_target_any(const SliceArgs &A, int k, int j, int &row0,
                                                 int &col0, bool &left, bool &conj,
                                                 float (&wx)[kSliceW], float (&wy)[kSliceW])
{
    if constexpr (UP) {
        slice_target_up<M>(A, k, j, row0, col0, left, conj, wx, wy);
    } else {
        conj = false;
        slice_target<M>(A, k, j, row0, col0, left, wx, wy);
    }
}

// fc * T, or fc * conj(T)
__device__ __forceinline__ float2 slice_scale(float2 fc, float2 t, bool conj)
{
    if (conj) t.y = -t.y;
    return make_float2(fc.x * t.x - fc.y * t.y, fc.x * t.y + fc.y * t.x);
}

// sum_b wy[b] sum_a wx[a] g[b S + a da], complex, times fac
__device__ __forceinline__ float2 slice_sum(const float2 *g, int S, int da,
                                            const float (&wx)[kSliceW],
                                            const float (&wy)[kSliceW], float2 fc)
{
    float tr = 0.f, ti = 0.f;
#pragma unroll
    for (int b = 0; b < kSliceW; ++b) {
        float rr = 0.f, ri = 0.f;
#pragma unroll
        for (int a = 0; a < kSliceW; ++a) {
            const float2 gv = g[b * S + a * da];
            rr = fmaf(wx[a], gv.x, rr);
            ri = fmaf(wx[a], gv.y, ri);
        }
        tr = fmaf(wy[b], rr, tr);
        ti = fmaf(wy[b], ri, ti);
    }
    return make_float2(fc.x * tr - fc.y * ti, fc.x * ti + fc.y * tr);
}

// Tap sums of two ray-adjacent slice samples A = (k, j) and B = (k, j + 1)
// whose footprints start DRA / DRB rows and DCA / DCB columns into their
// union box (each 0 or 1, one of each pair 0): every cell of the box is
// loaded once and added to the sample(s) whose 9 x 9 footprint holds it.
// The offsets are compile-time, so no weight is selected at run time.
template <int DRA, int DRB, int DCA, int DCB>
__device__ __forceinline__ void pair_taps(const float2 *__restrict__ g, int S, int da,
                                          const float (&wxA)[kSliceW], const float (&wyA)[kSliceW],
                                          const float (&wxB)[kSliceW], const float (&wyB)[kSliceW],
                                          float2 &tA, float2 &tB)
{
    constexpr int W = kSliceW;
    constexpr int NR = W + (DRA | DRB), NC = W + (DCA | DCB);
    float tAr = 0.f, tAi = 0.f, tBr = 0.f, tBi = 0.f;
#pragma unroll
    for (int b = 0; b < NR; ++b) {
        const bool rowA = b >= DRA && b < DRA + W, rowB = b >= DRB && b < DRB + W;
        float sAr = 0.f, sAi = 0.f, sBr = 0.f, sBi = 0.f;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const float2 gv = g[b * S + a * da];
            if (rowA && a >= DCA && a < DCA + W) {
                sAr = fmaf(wxA[a - DCA], gv.x, sAr);
                sAi = fmaf(wxA[a - DCA], gv.y, sAi);
            }
            if (rowB && a >= DCB && a < DCB + W) {
                sBr = fmaf(wxB[a - DCB], gv.x, sBr);
                sBi = fmaf(wxB[a - DCB], gv.y, sBi);
            }
        }
        if (rowA) {
            tAr = fmaf(wyA[b - DRA], sAr, tAr);
            tAi = fmaf(wyA[b - DRA], sAi, tAi);
        }
        if (rowB) {
            tBr = fmaf(wyB[b - DRB], sBr, tBr);
            tBi = fmaf(wyB[b - DRB], sBi, tBi);
        }
    }
    tA = make_float2(tAr, tAi);
    tB = make_float2(tBr, tBi);
}

// Two ray-adjacent slice samples (k, j) and (k, j + 1) of one half of the
// grid, whose footprints start at most one row and one column apart (the
// host pairs only such targets: consecutive samples on a ray are one grid
// cell apart): their union box of at most 10 x 10 taps is read once for
// both, against 162 reads for two separate samples.  The footprints' offsets
// in the box select one of nine compile-time tap patterns; the host groups
// the pairs so that every warp takes one pattern.
template <int M, bool UP>
__device__ __forceinline__ void slice_pair(const SliceArgs &A, const float2 *G, int S, int k,
                                           int j, float2 &outA, float2 &outB)
{
    constexpr int W = kSliceW;
    float wxA[W], wyA[W], wxB[W], wyB[W];
    int rA, cA, rB, cB;
    bool lA, lB, zA, zB;
    slice_target_any<M, UP>(A, k, j, rA, cA, lA, zA, wxA, wyA);
    slice_target_any<M, UP>(A, k, j + 1, rB, cB, lB, zB, wxB, wyB);
    const int da = lA ? 1 : -1;  // both in the same half (host-checked)
    const int r0 = min(rA, rB);
    const int c0 = lA ? min(cA, cB) : max(cA, cB);
    // pattern: rows (A below B, B below A, level), columns likewise
    const int pr = rA > rB ? 1 : (rB > rA ? 2 : 0);
    const int pc = cA != c0 ? 1 : (cB != c0 ? 2 : 0);
    const float2 *g = G + r0 * S + c0;
    float2 tA, tB;
#define SW_PAIR_CASE(PR, PC, DRA, DRB, DCA, DCB)                                          \
    case PR * 3 + PC:                                                                      \
        pair_taps<DRA, DRB, DCA, DCB>(g, S, da, wxA, wyA, wxB, wyB, tA, tB);              \
        break;
    switch (pr * 3 + pc) {
        SW_PAIR_CASE(0, 0, 0, 0, 0, 0)
        SW_PAIR_CASE(0, 1, 0, 0, 1, 0)
        SW_PAIR_CASE(0, 2, 0, 0, 0, 1)
        SW_PAIR_CASE(1, 0, 1, 0, 0, 0)
        SW_PAIR_CASE(1, 1, 1, 0, 1, 0)
        SW_PAIR_CASE(1, 2, 1, 0, 0, 1)
        SW_PAIR_CASE(2, 0, 0, 1, 0, 0)
        SW_PAIR_CASE(2, 1, 0, 1, 1, 0)
        default: pair_taps<0, 1, 0, 1>(g, S, da, wxA, wyA, wxB, wyB, tA, tB); break;
    }
#undef SW_PAIR_CASE
    const int nj = (UP ? 32 : 16) * M + 1;
    const float2 fa = __ldg(A.fac + (size_t)k * nj + j), fb = __ldg(A.fac + (size_t)k * nj + j + 1);
    outA = slice_scale(fa, tA, zA);
    outB = slice_scale(fb, tB, zB);
}

// Phase C for the angles [k0, k0 + BATCH) of the grid G (shared memory):
// the slice samples into Xs [BATCH][B/2 + 1]; ends with a block barrier.
// An entry with kSlicePairBit set computes the pair (j, j + 1).  UP: G is
// the grid of an image of side L/2 (N = 32 M = B/2 points), the samples
// j <= N those of its 2 x 2 upsampled image (slice_target_up).
template <int M, int BATCH, bool UP = false>
__device__ __forceinline__ void slice_samples(const SliceArgs &A, const float2 *G, float2 *Xs,
                                              int k0, int bi)
{
    constexpr int N = 32 * M;
    const int nh = A.nh;
    const int S = slice_stride(N);
    const int nj = (UP ? N : N / 2) + 1;
    // rows of angles beyond nh (last batch) read as zero
    for (int it = threadIdx.x + (nh - k0) * nj; it < BATCH * nj; it += blockDim.x)
        Xs[it] = make_float2(0.f, 0.f);
    const int g0 = __ldg(A.goff + bi), ng = __ldg(A.goff + bi + 1) - g0;
    for (int slot = threadIdx.x; slot < ng * 16; slot += blockDim.x) {
        const unsigned ent = __ldg(A.gtab + (size_t)(g0 + (slot >> 4)) * 16 + (slot & 15));
        if (ent == 0xFFFFu) continue;
        const int kk = (int)((ent >> 8) & 63u), j = (int)(ent & 255u);
        const int k = k0 + kk;
        if (ent & kSlicePairBit) {
            float2 xa, xb;
            slice_pair<M, UP>(A, G, S, k, j, xa, xb);
            Xs[kk * nj + j] = xa;
            Xs[kk * nj + j + 1] = xb;
            continue;
        }
        float wx[kSliceW], wy[kSliceW];
        int row0, col0;
        bool left, conj;
        slice_target_any<M, UP>(A, k, j, row0, col0, left, conj, wx, wy);
        float2 fc = __ldg(A.fac + (size_t)k * nj + j);
        // fc conj(T) = conj(conj(fc) T)
        if (conj) fc.y = -fc.y;
        float2 x = slice_sum(G + row0 * S + col0, S, left ? 1 : -1, wx, wy, fc);
        if (conj) x.y = -x.y;
        Xs[kk * nj + j] = x;
    }
    __syncthreads();
}

// Phase D for the angles [k0, k0 + BATCH) of image gi from the slice samples
// Xs; tw in shared memory; BATCH / 2 warps.  Ends with a block barrier.
template <int M, int BATCH>
__device__ __forceinline__ void slice_rows_out(const SliceArgs &A, float2 *Xs, const float2 *tw,
                                               int gi, int k0, int warp, int lane)
{
    constexpr int N = 32 * M;
    const int nh = A.nh;
    const int nj = N / 2 + 1;
    const float invB = 1.f / (float)N;
    const int nrow = A.full_n ? 2 * nh : nh;
    float *outi = A.out + (size_t)gi * nrow * N;
    // D: warp w inverse-transforms the angles ka = 2w, kb = 2w + 1 of the
    // batch as Y_j = X_a + i X_b, Y_{B-j} = conj X_a + i conj X_b
    // (Y_0, Y_{B/2}: real parts), then writes both rows
    const int ka = 2 * warp;
    if (ka < BATCH && k0 + ka < nh) {
        const float2 *Xa = Xs + ka * nj, *Xb = Xa + nj;
        float2 v[M];
#pragma unroll
        for (int n1 = 0; n1 < M; ++n1) {
            const int n = 32 * n1 + lane;
            const int j = n <= N / 2 ? n : N - n;
            const float2 a = Xa[j], b = Xb[j];
            if (n == 0 || 2 * n == N) v[n1] = make_float2(a.x, b.x);
            else if (n < N / 2) v[n1] = make_float2(a.x - b.y, a.y + b.x);
            else v[n1] = make_float2(a.x + b.y, b.x - a.y);
        }
        __syncwarp();
        warp_ifft<M>(v, tw, lane);
        // stage the two rows in this warp's own sample rows (2 nj >= B + 2)
        float *stw = reinterpret_cast<float *>(Xs + ka * nj);
        const int kb = M * brev5(lane);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) {
            stw[k1 + kb] = v[k1].x * invB;
            stw[N + k1 + kb] = v[k1].y * invB;
        }
        __syncwarp();
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int k = k0 + ka + h2;
            if (k >= nh) break;
            float *o = outi + (size_t)k * N;
            float *om = outi + (size_t)(nh + k) * N + (N - 1);
            for (int b = lane; b < N; b += 32) {
                float val = stw[h2 * N + b];
                if (A.clip) val = fmaxf(val, 0.f);
                o[b] = val;
                if (A.full_n) om[-b] = val;
            }
        }
    }
    __syncthreads();
}

// L <= 128: one CTA per image, the grid in shared memory.
template <int M>
__global__ void __launch_bounds__(kSliceThreads, 1) k_project_slice(SliceArgs A)
{
    constexpr int N = 32 * M;
    extern __shared__ float2 sms[];
    const int nj = N / 2 + 1;
    float2 *G = sms;                                        // [rows][S] grid
    float2 *Xs = G + slice_rows(N) * slice_stride(N);       // [kSliceBatch][nj]
    float2 *tw = Xs + kSliceBatch * nj;                     // [N]
    __shared__ int s_bad, s_mass;
    const int gi = A.img_off + blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_mass = 0;
        // one CTA per SM: the image that starts about one CTA lifetime from
        // now is pulled into L2, so that its phase-A loads hit there
        if (A.pf_ahead > 0 && blockIdx.x + A.pf_ahead < gridDim.x)
            prefetch_l2(image_of(A, gi + A.pf_ahead), sizeof(float) * A.srcL * A.srcL);
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = A.tw[i];
    __syncthreads();
    int bad = 0, mass = 0;
    slice_grid<M>(A, image_of(A, gi), G, tw, warp, kSliceThreads / 32, lane, bad, mass);
    if (bad) atomicOr(&s_bad, 1);
    if (mass) atomicOr(&s_mass, 1);
    __syncthreads();
    if (threadIdx.x == 0) A.status[gi] = (s_bad || !s_mass) ? 1 : 0;
    for (int k0 = 0; k0 < A.nh; k0 += kSliceBatch) {
        slice_samples<M, kSliceBatch>(A, G, Xs, k0, k0 / kSliceBatch);
        slice_rows_out<M, kSliceBatch>(A, Xs, tw, gi, k0, warp, lane);
    }
}

// Images of side L/2 upsampled 2 x 2 (128 < L): one CTA per image with the
// grid of the L/2 image (N = 32 MG = B/2 points, A.L = A.srcL = L/2) in
// shared memory, the slice samples j <= N of the L x L image from it in
// kUpBatch-angle batches (slice_samples<UP>), and rows of B = 2 N bins.
template <int MG>
__global__ void __launch_bounds__(kSliceThreads, 1) k_project_slice_up(SliceArgs A)
{
    constexpr int N = 32 * MG;
    constexpr int nj = N + 1;
    extern __shared__ float2 sms[];
    float2 *G = sms;                                        // [rows][S] grid
    float2 *Xs = G + slice_rows(N) * slice_stride(N);       // [kUpBatch][nj]
    float2 *tw = Xs + kUpBatch * nj;                        // [N]
    float2 *tw2 = tw + N;                                   // [2 N]
    __shared__ int s_bad, s_mass;
    const int gi = A.img_off + blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_mass = 0;
        if (A.pf_ahead > 0 && blockIdx.x + A.pf_ahead < gridDim.x)
            prefetch_l2(image_of(A, gi + A.pf_ahead), sizeof(float) * A.srcL * A.srcL);
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = A.tw[i];
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) tw2[i] = A.tw2[i];
    __syncthreads();
    int bad = 0, mass = 0;
    slice_grid<MG>(A, image_of(A, gi), G, tw, warp, kSliceThreads / 32, lane, bad, mass);
    if (bad) atomicOr(&s_bad, 1);
    if (mass) atomicOr(&s_mass, 1);
    __syncthreads();
    if (threadIdx.x == 0) A.status[gi] = (s_bad || !s_mass) ? 1 : 0;
    for (int k0 = 0; k0 < A.nh; k0 += kUpBatch) {
        slice_samples<MG, kUpBatch, true>(A, G, Xs, k0, k0 / kUpBatch);
        slice_rows_out<2 * MG, kUpBatch>(A, Xs, tw2, gi, k0, warp, lane);
    }
}

// 128 < L: the grid of image img_off + blockIdx.x into A.grid[blockIdx.x].
template <int M>
__global__ void __launch_bounds__(kBigThreads, 2) k_slice_grid(SliceArgs A)
{
    constexpr int N = 32 * M;
    __shared__ float2 tw[N];
    __shared__ int s_bad, s_mass;
    const int gi = A.img_off + blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_mass = 0;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = A.tw[i];
    __syncthreads();
    extern __shared__ float stg[];  // [2][L][33] image bands (not upsampled)
    float2 *G = A.grid + (size_t)blockIdx.x * slice_rows(N) * slice_stride(N);
    int bad = 0, mass = 0;
    slice_grid<M>(A, image_of(A, gi), G, tw, warp, kBigThreads / 32, lane, bad, mass,
                  A.srcL == A.L ? stg : nullptr);
    if (bad) atomicOr(&s_bad, 1);
    if (mass) atomicOr(&s_mass, 1);
    __syncthreads();
    if (threadIdx.x == 0) A.status[gi] = (s_bad || !s_mass) ? 1 : 0;
}

// 128 < L: the slice samples whose footprints start in tile blockIdx.x of
// the grid A.grid[blockIdx.y], with the tile and its halo in shared memory,
// into A.xs[blockIdx.y].
template <int M>
__global__ void __launch_bounds__(kBigThreads) k_slice_tile(SliceArgs A)
{
    constexpr int N = 32 * M;
    constexpr int TS = kSliceTileSpan, RS = kSliceTileRS;
    __shared__ float2 T[TS * RS];
    const int rows = slice_rows(N), S = slice_stride(N), nj = N / 2 + 1;
    const int tile = blockIdx.x;
    const int r0 = (tile / slice_tiles_x(N)) * kSliceTile, c0 = (tile % slice_tiles_x(N)) * kSliceTile;
    const int g0 = __ldg(A.toff + tile), ng = __ldg(A.toff + tile + 1) - g0;
    if (ng == 0) return;  // no footprint starts here (whole CTA)
    const float2 *G = A.grid + (size_t)blockIdx.y * rows * S;
    float2 *X = A.xs + (size_t)blockIdx.y * A.nh * nj;
    for (int idx = threadIdx.x; idx < TS * TS; idx += blockDim.x) {
        const int r = idx / TS, c = idx % TS;
        const int gr = r0 + r, gc = c0 + c;
        T[r * RS + c] = (gr < rows && gc < S) ? G[(size_t)gr * S + gc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int slot = threadIdx.x; slot < ng * 16; slot += blockDim.x) {
        const uint32_t ent = __ldg(A.ttab + (size_t)(g0 + (slot >> 4)) * 16 + (slot & 15));
        if (ent == 0xFFFFFFFFu) continue;
        const int k = (int)(ent >> 16), j = (int)(ent & 0xFFFFu);
        float wx[kSliceW], wy[kSliceW];
        int row0, col0;
        bool left;
        slice_target<M>(A, k, j, row0, col0, left, wx, wy);
        const int da = left ? 1 : -1;
        const int lr = row0 - r0, lc = col0 - c0;
        const int cmin = left ? lc : lc - (kSliceW - 1);
        const float2 fc = __ldg(A.fac + (size_t)k * nj + j);
        // the host assigned the footprint to this tile; should the rounding
        // ever place it elsewhere, the taps are read from the global grid
        const bool inside = lr >= 0 && lr + kSliceW <= TS && cmin >= 0 && cmin + kSliceW <= TS;
        X[(size_t)k * nj + j] = inside ? slice_sum(T + lr * RS + lc, RS, da, wx, wy, fc)
                                       : slice_sum(G + (size_t)row0 * S + col0, S, da, wx, wy, fc);
    }
}

// 128 < L: rows of angle batch blockIdx.x of image img_off + blockIdx.y from
// the slice samples A.xs[blockIdx.y].
template <int M>
__global__ void __launch_bounds__(kBigThreads, 2) k_slice_rows(SliceArgs A)
{
    constexpr int N = 32 * M;
    constexpr int nj = N / 2 + 1;
    extern __shared__ float2 sms[];
    float2 *Xs = sms;                   // [kBigBatch][nj]
    float2 *tw = Xs + kBigBatch * nj;   // [N]
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = A.tw[i];
    const int k0 = blockIdx.x * kBigBatch;
    const float2 *X = A.xs + ((size_t)blockIdx.y * A.nh + k0) * nj;
    const int valid = min(kBigBatch, A.nh - k0) * nj;
    for (int it = threadIdx.x; it < kBigBatch * nj; it += blockDim.x)
        Xs[it] = it < valid ? X[it] : make_float2(0.f, 0.f);
    __syncthreads();
    slice_rows_out<M, kBigBatch>(A, Xs, tw, A.img_off + blockIdx.y, k0, threadIdx.x >> 5,
                                 threadIdx.x & 31);
}

template <int M>
cudaError_t launch_small(SliceArgs a, int nb, cudaStream_t st)
{
    const size_t smem = slice_smem_bytes(32 * M);
    cudaError_t e = cudaFuncSetAttribute(k_project_slice<M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        a.pf_ahead = sms;  // resident CTAs: one per SM
    k_project_slice<M><<<nb, kSliceThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int MG>
cudaError_t launch_up(SliceArgs a, int nb, cudaStream_t st)
{
    const size_t smem = slice_up_smem_bytes(64 * MG);
    cudaError_t e = cudaFuncSetAttribute(k_project_slice_up<MG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        a.pf_ahead = sms;
    k_project_slice_up<MG><<<nb, kSliceThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int M>
cudaError_t launch_big(SliceArgs a, int nb, int chunk, cudaStream_t st)
{
    constexpr int N = 32 * M;
    const int nbatch = (a.nh + kBigBatch - 1) / kBigBatch;
    const int ntiles = slice_tiles_y(N) * slice_tiles_x(N);
    const size_t smem = sizeof(float2) * ((size_t)kBigBatch * (N / 2 + 1) + N);
    cudaError_t e = cudaFuncSetAttribute(k_slice_rows<M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // two 32-column bands of the image (rows 33 floats apart) when not upsampled
    const size_t smem_grid = a.srcL == a.L ? sizeof(float) * 2 * (size_t)a.L * 33 : 0;
    e = cudaFuncSetAttribute(k_slice_grid<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_grid);
    if (e != cudaSuccess) return e;
    // chunks of equal size (at most `chunk`): no small last chunk whose
    // launches would leave most SMs idle
    const int nchunks = (nb + chunk - 1) / chunk;
    chunk = (nb + nchunks - 1) / nchunks;
    for (int i0 = 0; i0 < nb; i0 += chunk) {
        const int cnt = std::min(chunk, nb - i0);
        a.img_off = i0;
        k_slice_grid<M><<<cnt, kBigThreads, smem_grid, st>>>(a);
        k_slice_tile<M><<<dim3(ntiles, cnt), kBigThreads, 0, st>>>(a);
        k_slice_rows<M><<<dim3(nbatch, cnt), kBigThreads, smem, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

int slice_default_bins(int L, int min_bins)
{
    const int need = std::max(min_bins, (3 * L + 1) / 2);  // >= the default bins and 1.5 L
    int m = (need + 31) / 32;
    if (m > 6) m = m <= 8 ? 8 : (m <= 10 ? 10 : 12);  // grids in global memory: 256, 320, 384
    return 32 * m;
}

bool slice_bins_supported(int L, int B)
{
    if (B % 32 || 2 * B < 3 * L) return false;
    const int m = B / 32;
    return L <= 128 ? (m >= 1 && m <= 6 && slice_smem_bytes(B) <= kSliceSmemMax)
                    : (L <= 256 && (m == 8 || m == 10 || m == 12));
}

size_t slice_smem_bytes(int B)
{
    return sizeof(float2) * ((size_t)slice_rows(B) * slice_stride(B) +
                             (size_t)kSliceBatch * (B / 2 + 1) + (size_t)B);
}

int slice_batch_of(int L) { return L <= 128 ? kSliceBatch : kBigBatch; }

size_t slice_up_smem_bytes(int B)
{
    const int N = B / 2;
    return sizeof(float2) * ((size_t)slice_rows(N) * slice_stride(N) +
                             (size_t)kUpBatch * (N + 1) + 3 * (size_t)N);
}

bool slice_up_supported(int L, int B)
{
    return L > 128 && (L & 1) == 0 && slice_bins_supported(L, B) && (B / 2) % 32 == 0 &&
           slice_bins_supported(L / 2, B / 2) && slice_up_smem_bytes(B) <= kSliceSmemMax;
}

size_t slice_scratch_bytes(int L, int B, int nb, int nh)
{
    if (L <= 128) return 0;
    return sizeof(float2) * ((size_t)slice_rows(B) * slice_stride(B) + (size_t)nh * (B / 2 + 1)) *
           (size_t)std::min(nb, kSliceChunk);
}

cudaError_t launch_project_slice(const float *img, int nb, int L, int srcL, int nh, int B,
                                 const float2 *cs, const float *psi_inv, const float2 *fac,
                                 const uint16_t *gtab, const int *goff, const uint32_t *ttab,
                                 const int *toff, const SliceCoef &coef, const float2 *tw,
                                 float2 *scratch, int clip, float *out, int full_n,
                                 int32_t *status, cudaStream_t st, const float *img2,
                                 int nb_first)
{
    if (nb <= 0) return cudaSuccess;
    if (!slice_bins_supported(L, B)) return cudaErrorInvalidValue;
    SliceArgs a;
    a.img = img;
    a.img2 = img2 ? img2 : img;
    a.nb1 = (img2 && nb_first >= 0) ? nb_first : nb;
    a.img_off = 0;
    a.pf_ahead = 0;
    a.L = L;
    a.srcL = srcL;
    a.nh = nh;
    a.coef = coef;
    a.fac = fac;
    a.gtab = gtab;
    a.goff = goff;
    a.tw = tw;
    a.tw2 = nullptr;
    a.grid = scratch;
    a.xs = scratch ? scratch + (size_t)slice_rows(B) * slice_stride(B) * std::min(nb, kSliceChunk)
                   : nullptr;
    a.ttab = ttab;
    a.toff = toff;
    a.clip = clip;
    a.full_n = full_n;
    a.cs = cs;
    a.psi_inv = psi_inv;
    a.out = out;
    a.status = status;
    if (L > 128) {
        if (!scratch || !ttab || !toff) return cudaErrorInvalidValue;
        switch (B / 32) {
        case 8: return launch_big<8>(a, nb, kSliceChunk, st);
        case 10: return launch_big<10>(a, nb, kSliceChunk, st);
        case 12: return launch_big<12>(a, nb, kSliceChunk, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (B / 32) {
    case 1: return launch_small<1>(a, nb, st);
    case 2: return launch_small<2>(a, nb, st);
    case 3: return launch_small<3>(a, nb, st);
    case 4: return launch_small<4>(a, nb, st);
    case 5: return launch_small<5>(a, nb, st);
    case 6: return launch_small<6>(a, nb, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_project_slice_up(const float *img, int nb, int L, int nh, int B,
                                    const float2 *cs, const SliceUpTables &up,
                                    const SliceCoef &coef, const float2 *tw_rows, int clip,
                                    float *out, int full_n, int32_t *status, cudaStream_t st,
                                    const float *img2, int nb_first)
{
    if (nb <= 0) return cudaSuccess;
    if (!slice_up_supported(L, B) || !up.psi_inv || !up.fac || !up.gtab || !up.goff || !up.tw ||
        !tw_rows)
        return cudaErrorInvalidValue;
    SliceArgs a{};
    a.img = img;
    a.img2 = img2 ? img2 : img;
    a.nb1 = (img2 && nb_first >= 0) ? nb_first : nb;
    a.img_off = 0;
    a.pf_ahead = 0;
    a.L = L / 2;
    a.srcL = L / 2;
    a.nh = nh;
    a.coef = coef;
    a.fac = up.fac;
    a.gtab = up.gtab;
    a.goff = up.goff;
    a.tw = up.tw;
    a.tw2 = tw_rows;
    a.grid = nullptr;
    a.xs = nullptr;
    a.ttab = nullptr;
    a.toff = nullptr;
    a.clip = clip;
    a.full_n = full_n;
    a.cs = cs;
    a.psi_inv = up.psi_inv;
    a.out = out;
    a.status = status;
    switch (B / 64) {
    case 4: return launch_up<4>(a, nb, st);
    case 5: return launch_up<5>(a, nb, st);
    case 6: return launch_up<6>(a, nb, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace swk
