// sw_decide.cu -- second half of the FFT cross-correlation of Sec. 2.3
// ("Fast computation over rotations") and the alignment decision
// (Eq. optimal_rotation, Eq. discrete_rot_sw2).
//
// For a pair (i, j) with correlation spectra C(k'), k' = 1..n/2:
//   corr'(l) = (1/n) sum_{k' != 0} C(k') e^{2 pi i k' l / n}     (inverse FFT)
//   n M D_T(l) = n |m_i - m_j|^2 + N_i + N_j - 2 corr'(l)
// where m is the profile (mean over angle of each quantile level), N the
// centred, mean-free quantile norm, and the k' = 0 part n|m_i - m_j|^2 is a
// direct difference.  Without translation the distance is
// D_0(l) = D_T(l) + |s*(l)|^2 / 2, s*(l) = a_i - R_{alpha_l} a_j.
// l* = argmin (lowest l on ties) is taken on FP32 values; the distance at l*
// is formed in FP64.
//
// Two real correlation curves are packed in one complex inverse FFT (the
// curves are real, so the spectrum of c_a + i c_b is C_a + i C_b extended by
// Hermitian symmetry).  Two forms:
//  - register form (n = 64, 128, 256, 512): one CTA per (query, 16
//    templates), the block of spectra staged in shared memory by cp.async,
//    then one warp per curve pair: the length-n transform lives in the
//    warp's registers (an in-lane radix-2 pass, twiddles, five shuffle
//    stages), and the argmin is a warp reduction.  No block barrier after
//    the staging.
//  - shared-memory form (any n): one CTA per (query, 2*nsig templates), the
//    mixed-radix Stockham FFT of the library over nsig signals.
#include "sw_internal.cuh"
#include "swalign.h"

namespace swk {
namespace {

constexpr int kDecThreads = 256;

// Shift restriction (FP64): (sx, sy) holds the closed-form optimum c.
// tmode 0 (rotation only): the shift is 0 and d grows by rho |c|^2;
// tmode 2 (grid): the shift is the grid point g nearest c (clamped to
// |i|, |j| <= K) and d grows by rho |g - c|^2; tmode 1: unchanged.
__device__ __forceinline__ void restrict_shift(int tmode, int K, double step, double rho,
                                               double &sx, double &sy, double &d)
{
    if (tmode == 0) {
        d += rho * (sx * sx + sy * sy);
        sx = sy = 0.0;
    } else if (tmode == 2) {
        const double gx = fmin(fmax(rint(sx / step), -(double)K), (double)K) * step;
        const double gy = fmin(fmax(rint(sy / step), -(double)K), (double)K) * step;
        d += rho * ((sx - gx) * (sx - gx) + (sy - gy) * (sy - gy));
        sx = gx;
        sy = gy;
    }
}

// Centre of image idx for the decision: parts = 1: (a, 0); parts = 2 (two
// parts with vectors a+ and a-, centre array [..][2][2]): abar = (a+ + a-)/2
// (the joint translation is s* = abar_i - R abar_j) and d = a+ - a-.
__device__ __forceinline__ void centre_of(const double *ctr, int idx, int parts, double &ax,
                                          double &ay, double &dx, double &dy)
{
    if (parts == 1) {
        ax = ctr[2 * idx];
        ay = ctr[2 * idx + 1];
        dx = dy = 0.0;
    } else {
        const double *c = ctr + 4 * (size_t)idx;
        ax = 0.5 * (c[0] + c[2]);
        ay = 0.5 * (c[1] + c[3]);
        dx = c[0] - c[2];
        dy = c[1] - c[3];
    }
}

// Terms of the argmin key that depend on the rotation (FP32: they only rank
// the rotations; the distance at l* is formed again in FP64).
struct XtraTerms {
    int tmode;         // 0 rotation only, 1 closed-form shift, 2 shift grid
    bool rot_t;        // a shift term is present
    float gstep, ginv, gk;
    float hnm, qnm;    // (1/2 or 1) n M and n M / 4
    float aix, aiy, dix, diy;
};

// The query's centre (aix, aiy, dix, diy) in FP32.
template <int PARTS, bool XTRA>
__device__ __forceinline__ XtraTerms xtra_terms(const DecideArgs &A, float aix, float aiy,
                                                float dix, float diy)
{
    XtraTerms X;
    X.tmode = !XTRA ? 1 : (!A.translation ? 0 : (A.grid_k > 0 ? 2 : 1));
    X.rot_t = XTRA && X.tmode != 1;
    X.gstep = A.gstep;
    X.ginv = A.ginv;
    X.gk = A.gk;
    X.hnm = A.hnm;
    X.qnm = A.qnm;
    X.aix = aix;
    X.aiy = aiy;
    X.dix = dix;
    X.diy = diy;
    return X;
}

// Key k of one pair at alpha_l = (c, sn) plus rc |s - c(l)|^2, c(l) =
// abar_i - R abar_j, s = 0 (rotation only) or the grid point nearest c(l),
// and (two parts) |d_i - R d_j|^2 / 4 scaled by n M.  (ax, ay), (ex, ey):
// the template's abar and d.
template <int PARTS>
__device__ __forceinline__ float xtra_key(float k, const XtraTerms &X, float c, float sn,
                                          float ax, float ay, float ex, float ey)
{
    if (X.rot_t) {
        float sx = X.aix - (c * ax - sn * ay), sy = X.aiy - (sn * ax + c * ay);
        if (X.tmode == 2) {
            sx -= fminf(fmaxf(rintf(sx * X.ginv), -X.gk), X.gk) * X.gstep;
            sy -= fminf(fmaxf(rintf(sy * X.ginv), -X.gk), X.gk) * X.gstep;
        }
        k = fmaf(X.hnm, sx * sx + sy * sy, k);
    }
    if (PARTS == 2) {
        const float sx = X.dix - (c * ex - sn * ey), sy = X.diy - (sn * ex + c * ey);
        k = fmaf(X.qnm, sx * sx + sy * sy, k);
    }
    return k;
}

// FP64 distance and shift of a pair at rotation l from rval = n corr(l);
// base = n |m_i - m_j|^2 + N_i + N_j.
template <int PARTS>
__device__ __forceinline__ double pair_distance(const DecideArgs &A, int l, float rval,
                                                double base, int tmode, double aix, double aiy,
                                                double dix, double diy, double ajx, double ajy,
                                                double djx, double djy, double &sx, double &sy)
{
    const double corr = (double)rval * A.inv_n;
    const double2 c = A.cs64[l];
    sx = aix - (c.x * ajx - c.y * ajy);
    sy = aiy - (c.y * ajx + c.x * ajy);
    double d = (base - 2.0 * corr) * A.inv_nM;
    if (PARTS == 2) {
        const double ex = dix - (c.x * djx - c.y * djy);
        const double ey = diy - (c.y * djx + c.x * djy);
        d += 0.25 * (ex * ex + ey * ey);
    }
    restrict_shift(tmode, A.grid_k, A.grid_step, PARTS == 2 ? 1.0 : 0.5, sx, sy, d);
    return d;
}

// The result of pair (i, j): rotation bl (>= n when every key was NaN),
// rval = n corr(bl), delta = n |m_i - m_j|^2, bad_t: template j unusable.
template <int PARTS>
__device__ __forceinline__ void write_result(const DecideArgs &A, int i, int j, int bl,
                                             float rval, float delta, int bad_t, int tmode,
                                             double aix, double aiy, double dix, double diy)
{
    if (bl >= A.n) bl = 0;  // keep the index in range
    const int st = A.st_q[i] ? 1 : (bad_t ? 2 : ((A.dev_err && *A.dev_err) ? 3 : 0));
    sw_result r;
    if (st) {
        const double nan = __longlong_as_double(0x7ff8000000000000ULL);
        r.best_l = -1;
        r.status = st;
        r.angle_rad = __int_as_float(0x7fc00000);
        r.shift[0] = r.shift[1] = nan;
        r.d2 = nan;
    } else {
        double ajx, ajy, djx, djy;
        centre_of(A.ctr_t, j, PARTS, ajx, ajy, djx, djy);
        const double base = (double)delta + A.norm_q[i] + A.norm_t[j];
        double sx, sy;
        r.d2 = pair_distance<PARTS>(A, bl, rval, base, tmode, aix, aiy, dix, diy, ajx, ajy, djx,
                                    djy, sx, sy);
        r.best_l = bl;
        r.status = 0;
        r.angle_rad = (float)(A.dalpha * bl);
        r.shift[0] = sx;
        r.shift[1] = sy;
    }
    r.template_index = j;
    reinterpret_cast<sw_result *>(A.out)[(size_t)i * A.Nt + j] = r;
}

// Point l of the full curve of pair (0, 0) (single-pair call).
template <int PARTS>
__device__ __forceinline__ void curve_point(const DecideArgs &A, int l, float rval, double base,
                                            int st, int tmode, double aix, double aiy, double dix,
                                            double diy, double ajx, double ajy, double djx,
                                            double djy)
{
    double sx, sy;
    const double d = pair_distance<PARTS>(A, l, rval, base, tmode, aix, aiy, dix, diy, ajx, ajy,
                                          djx, djy, sx, sy);
    A.curve[l] = st ? __longlong_as_double(0x7ff8000000000000ULL) : d;
    if (A.shifts) {
        A.shifts[2 * l] = sx;
        A.shifts[2 * l + 1] = sy;
    }
}

// XTRA: a rotation-dependent term is present (rotation only, a translation
// grid, or two parts); without it (sliced W2 with the closed-form
// translation) the argmin reads the correlation alone.
template <int nsig, int PARTS, bool XTRA>
__global__ void __launch_bounds__(kDecThreads, XTRA ? 5 : 6)
k_decide(DecideArgs A, FftPlan plan, const float2 *__restrict__ tw)
{
    constexpr int NP = 2 * nsig;                               // pairs per CTA
    constexpr int NW = kDecThreads / 32;
    extern __shared__ float2 smd[];
    const int n = A.n, M = A.M, nh = n / 2;
    float2 *b0 = smd;
    float2 *b1 = b0 + n * nsig;
    float2 *tws = b1 + n * nsig;                              // [n] twiddles
    float *prof_i = reinterpret_cast<float *>(tws + n);       // [M]
    __shared__ float delta[NP];
    __shared__ int stt[NP];
    __shared__ float red_key[NW][NP];
    __shared__ int red_l[NW][NP];
    const int i = blockIdx.x;
    const int j0 = blockIdx.y * NP;
    const int Nq = A.Nq, Nt = A.Nt;

    for (int t = threadIdx.x; t < n; t += blockDim.x) tws[t] = tw[t];
    for (int p = threadIdx.x; p < M; p += blockDim.x) prof_i[p] = A.prof_q[(size_t)i * M + p];
    if (threadIdx.x < NP) {
        const int j = j0 + threadIdx.x;
        stt[threadIdx.x] = j < Nt ? A.st_t[j] : 1;
    }
    __syncthreads();
    // ---- Hermitian-extended spectra of two pairs per signal.  Each thread
    // reads C(k') of two adjacent templates with one 16-byte load and writes
    // Z(k') and Z(n - k').  Unusable templates contribute zeros, so that their
    // NaNs cannot reach the partner pair through the FFT.
    const float2 *Ci = A.C + (size_t)i * Nt;
    const size_t fs = (size_t)Nq * Nt;
    const bool vec = (Nt & 1) == 0;  // C rows of even length keep 16-byte alignment
#pragma unroll 4
    for (int t = threadIdx.x; t < (nh + 1) * nsig; t += blockDim.x) {
        const int kf = t / nsig, s = t % nsig;
        const int ja = j0 + 2 * s, jb = ja + 1;
        float2 Xa = make_float2(0.f, 0.f), Xb = make_float2(0.f, 0.f);
        if (kf != 0) {
            const float2 *Cm = Ci + (size_t)(kf - 1) * fs;
            if (vec && jb < Nt) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(Cm + ja));
                Xa = make_float2(v.x, v.y);
                Xb = make_float2(v.z, v.w);
            } else {
                if (ja < Nt) Xa = Cm[ja];
                if (jb < Nt) Xb = Cm[jb];
            }
            if (stt[2 * s]) Xa = make_float2(0.f, 0.f);
            if (stt[2 * s + 1]) Xb = make_float2(0.f, 0.f);
        }
        if (kf == 0) {
            b0[s] = make_float2(0.f, 0.f);
        } else if (kf == nh) {
            b0[kf * nsig + s] = make_float2(Xa.x, Xb.x);  // real parts
        } else {
            b0[kf * nsig + s] = make_float2(Xa.x - Xb.y, Xa.y + Xb.x);        // Xa + i Xb
            b0[(n - kf) * nsig + s] = make_float2(Xa.x + Xb.y, Xb.x - Xa.y);  // conj Xa + i conj Xb
        }
    }
    __syncthreads();
    const float2 *R = fft_smem<nsig, +1>(b0, b1, plan, tws);  // R[l][s] = n (corr_a + i corr_b)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- k' = 0 part: n |m_i - m_j|^2
    for (int pr = warp; pr < NP; pr += NW) {
        const int j = j0 + pr;
        float sacc = 0.f;
        if (j < Nt) {
            const float *pj = A.prof_t + (size_t)j * M;
            for (int p = lane; p < M; p += 32) {
                const float d = prof_i[p] - pj[p];
                sacc = fmaf(d, d, sacc);
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
        if (lane == 0) delta[pr] = sacc * (float)n;
    }

    // ---- argmin over l (FP32 keys, lowest l on ties).  Thread (s, lq) scans
    // l = lq, lq + LQ, ... for both pairs of signal s: a warp then reads 32
    // consecutive complex values (conflict-free).
    double aix, aiy, dix, diy;
    centre_of(A.ctr_q, i, PARTS, aix, aiy, dix, diy);
    const XtraTerms X = xtra_terms<PARTS, XTRA>(A, (float)aix, (float)aiy, (float)dix, (float)diy);
    const float invn = 1.f / (float)n;
    constexpr int LQ = kDecThreads / nsig;
    const int s = threadIdx.x % nsig, lq = threadIdx.x / nsig;
    float best0 = __int_as_float(0x7f800000), best1 = best0;
    int bl0 = 0x7fffffff, bl1 = 0x7fffffff;
    const bool x_t = PARTS == 2;
    float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, ex0 = 0.f, ey0 = 0.f, ex1 = 0.f, ey1 = 0.f;
    if (X.rot_t || x_t) {
        const int ja = min(j0 + 2 * s, Nt - 1), jb = min(j0 + 2 * s + 1, Nt - 1);
        double x, y, u, v;
        centre_of(A.ctr_t, ja, PARTS, x, y, u, v);
        ax0 = (float)x, ay0 = (float)y, ex0 = (float)u, ey0 = (float)v;
        centre_of(A.ctr_t, jb, PARTS, x, y, u, v);
        ax1 = (float)x, ay1 = (float)y, ex1 = (float)u, ey1 = (float)v;
    }
    for (int l = lq; l < n; l += LQ) {
        const float2 z = R[l * nsig + s];
        float k0 = -2.f * z.x * invn, k1 = -2.f * z.y * invn;
        if (X.rot_t || x_t) {
            const float2 w = tws[l];  // (cos alpha_l, -sin alpha_l)
            k0 = xtra_key<PARTS>(k0, X, w.x, -w.y, ax0, ay0, ex0, ey0);
            k1 = xtra_key<PARTS>(k1, X, w.x, -w.y, ax1, ay1, ex1, ey1);
        }
        if (k0 < best0) { best0 = k0; bl0 = l; }   // l increases: ties keep the lowest
        if (k1 < best1) { best1 = k1; bl1 = l; }
    }
    // reduce over the lanes of this warp that share s (lane bits above log2 nsig)
#pragma unroll
    for (int off = nsig; off < 32; off <<= 1) {
        const float o0 = __shfl_xor_sync(0xffffffffu, best0, off);
        const int q0 = __shfl_xor_sync(0xffffffffu, bl0, off);
        const float o1 = __shfl_xor_sync(0xffffffffu, best1, off);
        const int q1 = __shfl_xor_sync(0xffffffffu, bl1, off);
        if (o0 < best0 || (o0 == best0 && q0 < bl0)) { best0 = o0; bl0 = q0; }
        if (o1 < best1 || (o1 == best1 && q1 < bl1)) { best1 = o1; bl1 = q1; }
    }
    if (lane < nsig) {
        red_key[warp][2 * s] = best0;
        red_l[warp][2 * s] = bl0;
        red_key[warp][2 * s + 1] = best1;
        red_l[warp][2 * s + 1] = bl1;
    }
    __syncthreads();

    // ---- one thread per pair: combine warps, FP64 distance at l*
    if (threadIdx.x < NP) {
        const int pr = threadIdx.x;
        const int j = j0 + pr;
        if (j < Nt) {
            float bk = red_key[0][pr];
            int bl = red_l[0][pr];
            for (int w = 1; w < NW; ++w) {
                const float k = red_key[w][pr];
                const int l = red_l[w][pr];
                if (k < bk || (k == bk && l < bl)) { bk = k; bl = l; }
            }
            const float2 z = R[(bl < n ? bl : 0) * nsig + (pr >> 1)];
            write_result<PARTS>(A, i, j, bl, (pr & 1) ? z.y : z.x, delta[pr], stt[pr], X.tmode,
                                aix, aiy, dix, diy);
        }
    }
    // ---- full curve of pair (0, 0) (single-pair call)
    if (A.curve && i == 0 && j0 == 0) {
        double ajx, ajy, djx, djy;
        centre_of(A.ctr_t, 0, PARTS, ajx, ajy, djx, djy);
        const double base = (double)delta[0] + A.norm_q[0] + A.norm_t[0];
        const int st = A.st_q[0] || stt[0] || (A.dev_err && *A.dev_err);
        for (int l = threadIdx.x; l < n; l += blockDim.x)
            curve_point<PARTS>(A, l, R[l * nsig].x, base, st, X.tmode, aix, aiy, dix, diy, ajx,
                               ajy, djx, djy);
    }
}

// ---------------------------------------------------------------------------
// Register form.
constexpr int kRegThreads = 256;   // 8 warps, one curve pair (two templates) each
constexpr int kRegTemplates = 16;  // templates per CTA
constexpr int kRegRow = 9;         // float4 per staged frequency: 16 complex + 16 bytes of pad

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
                 : "memory");
}

// Radix-2 decimation-in-time stages of span LEN, 2 LEN, ..., MW over a[] (bit-
// reversed input): a[b + j] +- e^{+2 pi i j / LEN} a[b + j + LEN / 2].
template <int MW, int LEN>
__device__ __forceinline__ void lane_stages(float2 (&a)[MW], const float2 *__restrict__ tw)
{
    constexpr int n = 32 * MW, hl = LEN / 2;
#pragma unroll
    for (int b = 0; b < MW; b += LEN) {
#pragma unroll
        for (int j = 0; j < hl; ++j) {
            float2 x = a[b + j + hl];
            if (j == 0) {
            } else if (4 * j == LEN) {
                x = make_float2(-x.y, x.x);  // e^{+i pi / 2}
            } else {
                x = cmul(x, cconj(tw[j * (n / LEN)]));
            }
            const float2 u = a[b + j];
            a[b + j] = cadd(u, x);
            a[b + j + hl] = csub(u, x);
        }
    }
    if constexpr (2 * LEN <= MW) lane_stages<MW, 2 * LEN>(a, tw);
}

// Unnormalised inverse DFT of length n = 32 MW (MW a power of two <= 16) held
// by one warp, X(q) = sum_t x(t) e^{+2 pi i t q / n}.  In: v[t1] = x(32 t1 +
// lane).  Out: v[k1] = X(k1 + MW brev5(lane)).  tw[q] = e^{-2 pi i q / n}.
// With t = 32 t1 + lane and q = k1 + MW q2 the kernel factors into an MW-point
// transform over t1 in each lane (radix 2, decimation in time), the twiddles
// e^{+2 pi i lane k1 / n}, and a 32-point transform over the lanes (five
// radix-2 decimation-in-frequency stages, outputs in bit-reversed lanes).
template <int MW>
__device__ __forceinline__ void reg_ifft(float2 (&v)[MW], const float2 *__restrict__ tw, int lane)
{
    constexpr int LG = MW == 1 ? 0 : MW == 2 ? 1 : MW == 4 ? 2 : MW == 8 ? 3 : 4;
    static_assert((1 << LG) == MW, "MW must be 1, 2, 4, 8 or 16");
    float2 a[MW];
#pragma unroll
    for (int t = 0; t < MW; ++t) {
        int r = 0;  // t with its LG bits reversed
#pragma unroll
        for (int b = 0; b < LG; ++b) r |= ((t >> b) & 1) << (LG - 1 - b);
        a[r] = v[t];
    }
    lane_stages<MW, 2>(a, tw);
#pragma unroll
    for (int k1 = 1; k1 < MW; ++k1) a[k1] = cmul(a[k1], cconj(tw[lane * k1]));
    warp_lane_stages<MW>(a, tw, lane);
#pragma unroll
    for (int k1 = 0; k1 < MW; ++k1) v[k1] = a[k1];
}

// Unnormalised inverse DFT of length n = 30 MW (MW even, at most 16) held by
// lanes 0..29 of a warp, X(q) = sum_t x(t) e^{+2 pi i t q / n}.  In: v[t1] =
// x(30 t1 + lane).  Out: v[k1] = X(k1 + MW q2(lane)), q2 = lane30_q(lane).
// tw[q] = e^{-2 pi i q / n}.  Four-step as reg_ifft: an MW-point mixed-radix
// DFT over t1 in each lane, the twiddles e^{+2 pi i lane k1 / n}, and a
// 30-point transform over the lanes in three decimation-in-frequency stages
// (radix 2 over lanes 15 apart, radix 3 over lanes 5 apart in each block of
// 15, radix 5 over adjacent lanes in each block of 5): the lane u + S m of a
// stage of radix r and span S keeps its own output digit m,
//   z = e^{+2 pi i u m / (r S)} sum_j y(u + S j) e^{+2 pi i j m / r},
// so lane m3 + 5 m2 + 15 m ends with the output q2 = m + 2 m2 + 6 m3.
// Lanes 30 and 31 compute nothing of use (they read their own values).
__device__ __forceinline__ int lane30_q(int lane)
{
    return lane / 15 + 2 * ((lane % 15) / 5) + 6 * (lane % 5);
}
__device__ __forceinline__ int lane30_of_q(int q)
{
    return (q / 6) + 5 * ((q / 2) % 3) + 15 * (q % 2);
}
// e^{+2 pi i x / r} from the n-point table (r divides n, 0 <= x < r)
__device__ __forceinline__ float2 root_of(const float2 *tw, int x, int r, int n)
{
    return cconj(tw[x * (n / r)]);
}
template <int MW>
__device__ __forceinline__ void reg_ifft30(float2 (&v)[MW], const float2 *__restrict__ tw, int lane)
{
    constexpr int n = 30 * MW;
    lane_dft<MW, 30>(v, tw);
    const int ln = lane < 30 ? lane : 0;
#pragma unroll
    for (int k1 = 1; k1 < MW; ++k1) v[k1] = cmul(v[k1], cconj(tw[ln * k1]));
    // radix 2, span 15: lane u + 15 m
    {
        const int m = ln / 15, u = ln % 15;
        const int src = lane < 30 ? (m ? lane - 15 : lane + 15) : lane;
        const float2 w = root_of(tw, u * m, 30, n);
#pragma unroll
        for (int k1 = 0; k1 < MW; ++k1) {
            const float2 o = make_float2(__shfl_sync(0xffffffffu, v[k1].x, src),
                                         __shfl_sync(0xffffffffu, v[k1].y, src));
            // m = 0: y0 + y1 (own + other); m = 1: y0 - y1 (other - own)
            const float2 z = m ? csub(o, v[k1]) : cadd(v[k1], o);
            v[k1] = m ? cmul(z, w) : z;
        }
    }
    // radix 3, span 5, in blocks of 15: lane b + v + 5 m2
    {
        const int b = ln - ln % 15, u = ln % 15, m2 = u / 5, vv = u % 5;
        const int s1 = lane < 30 ? b + vv + 5 * ((m2 + 1) % 3) : lane;
        const int s2 = lane < 30 ? b + vv + 5 * ((m2 + 2) % 3) : lane;
        // inputs j = m2 (own), m2 + 1, m2 + 2 (mod 3), weighted e^{+2 pi i j m2 / 3}
        const float2 c1 = root_of(tw, ((m2 + 1) % 3) * m2 % 3, 3, n);
        const float2 c2 = root_of(tw, ((m2 + 2) % 3) * m2 % 3, 3, n);
        const float2 c0 = root_of(tw, m2 * m2 % 3, 3, n);
        const float2 w = root_of(tw, vv * m2, 15, n);
#pragma unroll
        for (int k1 = 0; k1 < MW; ++k1) {
            const float2 o1 = make_float2(__shfl_sync(0xffffffffu, v[k1].x, s1),
                                          __shfl_sync(0xffffffffu, v[k1].y, s1));
            const float2 o2 = make_float2(__shfl_sync(0xffffffffu, v[k1].x, s2),
                                          __shfl_sync(0xffffffffu, v[k1].y, s2));
            const float2 z = cadd(cadd(cmul(v[k1], c0), cmul(o1, c1)), cmul(o2, c2));
            v[k1] = cmul(z, w);
        }
    }
    // radix 5, span 1, in blocks of 5: lane b + m3
    {
        const int b = ln - ln % 5, m3 = ln % 5;
        int src[4];
        float2 c[5];
        c[0] = root_of(tw, m3 * m3 % 5, 5, n);
#pragma unroll
        for (int d = 1; d < 5; ++d) {
            const int j = (m3 + d) % 5;
            src[d - 1] = lane < 30 ? b + j : lane;
            c[d] = root_of(tw, j * m3 % 5, 5, n);
        }
#pragma unroll
        for (int k1 = 0; k1 < MW; ++k1) {
            float2 z = cmul(v[k1], c[0]);
#pragma unroll
            for (int d = 1; d < 5; ++d) {
                const float2 o = make_float2(__shfl_sync(0xffffffffu, v[k1].x, src[d - 1]),
                                             __shfl_sync(0xffffffffu, v[k1].y, src[d - 1]));
                z = cadd(z, cmul(o, c[d]));
            }
            v[k1] = z;
        }
    }
}

// Integer image of a float that preserves its order, -0 taken as +0 and NaN
// above everything.
__device__ __forceinline__ int ordered_key(float x)
{
    x = x + 0.f;  // -0 -> +0 (equal keys must map to one integer)
    const int i = __float_as_int(x);
    return x != x ? 0x7fffffff : (i >= 0 ? i : i ^ 0x7fffffff);
}

// Warp-wide argmin: every lane offers (key, l); returns the lowest l among
// the lanes holding the smallest key (a NaN key loses to any other).
__device__ __forceinline__ int warp_argmin(float key, int l)
{
    const int k = ~ordered_key(key);  // order-reversing
    const int kmax = __reduce_max_sync(0xffffffffu, k);
    return (int)__reduce_min_sync(0xffffffffu, (unsigned)(k == kmax ? l : 0x7fffffff));
}

// Issue the copies of the block (query i, templates j0 .. j0 + 15) into buf
// (the caller commits the cp.async group).  Templates past Nt are
// zero-filled; even Nt keeps every row 16-byte aligned.
template <int NH>
__device__ __forceinline__ void stage_block(const DecideArgs &A, int i, int j0, float4 *buf,
                                            int tid)
{
    const int Nq = A.Nq, Nt = A.Nt;
    const size_t fs = (size_t)Nq * Nt;
    const float2 *Ci = A.C + (size_t)i * Nt + j0;
    if ((Nt & 1) == 0) {
        for (int c = tid; c < NH * 8; c += kRegThreads) {
            const int f = c >> 3, col = c & 7;
            const int valid = min(max(Nt - (j0 + 2 * col), 0), 2);
            const float2 *src = valid ? Ci + (size_t)f * fs + 2 * col : A.C;
            cp_async16(buf + f * kRegRow + col, src, 8 * valid);
        }
    } else {
        for (int c = tid; c < NH * 16; c += kRegThreads) {
            const int f = c >> 4, col = c & 15;
            const bool valid = j0 + col < Nt;
            const float2 *src = valid ? Ci + (size_t)f * fs + col : A.C;
            cp_async8(reinterpret_cast<float2 *>(buf + f * kRegRow) + col, src, valid ? 8 : 0);
        }
    }
}

// The staging buffer of n/2 rows, then the twiddles and the query's profile.
size_t reg_smem_bytes(int n, int M)
{
    return sizeof(float4) * (size_t)(n / 2) * kRegRow + sizeof(float2) * (size_t)n +
           sizeof(float) * (size_t)M;
}

// One CTA per (query i, templates j0 .. j0 + 15).  LANES = 32: n = 32 MW
// (powers of two); LANES = 30: n = 30 MW on lanes 0..29 (reg_ifft30).  At
// MW = 12 (n = 360) four CTAs per SM (64 registers, no spills) beat two
// (0.137 against 0.177 ms for 128 x 1000 pairs).
template <int MW, int PARTS, bool XTRA, int LANES = 32>
__global__ void __launch_bounds__(kRegThreads, MW <= 8 ? (XTRA || PARTS == 2 ? 4 : 6) : (MW == 12 ? 4 : 2))
k_decide_reg(DecideArgs A, const float2 *__restrict__ tw)
{
    constexpr int n = LANES * MW, nh = n / 2;
    static_assert(LANES == 32 || (LANES == 30 && MW % 2 == 0), "n = 32 MW or 30 MW (MW even)");
    extern __shared__ float4 smr[];
    float4 *sC = smr;                                             // [nh][kRegRow]
    float2 *tws = reinterpret_cast<float2 *>(sC + nh * kRegRow);  // [n]
    float *prof_i = reinterpret_cast<float *>(tws + n);           // [M]
    __shared__ int stt[kRegTemplates];
    __shared__ float4 ctr_f[kRegTemplates + 1];  // FP32 centres (abar, d): templates, then the query
    __shared__ int res_l[kRegTemplates];         // per template: l*, n corr(l*), n |m_i - m_j|^2
    __shared__ float res_v[kRegTemplates], res_d[kRegTemplates];
    const int Nt = A.Nt, M = A.M;
    const int i = blockIdx.x, j0 = blockIdx.y * kRegTemplates;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = warp;  // this warp's templates: j0 + 2s (real part), j0 + 2s + 1 (imaginary)

    // ---- stage C(k', i, j0 .. j0 + 15), k' = 1..n/2 (row k' - 1)
    stage_block<nh>(A, i, j0, sC, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int t = tid; t < n; t += kRegThreads) tws[t] = tw[t];
    for (int p = tid; p < M; p += kRegThreads) prof_i[p] = A.prof_q[(size_t)i * M + p];
    if (tid < kRegTemplates) {
        const int j = j0 + tid;
        stt[tid] = j < Nt ? A.st_t[j] : 1;
    }
    if ((XTRA || PARTS == 2) && tid <= kRegTemplates) {
        // the keys' centres, converted once per CTA (not per warp)
        double x, y, u, w;
        if (tid < kRegTemplates) centre_of(A.ctr_t, min(j0 + tid, Nt - 1), PARTS, x, y, u, w);
        else centre_of(A.ctr_q, i, PARTS, x, y, u, w);
        ctr_f[tid] = make_float4((float)x, (float)y, (float)u, (float)w);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    const int ja = j0 + 2 * s, jb = ja + 1;
    // k' = 0 part: n |m_i - m_j|^2
    // (half-warp h takes template ja + h)
    float dsum = 0.f;
    {
        const int jh = lane < 16 ? ja : jb;
        if (jh < Nt) {
            const float *ph = A.prof_t + (size_t)jh * M;
            for (int p = lane & 15; p < M; p += 16) {
                const float d = prof_i[p] - __ldg(ph + p);
                dsum = fmaf(d, d, dsum);
            }
        }
#pragma unroll
        for (int off = 8; off; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
    }
    const float da = __shfl_sync(0xffffffffu, dsum, 0) * (float)n;
    const float db = __shfl_sync(0xffffffffu, dsum, 16) * (float)n;

    // Hermitian-extended spectrum Z(t) = C_a(t) + i C_b(t) (t < n/2),
    // conj C_a(n - t) + i conj C_b(n - t) (t > n/2), real parts at n/2, 0
    // at 0; unusable templates contribute zeros (their NaNs stay out of
    // the partner)
    const bool za = stt[2 * s] != 0, zb = stt[2 * s + 1] != 0;
    const bool live = lane < LANES;  // lanes that hold samples of the transform
    float2 v[MW];
#pragma unroll
    for (int m = 0; m < MW; ++m) {
        const int t = LANES * m + lane;
        const int kf = m < MW / 2 ? t : n - t;
        float4 X = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live && kf != 0) X = sC[(kf - 1) * kRegRow + s];
        if (za) X.x = X.y = 0.f;
        if (zb) X.z = X.w = 0.f;
        if (m < MW / 2)
            v[m] = make_float2(X.x - X.w, X.y + X.z);  // kf = 0 gives 0
        else if (m == MW / 2 && lane == 0)
            v[m] = make_float2(X.x, X.z);
        else
            v[m] = make_float2(X.x + X.w, X.z - X.y);
    }
    // v[k1] = n (corr_a + i corr_b) at l = k1 + MW q2(lane)
    if constexpr (LANES == 32) reg_ifft<MW>(v, tws, lane);
    else reg_ifft30<MW>(v, tws, lane);

    // ---- argmin over l (FP32 keys, lowest l on ties), carrying n corr(l)
    const bool x_t = PARTS == 2;
    float4 cq = make_float4(0.f, 0.f, 0.f, 0.f), c0 = cq, c1 = cq;
    if (XTRA || x_t) {
        cq = ctr_f[kRegTemplates];
        c0 = ctr_f[2 * s];
        c1 = ctr_f[2 * s + 1];
    }
    const XtraTerms X = xtra_terms<PARTS, XTRA>(A, cq.x, cq.y, cq.z, cq.w);
    // Per lane the lowest l of its best key (l grows with k1), then two warp
    // reductions on order-preserving integer images of the keys: the best
    // key, then the lowest l holding it.  NaN keys never win (unless all are).
    float best0, best1, rv0, rv1;  // per lane: best key, and n corr at its l
    int bl0, bl1;
    const int lb = MW * (LANES == 32 ? brev5(lane) : (live ? lane30_q(lane) : 0));
    if (!X.rot_t && !x_t) {
        // key = -2 corr(l) / n: the smallest key is the largest n corr(l)
        // (exactly so for n a power of two; for n = 30 MW the keys are
        // compared as -n corr, the same order up to the scaling's rounding,
        // which is monotone)
        rv0 = rv1 = __int_as_float(0xff800000);  // -inf: NaN values never replace it
        bl0 = bl1 = lb;
        if (live) {
#pragma unroll
            for (int k1 = 0; k1 < MW; ++k1) {
                if (v[k1].x > rv0) { rv0 = v[k1].x; bl0 = k1 + lb; }
                if (v[k1].y > rv1) { rv1 = v[k1].y; bl1 = k1 + lb; }
            }
        }
        best0 = -rv0;
        best1 = -rv1;
    } else {
        const float invn = 1.f / (float)n;
        best0 = best1 = __int_as_float(0x7f800000);
        rv0 = v[0].x;
        rv1 = v[0].y;
        bl0 = bl1 = lb;
#pragma unroll
        for (int k1 = 0; k1 < MW; ++k1) {
            if (!live) break;
            const int l = k1 + lb;
            const float2 z = v[k1];
            const float2 w = tws[l];  // (cos alpha_l, -sin alpha_l)
            const float k0 = xtra_key<PARTS>(-2.f * z.x * invn, X, w.x, -w.y, c0.x, c0.y, c0.z, c0.w);
            const float kb = xtra_key<PARTS>(-2.f * z.y * invn, X, w.x, -w.y, c1.x, c1.y, c1.z, c1.w);
            if (k0 < best0) { best0 = k0; bl0 = l; rv0 = z.x; }
            if (kb < best1) { best1 = kb; bl1 = l; rv1 = z.y; }
        }
    }
    // the lane holding l* has l* as its own best: n corr(l*) comes from it
    bl0 = warp_argmin(best0, bl0);
    bl1 = warp_argmin(best1, bl1);
    rv0 = __shfl_sync(0xffffffffu, rv0, LANES == 32 ? brev5(bl0 / MW) : lane30_of_q(bl0 / MW));
    rv1 = __shfl_sync(0xffffffffu, rv1, LANES == 32 ? brev5(bl1 / MW) : lane30_of_q(bl1 / MW));
    if (lane < 2) {
        res_l[2 * s + lane] = lane ? bl1 : bl0;
        res_v[2 * s + lane] = lane ? rv1 : rv0;
        res_d[2 * s + lane] = lane ? db : da;
    }
    double aix, aiy, dix, diy;
    // ---- full curve of pair (0, 0) (single-pair call)
    if (A.curve && i == 0 && j0 == 0 && s == 0) {
        centre_of(A.ctr_q, i, PARTS, aix, aiy, dix, diy);
        double ajx, ajy, djx, djy;
        centre_of(A.ctr_t, 0, PARTS, ajx, ajy, djx, djy);
        const double base = (double)da + A.norm_q[0] + A.norm_t[0];
        const int st = A.st_q[0] || stt[0] || (A.dev_err && *A.dev_err);
        if (live) {
#pragma unroll
            for (int k1 = 0; k1 < MW; ++k1)
                curve_point<PARTS>(A, k1 + lb, v[k1].x, base, st, X.tmode, aix, aiy, dix, diy,
                                   ajx, ajy, djx, djy);
        }
    }
    // every warp has posted its pairs
    __syncthreads();
    // ---- FP64 distance at l*: one lane per template, all in warp 0 (the
    // FP64 pipe is narrow: its instructions are issued once per 16 pairs)
    if (warp == 0 && lane < kRegTemplates && j0 + lane < Nt) {
        centre_of(A.ctr_q, i, PARTS, aix, aiy, dix, diy);
        write_result<PARTS>(A, i, j0 + lane, res_l[lane], res_v[lane], res_d[lane],
                            stt[lane], X.tmode, aix, aiy, dix, diy);
    }
}

// Best template per query: lowest d2 among usable templates, lowest j on ties.
__global__ void k_best_template(const sw_result *__restrict__ all, int Nq, int Nt,
                                sw_result *__restrict__ out)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= Nq) return;
    const sw_result *row = all + (size_t)warp * Nt;
    double best = __longlong_as_double(0x7ff0000000000000ULL);
    int bj = 0x7fffffff;
    int qbad = 0;
    for (int j = lane; j < Nt; j += 32) {
        const sw_result r = row[j];
        if (r.status == 1) qbad = 1;
        if (r.status == 0 && (r.d2 < best || (r.d2 == best && j < bj))) {
            best = r.d2;
            bj = j;
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
        qbad |= __shfl_xor_sync(0xffffffffu, qbad, off);
        if (ob < best || (ob == best && oj < bj)) {
            best = ob;
            bj = oj;
        }
    }
    if (lane == 0) {
        sw_result r;
        if (bj == 0x7fffffff) {
            const double nan = __longlong_as_double(0x7ff8000000000000ULL);
            r.best_l = -1;
            r.status = qbad || Nt == 0 ? 1 : 2;
            r.angle_rad = __int_as_float(0x7fc00000);
            r.template_index = -1;
            r.shift[0] = r.shift[1] = nan;
            r.d2 = nan;
        } else {
            r = row[bj];
            r.template_index = bj;
        }
        out[warp] = r;
    }
}

}  // namespace

bool decide_reg_ok(int n)
{
    return n == 64 || n == 128 || n == 256 || n == 512 ||  // 32 lanes
           n == 60 || n == 120 || n == 180 || n == 240 || n == 360 || n == 480;  // 30 lanes
}

cudaError_t launch_decide(const DecideArgs &args, const FftPlan &plan, const float2 *tw,
                          cudaStream_t st, int nsig_req)
{
    if (args.Nq <= 0 || args.Nt <= 0) return cudaSuccess;
    DecideArgs a = args;
    if (a.parts != 1 && (a.parts != 2 || a.M % 2)) return cudaErrorInvalidValue;
    if (a.grid_k > 0 && !(a.grid_step > 0.0)) return cudaErrorInvalidValue;
    a.inv_n = 1.0 / a.n;
    a.inv_nM = 1.0 / ((double)a.n * (a.M / a.parts));
    a.dalpha = 6.283185307179586 / a.n;
    const double nM = (double)a.n * (a.M / a.parts);  // the levels per part
    a.hnm = (a.parts == 2 ? 1.f : 0.5f) * (float)nM;
    a.qnm = 0.25f * (float)nM;
    a.gstep = (float)a.grid_step;
    a.ginv = a.grid_k > 0 ? (float)(1.0 / a.grid_step) : 0.f;
    a.gk = (float)a.grid_k;
    if (decide_reg_ok(a.n) && (nsig_req == 0 || nsig_req == 1)) {
        const size_t smem = reg_smem_bytes(a.n, a.M);
        dim3 grid(a.Nq, (a.Nt + kRegTemplates - 1) / kRegTemplates);
#define SW_REG_LAUNCH(MW, P, X, LN)                                                         \
    do {                                                                                    \
        cudaFuncSetAttribute(k_decide_reg<MW, P, X, LN>,                                    \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
        k_decide_reg<MW, P, X, LN><<<grid, kRegThreads, smem, st>>>(a, tw);                 \
    } while (0)
#define SW_REG_FORMS(MW, LN)                                                                \
    do {                                                                                    \
        if (a.parts == 1 && a.translation && a.grid_k == 0) SW_REG_LAUNCH(MW, 1, false, LN); \
        else if (a.parts == 1) SW_REG_LAUNCH(MW, 1, true, LN);                              \
        else SW_REG_LAUNCH(MW, 2, true, LN);                                                \
    } while (0)
        switch (a.n) {
        case 64: SW_REG_FORMS(2, 32); break;
        case 128: SW_REG_FORMS(4, 32); break;
        case 256: SW_REG_FORMS(8, 32); break;
        case 512: SW_REG_FORMS(16, 32); break;
        case 60: SW_REG_FORMS(2, 30); break;
        case 120: SW_REG_FORMS(4, 30); break;
        case 180: SW_REG_FORMS(6, 30); break;
        case 240: SW_REG_FORMS(8, 30); break;
        case 360: SW_REG_FORMS(12, 30); break;
        default: SW_REG_FORMS(16, 30); break;  // 480
        }
#undef SW_REG_FORMS
#undef SW_REG_LAUNCH
        return cudaGetLastError();
    }
    // shared-memory form: 8 signals (16 pairs) per CTA keeps the shared
    // footprint small enough for several CTAs per SM; 4 at n = 1024.  A
    // requested width is taken when its buffers fit (2 n nsig complex values).
    int nsig = a.n <= 512 ? 8 : 4;
    if ((nsig_req == 4 || nsig_req == 8 || nsig_req == 16) && (size_t)a.n * nsig_req <= 8192)
        nsig = nsig_req;
    const size_t smem = sizeof(float2) * ((size_t)2 * a.n * nsig + a.n) + sizeof(float) * a.M;
    dim3 grid(a.Nq, (a.Nt + 2 * nsig - 1) / (2 * nsig));  // queries on x (no 65535 cap)
#define SW_DEC_LAUNCH(NS, P, X)                                                              \
    do {                                                                                    \
        cudaFuncSetAttribute(k_decide<NS, P, X>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             200 * 1024);                                                   \
        k_decide<NS, P, X><<<grid, kDecThreads, smem, st>>>(a, plan, tw);                   \
    } while (0)
    const bool plain = a.parts == 1 && a.translation && a.grid_k == 0;
    if (plain) {
        if (nsig == 16) SW_DEC_LAUNCH(16, 1, false);
        else if (nsig == 8) SW_DEC_LAUNCH(8, 1, false);
        else SW_DEC_LAUNCH(4, 1, false);
    } else if (a.parts == 1) {
        if (nsig == 16) SW_DEC_LAUNCH(16, 1, true);
        else if (nsig == 8) SW_DEC_LAUNCH(8, 1, true);
        else SW_DEC_LAUNCH(4, 1, true);
    } else {
        if (nsig == 16) SW_DEC_LAUNCH(16, 2, true);
        else if (nsig == 8) SW_DEC_LAUNCH(8, 2, true);
        else SW_DEC_LAUNCH(4, 2, true);
    }
#undef SW_DEC_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_best_template(const void *all, int Nq, int Nt, void *out, cudaStream_t st)
{
    if (Nq <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (Nq * 32 + threads - 1) / threads;
    k_best_template<<<blocks, threads, 0, st>>>(reinterpret_cast<const sw_result *>(all), Nq,
                                                Nt, reinterpret_cast<sw_result *>(out));
    return cudaGetLastError();
}

}  // namespace swk
