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
// Design: one CTA per (query, 2*nsig templates); two real correlation
// curves are packed in one complex inverse FFT (the curves are real, so the
// spectrum of c_a + i c_b is C_a + i C_b extended by Hermitian symmetry).
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
    // the distance's M is the levels per part (parts = 2: ramp-filtered)
    const double nM = (double)n * (M / PARTS);
    double aix, aiy, dix, diy;
    centre_of(A.ctr_q, i, PARTS, aix, aiy, dix, diy);
    const float invn = 1.f / (float)n;
    constexpr int LQ = kDecThreads / nsig;
    const int s = threadIdx.x % nsig, lq = threadIdx.x / nsig;
    float best0 = __int_as_float(0x7f800000), best1 = best0;
    int bl0 = 0x7fffffff, bl1 = 0x7fffffff;
    // rotation-dependent terms of the two pairs: rc |s - c|^2 with
    // c = abar_i - R abar_j and s = 0 (rotation only) or the grid point
    // nearest c (translation on a grid), and xc |d_i - R d_j|^2 (two parts)
    const int tmode = !XTRA ? 1 : (!A.translation ? 0 : (A.grid_k > 0 ? 2 : 1));
    const bool rot_t = XTRA && tmode != 1, x_t = PARTS == 2;
    const float gstep = (float)A.grid_step, ginv = tmode == 2 ? (float)(1.0 / A.grid_step) : 0.f;
    const float gk = (float)A.grid_k;
    float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, ex0 = 0.f, ey0 = 0.f, ex1 = 0.f, ey1 = 0.f;
    if (rot_t || x_t) {
        const int ja = min(j0 + 2 * s, Nt - 1), jb = min(j0 + 2 * s + 1, Nt - 1);
        double x, y, u, v;
        centre_of(A.ctr_t, ja, PARTS, x, y, u, v);
        ax0 = (float)x, ay0 = (float)y, ex0 = (float)u, ey0 = (float)v;
        centre_of(A.ctr_t, jb, PARTS, x, y, u, v);
        ax1 = (float)x, ay1 = (float)y, ex1 = (float)u, ey1 = (float)v;
    }
    const float hnm = (PARTS == 2 ? 1.f : 0.5f) * (float)nM;
    const float qnm = 0.25f * (float)nM;
    for (int l = lq; l < n; l += LQ) {
        const float2 z = R[l * nsig + s];
        float k0 = -2.f * z.x * invn, k1 = -2.f * z.y * invn;
        if (rot_t || x_t) {
            const float2 w = tws[l];  // (cos alpha_l, -sin alpha_l)
            const float c = w.x, sn = -w.y;
            if (rot_t) {
                float sx = (float)aix - (c * ax0 - sn * ay0), sy = (float)aiy - (sn * ax0 + c * ay0);
                if (tmode == 2) {
                    sx -= fminf(fmaxf(rintf(sx * ginv), -gk), gk) * gstep;
                    sy -= fminf(fmaxf(rintf(sy * ginv), -gk), gk) * gstep;
                }
                k0 = fmaf(hnm, sx * sx + sy * sy, k0);
                sx = (float)aix - (c * ax1 - sn * ay1);
                sy = (float)aiy - (sn * ax1 + c * ay1);
                if (tmode == 2) {
                    sx -= fminf(fmaxf(rintf(sx * ginv), -gk), gk) * gstep;
                    sy -= fminf(fmaxf(rintf(sy * ginv), -gk), gk) * gstep;
                }
                k1 = fmaf(hnm, sx * sx + sy * sy, k1);
            }
            if (x_t) {
                float sx = (float)dix - (c * ex0 - sn * ey0), sy = (float)diy - (sn * ex0 + c * ey0);
                k0 = fmaf(qnm, sx * sx + sy * sy, k0);
                sx = (float)dix - (c * ex1 - sn * ey1);
                sy = (float)diy - (sn * ex1 + c * ey1);
                k1 = fmaf(qnm, sx * sx + sy * sy, k1);
            }
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
            if (bl >= n) bl = 0;  // every key NaN (unusable input): keep the index in range
            const int sg = pr >> 1, comp = pr & 1;
            double ajx, ajy, djx, djy;
            centre_of(A.ctr_t, j, PARTS, ajx, ajy, djx, djy);
            const double base = (double)delta[pr] + A.norm_q[i] + A.norm_t[j];
            const int st = A.st_q[i] ? 1 : (stt[pr] ? 2 : ((A.dev_err && *A.dev_err) ? 3 : 0));
            sw_result r;
            if (st) {
                const double nan = __longlong_as_double(0x7ff8000000000000ULL);
                r.best_l = -1;
                r.status = st;
                r.angle_rad = __int_as_float(0x7fc00000);
                r.shift[0] = r.shift[1] = nan;
                r.d2 = nan;
            } else {
                const float2 z = R[bl * nsig + sg];
                const double corr = (double)(comp ? z.y : z.x) * A.inv_n;
                const double2 c = A.cs64[bl];
                double sx = aix - (c.x * ajx - c.y * ajy);
                double sy = aiy - (c.y * ajx + c.x * ajy);
                double d = (base - 2.0 * corr) * A.inv_nM;
                if (x_t) {
                    const double ex = dix - (c.x * djx - c.y * djy);
                    const double ey = diy - (c.y * djx + c.x * djy);
                    d += 0.25 * (ex * ex + ey * ey);
                }
                restrict_shift(tmode, A.grid_k, A.grid_step, PARTS == 2 ? 1.0 : 0.5, sx, sy, d);
                r.best_l = bl;
                r.status = 0;
                r.angle_rad = (float)(A.dalpha * bl);
                r.shift[0] = sx;
                r.shift[1] = sy;
                r.d2 = d;
            }
            r.reserved = 0.f;
            reinterpret_cast<sw_result *>(A.out)[(size_t)i * Nt + j] = r;
        }
    }
    // ---- full curve of pair (0, 0) (single-pair call)
    if (A.curve && i == 0 && j0 == 0) {
        double ajx, ajy, djx, djy;
        centre_of(A.ctr_t, 0, PARTS, ajx, ajy, djx, djy);
        const double base = (double)delta[0] + A.norm_q[0] + A.norm_t[0];
        const int st = A.st_q[0] || stt[0] || (A.dev_err && *A.dev_err);
        for (int l = threadIdx.x; l < n; l += blockDim.x) {
            const double corr = (double)R[l * nsig].x * A.inv_n;
            const double2 c = A.cs64[l];
            double sx = aix - (c.x * ajx - c.y * ajy);
            double sy = aiy - (c.y * ajx + c.x * ajy);
            double d = (base - 2.0 * corr) * A.inv_nM;
            if (x_t) {
                const double ex = dix - (c.x * djx - c.y * djy);
                const double ey = diy - (c.y * djx + c.x * djy);
                d += 0.25 * (ex * ex + ey * ey);
            }
            restrict_shift(tmode, A.grid_k, A.grid_step, PARTS == 2 ? 1.0 : 0.5, sx, sy, d);
            A.curve[l] = st ? __longlong_as_double(0x7ff8000000000000ULL) : d;
            if (A.shifts) {
                A.shifts[2 * l] = sx;
                A.shifts[2 * l + 1] = sy;
            }
        }
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
            r.reserved = -1.f;
            r.shift[0] = r.shift[1] = nan;
            r.d2 = nan;
        } else {
            r = row[bj];
            r.reserved = (float)bj;
        }
        out[warp] = r;
    }
}

}  // namespace

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
    // 8 signals (16 pairs) per CTA keeps the shared footprint small enough
    // for several CTAs per SM; 4 at n = 1024.  A requested width is taken
    // when its buffers fit (2 n nsig complex values).
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
