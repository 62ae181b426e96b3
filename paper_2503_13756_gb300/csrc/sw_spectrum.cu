// sw_spectrum.cu -- angle spectra of the quantile functions: the first half
// of the FFT cross-correlation of Sec. 2.3 ("Fast computation over
// rotations": the correlation along angle of every row of U_I and V_I is
// computed with the FFT), plus the translation centring.
//
// For level p, the quantiles u_pk (k = 0..n-1) are transformed over k:
//   Qhat(k', p) = sum_k u~_pk e^{-2 pi i k k'/n},  u~_pk = u_pk - <a, theta_k>,
// with a = (2/n) sum_k ubar_k theta_k.  Centring only changes k' = 1 (and
// n-1): Qhat(1, p) -= c1 with c1 = mean_p Qhat_u(1, p) = (n/2)(a_x - i a_y),
// so it is applied after the transform with no second pass over the data.
// The k' = 0 term (n times the mean over angle of each level, the "profile")
// is kept apart, so that the rotation-invariant part of the distance is
// computed later as a direct difference instead of a cancelling sum.
//
// Design (GB300): one CTA per image; levels are taken 2*nsig at a time, two
// real levels packed into one complex signal, FFT'd by the shared-memory
// Stockham FFT and unpacked by Hermitian symmetry.  The batches are staged
// by cp.async into two buffers, so that batch b + 1 is in flight while batch
// b is transformed and written.  Norms are accumulated in double-float.
// Optional BF16/FP16 copies feed the tensor-core GEMM, with their norms taken
// from the rounded values so that self-distances cancel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int kSpecThreads = 256;
constexpr size_t kSmemOptIn = 227 * 1024;  // dynamic shared memory a CTA may opt in to

template <typename T>
__device__ __forceinline__ T to_lp(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_lp<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_lp<__half>(float x) { return __float2half_rn(x); }
template <typename T>
__device__ __forceinline__ float from_lp(T x);
template <>
__device__ __forceinline__ float from_lp<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float from_lp<__half>(__half x) { return __half2float(x); }

struct SpecOut {
    float *spec32;
    size_t fstride;
    void *lp_q;
    size_t lpq_fstride;
    void *lp_t;
    size_t lpt_fstride;
    int Nq;
    int ldk;    // low-precision segment length (>= 2M, zero padded)
    int lp;     // write low-precision copies (queries to lp_q, templates to lp_t)
    int split;  // FP16 hi/lo split: rows of 2 segments [hi | lo]
};

// Compensated (Kahan) sum of nonnegative terms, kept as (sum, -compensation):
// the value is a.hi + a.lo, within about 2 ulp of the exact sum.
__device__ __forceinline__ void kahan_add(DF &a, float x)
{
    const float y = x + a.lo;
    const float t = a.hi + y;
    a.lo = y - (t - a.hi);
    a.hi = t;
}

// Writes Qhat(kf, p) (kf >= 1) for image img and adds its |.|^2 (weight w)
// to acc32 (FP32 values) and acc16 (the low-precision values the GEMM sees).
template <typename T>
__device__ __forceinline__ void emit(const SpecOut &o, int img, int M, int kf, int p, float2 X,
                                     float w, DF &acc32, DF &acc16)
{
    kahan_add(acc32, w * fmaf(X.x, X.x, X.y * X.y));
    if (!o.lp) {
        float *row = o.spec32 + (size_t)(kf - 1) * o.fstride + (size_t)img * 2 * M;
        row[p] = X.x;
        row[M + p] = X.y;
        return;
    }
    const T re = to_lp<T>(X.x), im = to_lp<T>(X.y);
    const float rf = from_lp<T>(re), imf = from_lp<T>(im);
    const T nim = to_lp<T>(-imf);
    const bool tmpl = img >= o.Nq;
    const int seg = o.ldk;                     // one [re|im|0] segment
    const int row_len = o.split ? 2 * seg : seg;
    T *r = tmpl ? reinterpret_cast<T *>(o.lp_t) + (size_t)(kf - 1) * o.lpt_fstride +
                      (size_t)(2 * (img - o.Nq)) * row_len
                : reinterpret_cast<T *>(o.lp_q) + (size_t)(kf - 1) * o.lpq_fstride +
                      (size_t)img * row_len;
    if (!o.split) {
        kahan_add(acc16, w * fmaf(rf, rf, imf * imf));
        r[p] = re;
        r[M + p] = im;
        if (tmpl) {
            r[row_len + p] = nim;  // row 2j+1: [ -im | re | 0 ]
            r[row_len + M + p] = re;
        }
        return;
    }
    // FP16 split: lo = x - hi, exact in FP32, rounded to FP16; rows [hi | lo]
    // (the correlation reads segments hi hi, hi lo, lo hi of its operands)
    const T rel = to_lp<T>(X.x - rf), iml = to_lp<T>(X.y - imf);
    r[p] = re;
    r[M + p] = im;
    r[seg + p] = rel;
    r[seg + M + p] = iml;
    if (tmpl) {  // row 2j+1: [-im | re]
        const T nrel = to_lp<T>(-(X.y - imf));
        T *r2 = r + row_len;
        r2[p] = nim;
        r2[M + p] = re;
        r2[seg + p] = nrel;
        r2[seg + M + p] = rel;
    }
}

template <typename T>
struct Pair2;
template <>
struct Pair2<__half> {
    using V = __half2;
    static __device__ __forceinline__ V make(__half a, __half b) { return __halves2half2(a, b); }
};
template <>
struct Pair2<__nv_bfloat16> {
    using V = __nv_bfloat162;
    static __device__ __forceinline__ V make(__nv_bfloat16 a, __nv_bfloat16 b)
    {
        return __halves2bfloat162(a, b);
    }
};

// emit for the two levels pa (even) and pa + 1 of one frequency at once, M
// even: every row segment then takes the pair as one 4-byte store (FP32
// rows: one 8-byte store), the same values as two emit calls.
template <typename T>
__device__ __forceinline__ void emit2(const SpecOut &o, int img, int M, int kf, int pa, float2 Xa,
                                      float2 Xb, float w, DF &acc32, DF &acc16)
{
    kahan_add(acc32, w * fmaf(Xa.x, Xa.x, Xa.y * Xa.y));
    kahan_add(acc32, w * fmaf(Xb.x, Xb.x, Xb.y * Xb.y));
    if (!o.lp) {
        float *row = o.spec32 + (size_t)(kf - 1) * o.fstride + (size_t)img * 2 * M;
        *reinterpret_cast<float2 *>(row + pa) = make_float2(Xa.x, Xb.x);
        *reinterpret_cast<float2 *>(row + M + pa) = make_float2(Xa.y, Xb.y);
        return;
    }
    using P = Pair2<T>;
    using V = typename P::V;
    const T rea = to_lp<T>(Xa.x), ima = to_lp<T>(Xa.y), reb = to_lp<T>(Xb.x), imb = to_lp<T>(Xb.y);
    const float rfa = from_lp<T>(rea), imfa = from_lp<T>(ima);
    const float rfb = from_lp<T>(reb), imfb = from_lp<T>(imb);
    const bool tmpl = img >= o.Nq;
    const int seg = o.ldk;
    const int row_len = o.split ? 2 * seg : seg;
    T *r = tmpl ? reinterpret_cast<T *>(o.lp_t) + (size_t)(kf - 1) * o.lpt_fstride +
                      (size_t)(2 * (img - o.Nq)) * row_len
                : reinterpret_cast<T *>(o.lp_q) + (size_t)(kf - 1) * o.lpq_fstride +
                      (size_t)img * row_len;
    auto put = [](T *dst, V v) { *reinterpret_cast<V *>(dst) = v; };
    const V re2 = P::make(rea, reb), im2 = P::make(ima, imb);
    const V nim2 = P::make(to_lp<T>(-imfa), to_lp<T>(-imfb));
    if (!o.split) {
        kahan_add(acc16, w * fmaf(rfa, rfa, imfa * imfa));
        kahan_add(acc16, w * fmaf(rfb, rfb, imfb * imfb));
        put(r + pa, re2);
        put(r + M + pa, im2);
        if (tmpl) {
            put(r + row_len + pa, nim2);  // row 2j+1: [ -im | re | 0 ]
            put(r + row_len + M + pa, re2);
        }
        return;
    }
    // FP16 split: lo = x - hi, exact in FP32, rounded to FP16
    const V rel2 = P::make(to_lp<T>(Xa.x - rfa), to_lp<T>(Xb.x - rfb));
    const V iml2 = P::make(to_lp<T>(Xa.y - imfa), to_lp<T>(Xb.y - imfb));
    put(r + pa, re2);  // [hi | lo]
    put(r + M + pa, im2);
    put(r + seg + pa, rel2);
    put(r + seg + M + pa, iml2);
    if (tmpl) {  // row 2j+1: [-im | re]
        const V nrel2 = P::make(to_lp<T>(-(Xa.y - imfa)), to_lp<T>(-(Xb.y - imfb)));
        T *r2 = r + row_len;
        put(r2 + pa, nim2);
        put(r2 + M + pa, re2);
        put(r2 + seg + pa, nrel2);
        put(r2 + seg + M + pa, rel2);
    }
}

__device__ __forceinline__ void cpa16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
                 : "memory");
}

// Issue the copies of the level batch [p0, p0 + 2 nsig) of image qi into
// buf: signal s of angle k is buf[k nsig + s] = (level p0 + 2s, p0 + 2s + 1);
// levels past M are zero-filled.  With one part and M % 4 == 0 every angle's
// slice is whole 16-byte chunks; otherwise one 4-byte copy per level.
template <int nsig>
__device__ __forceinline__ void stage_levels(const float *__restrict__ qi, int n, int M, int Mp,
                                             int parts, int p0, float2 *buf)
{
    if (parts == 1 && (M & 3) == 0) {
        constexpr int CH = nsig / 2;  // 16-byte chunks (4 levels) per angle
        for (int c = threadIdx.x; c < n * CH; c += blockDim.x) {
            const int k = c / CH, h = c % CH;
            const int p = p0 + 4 * h;
            const int valid = min(max(M - p, 0), 4);
            const float *src = valid ? qi + (size_t)k * M + p : qi;
            cpa16(buf + k * nsig + 2 * h, src, 4 * valid);
        }
    } else {
        for (int c = threadIdx.x; c < n * 2 * nsig; c += blockDim.x) {
            const int k = c / (2 * nsig), e = c % (2 * nsig);
            const int p = p0 + e;
            const float *src = qi;
            if (p < M)
                src = parts == 1 ? qi + (size_t)k * M + p
                                 : qi + (size_t)(p / Mp) * n * Mp + (size_t)k * Mp + p % Mp;
            cpa4(reinterpret_cast<float *>(buf + k * nsig) + e, src, p < M ? 4 : 0);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename T, int nsig>
__global__ void __launch_bounds__(kSpecThreads)
k_spectrum(const float *__restrict__ q, int n, int M, FftPlan plan, const float2 *__restrict__ tw,
           SpecOut o, float *__restrict__ prof, double *__restrict__ center,
           double *__restrict__ norm32, double *__restrict__ norm16, int parts)
{
    // M levels in all; with parts = 2 (ramp-filtered distance) the levels
    // [0, M/2) and [M/2, M) are the quantiles of the positive and negative
    // parts, stored as [parts][n][M/2], and each part is centred by its own
    // vector.
    extern __shared__ __align__(16) float2 smc[];
    // two batch buffers: the staged input of the FFT and its other buffer;
    // once a batch's transform is done, the buffer it did not end in takes
    // the next batch's copies while the unpack reads the result
    float2 *bufA = smc;                  // [n nsig]
    float2 *bufB = bufA + n * nsig;      // [n nsig]
    float2 *x1 = bufB + n * nsig;        // [M] Qhat(1, p) before centring
    float2 *tws = x1 + M;                // [n] twiddles
    __shared__ double red[2][kSpecThreads / 32];
    __shared__ double s_c1[2][2];
    const int Mp = M / parts;  // levels per part
    const int img = blockIdx.x;
    const float *qi = q + (size_t)img * n * M;
    stage_levels<nsig>(qi, n, M, Mp, parts, 0, bufA);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tws[i] = tw[i];
    const int nh = n / 2;
    // norms as compensated (Kahan) FP32 sums: FP64 arithmetic is scarce on
    // this part
    DF acc32 = {0.f, 0.f}, acc16 = {0.f, 0.f};
    const float invn = 1.f / (float)n;

    float2 *cur = bufA, *oth = bufB;
    for (int p0 = 0; p0 < M; p0 += 2 * nsig) {
        // ---- batch: levels (p0 + 2s, p0 + 2s + 1) as signal s (re, im)
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        float2 *R = fft_smem<nsig, -1>(cur, oth, plan, tws);
        // the next batch goes to the buffer the transform did not end in
        // (fft_smem ends with a block barrier: both buffers' readers are done)
        float2 *nxt = R == cur ? oth : cur;
        if (p0 + 2 * nsig < M) stage_levels<nsig>(qi, n, M, Mp, parts, p0 + 2 * nsig, nxt);
        cur = nxt;
        oth = R;
        // ---- unpack two real spectra per signal, k' = 0..n/2
        for (int t = threadIdx.x; t < (nh + 1) * nsig; t += blockDim.x) {
            const int kf = t / nsig, s = t % nsig;
            const float2 Z = R[kf * nsig + s];
            const float2 Zc = cconj(R[((n - kf) % n) * nsig + s]);
            // Xa = (Z + conj Z(n-k))/2, Xb = (Z - conj Z(n-k)) / (2i)
            const float2 Xa = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
            const float2 dz = make_float2(0.5f * (Z.x - Zc.x), 0.5f * (Z.y - Zc.y));
            const float2 Xb = make_float2(dz.y, -dz.x);
            const int pa = p0 + 2 * s, pb = pa + 1;
            if (kf >= 2 && (M & 1) == 0 && pb < M) {
                // both levels at once (pa even, M even: 4-byte aligned pairs)
                float2 A = Xa, Bv = Xb;
                if (kf == nh) A.y = Bv.y = 0.f;  // Nyquist term of a real signal
                emit2<T>(o, img, M, kf, pa, A, Bv, kf == nh ? 1.f : 2.f, acc32, acc16);
                continue;
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int p = h2 ? pb : pa;
                if (p >= M) continue;
                float2 X = h2 ? Xb : Xa;
                if (kf == 0) {
                    prof[(size_t)img * M + p] = X.x * invn;
                } else if (kf == 1) {
                    x1[p] = X;
                } else {
                    if (kf == nh) X.y = 0.f;  // Nyquist term of a real signal
                    const float w = kf == nh ? 1.f : 2.f;
                    emit<T>(o, img, M, kf, p, X, w, acc32, acc16);
                }
            }
        }
        __syncthreads();
    }
    // ---- centring, per part: c1 = mean_p Qhat_u(1, p);  a = (2/n)(Re c1, -Im c1)
    for (int part = 0; part < parts; ++part) {
        double cr = 0.0, ci = 0.0;
        for (int p = part * Mp + threadIdx.x; p < (part + 1) * Mp; p += blockDim.x) {
            cr += x1[p].x;
            ci += x1[p].y;
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            cr += __shfl_xor_sync(0xffffffffu, cr, off);
            ci += __shfl_xor_sync(0xffffffffu, ci, off);
        }
        if (lane == 0) {
            red[0][warp] = cr;
            red[1][warp] = ci;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sr = 0.0, si = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                sr += red[0][w];
                si += red[1][w];
            }
            s_c1[part][0] = sr / Mp;
            s_c1[part][1] = si / Mp;
            double *cimg = center + 2 * ((size_t)img * parts + part);
            cimg[0] = 2.0 * s_c1[part][0] / n;
            cimg[1] = -2.0 * s_c1[part][1] / n;
        }
        __syncthreads();
    }
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
        const int part = p / Mp;
        const float c1r = (float)s_c1[part][0], c1i = (float)s_c1[part][1];
        const float2 X = make_float2(x1[p].x - c1r, x1[p].y - c1i);
        emit<T>(o, img, M, 1, p, X, 2.f, acc32, acc16);  // n >= 4: k' = 1 < n/2
    }
    // ---- zero padding of the low-precision rows: [2M, ldk) of every segment
    if (o.lp && o.ldk > 2 * M) {
        const int pad = o.ldk - 2 * M;
        const bool tmpl = img >= o.Nq;
        const int nseg = o.split ? 2 : 1;
        const int row_len = nseg * o.ldk;
        const int rows = tmpl ? 2 : 1;
        const int per_f = rows * nseg * pad;
        for (int t = threadIdx.x; t < nh * per_f; t += blockDim.x) {
            const int kf = 1 + t / per_f, rem = t % per_f;
            const int rr = rem / (nseg * pad), sg = (rem / pad) % nseg, e = 2 * M + rem % pad;
            T *r = tmpl ? reinterpret_cast<T *>(o.lp_t) + (size_t)(kf - 1) * o.lpt_fstride +
                              (size_t)(2 * (img - o.Nq) + rr) * row_len
                        : reinterpret_cast<T *>(o.lp_q) + (size_t)(kf - 1) * o.lpq_fstride +
                              (size_t)img * row_len;
            r[sg * o.ldk + e] = to_lp<T>(0.f);
        }
    }
    // ---- norms: Parseval over k' != 0 of the centred spectra, / n
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double a32 = (double)acc32.hi + (double)acc32.lo;
    double a16 = (double)acc16.hi + (double)acc16.lo;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        a32 += __shfl_xor_sync(0xffffffffu, a32, off);
        a16 += __shfl_xor_sync(0xffffffffu, a16, off);
    }
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = a32;
        red[1][warp] = a16;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s32 = 0.0, s16 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s32 += red[0][w];
            s16 += red[1][w];
        }
        norm32[img] = s32 / n;
        if (norm16) norm16[img] = s16 / n;
    }
}

}  // namespace

cudaError_t launch_spectrum(const float *q, int nb, int n, int M, const FftPlan &plan,
                            const float2 *tw, float *spec32, size_t fstride, int lp_kind,
                            void *lp_q, size_t lpq_fstride, void *lp_t, size_t lpt_fstride,
                            int Nq, float *prof, double *center, double *norm32,
                            double *norm16, cudaStream_t st, int nsig_req, int parts)
{
    if (parts != 1 && (parts != 2 || M % 2)) return cudaErrorInvalidValue;
    if (nb <= 0) return cudaSuccess;
    // signals per FFT batch: 16 by default, 8 at n = 1024; a requested
    // width is taken when its buffers fit (2 n nsig complex values)
    int nsig = n <= 512 ? 16 : 8;
    if ((nsig_req == 4 || nsig_req == 8 || nsig_req == 16) && (size_t)n * nsig_req <= 8192)
        nsig = nsig_req;
    // two batch buffers (the staged input and the FFT's other buffer),
    // within the 227 KB a CTA can hold
    auto smem_of = [&](int ns) { return sizeof(float2) * ((size_t)2 * n * ns + M + n); };
    while (nsig > 4 && smem_of(nsig) > kSmemOptIn) nsig /= 2;
    const size_t smem = smem_of(nsig);
    if (smem > kSmemOptIn) return cudaErrorInvalidValue;
    SpecOut o{spec32, fstride, lp_q, lpq_fstride, lp_t, lpt_fstride, Nq, tc_ldk(M),
              lp_kind != 0, lp_kind == 3};
#define SW_SPEC_LAUNCH(T, NS)                                                                    \
    do {                                                                                        \
        cudaFuncSetAttribute(k_spectrum<T, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)smem);                                                        \
        k_spectrum<T, NS><<<nb, kSpecThreads, smem, st>>>(q, n, M, plan, tw, o, prof, center,  \
                                                          norm32, norm16, parts);               \
    } while (0)
    if (lp_kind == 2 || lp_kind == 3) {
        if (nsig == 16) SW_SPEC_LAUNCH(__half, 16);
        else if (nsig == 8) SW_SPEC_LAUNCH(__half, 8);
        else SW_SPEC_LAUNCH(__half, 4);
    } else {
        if (nsig == 16) SW_SPEC_LAUNCH(__nv_bfloat16, 16);
        else if (nsig == 8) SW_SPEC_LAUNCH(__nv_bfloat16, 8);
        else SW_SPEC_LAUNCH(__nv_bfloat16, 4);
    }
#undef SW_SPEC_LAUNCH
    return cudaGetLastError();
}

}  // namespace swk
