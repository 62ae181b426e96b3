// sw_project.cu -- Radon projection of images at nh = n/2 angles in [0, pi)
// (Eq. radon_transform, Sec. 2.1; Sec. 2.3 "Computation"), as a
// pixel-driven linear splat: a cell at (x, y) with value f adds
// f * max(0, 1 - |u - b|) to bin b, u = <(x,y), theta>/h + (B-1)/2.
// The angles theta + pi are the mirror images (P_{theta+pi} f(s) = P_theta f(-s))
// and are not recomputed.
//
// Design (GB300): the splat is evaluated as a deterministic gather.  A warp
// owns one angle and 32 consecutive bins; each lane walks the rows (or the
// columns, when the direction is closer to the y axis) of an image held in
// shared memory and sums the <= 3 cells whose projection falls within one
// bin of its own.  No atomics, so results are bitwise reproducible and
// independent of batching.  Rows whose projection misses the warp's 32 bins
// are skipped.  When n % 4 == 0 and the image fits in shared memory
// (k_project4), one set of weights serves four angles through the square's
// symmetries; otherwise (k_project) images are processed tile by tile with
// zero borders, accumulating in shared memory.
#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int kProjThreads = 512;
constexpr int kPad = 2;  // zero border (cells) around the staged tile

struct TileGeom {
    int T;   // tile side
    int S;   // row stride of the staged tile (odd, >= T + 2*kPad)
    int nt;  // tiles per side
};

__host__ __device__ inline TileGeom tile_geom(int L)
{
    TileGeom g;
    g.T = L <= 128 ? L : 128;
    g.nt = (L + g.T - 1) / g.T;
    g.S = g.T + 2 * kPad;
    if ((g.S & 1) == 0) g.S += 1;
    return g;
}

__global__ void __launch_bounds__(kProjThreads)
k_project(const float *__restrict__ img, int L, int srcL, int nh, int B, int G,
          const float2 *__restrict__ cs, float *__restrict__ out, int full_n,
          int32_t *__restrict__ status, const float *__restrict__ img2, int nb1)
{
    extern __shared__ float smem[];
    const TileGeom tg = tile_geom(L);
    const int T = tg.T, S = tg.S;
    const int rowsT = T + 2 * kPad;
    float *tile = smem;                      // [rowsT][S]
    const int Bp = (B + 31) & ~31;
    float *acc = tile + rowsT * S;           // [G][Bp]
    __shared__ int s_bad, s_mass;

    const int imgi = blockIdx.y;
    const int k0 = blockIdx.x * G;
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // images [0, nb1) from img, the rest from img2 (two batches in one launch)
    const float *src = imgi < nb1 ? img + (size_t)imgi * srcL * srcL
                                  : img2 + (size_t)(imgi - nb1) * srcL * srcL;

    if (threadIdx.x == 0) {
        s_bad = 0;
        s_mass = 0;
    }
    for (int i = threadIdx.x; i < G * Bp; i += blockDim.x) acc[i] = 0.f;

    const float half_L1 = 0.5f * (float)(L - 1);
    const float half_B1 = 0.5f * (float)(B - 1);
    const int ngroups = Bp >> 5;
    const int nitems = G * ngroups;
    int bad = 0, mass = 0;

    for (int tr = 0; tr < tg.nt; ++tr) {
        for (int tc = 0; tc < tg.nt; ++tc) {
            __syncthreads();
            // ---- stage tile (rows tr*T.., cols tc*T..) with a zero border
            for (int idx = threadIdx.x; idx < rowsT * S; idx += blockDim.x) {
                const int rr = idx / S - kPad, cc = idx % S - kPad;
                const int r = tr * T + rr, c = tc * T + cc;
                float v = 0.f;
                if (rr >= 0 && rr < T && cc >= 0 && cc < T && r < L && c < L) {
                    if (srcL == L) v = __ldg(src + (size_t)r * L + c);
                    else v = 0.25f * __ldg(src + (size_t)(r >> 1) * srcL + (c >> 1));
                    if (!isfinite(v)) {
                        bad = 1;
                        v = 0.f;
                    }
                    v = fmaxf(v, 0.f);
                    mass |= v > 0.f;
                }
                tile[idx] = v;
            }
            __syncthreads();
            // ---- warp items: (angle a, bin group g)
            const float q0 = (float)(tc * T) - half_L1;  // centred x of tile column 0
            const float m0 = (float)(tr * T) - half_L1;  // centred y of tile row 0
            for (int it = warp; it < nitems; it += nwarps) {
                const int a = it / ngroups, g = it % ngroups;
                const int k = k0 + a;
                if (k >= nh) continue;
                const float2 t = cs[k];
                const bool rowmode = fabsf(t.x) >= fabsf(t.y);
                // minor index q runs along x in row mode (y in column mode)
                const float kq = rowmode ? t.x : t.y;
                const float km = rowmode ? t.y : t.x;
                const float qc0 = rowmode ? q0 : m0;  // centred coord of minor index 0
                const float mc0 = rowmode ? m0 : q0;  // centred coord of major index 0
                const int sq = rowmode ? 1 : S;       // smem stride of the minor index
                const int sm = rowmode ? S : 1;       // smem stride of the major index
                const int b0 = g << 5;
                // rows whose projection can reach bins [b0-1, b0+32]:
                // u(q, m) = q kq + m km + U0, q in [0, T), m in [0, T)
                const float U0 = fmaf(qc0, kq, fmaf(mc0, km, half_B1));
                const float ext = (float)(T - 1) * kq;
                const float umin = U0 + fminf(0.f, ext), umax = U0 + fmaxf(0.f, ext);
                int mlo = 0, mhi = T - 1;
                if (fabsf(km) > 1e-6f) {
                    // need umin + m km <= b0 + 32 and umax + m km >= b0 - 1
                    float ma = ((float)b0 + 32.f - umin) / km;
                    float mb = ((float)b0 - 1.f - umax) / km;
                    float lo = fminf(ma, mb), hi = fmaxf(ma, mb);
                    lo = fmaxf(lo - 1.f, 0.f);
                    hi = fminf(hi + 1.f, (float)(T - 1));
                    if (lo > hi) continue;
                    mlo = (int)lo;
                    mhi = (int)hi;
                } else if (umax < (float)b0 - 1.f || umin > (float)b0 + 32.f) {
                    continue;
                }
                const int b = b0 + lane;
                // d(q, m) = u(q, m) - b = q kq + beta_m
                const float Ab = fmaf(qc0, kq, half_B1 - (float)b);
                const float invk = 1.f / kq;
                const float cw = -1.f / fabsf(kq);
                float sum = 0.f;
                for (int m = mlo; m <= mhi; ++m) {
                    const float beta = fmaf(mc0 + (float)m, km, Ab);
                    const float qlo = fmaf(-beta, invk, cw);  // window (qlo, qlo + 2/|kq|)
                    float qs = floorf(qlo) + 1.f;
                    qs = fminf(fmaxf(qs, -2.f), (float)(T - 1));
                    const int qi = (int)qs;
                    const float d0 = fmaf(qs, kq, beta);
                    const float d1 = d0 + kq, d2 = d1 + kq;
                    const float *p = tile + (m + kPad) * sm + (qi + kPad) * sq;
                    const float w0 = fmaxf(0.f, 1.f - fabsf(d0));
                    const float w1 = fmaxf(0.f, 1.f - fabsf(d1));
                    const float w2 = fmaxf(0.f, 1.f - fabsf(d2));
                    sum = fmaf(w0, p[0], sum);
                    sum = fmaf(w1, p[sq], sum);
                    sum = fmaf(w2, p[2 * sq], sum);
                }
                acc[a * Bp + b] += sum;
            }
        }
    }
    // ---- image status (every block of an image computes the same flags)
    if (bad) atomicOr(&s_bad, 1);
    if (mass) atomicOr(&s_mass, 1);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) status[imgi] = (s_bad || !s_mass) ? 1 : 0;
    // ---- write
    const int nrow = full_n ? 2 * nh : nh;
    for (int i = threadIdx.x; i < G * B; i += blockDim.x) {
        const int a = i / B, b = i % B;
        const int k = k0 + a;
        if (k >= nh) continue;
        const float v = acc[a * Bp + b];
        float *o = out + ((size_t)imgi * nrow + k) * B;
        o[b] = v;
        if (full_n) o[(size_t)nh * B + (B - 1 - b)] = v;
    }
}

// ---------------------------------------------------------------------------
// Four angles per set of weights.  For theta in [0, pi/4] the angles
// pi/2 - theta, pi/2 + theta and pi - theta are theta applied to exact cell
// permutations of the image (transpose and flips), so the splat weights of a
// cell of the canonical frame serve all four:
//   view 1: F[m][q]        -> angle k
//   view 2: F[q][m]        -> angle n/4 - k
//   view 3: F[q][L-1-m]    -> angle n/4 + k
//   view 4: F[m][L-1-q]    -> angle n/2 - k
// for canonical k with 8k <= n (needs n % 4 == 0).  Duplicates (k = 0, 8k = n)
// are written once.  The image sits in shared memory with a zero border of
// two cells, so every view reads it in place.
//
// BANDED (images too large for shared memory): the CTA holds the rows
// [r0, r1) of the image only (blockIdx.z = band, two bands).  Its rows give
// views 1 and 4 of the canonical rows m in the band, and, as rows q of
// views 2 and 3, their cells' share of every canonical row m; cells outside
// the band read as zero.  The two bands' partial sums are added into the
// output (zeroed by the launcher): two addends onto an exact zero give the
// same sum in either order, so the result stays deterministic.
constexpr int kMaxL4 = 200;

template <bool BANDED>
__global__ void __launch_bounds__(kProjThreads)
k_project4(const float *__restrict__ img, int L, int srcL, int n, int B, int per, int kc,
           const float2 *__restrict__ cs, float *__restrict__ out, int full_n,
           int32_t *__restrict__ status, int band_rows, const float *__restrict__ img2, int nb1)
{
    // this CTA's canonical angles: [kc0, kc0 + kcn)
    const int kc0 = blockIdx.x * per;
    const int kcn = min(per, kc - kc0);
    extern __shared__ float tile[];
    const int S = ((L + 2 * kPad) & 1) ? L + 2 * kPad : L + 2 * kPad + 1;
    const int r0 = BANDED ? blockIdx.z * band_rows : 0;
    const int r1 = BANDED ? min(L, r0 + band_rows) : L;
    const int rowsT = (r1 - r0) + 2 * kPad;
    __shared__ int s_bad, s_mass;
    const int imgi = blockIdx.y;
    // images [0, nb1) from img, the rest from img2 (two batches in one launch)
    const float *src = imgi < nb1 ? img + (size_t)imgi * srcL * srcL
                                  : img2 + (size_t)(imgi - nb1) * srcL * srcL;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_mass = 0;
    }
    __syncthreads();
    int bad = 0, mass = 0;
    for (int idx = threadIdx.x; idx < rowsT * S; idx += blockDim.x) {
        const int r = idx / S - kPad + r0, c = idx % S - kPad;
        float v = 0.f;
        if (r >= r0 && r < r1 && c >= 0 && c < L) {
            if (srcL == L) v = __ldg(src + (size_t)r * L + c);
            else v = 0.25f * __ldg(src + (size_t)(r >> 1) * srcL + (c >> 1));
            if (!isfinite(v)) {
                bad = 1;
                v = 0.f;
            }
            v = fmaxf(v, 0.f);
            mass |= v > 0.f;
        }
        tile[idx] = v;
    }
    if (bad) atomicOr(&s_bad, 1);
    if (mass) atomicOr(&s_mass, 1);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!BANDED) status[imgi] = (s_bad || !s_mass) ? 1 : 0;
        else if (s_bad) atomicOr(status + imgi, 1);  // no mass: flagged by the quantiles
    }

    const int nh = n / 2, n4 = n / 4;
    const int nrow = full_n ? n : nh;
    const int Bp = (B + 31) & ~31;
    const int ngroups = Bp >> 5;
    const int nitems = kcn * ngroups;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const float c0 = 0.5f * (float)(L - 1);
    const float half_B1 = 0.5f * (float)(B - 1);
    float *outi = out + (size_t)imgi * nrow * B;
    // tile row of image row r (views 1, 4 read rows m; views 2, 3 rows q)
    const float *trow = tile + (kPad - r0) * S + kPad;

    for (int it = warp; it < nitems; it += nwarps) {
        const int k = kc0 + it / ngroups, g = it % ngroups;
        const float2 t = cs[k];  // cos >= sin >= 0
        const float kq = t.x, km = t.y;
        const int b0 = g << 5;
        // u(q, m) = q kq + m km + U0 on the canonical frame, q, m in [0, L)
        const float U0 = fmaf(-c0, kq, fmaf(-c0, km, half_B1));
        const float ext = (float)(L - 1) * kq;
        // rows m that can reach bins [b0-1, b0+32] (views 1, 4: any q; views
        // 2, 3 in a band: q in [r0, r1)); an empty range still writes its
        // (zero) bins below
        int mlo = 0, mhi = L - 1, nlo = 0, nhi = L - 1;
        if (km > 1e-6f) {
            float hi = ((float)b0 + 32.f - U0) / km;
            float lo = ((float)b0 - 1.f - U0 - ext) / km;
            lo = fmaxf(floorf(lo) - 1.f, 0.f);
            hi = fminf(ceilf(hi) + 1.f, (float)(L - 1));
            mlo = (int)lo;
            mhi = lo > hi ? mlo - 1 : (int)hi;
            if (BANDED) {
                float h2 = ((float)b0 + 32.f - U0 - (float)r0 * kq) / km;
                float l2 = ((float)b0 - 1.f - U0 - (float)(r1 - 1) * kq) / km;
                l2 = fmaxf(floorf(l2) - 1.f, 0.f);
                h2 = fminf(ceilf(h2) + 1.f, (float)(L - 1));
                nlo = (int)l2;
                nhi = l2 > h2 ? nlo - 1 : (int)h2;
            }
        } else if (U0 + ext < (float)b0 - 1.f || U0 > (float)b0 + 32.f) {
            mhi = -1;
            nhi = -1;
        }
        int m14lo = mlo, m14hi = mhi, m23lo = mlo, m23hi = mhi;
        if (BANDED) {
            m14lo = max(mlo, r0);
            m14hi = min(mhi, r1 - 1);
            m23lo = max(mlo, nlo);
            m23hi = min(mhi, nhi);
        }
        const int mfrom = min(m14lo, m23lo), mto = max(m14hi, m23hi);
        const int b = b0 + lane;
        const float Ab = fmaf(-c0, kq, half_B1 - (float)b);
        const float invk = 1.f / kq;
        float s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
        for (int m = mfrom; m <= mto; ++m) {
            const float beta = fmaf((float)m - c0, km, Ab);  // d(q) = q kq + beta
            const float qlo = fmaf(-beta, invk, -invk);       // window (qlo, qlo + 2/kq)
            const float qf = floorf(qlo) + 1.f;
            if (!BANDED || (m >= m14lo && m <= m14hi)) {
                const float qs = fminf(fmaxf(qf, -2.f), (float)(L - 1));
                const int qi = __float_as_int(qs + 12582912.f) - 0x4B400000;  // exact small int
                const float d0 = fmaf(qs, kq, beta), d1 = d0 + kq, d2 = d1 + kq;
                const float w0 = fmaxf(0.f, 1.f - fabsf(d0));
                const float w1 = fmaxf(0.f, 1.f - fabsf(d1));
                const float w2 = fmaxf(0.f, 1.f - fabsf(d2));
                const float *r1p = trow + m * S + qi;
                const float *r4p = trow + m * S + (L - 1 - qi);
                s1 = fmaf(w0, r1p[0], s1);
                s4 = fmaf(w0, r4p[0], s4);
                s1 = fmaf(w1, r1p[1], s1);
                s4 = fmaf(w1, r4p[-1], s4);
                s1 = fmaf(w2, r1p[2], s1);
                s4 = fmaf(w2, r4p[-2], s4);
                if (!BANDED) {  // same cells as rows q: views 2, 3 share the weights
                    const float *r2p = trow + qi * S + m;
                    const float *r3p = trow + qi * S + (L - 1 - m);
                    s2 = fmaf(w0, r2p[0], s2);
                    s3 = fmaf(w0, r3p[0], s3);
                    s2 = fmaf(w1, r2p[S], s2);
                    s3 = fmaf(w1, r3p[S], s3);
                    s2 = fmaf(w2, r2p[2 * S], s2);
                    s3 = fmaf(w2, r3p[2 * S], s3);
                }
            }
            if (BANDED && m >= m23lo && m <= m23hi) {
                // rows q of views 2, 3 clamped to the band's tile rows
                const float qs = fminf(fmaxf(qf, (float)(r0 - 2)), (float)(r1 - 1));
                const int qi = __float_as_int(qs + 12582912.f) - 0x4B400000;
                const float d0 = fmaf(qs, kq, beta), d1 = d0 + kq, d2 = d1 + kq;
                const float w0 = fmaxf(0.f, 1.f - fabsf(d0));
                const float w1 = fmaxf(0.f, 1.f - fabsf(d1));
                const float w2 = fmaxf(0.f, 1.f - fabsf(d2));
                const float *r2p = trow + qi * S + m;
                const float *r3p = trow + qi * S + (L - 1 - m);
                s2 = fmaf(w0, r2p[0], s2);
                s3 = fmaf(w0, r3p[0], s3);
                s2 = fmaf(w1, r2p[S], s2);
                s3 = fmaf(w1, r3p[S], s3);
                s2 = fmaf(w2, r2p[2 * S], s2);
                s3 = fmaf(w2, r3p[2 * S], s3);
            }
        }
        if (b >= B) continue;
        const int angle[4] = {k, n4 - k, n4 + k, nh - k};
        const bool keep[4] = {true, 8 * k != n, k != 0, k != 0 && 8 * k != n};
        const float val[4] = {s1, s2, s3, s4};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (!keep[v]) continue;
            float *o = outi + (size_t)angle[v] * B;
            if (BANDED) {
                atomicAdd(o + b, val[v]);
                if (full_n) atomicAdd(o + (size_t)nh * B + (B - 1 - b), val[v]);
            } else {
                o[b] = val[v];
                if (full_n) o[(size_t)nh * B + (B - 1 - b)] = val[v];
            }
        }
    }
}

// Ingest (row a1 of the path): the clipped mass m = sum max(pixel, 0) of
// each image in FP64 and its normalising scale 1 / m (Sec. 1.1: images are
// probability densities; Sec. 5.4's g+ rule clips negatives).  One CTA per
// image; NaN for an image with no positive mass or a non-finite pixel.
constexpr int kScaleThreads = 256;

__global__ void __launch_bounds__(kScaleThreads) k_image_scale(const float *__restrict__ img,
                                                                int L, double *__restrict__ scale)
{
    const float *im = img + (size_t)blockIdx.x * L * L;
    const int np = L * L;
    double m = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < np; i += kScaleThreads) {
        const float x = __ldg(im + i);
        if (!isfinite(x)) bad = 1;
        else if (x > 0.f) m += (double)x;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, off);
        bad |= __shfl_xor_sync(0xffffffffu, bad, off);
    }
    __shared__ double sm[kScaleThreads / 32];
    __shared__ int sb[kScaleThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sm[w] = m;
        sb[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int b = 0;
        for (int i = 0; i < kScaleThreads / 32; ++i) {  // fixed order: reproducible
            t += sm[i];
            b |= sb[i];
        }
        scale[blockIdx.x] = (b || !(t > 0.0)) ? __longlong_as_double(0x7ff8000000000000ULL)
                                               : 1.0 / t;
    }
}

}  // namespace

cudaError_t launch_image_scale(const float *img, int nb, int L, double *scale, cudaStream_t st)
{
    if (nb <= 0) return cudaSuccess;
    k_image_scale<<<nb, kScaleThreads, 0, st>>>(img, L, scale);
    return cudaGetLastError();
}

cudaError_t launch_project(const float *img, int nb, int L, int srcL, int nh, int B,
                           const float2 *cs, float *out, int full_n, int32_t *status,
                           cudaStream_t st, int want_ctas, const float *img2, int nb_first)
{
    if (nb <= 0) return cudaSuccess;
    const int nb1 = (img2 && nb_first >= 0) ? nb_first : nb;
    const int n = 2 * nh;
    // four-view kernel: the whole image in shared memory up to L = 200;
    // beyond, two row bands per image while a band fits in 200 KB (L <= 312)
    const int S4 = ((L + 2 * kPad) & 1) ? L + 2 * kPad : L + 2 * kPad + 1;
    const int band = (L + 1) / 2;
    const size_t band_smem = sizeof(float) * (size_t)(band + 2 * kPad) * S4;
    const bool banded = L > kMaxL4 && band_smem <= 200 * 1024;
    if (n % 4 == 0 && (L <= kMaxL4 || banded)) {
        // canonical angles k = 0..n/8; split over CTAs when the batch is
        // small.  Default target: ~3 resident CTAs per SM on 152 SMs.
        const int kc = n / 8 + 1;
        const int want = want_ctas > 0 ? want_ctas : 456;
        const int nbands = banded ? 2 : 1;
        int groups = nb * nbands >= want ? 1 : (want + nb * nbands - 1) / (nb * nbands);
        if (groups > kc) groups = kc;
        const int per = (kc + groups - 1) / groups;
        groups = (kc + per - 1) / per;
        dim3 grid(groups, nb, nbands);
        if (!banded) {
            const size_t smem = sizeof(float) * (size_t)(L + 2 * kPad) * S4;
            cudaFuncSetAttribute(k_project4<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
            k_project4<false><<<grid, kProjThreads, smem, st>>>(img, L, srcL, n, B, per, kc, cs,
                                                                out, full_n, status, L, img2,
                                                                nb1);
        } else {
            const size_t rows = (size_t)nb * (full_n ? n : nh) * B;
            cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * rows, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t) * nb, st);
            if (e != cudaSuccess) return e;
            cudaFuncSetAttribute(k_project4<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
            k_project4<true><<<grid, kProjThreads, band_smem, st>>>(img, L, srcL, n, B, per, kc,
                                                                    cs, out, full_n, status, band,
                                                                    img2, nb1);
        }
        return cudaGetLastError();
    }
    const TileGeom tg = tile_geom(L);
    const int Bp = (B + 31) & ~31;
    int G = 16;
    if (nh < G) G = nh;
    const size_t smem = sizeof(float) * ((size_t)(tg.T + 2 * kPad) * tg.S + (size_t)G * Bp);
    cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    dim3 grid((nh + G - 1) / G, nb);
    k_project<<<grid, kProjThreads, smem, st>>>(img, L, srcL, nh, B, G, cs, out, full_n, status,
                                                img2, nb1);
    return cudaGetLastError();
}

}  // namespace swk
