// sw_quantile.cu -- quantile functions of the projections (Sec. 2.3
// "Computation": CDF by cumulative sum, ICDF by linear interpolation;
// Eq. inv_cdf read with the ">=" of App. A.1.1).
//
// For one projection U[0..B) with nodes e_j = (j - B/2) h:
//   F_0 = 0, F_j = sum_{b<j} U_b,  tau_p = z_p F_B,
//   j* = min{ j >= 1 : F_j >= tau_p },
//   Q(z_p) = e_{j*-1} + h (tau_p - F_{j*-1}) / U_{j*-1};
// at tau = 0 (level p = 0 under the p/M rule) every t qualifies and Q is the
// left end of the domain, e_0.
//
// Design (GB300): one warp per projection, four projections per warp, the next
// one staged by cp.async while the current one is computed.  The CDF is a warp
// scan of double-float partial sums (TwoSum-compensated FP32) kept in shared
// memory, so that tau - F_{j-1} keeps ~48 bits even where it cancels; each
// lane then binary-searches its levels.  No FP64 on this path.
#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int kQThreads = 256;  // 8 warps

// a + b for double-floats of non-negative value (every partial sum of a
// projection row): TwoSum of the leading parts, then the tails, then a
// Fast2Sum renormalisation -- exact, since without cancellation the tail
// sum is below an ulp and a half of the leading sum, which Fast2Sum needs.
// The same (hi, lo) as df_add with its second TwoSum, in three fewer flops.
__device__ __forceinline__ DF df_add_nonneg(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo);
    const float hi = s.hi + e;
    return {hi, e - (hi - s.hi)};
}
constexpr int kQRows = 4;       // projections per warp: the next is staged while one is computed

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}

// Issue the copies of projection k of image imgi into U (reversed for the
// mirrored half: row k + n/2 of a half projection is row k read backwards).
__device__ __forceinline__ void stage_row(float *U, const float *__restrict__ proj, int n, int B,
                                          int half, int imgi, int k, int lane)
{
    const int nh = n / 2;
    const bool mirror = half && k >= nh;
    const float *row = half ? proj + ((size_t)imgi * nh + (mirror ? k - nh : k)) * B
                            : proj + ((size_t)imgi * n + k) * B;
    for (int b = lane; b < B; b += 32) cp_async4(U + b, mirror ? row + B - 1 - b : row + b);
}

__global__ void __launch_bounds__(kQThreads)
k_quantiles(const float *__restrict__ proj, int n, int B, int M, float h, int level_rule,
            int half, int mirror_out, float *__restrict__ q, int32_t *__restrict__ status,
            int status_shift)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int imgi = blockIdx.y;
    const int nrows = mirror_out ? n / 2 : n;
    const int k0 = (blockIdx.x * nw + warp) * kQRows;
    if (k0 >= nrows) return;  // whole warp leaves; no block barrier below
    const int kend = min(nrows, k0 + kQRows);
    // per warp: two U buffers (B+1 floats, padded to even) then F (B+1
    // float2) and the quantiles: every region and every F starts 8-byte aligned
    const int ue = (B + 1) + ((B + 1) & 1);
    const int stride = 2 * ue + 2 * (B + 1) + M + (M & 1);
    float *Ubuf = sm + warp * stride;                            // [2][ue]
    float2 *F = reinterpret_cast<float2 *>(Ubuf + 2 * ue);       // [B+1] (hi, lo)
    float *qb = reinterpret_cast<float *>(F + (B + 1));          // [M] this projection's quantiles
    stage_row(Ubuf, proj, n, B, half, imgi, k0, lane);
    asm volatile("cp.async.commit_group;" ::: "memory");

    for (int k = k0, r = 0; k < kend; ++k, ++r) {
        if (k + 1 < kend) stage_row(Ubuf + ((r + 1) & 1) * ue, proj, n, B, half, imgi, k + 1, lane);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // projection k has landed
        __syncwarp();
        const float *U = Ubuf + (r & 1) * ue;

        // ---- compensated prefix sums: lane owns bins [c0, c1)
        const int C = (B + 31) / 32;
        const int c0 = min(B, lane * C), c1 = min(B, c0 + C);
        DF s = {0.f, 0.f};
        for (int b = c0; b < c1; ++b) s = df_add_nonneg(s, DF{U[b], 0.f});
        // inclusive warp scan of the lane sums
        DF inc = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            DF o;
            o.hi = __shfl_up_sync(0xffffffffu, inc.hi, off);
            o.lo = __shfl_up_sync(0xffffffffu, inc.lo, off);
            if (lane >= off) inc = df_add_nonneg(o, inc);
        }
        DF run;
        run.hi = __shfl_up_sync(0xffffffffu, inc.hi, 1);
        run.lo = __shfl_up_sync(0xffffffffu, inc.lo, 1);
        if (lane == 0) {
            run = {0.f, 0.f};
            F[0] = make_float2(0.f, 0.f);
        }
        for (int b = c0; b < c1; ++b) {
            run = df_add_nonneg(run, DF{U[b], 0.f});
            F[b + 1] = make_float2(run.hi, run.lo);
        }
        __syncwarp();
        const DF total = {F[B].x, F[B].y};
        float *qo = q + ((size_t)imgi * n + k) * M;
        if (!(total.hi > 0.f) || !isfinite(total.hi)) {
            for (int p = lane; p < M; p += 32) qo[p] = __int_as_float(0x7fc00000);
            if (mirror_out) {
                float *qm = q + ((size_t)imgi * n + k + n / 2) * M;
                for (int p = lane; p < M; p += 32) qm[p] = __int_as_float(0x7fc00000);
            }
            if (lane == 0) atomicOr(status + (imgi >> status_shift), 1);
        } else {
            const float dz = level_rule == 0 ? 2.f * M : (float)M;
            const float inv_dz = 1.f / dz;
            // lane owns levels [pb, pe): one binary search, then a forward walk
            // (the levels increase, so j* never decreases)
            const int P = (M + 31) / 32;
            const int pb = min(M, lane * P), pe = min(M, pb + P);
            int j = 1;
            for (int p = pb; p < pe; ++p) {
                // tau = z_p F_B with z_p = (2p+1)/(2M) or p/M, formed exactly
                const float kz = level_rule == 0 ? 2.f * p + 1.f : (float)p;
                float Q;
                if (kz == 0.f) {
                    Q = -0.5f * (float)B * h;  // inf{t : F(t) >= 0}: the domain's left end e_0
                } else {
                    const DF tau = df_scale_ratio(total, kz, dz, inv_dz);
                    if (p == pb || (level_rule == 1 && p == 1)) {
                        int lo = 1, hi = B;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            const float2 f = F[mid];
                            if (df_ge(DF{f.x, f.y}, tau)) hi = mid;
                            else lo = mid + 1;
                        }
                        j = lo;
                    } else {
                        while (j < B) {
                            const float2 f = F[j];
                            if (df_ge(DF{f.x, f.y}, tau)) break;
                            ++j;
                        }
                    }
                    const float2 fj = F[j - 1];
                    const float num = (tau.hi - fj.x) + (tau.lo - fj.y);
                    const float den = U[j - 1];
                    // the fraction only scales h: a fast divide (error ~2 ulp) is ample
                    float frac = den > 0.f ? __fdividef(num, den) : 0.f;
                    frac = fminf(fmaxf(frac, 0.f), 1.f);
                    const float ej = ((float)(j - 1) - 0.5f * (float)B) * h;
                    Q = fmaf(h, frac, ej);
                }
                qb[p] = Q;
            }
            __syncwarp();
            for (int p = lane; p < M; p += 32) qo[p] = qb[p];
            if (mirror_out) {
                // theta + pi: the mirrored histogram has Q'(z) = -Q(1 - z), and
                // with midpoint levels 1 - z_p = z_{M-1-p}
                float *qm = q + ((size_t)imgi * n + k + n / 2) * M;
                for (int p = lane; p < M; p += 32) qm[p] = -qb[M - 1 - p];
            }
        }
        __syncwarp();  // U, F and qb are free for the next projection
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Centring vector and centred norm (public sw_quantiles outputs).  One block
// per image; FP64 accumulation.
__global__ void k_center_norm(const float *__restrict__ q, int n, int M,
                              const double2 *__restrict__ cs64, double *__restrict__ center,
                              double *__restrict__ norm)
{
    __shared__ double red[3][32];
    __shared__ double s_a[2];
    const int imgi = blockIdx.x;
    const float *qi = q + (size_t)imgi * n * M;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // a = (2/n) sum_k ubar_k (cos, sin),  ubar_k = mean_p q[k][p]
    double ax = 0.0, ay = 0.0;
    for (int k = warp; k < n; k += nw) {
        double s = 0.0;
        for (int p = lane; p < M; p += 32) s += (double)qi[(size_t)k * M + p];
#pragma unroll
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        const double ub = s / M;
        ax += ub * cs64[k].x;
        ay += ub * cs64[k].y;
    }
    if (lane == 0) {
        red[0][warp] = ax;
        red[1][warp] = ay;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sx = 0.0, sy = 0.0;
        for (int w = 0; w < nw; ++w) {
            sx += red[0][w];
            sy += red[1][w];
        }
        s_a[0] = sx * 2.0 / n;
        s_a[1] = sy * 2.0 / n;
    }
    __syncthreads();
    const double a0 = s_a[0], a1 = s_a[1];
    double acc = 0.0;
    for (int k = warp; k < n; k += nw) {
        const double off = a0 * cs64[k].x + a1 * cs64[k].y;
        for (int p = lane; p < M; p += 32) {
            const double d = (double)qi[(size_t)k * M + p] - off;
            acc += d * d;
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) red[2][warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[2][w];
        if (center) {
            center[2 * imgi] = a0;
            center[2 * imgi + 1] = a1;
        }
        if (norm) norm[imgi] = s;
    }
}

}  // namespace

cudaError_t launch_quantiles(const float *proj, int nb, int n, int B, int M, float h,
                             int level_rule, int half, float *q, int32_t *status,
                             cudaStream_t st, int status_shift)
{
    if (nb <= 0) return cudaSuccess;
    const int nw = kQThreads / 32;
    const int ue = (B + 1) + ((B + 1) & 1);
    const size_t smem = sizeof(float) * (size_t)nw * (2 * ue + 2 * (B + 1) + M + (M & 1));
    // with half projections and midpoint levels, angles k and k + n/2 come
    // from one quantile computation
    const int mirror = half && level_rule == 0;
    const int nang = mirror ? n / 2 : n;
    cudaFuncSetAttribute(k_quantiles, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    dim3 grid((nang + nw * kQRows - 1) / (nw * kQRows), nb);
    k_quantiles<<<grid, kQThreads, smem, st>>>(proj, n, B, M, h, level_rule, half, mirror, q,
                                                status, status_shift);
    return cudaGetLastError();
}

cudaError_t launch_center_norm(const float *q, int nb, int n, int M, const double2 *cs64,
                               double *center, double *norm, cudaStream_t st)
{
    if (nb <= 0) return cudaSuccess;
    k_center_norm<<<nb, 256, 0, st>>>(q, n, M, cs64, center, norm);
    return cudaGetLastError();
}

}  // namespace swk
