// sw_msw.cu -- max-sliced W2 over rotations (Eq. max_sliced_wasserstein):
//   D(l) = max_k (1/M) sum_p (u_pk - v_{p,(k-l) mod n})^2
// over the (optionally centred) quantiles of two images.  The cyclic
// cross-correlation does not apply to a maximum, so every (k, k') column
// pair is formed: O(n^2 M) per pair.
//
// Design (GB300): the per-angle terms are squared differences summed
// directly in FP32 (no Gram-matrix cancellation).  One CTA takes one pair
// and a block of R rows k of the query against all n columns k' of the
// template, staging the query rows [R][PC] and the template columns
// transposed [PC][n+1] in shared memory, PC levels at a time; each thread
// owns the columns k' = t, t + 256, ... and R accumulators per column.  The
// block's terms then go to shared memory, each thread takes rotations
// l = t, t + 256, ... and the maximum over its rows of E[k][(k - l) mod n],
// and the blocks of a pair meet in an atomic max on the pair's curve (the
// terms are >= 0, so their float bits order as integers; the maximum does
// not depend on the order).  A second kernel takes the argmin per pair.
#include "sw_internal.cuh"
#include "swalign.h"

namespace swk {
namespace {

constexpr int kMswThreads = 256;
constexpr int kMswPC = 32;  // levels per stage (a multiple of 4)

template <int R, int NC>
__global__ void __launch_bounds__(kMswThreads)
k_msw(MswArgs A)
{
    extern __shared__ float sms[];
    const int n = A.n, M = A.M;
    const int np1 = n + 1;
    float *Us = sms;                   // [R][kMswPC]
    float *Vt = Us + R * kMswPC;       // [kMswPC][n + 1]
    float *Eb = Vt + kMswPC * np1;     // [R][n]
    float *offt = Eb + R * n;          // [n] template column offsets
    __shared__ float offq[R];
    const int pair = blockIdx.x;
    const int i = pair / A.Nt, j = pair % A.Nt;
    const int k0 = blockIdx.y * R;
    const int t = threadIdx.x;
    const float *Qi = A.q + (size_t)i * n * M;
    const float *Qj = A.t + (size_t)j * n * M;
    // centring offsets <a, e_k> (translation): query rows here, template
    // columns folded into the staging below
    const double2 *cs = A.cs64;
    const double aix = A.translation ? A.ctr_q[2 * i] : 0.0;
    const double aiy = A.translation ? A.ctr_q[2 * i + 1] : 0.0;
    const double ajx = A.translation ? A.ctr_t[2 * j] : 0.0;
    const double ajy = A.translation ? A.ctr_t[2 * j + 1] : 0.0;
    if (t < R) {
        const int k = k0 + t;
        offq[t] = k < n ? (float)(aix * cs[k].x + aiy * cs[k].y) : 0.f;
    }
    // once per column (FP64 is scarce: not once per staged level)
    for (int kk = t; kk < n; kk += kMswThreads)
        offt[kk] = A.translation ? (float)(ajx * cs[kk].x + ajy * cs[kk].y) : 0.f;
    float acc[NC][R];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[c][r] = 0.f;
    __syncthreads();
    for (int p0 = 0; p0 < M; p0 += kMswPC) {
        const int pc = min(kMswPC, M - p0);
        // query rows: Us[r][p] (zero outside), centred
        for (int e = t; e < R * kMswPC; e += kMswThreads) {
            const int r = e / kMswPC, p = e % kMswPC, k = k0 + r;
            Us[e] = (k < n && p < pc) ? Qi[(size_t)k * M + p0 + p] - offq[r] : 0.f;
        }
        // template columns transposed: Vt[p][k'] (zero outside), centred
        for (int e = t; e < n * kMswPC; e += kMswThreads) {
            const int kk = e / kMswPC, p = e % kMswPC;
            float v = 0.f;
            if (p < pc) v = Qj[(size_t)kk * M + p0 + p] - offt[kk];
            Vt[p * np1 + kk] = v;
        }
        __syncthreads();
        // four levels at a time: one 16-byte read of each query row (the
        // staged tiles are zero past pc, and zeros add nothing)
        for (int p = 0; p < pc; p += 4) {
            float v[NC][4];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int kk = t + c * kMswThreads;
#pragma unroll
                for (int q = 0; q < 4; ++q) v[c][q] = kk < n ? Vt[(p + q) * np1 + kk] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float4 u = *reinterpret_cast<const float4 *>(Us + r * kMswPC + p);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float d = u.x - v[c][0];
                    acc[c][r] = fmaf(d, d, acc[c][r]);
                    d = u.y - v[c][1];
                    acc[c][r] = fmaf(d, d, acc[c][r]);
                    d = u.z - v[c][2];
                    acc[c][r] = fmaf(d, d, acc[c][r]);
                    d = u.w - v[c][3];
                    acc[c][r] = fmaf(d, d, acc[c][r]);
                }
            }
        }
        __syncthreads();
    }
    // ---- block terms to shared memory, then diagonal maxima per rotation
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int kk = t + c * kMswThreads;
        if (kk < n)
#pragma unroll
            for (int r = 0; r < R; ++r) Eb[r * n + kk] = acc[c][r];
    }
    __syncthreads();
    const int rows = min(R, n - k0);
    unsigned *curve = reinterpret_cast<unsigned *>(A.curve) + (size_t)pair * n;
    for (int l = t; l < n; l += kMswThreads) {
        float mx = 0.f;
        for (int r = 0; r < rows; ++r) {
            int kk = k0 + r - l;
            kk += kk < 0 ? n : 0;
            mx = fmaxf(mx, Eb[r * n + kk]);
        }
        atomicMax(curve + l, __float_as_uint(mx));
    }
}

// argmin over l (lowest l on ties), one warp per pair
__global__ void k_msw_decide(MswArgs A)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int pairs = A.Nq * A.Nt;
    if (warp >= pairs) return;
    const int i = warp / A.Nt, j = warp % A.Nt, n = A.n;
    const float *cv = A.curve + (size_t)warp * n;
    float best = __int_as_float(0x7f800000);
    int bl = 0x7fffffff;
    for (int l = lane; l < n; l += 32) {
        const float v = cv[l];
        if (v < best) {  // l increases: ties keep the lowest
            best = v;
            bl = l;
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
        if (ob < best || (ob == best && ol < bl)) {
            best = ob;
            bl = ol;
        }
    }
    const double invM = 1.0 / A.M;
    const int st = A.st_q[i] ? 1 : (A.st_t[j] ? 2 : 0);
    auto shift_at = [&](int l, double &sx, double &sy) {
        sx = sy = 0.0;
        if (A.translation) {
            const double2 c = A.cs64[l];
            const double ajx = A.ctr_t[2 * j], ajy = A.ctr_t[2 * j + 1];
            sx = A.ctr_q[2 * i] - (c.x * ajx - c.y * ajy);
            sy = A.ctr_q[2 * i + 1] - (c.y * ajx + c.x * ajy);
        }
    };
    if (lane == 0) {
        sw_result r;
        if (st || bl >= n) {
            const double nan = __longlong_as_double(0x7ff8000000000000ULL);
            r.best_l = -1;
            r.status = st ? st : 1;
            r.angle_rad = __int_as_float(0x7fc00000);
            r.shift[0] = r.shift[1] = nan;
            r.d2 = nan;
        } else {
            r.best_l = bl;
            r.status = 0;
            r.angle_rad = (float)(A.dalpha * bl);
            shift_at(bl, r.shift[0], r.shift[1]);
            r.d2 = (double)best * invM;
        }
        r.template_index = j;
        reinterpret_cast<sw_result *>(A.out)[warp] = r;
    }
    if (A.full && warp == 0) {
        const int bad = st != 0;
        for (int l = lane; l < n; l += 32) {
            A.full[l] = bad ? __longlong_as_double(0x7ff8000000000000ULL) : (double)cv[l] * invM;
            if (A.shifts) shift_at(l, A.shifts[2 * l], A.shifts[2 * l + 1]);
        }
    }
}

template <int R, int NC>
cudaError_t launch_rows(const MswArgs &a, cudaStream_t st)
{
    const size_t smem = sizeof(float) * ((size_t)R * kMswPC + (size_t)kMswPC * (a.n + 1) +
                                         (size_t)R * a.n + a.n);
    cudaFuncSetAttribute(k_msw<R, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    dim3 grid(a.Nq * a.Nt, (a.n + R - 1) / R);
    k_msw<R, NC><<<grid, kMswThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_msw(const MswArgs &args, cudaStream_t st)
{
    if (args.Nq <= 0 || args.Nt <= 0) return cudaSuccess;
    if (args.n > 1024 || (size_t)args.Nq * args.Nt > 0x7fffffffu) return cudaErrorInvalidValue;
    MswArgs a = args;
    a.dalpha = 6.283185307179586 / a.n;
    cudaError_t e = cudaMemsetAsync(a.curve, 0, sizeof(float) * (size_t)a.Nq * a.Nt * a.n, st);
    if (e != cudaSuccess) return e;
    if (a.n <= 256) e = launch_rows<64, 1>(a, st);
    else if (a.n <= 512) e = launch_rows<32, 2>(a, st);
    else e = launch_rows<16, 4>(a, st);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const long long warps = (long long)a.Nq * a.Nt;
    k_msw_decide<<<(unsigned)((warps * 32 + threads - 1) / threads), threads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace swk
