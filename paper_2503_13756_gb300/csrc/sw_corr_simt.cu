// sw_corr_simt.cu -- FP32 correlation of angle spectra on the CUDA cores:
// the "products summed over rows" step of the FFT cross-correlation of
// Sec. 2.3 ("Fast computation over rotations"), written as one complex
// product-sum per frequency and pair:
//   C_ij(k') = sum_p Qhat_i(k', p) conj(Qhat_j(k', p))
//            = sum_p (a_i a_j + b_i b_j) + i (b_i a_j - a_i b_j),  Qhat = a + i b.
// This is a batched GEMM over frequencies; the FP32 path keeps it on FFMA
// so that the accumulation is full single precision.
//
// Design: 64 x 64 pair tile per CTA, 4 x 4 pairs per thread, levels staged
// 16 at a time in shared memory (transposed so that each thread reads four
// consecutive queries or templates as one float4), register double-buffer
// of the next stage.
#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int TM = 64, TN = 64, KP = 16;

__global__ void __launch_bounds__(256)
k_corr_simt(const float *__restrict__ X, size_t xf, const float *__restrict__ Y, size_t yf,
            int Nq, int Nt, int M, float2 *__restrict__ C)
{
    __shared__ __align__(16) float qa[KP][TM], qb[KP][TM], ta[KP][TN], tb[KP][TN];
    const int f = blockIdx.z;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    const float *Xf = X + (size_t)f * xf;
    const float *Yf = Y + (size_t)f * yf;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // loader mapping: row r = t / 4 (0..63), levels (t % 4) * 4 .. +3
    const int lr = threadIdx.x >> 2, lp = (threadIdx.x & 3) * 4;
    const int gi = i0 + lr, gj = j0 + lr;
    const float *xrow = gi < Nq ? Xf + (size_t)gi * 2 * M : nullptr;
    const float *yrow = gj < Nt ? Yf + (size_t)gj * 2 * M : nullptr;

    float vqa[4], vqb[4], vta[4], vtb[4];
    auto fetch = [&](int p0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + lp + u;
            const bool okp = p < M;
            vqa[u] = (xrow && okp) ? __ldg(xrow + p) : 0.f;
            vqb[u] = (xrow && okp) ? __ldg(xrow + M + p) : 0.f;
            vta[u] = (yrow && okp) ? __ldg(yrow + p) : 0.f;
            vtb[u] = (yrow && okp) ? __ldg(yrow + M + p) : 0.f;
        }
    };

    float re[4][4], im[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) re[a][b] = im[a][b] = 0.f;

    fetch(0);
    for (int p0 = 0; p0 < M; p0 += KP) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            qa[lp + u][lr] = vqa[u];
            qb[lp + u][lr] = vqb[u];
            ta[lp + u][lr] = vta[u];
            tb[lp + u][lr] = vtb[u];
        }
        __syncthreads();
        if (p0 + KP < M) fetch(p0 + KP);
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            const float4 xa = *reinterpret_cast<const float4 *>(&qa[p][ty * 4]);
            const float4 xb = *reinterpret_cast<const float4 *>(&qb[p][ty * 4]);
            const float4 ya = *reinterpret_cast<const float4 *>(&ta[p][tx * 4]);
            const float4 yb = *reinterpret_cast<const float4 *>(&tb[p][tx * 4]);
            const float A[4] = {xa.x, xa.y, xa.z, xa.w}, Bq[4] = {xb.x, xb.y, xb.z, xb.w};
            const float Ca[4] = {ya.x, ya.y, ya.z, ya.w}, Cb[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    re[a][b] = fmaf(A[a], Ca[b], fmaf(Bq[a], Cb[b], re[a][b]));
                    im[a][b] = fmaf(Bq[a], Ca[b], fmaf(-A[a], Cb[b], im[a][b]));
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty * 4 + a;
        if (i >= Nq) continue;
        float2 *crow = C + ((size_t)f * Nq + i) * Nt;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + tx * 4 + b;
            if (j < Nt) crow[j] = make_float2(re[a][b], im[a][b]);
        }
    }
}

}  // namespace

cudaError_t launch_corr_simt(const float *X, size_t xf, const float *Y, size_t yf, int Nq,
                             int Nt, int M, int nf, float2 *C, cudaStream_t st)
{
    if (Nq <= 0 || Nt <= 0 || nf <= 0) return cudaSuccess;
    dim3 grid((Nt + TN - 1) / TN, (Nq + TM - 1) / TM, nf);
    k_corr_simt<<<grid, 256, 0, st>>>(X, xf, Y, yf, Nq, Nt, M, C);
    return cudaGetLastError();
}

}  // namespace swk
