// sw_ramp.cu -- ramp filter and positive/negative split of the projections
// for the ramp-filtered sliced W2 (Sec. 2.1 "High-pass filter (optional)",
// Eq. 1d_ift_ramp and Eq. line_decomp; the negative part is taken as the
// absolute value max(-mu~, 0), as in the appendix on ramp-filtered
// distances, and each part is normalised later by its own mass).
//
// Each projection row U[0..B) is filtered circularly on its bin grid:
//   Ut = IDFT_B( |xi_j| DFT_B(U) ),  |xi_j| = min(j, B - j),
// then split into Ut+ = max(Ut, 0) and Ut- = max(-Ut, 0).
//
// Design (GB300): one CTA per image; rows are taken 2*nsig at a time, two
// real rows packed into one complex signal.  The filter is real and even, so
// filtering the packed signal filters both rows at once (the real part holds
// one filtered row, the imaginary part the other): forward FFT, scale by
// |xi_j| / B, inverse FFT, all in shared memory with the Stockham FFT.
#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int kRampThreads = 256;
#ifndef RAMP_NSIG_MAX
#define RAMP_NSIG_MAX 8
#endif

template <int nsig>
__global__ void __launch_bounds__(kRampThreads)
k_ramp(const float *__restrict__ proj, int nh, int B, FftPlan plan,
       const float2 *__restrict__ tw, float *__restrict__ parts)
{
    extern __shared__ float2 smr[];
    float2 *b0 = smr;
    float2 *b1 = b0 + B * nsig;
    float2 *tws = b1 + B * nsig;                            // [B]
    float *tile = reinterpret_cast<float *>(tws + B);       // [2 nsig][B + 1] rows of the chunk
    const int TS = B + 1;  // odd row stride (B is even): column reads hit distinct banks
    for (int i = threadIdx.x; i < B; i += blockDim.x) tws[i] = tw[i];
    const int img = blockIdx.x;
    const float *U = proj + (size_t)img * nh * B;
    float *Pp = parts + (size_t)img * 2 * nh * B;  // part 0 (positive)
    float *Pm = Pp + (size_t)nh * B;                // part 1 (negative)
    const float invB = 1.f / (float)B;
    for (int r0 = 0; r0 < nh; r0 += 2 * nsig) {
        const int rows = min(2 * nsig, nh - r0);
        // ---- load the chunk's rows (coalesced), then pack: signal s =
        // rows (2s, 2s + 1) as (re, im), element-major for the FFT
        for (int e = threadIdx.x; e < 2 * nsig * B; e += blockDim.x) {
            const int r = e / B, b = e - r * B;
            tile[r * TS + b] = r < rows ? U[(size_t)(r0 + r) * B + b] : 0.f;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < B * nsig; t += blockDim.x) {
            const int b = t / nsig, sg = t % nsig;
            b0[t] = make_float2(tile[(2 * sg) * TS + b], tile[(2 * sg + 1) * TS + b]);
        }
        __syncthreads();
        float2 *X = fft_smem<nsig, -1>(b0, b1, plan, tws);
        float2 *Y = X == b0 ? b1 : b0;
        for (int t = threadIdx.x; t < B * nsig; t += blockDim.x) {
            const int j = t / nsig;
            const float w = (float)min(j, B - j) * invB;
            X[t] = make_float2(w * X[t].x, w * X[t].y);
        }
        __syncthreads();
        const float2 *R = fft_smem<nsig, +1>(X, Y, plan, tws);
        // ---- unpack to rows, then split and write (coalesced)
        for (int t = threadIdx.x; t < B * nsig; t += blockDim.x) {
            const int b = t / nsig, sg = t % nsig;
            const float2 v = R[t];
            tile[(2 * sg) * TS + b] = v.x;
            tile[(2 * sg + 1) * TS + b] = v.y;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * B; e += blockDim.x) {
            const int r = e / B, b = e - r * B;
            const float v = tile[r * TS + b];
            Pp[(size_t)(r0 + r) * B + b] = fmaxf(v, 0.f);
            Pm[(size_t)(r0 + r) * B + b] = fmaxf(-v, 0.f);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_ramp(const float *proj, int nb, int nh, int B, const FftPlan &plan,
                        const float2 *tw, float *parts, cudaStream_t st)
{
    if (nb <= 0) return cudaSuccess;
    if (plan.n != B) return cudaErrorInvalidValue;
    // the widest signal batch (up to RAMP_NSIG_MAX) whose buffers fit 200 KB
    auto smem_of = [&](int ns) {
        return sizeof(float2) * ((size_t)2 * B * ns + B) + sizeof(float) * (size_t)2 * ns * (B + 1);
    };
    int nsig = RAMP_NSIG_MAX;
    while (nsig > 2 && smem_of(nsig) > 200 * 1024) nsig /= 2;
    if (smem_of(nsig) > 200 * 1024) return cudaErrorInvalidValue;
    const size_t smem = smem_of(nsig);
#define SW_RAMP_LAUNCH(NS)                                                                     \
    do {                                                                                      \
        cudaFuncSetAttribute(k_ramp<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                             200 * 1024);                                                     \
        k_ramp<NS><<<nb, kRampThreads, smem, st>>>(proj, nh, B, plan, tw, parts);             \
    } while (0)
    if (nsig == 16) SW_RAMP_LAUNCH(16);
    else if (nsig == 8) SW_RAMP_LAUNCH(8);
    else if (nsig == 4) SW_RAMP_LAUNCH(4);
    else SW_RAMP_LAUNCH(2);
#undef SW_RAMP_LAUNCH
    return cudaGetLastError();
}

}  // namespace swk
