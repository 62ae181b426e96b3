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

template <int nsig>
__global__ void __launch_bounds__(kRampThreads)
k_ramp(const float *__restrict__ proj, int nh, int B, FftPlan plan,
       const float2 *__restrict__ tw, float *__restrict__ parts)
{
    extern __shared__ float2 smr[];
    float2 *b0 = smr;
    float2 *b1 = b0 + B * nsig;
    float2 *tws = b1 + B * nsig;  // [B]
    for (int i = threadIdx.x; i < B; i += blockDim.x) tws[i] = tw[i];
    const int img = blockIdx.x;
    const float *U = proj + (size_t)img * nh * B;
    float *Pp = parts + (size_t)img * 2 * nh * B;  // part 0 (positive)
    float *Pm = Pp + (size_t)nh * B;                // part 1 (negative)
    const float invB = 1.f / (float)B;
    for (int r0 = 0; r0 < nh; r0 += 2 * nsig) {
        // ---- load: signal s = rows (r0 + 2s, r0 + 2s + 1) as (re, im)
        for (int t = threadIdx.x; t < B * nsig; t += blockDim.x) {
            const int b = t / nsig, s = t % nsig;
            const int ra = r0 + 2 * s, rb = ra + 1;
            const float xr = ra < nh ? U[(size_t)ra * B + b] : 0.f;
            const float xi = rb < nh ? U[(size_t)rb * B + b] : 0.f;
            b0[t] = make_float2(xr, xi);
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
        // ---- split and write
        for (int t = threadIdx.x; t < B * nsig; t += blockDim.x) {
            const int b = t / nsig, s = t % nsig;
            const int ra = r0 + 2 * s, rb = ra + 1;
            const float2 v = R[t];
            if (ra < nh) {
                Pp[(size_t)ra * B + b] = fmaxf(v.x, 0.f);
                Pm[(size_t)ra * B + b] = fmaxf(-v.x, 0.f);
            }
            if (rb < nh) {
                Pp[(size_t)rb * B + b] = fmaxf(v.y, 0.f);
                Pm[(size_t)rb * B + b] = fmaxf(-v.y, 0.f);
            }
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
    const int nsig = B <= 512 ? 16 : 4;
    const size_t smem = sizeof(float2) * ((size_t)2 * B * nsig + B);
    if (nsig == 16) {
        cudaFuncSetAttribute(k_ramp<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        k_ramp<16><<<nb, kRampThreads, smem, st>>>(proj, nh, B, plan, tw, parts);
    } else {
        cudaFuncSetAttribute(k_ramp<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        k_ramp<4><<<nb, kRampThreads, smem, st>>>(proj, nh, B, plan, tw, parts);
    }
    return cudaGetLastError();
}

}  // namespace swk
