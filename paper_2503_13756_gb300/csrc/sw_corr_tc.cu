// sw_corr_tc.cu -- the per-frequency correlation GEMM on the 5th-generation
// tensor cores (tcgen05), BF16 or FP16 operands with FP32 accumulation.
//
// This is the "products summed over rows" step of the FFT cross-correlation
// (Sec. 2.3, "Fast computation over rotations"), for many pairs at once:
//   C_ij(k') = sum_p Qhat_i(k',p) conj(Qhat_j(k',p)),  k' = 1..n/2,
// embedded in real arithmetic as D_f = A_f B_f^T with
//   A_f row i   = [Re Qhat_i | Im Qhat_i | 0...]                 (queries)
//   B_f row 2j  = [Re Qhat_j | Im Qhat_j | 0...]                 (templates)
//   B_f row 2j+1= [-Im Qhat_j | Re Qhat_j | 0...]
// so that D_f[i][2j] = Re C_ij(f) and D_f[i][2j+1] = Im C_ij(f): row i of D_f
// is exactly the float2 row C[f][i][0..Nt) that the decision kernel reads.
// Rows are K-major with K = ldk (2M rounded up to 64, zero padded).
//
// Design: persistent CTAs, one per SM, each walking output tiles of
// 128 queries x BN columns (BN / 2 templates) for one frequency; BN is 256 or
// 128 (the autotuner's choice: 128 when fewer templates would leave half of a
// 256-wide tile as padding).  Warp 0 issues TMA loads (128-byte swizzle, 3-D
// maps over frequency) into a 4-stage ring of 64-wide K slices; warp 1 owns
// the 2 BN-column TMEM allocation and one lane issues tcgen05.mma (M=128,
// N=BN, K=16) into one of two TMEM accumulators; the epilogue warps drain
// the other accumulator with tcgen05.ld, so the epilogue of one tile
// overlaps the MMAs of the next.  BF16 / FP16 (one K pass per tile) take
// eight epilogue warps, two per TMEM lane quarter each draining half of the
// tile's columns, with a 3-stage ring at BN = 256 to leave room for their
// store buffers.  The FP16 split (three products per tile) loads each K
// slice's four operand segments (A hi, A lo, B hi, B lo) into one stage and
// issues the three products' MMAs from it, so each segment is read once per
// tile instead of the hi segments twice (a third fewer operand bytes; two
// stages at BN = 256, three at 128), with four epilogue warps.  With Nt even each
// epilogue warp writes its 32 x 32 FP32 blocks into one of two 128-byte-
// swizzled shared-memory buffers and one lane stores them with a TMA tensor
// store (coalesced, clipped at the tensor's edges); odd Nt keeps per-lane
// stores of each row.  Every wait of one role on another gives up after a
// limit (a kernel argument: ~2 s of clock by default), sets *err and stops
// every role; the waits that let issued copies and MMAs land before the CTA
// ends keep the long limit, so nothing is in flight when TMEM is released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "sw_internal.cuh"

namespace swk {
namespace {

constexpr int BM = 128, BK = 64;                  // tile rows; BK bf16 = 128 B rows
constexpr int MAX_STAGES = 4;
constexpr int A_STAGE = BM * BK * 2;              // 16 KB
constexpr int EPI_BUF = 32 * 32 * 4;              // 4 KB: 32 rows x 32 FP32, 128-byte swizzle
// EPW epilogue warps per TMEM lane quarter (1 or 2)
template <int EPW> constexpr int tc_threads() { return 64 + 128 * EPW; }  // TMA, MMA, epilogue
template <int BN, int EPW, bool S4>
constexpr int stages()
{
    return S4 ? (BN == 256 ? 2 : 3) : ((BN == 256 && EPW == 2) ? 3 : 4);
}
template <int BN> constexpr int b_stage() { return BN * BK * 2; }  // 32 KB (BN 256), 16 KB
template <int BN> constexpr int tmem_cols() { return 2 * BN; }     // two BN-column accumulators
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz: default and drain limit

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Waits for the phase of `parity` to complete; false after `limit` cycles, or
// as soon as another role has given up (abort_flag != NULL and set).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          long long limit = WAIT_CYCLES)
{
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (abort_flag && *abort_flag) return false;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y,
                                             int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p)
{
    const uint64_t start = (smem_u32(p) & 0x3FFFFu) >> 4;
    return start | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct TcArgs {
    int Nq, Nt2, nf, kblocks;   // Nt2 = 2 Nt columns of D; kblocks: K slices of the product
    int segb;                   // K slices per operand segment (ldk / BK)
    int split;                  // FP16 split: rows [hi | lo]; the three products hi hi, hi lo,
                                // lo hi take A's segments 0, 0, 1 and B's 0, 1, 0
    int mtiles, ntiles;
    uint32_t idesc;
    float *C;                   // [nf][Nq][Nt2] fp32
    int *err;                   // set to 1 on a timed-out wait
    long long wait_cycles;      // limit of each wait of one role on another
    int stall;                  // test hook: issue no copies (the consumers' waits run out)
    int tma_store;              // C rows 16-byte aligned (Nt even): TMA stores through mapC
};

// S4: the FP16 split with the four segments of a K slice in one stage
// (args.kblocks = segb); otherwise one A and one B slice per stage.
template <int BN, int EPW, bool S4>
__global__ void __launch_bounds__(tc_threads<EPW>(), 1)
k_corr_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          const __grid_constant__ CUtensorMap mapC, TcArgs args)
{
    constexpr int B_STAGE = b_stage<BN>();
    constexpr int TMEM_COLS = tmem_cols<BN>();
    constexpr int STAGES = stages<BN, EPW, S4>();
    constexpr int EPI_WARPS = 4 * EPW;
    constexpr int A_ST = S4 ? 2 * A_STAGE : A_STAGE;  // one stage: [hi | lo] with S4
    constexpr int B_ST = S4 ? 2 * B_STAGE : B_STAGE;
    extern __shared__ uint8_t dsm[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t *sA = base;                       // STAGES x A_ST
    uint8_t *sB = base + STAGES * A_ST;       // STAGES x B_ST
    uint8_t *sE = sB + STAGES * B_ST;         // [EPI_WARPS][2] x 4 KB epilogue blocks (1 KB aligned)
    __shared__ __align__(8) uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_tiles = args.nf * args.mtiles * args.ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], EPI_WARPS);  // one arrival per epilogue warp
        }
        mbar_init(&done_bar, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    volatile int *abort_flag = &abort_s;

    auto give_up = [&]() {
        *abort_flag = 1;
        atomicExch(args.err, 1);
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < num_tiles && !*abort_flag && !args.stall;
                 t += gridDim.x) {
                const int nt = t % args.ntiles;
                const int mt = (t / args.ntiles) % args.mtiles;
                const int f = t / (args.ntiles * args.mtiles);
                for (int kb = 0; kb < args.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t round = it / STAGES;
                    if (!mbar_wait(&empty_bar[s], (round & 1) ^ 1, abort_flag, args.wait_cycles)) {
                        give_up();
                        break;
                    }
                    if constexpr (S4) {
                        // K slice kb: A hi, A lo, B hi, B lo
                        const int xh = kb * BK, xl = (args.segb + kb) * BK;
                        mbar_expect_tx(&full_bar[s], A_ST + B_ST);
                        tma_load_3d(sA + s * A_ST, &mapA, &full_bar[s], xh, mt * BM, f);
                        tma_load_3d(sA + s * A_ST + A_STAGE, &mapA, &full_bar[s], xl, mt * BM, f);
                        tma_load_3d(sB + s * B_ST, &mapB, &full_bar[s], xh, nt * BN, f);
                        tma_load_3d(sB + s * B_ST + B_STAGE, &mapB, &full_bar[s], xl, nt * BN, f);
                    } else {
                        // K slice kb of product term t: A's and B's segment for that term
                        const int t = kb / args.segb, kk = kb - t * args.segb;
                        const int xa = ((args.split && t == 2) ? args.segb + kk : kk) * BK;
                        const int xb = ((args.split && t == 1) ? args.segb + kk : kk) * BK;
                        mbar_expect_tx(&full_bar[s], A_STAGE + B_STAGE);
                        tma_load_3d(sA + s * A_STAGE, &mapA, &full_bar[s], xa, mt * BM, f);
                        tma_load_3d(sB + s * B_STAGE, &mapB, &full_bar[s], xb, nt * BN, f);
                    }
                }
            }
            // let every issued copy land before the CTA may exit (time-bounded
            // even when another role has given up)
            const int issued = it;
            for (int j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
                if (!mbar_wait(&full_bar[j % STAGES], (j / STAGES) & 1, nullptr)) give_up();
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            int it = 0, lt = 0;
            for (int t = blockIdx.x; t < num_tiles && !*abort_flag; t += gridDim.x, ++lt) {
                const int buf = lt & 1;
                const uint32_t use = lt >> 1;
                if (!mbar_wait(&tempty_bar[buf], (use & 1) ^ 1, abort_flag, args.wait_cycles)) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + buf * BN;
                bool ok = true;
                for (int kb = 0; kb < args.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&full_bar[s], (it / STAGES) & 1, abort_flag, args.wait_cycles)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if constexpr (S4) {
                        // hi hi, hi lo, lo hi from the stage's four segments
                        const uint64_t ah = smem_desc_sw128(sA + s * A_ST);
                        const uint64_t al = smem_desc_sw128(sA + s * A_ST + A_STAGE);
                        const uint64_t bh = smem_desc_sw128(sB + s * B_ST);
                        const uint64_t bl = smem_desc_sw128(sB + s * B_ST + B_STAGE);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_f16(d, ah + 2 * kk, bh + 2 * kk, args.idesc, (kb | kk) != 0);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_f16(d, ah + 2 * kk, bl + 2 * kk, args.idesc, true);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_f16(d, al + 2 * kk, bh + 2 * kk, args.idesc, true);
                    } else {
                        const uint64_t da = smem_desc_sw128(sA + s * A_STAGE);
                        const uint64_t db = smem_desc_sw128(sB + s * B_STAGE);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)  // +32 bytes along K per step
                            mma_f16(d, da + 2 * kk, db + 2 * kk, args.idesc, (kb | kk) != 0);
                    }
                    mma_commit(&empty_bar[s]);  // stage free once these MMAs finish
                }
                if (!ok) break;
                mma_commit(&tfull_bar[buf]);    // accumulator ready
            }
            // every MMA issued above has completed before TMEM can be freed
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0, nullptr)) give_up();
        }
    } else {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int ew = warp - 2;                // epilogue warp 0 .. EPI_WARPS - 1
        const int cbeg = (ew / 4) * (BN / EPW); // this warp's share of the columns
        const int row_in_tile = q * 32 + lane;
        uint8_t *myE = sE + ew * 2 * EPI_BUF;
        int lt = 0, chunk = 0;
        for (int t = blockIdx.x; t < num_tiles && !*abort_flag; t += gridDim.x, ++lt) {
            const int nt = t % args.ntiles;
            const int mt = (t / args.ntiles) % args.mtiles;
            const int f = t / (args.ntiles * args.mtiles);
            const int buf = lt & 1;
            if (!mbar_wait(&tfull_bar[buf], (lt >> 1) & 1, abort_flag, args.wait_cycles)) {
                give_up();
                break;
            }
            tc_fence_after();
            const int i = mt * BM + row_in_tile;
            float *crow = args.C + ((size_t)f * args.Nq + i) * args.Nt2 + (size_t)nt * BN;
            const int ncols = min(BN, args.Nt2 - nt * BN);
#pragma unroll 1
            for (int c0 = cbeg; c0 < cbeg + BN / EPW; c0 += 32) {
                uint32_t r[32];
                if (args.tma_store) {
                    // a box wholly past the tensor's edge holds nothing (warp-uniform)
                    const int x = nt * BN + c0, y = mt * BM + q * 32;
                    if (x >= args.Nt2 || y >= args.Nq) continue;
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + buf * BN + c0, r);
                    // the store issued two boxes ago read this buffer: it is done
                    uint8_t *eb = myE + (chunk & 1) * EPI_BUF;
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    __syncwarp();
                    // row `lane`, 16-byte chunk v at v ^ (row mod 8): the 128-byte
                    // swizzle of the tensor map; a quarter-warp fills 8 distinct chunks
                    float4 *rowp = reinterpret_cast<float4 *>(eb + lane * 128);
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        rowp[v ^ (lane & 7)] =
                            make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                        __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_3d(&mapC, eb, x, y, f);
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                    ++chunk;
                } else {
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + buf * BN + c0, r);
                    if (i < args.Nq && c0 < ncols) {
                        // rows are 2 Nt floats: 8-byte aligned (float2 per template)
                        if (c0 + 32 <= ncols) {
                            float2 *dst = reinterpret_cast<float2 *>(crow + c0);
#pragma unroll
                            for (int v = 0; v < 16; ++v)
                                dst[v] = make_float2(__uint_as_float(r[2 * v]),
                                                     __uint_as_float(r[2 * v + 1]));
                        } else {
#pragma unroll
                            for (int v = 0; v < 32; ++v)
                                if (c0 + v < ncols) crow[c0 + v] = __uint_as_float(r[v]);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty_bar[buf]);
        }
        // every TMA store of this warp has completed before the CTA ends
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// C as [nf][Nq][Nt2] FP32 in 32 x 32 boxes, 128-byte swizzle (Nt2 4 bytes a
// multiple of 16: Nt even).
bool make_map_c(CUtensorMap *m, float *C, uint64_t nt2, uint64_t nq, uint64_t nf)
{
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[3] = {nt2, nq, nf};
    const cuuint64_t strides[2] = {nt2 * 4, nt2 * 4 * nq};
    const cuuint32_t box[3] = {32, 32, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, C, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_map(CUtensorMap *m, const void *base, int kind, uint64_t ldk, uint64_t rows,
              uint64_t nf, uint32_t box_rows)
{
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[3] = {ldk, rows, nf};
    const cuuint64_t strides[2] = {ldk * 2, ldk * 2 * rows};
    const cuuint32_t box[3] = {(cuuint32_t)BK, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                           3, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int EPW, bool S4 = false>
cudaError_t launch_tile(const void *Xq, const void *Yt, int Nq, int Nt, int M, int nf, int kind,
                        float2 *C, int *err, int num_sms, cudaStream_t st, long long wait_cycles,
                        int stall)
{
    const int ldk = lp_row_len(M, kind);
    CUtensorMap ma, mb;
    if (!make_map(&ma, Xq, kind, ldk, (uint64_t)Nq, nf, BM) ||
        !make_map(&mb, Yt, kind, ldk, (uint64_t)2 * Nt, nf, BN))
        return cudaErrorInvalidValue;
    TcArgs a;
    a.Nq = Nq;
    a.Nt2 = 2 * Nt;
    a.nf = nf;
    a.segb = tc_ldk(M) / BK;
    a.split = kind == 3;
    a.kblocks = (a.split && !S4) ? 3 * a.segb : a.segb;
    a.mtiles = (Nq + BM - 1) / BM;
    a.ntiles = (2 * Nt + BN - 1) / BN;
    // kind::f16 instruction descriptor: FP32 accumulator, A/B BF16 (1) or
    // FP16 (0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
    const uint32_t fmt = kind == 1 ? 1u : 0u;  // BF16, else FP16 (plain or split)
    a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
              ((uint32_t)(BM >> 4) << 24);
    a.C = reinterpret_cast<float *>(C);
    a.err = err;
    a.wait_cycles = wait_cycles > 0 ? wait_cycles : WAIT_CYCLES;
    a.stall = stall;
    CUtensorMap mc;
    std::memset(&mc, 0, sizeof(mc));
    a.tma_store = (Nt % 2 == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0 &&
                   make_map_c(&mc, a.C, (uint64_t)2 * Nt, (uint64_t)Nq, (uint64_t)nf))
                      ? 1
                      : 0;
    const int per = S4 ? 2 : 1;  // segments of each operand per stage
    const size_t smem = (size_t)stages<BN, EPW, S4>() * per * (A_STAGE + b_stage<BN>()) +
                        4 * EPW * 2 * EPI_BUF + 1024;
    cudaFuncSetAttribute(k_corr_tc<BN, EPW, S4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    const int tiles = nf * a.mtiles * a.ntiles;
    const int grid = tiles < num_sms ? tiles : num_sms;
    k_corr_tc<BN, EPW, S4><<<grid, tc_threads<EPW>(), smem, st>>>(ma, mb, mc, a);
    return cudaGetLastError();
}

}  // namespace

int tc_ldk(int M) { return ((2 * M + BK - 1) / BK) * BK; }
int lp_row_len(int M, int lp_kind) { return lp_kind == 3 ? 2 * tc_ldk(M) : tc_ldk(M); }

cudaError_t launch_corr_tc(const void *Xq, const void *Yt, int Nq, int Nt, int M, int nf,
                           int kind, float2 *C, int *err, int num_sms, cudaStream_t st,
                           long long wait_cycles, int stall, int tile_n)
{
    if (Nq <= 0 || Nt <= 0 || nf <= 0) return cudaSuccess;
    // the FP16 split (kind 3): four segments per stage, four epilogue warps;
    // BF16 / FP16 drain with eight
    if (kind == 3)
        return tile_n == 128
                   ? launch_tile<128, 1, true>(Xq, Yt, Nq, Nt, M, nf, kind, C, err, num_sms, st,
                                               wait_cycles, stall)
                   : launch_tile<256, 1, true>(Xq, Yt, Nq, Nt, M, nf, kind, C, err, num_sms, st,
                                               wait_cycles, stall);
    return tile_n == 128 ? launch_tile<128, 2>(Xq, Yt, Nq, Nt, M, nf, kind, C, err, num_sms, st,
                                               wait_cycles, stall)
                         : launch_tile<256, 2>(Xq, Yt, Nq, Nt, M, nf, kind, C, err, num_sms, st,
                                               wait_cycles, stall);
}

}  // namespace swk
