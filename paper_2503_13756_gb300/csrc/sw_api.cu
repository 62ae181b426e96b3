// sw_api.cu -- the C ABI declared in include/swalign.h: argument checks,
// angle/twiddle tables, workspace and the launch sequence of each call.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <fstream>
#include <map>
#include <random>
#include <sstream>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sw_internal.cuh"
#include "sw_slice_plan.h"
#include "swalign.h"

using swk::FftPlan;

namespace {

// Angle tables for one n: theta_k = 2 pi k / n, k < n.  Built in FP64 from
// the first octant and completed by exact symmetries, so that cos/sin of
// k = n/4, n/2, 3n/4 are exactly 0 and +-1 and theta + pi is exactly -theta.
struct Tables {
    int n = 0;
    int variant = 0;  // radix order of the FFT plan (fft_plan)
    FftPlan plan{};
    float2 *cs = nullptr;     // [n] (cos, sin) fp32
    double2 *cs64 = nullptr;  // [n] (cos, sin) fp64
    float2 *tw = nullptr;     // [n] e^{-2 pi i m / n}
};

// Tables of the Fourier-slice projector for one (L, n, B): the oversampled
// grid N, the kernel shape beta, psi_inv [L] = 1 / Psi(c - floor(L/2)),
// where Psi(k) = integral over |u| <= W/2 of psi(u) e^{-2 pi i k u / N} du is
// the Fourier transform of psi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)), the
// tap-weight polynomials, and the per-target factor table fac [n/2][B/2 + 1].
struct SliceTables {
    int L = 0, n = 0, B = 0, N = 0;
    double beta = 0.0;
    swk::SliceCoef coef{};
    float *psi_inv = nullptr;
    float2 *fac = nullptr;
    uint16_t *gtab = nullptr;  // target groups per angle batch (launch_project_slice)
    int *goff = nullptr;
    uint32_t *ttab = nullptr;  // target groups per grid tile (L > 128)
    int *toff = nullptr;
    // images of side L/2 upsampled 2 x 2 (launch_project_slice_up; 128 < L)
    float *up_psi_inv = nullptr;
    float2 *up_fac = nullptr;
    uint16_t *up_gtab = nullptr;
    int *up_goff = nullptr;
    float2 *up_tw = nullptr;
    swk::SliceUpTables up() const { return {up_psi_inv, up_fac, up_gtab, up_goff, up_tw}; }
};

// Mixed-radix plan of length n.  The radix order is free (any order is a
// valid Stockham factorisation; only the rounding and the speed change).
// The power-of-two part is taken in radix-4 stages (variants 0-3), or in
// radix-8 stages with at most one radix-4 stage (variants 4-7; fewer passes
// over shared memory, more registers per item); the rest in 2, 3, 5.  Order
// (variant & 3): 0: the power-of-two stages first, then 2, 3, 5; 1: 2, 3, 5
// first, then the power-of-two stages; 2: power-of-two first, then 5, 3, 2;
// 3: 5, 3, 2 first, then the power-of-two stages.
constexpr int kPlanVariants = 8;

bool fft_plan(int n, FftPlan &p, int variant = 0)
{
    p.n = n;
    p.nst = 0;
    int m = n, npow = 0;
    int pow2[swk::kMaxStages];
    if (variant & 4)
        while (m % 8 == 0 && npow < swk::kMaxStages) {
            pow2[npow++] = 8;
            m /= 8;
        }
    while (m % 4 == 0 && npow < swk::kMaxStages) {
        pow2[npow++] = 4;
        m /= 4;
    }
    int rest[swk::kMaxStages], nrest = 0;
    const int order = variant & 3;
    const bool desc = order == 2 || order == 3;
    const int asc[3] = {2, 3, 5}, dsc[3] = {5, 3, 2};
    for (int q : desc ? dsc : asc)
        while (m % q == 0 && nrest < swk::kMaxStages) {
            rest[nrest++] = q;
            m /= q;
        }
    if (m != 1 || npow + nrest > swk::kMaxStages) return false;
    const bool pow2_first = order == 0 || order == 2;
    if (!pow2_first)
        for (int i = 0; i < nrest; ++i) p.radix[p.nst++] = rest[i];
    for (int i = 0; i < npow; ++i) p.radix[p.nst++] = pow2[i];
    if (pow2_first)
        for (int i = 0; i < nrest; ++i) p.radix[p.nst++] = rest[i];
    int Ns = 1;
    for (int st = 0; st < p.nst; ++st) {
        p.ns[st] = Ns;
        p.ns_rcp[st] = (unsigned)((((unsigned long long)1 << 32) + Ns - 1) / Ns);
        p.tstep[st] = n / (Ns * p.radix[st]);
        Ns *= p.radix[st];
    }
    return true;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Offsets of the batch workspace.
struct Layout {
    size_t status, proj, ramp, quant, spec32, lp_q, lp_t, prof, center, norm32, norm16, C,
        scratch, err, total;
};

bool smooth235(int n);

// Ramp-filtered sliced W2: the filter is circular on the bin grid, so the
// default bin count is the smallest even 2/3/5-smooth count >= the default
// B (the FFT's lengths).
int rfsw_default_bins(int L)
{
    int B = sw_default_bins(L);
    while (B % 2 || !smooth235(B)) ++B;
    return B;
}

int bins_of(const sw_params *p)
{
    if (p->n_bins > 0) return p->n_bins;
    if (p->projector == SW_PROJ_SLICE)
        return swk::slice_default_bins(p->L, sw_default_bins(p->L));
    return p->metric == SW_METRIC_RFSW2 ? rfsw_default_bins(p->L) : sw_default_bins(p->L);
}

// Quantile sets per image: 2 for the ramp-filtered distance (positive and
// negative parts), stored one after the other as levels [0, M) and [M, 2M).
int parts_of(const sw_params *p) { return p->metric == SW_METRIC_RFSW2 ? 2 : 1; }
int levels_of(const sw_params *p) { return p->n_levels * parts_of(p); }

// Low-precision spectra kind of a precision: 3 = FP16 split (FP32-accurate
// tensor-core path), 1 = BF16, 2 = FP16, 0 = none (CUDA-core FP32).
int lp_kind_of(int precision)
{
    switch (precision) {
    case SW_PREC_FP32: return 3;
    case SW_PREC_BF16: return 1;
    case SW_PREC_FP16: return 2;
    default: return 0;
    }
}

Layout batch_layout(const sw_params *p, int Nq, int Nt, int lp_kind, bool scratch)
{
    const size_t nimg = (size_t)Nq + Nt;
    const size_t n = p->n_theta, nh = n / 2, M = levels_of(p), B = bins_of(p);
    const size_t parts = parts_of(p);
    const bool msw = p->metric == SW_METRIC_MSW2;  // quantiles only, no spectra
    if (msw) lp_kind = 0;
    Layout l{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t row = lp_kind ? (size_t)swk::lp_row_len((int)M, lp_kind) : 0;
    l.status = take(4 * nimg);
    l.proj = take(4 * nimg * nh * B);
    l.ramp = take(parts == 2 ? 4 * nimg * 2 * nh * B : 0);
    l.quant = take(4 * nimg * n * M);
    l.spec32 = take(lp_kind || msw ? 0 : 4 * nh * nimg * 2 * M);
    l.lp_q = take(2 * nh * (size_t)Nq * row);
    l.lp_t = take(2 * nh * (size_t)2 * Nt * row);
    l.prof = take(4 * nimg * M);
    l.center = take(16 * parts * nimg);
    l.norm32 = take(8 * nimg);
    l.norm16 = take(8 * nimg);
    l.C = take(8 * nh * (size_t)Nq * Nt);
    l.scratch = take(scratch ? sizeof(sw_result) * (size_t)Nq * Nt : 0);
    l.err = take(sizeof(int));
    l.total = o;
    return l;
}

// Workspace of sw_bank_align: query-side buffers only, the correlation of
// Nq queries against Nt bank templates.
Layout bank_layout(const sw_params *p, int Nq, int Nt, bool scratch)
{
    const size_t n = p->n_theta, nh = n / 2, M = levels_of(p), B = bins_of(p);
    const size_t parts = parts_of(p);
    const int lp_kind = lp_kind_of(p->gemm_precision);
    const size_t row = lp_kind ? (size_t)swk::lp_row_len((int)M, lp_kind) : 0;
    Layout l{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at_ = o;
        o = align_up(o + bytes);
        return at_;
    };
    l.status = take(4 * (size_t)Nq);
    l.proj = take(4 * (size_t)Nq * nh * B);
    l.ramp = take(parts == 2 ? 4 * (size_t)Nq * 2 * nh * B : 0);
    l.quant = take(4 * (size_t)Nq * n * M);
    l.spec32 = take(lp_kind ? 0 : 4 * nh * (size_t)Nq * 2 * M);
    l.lp_q = take(2 * nh * (size_t)Nq * row);
    l.lp_t = take(0);
    l.prof = take(4 * (size_t)Nq * M);
    l.center = take(16 * parts * (size_t)Nq);
    l.norm32 = take(8 * (size_t)Nq);
    l.norm16 = take(8 * (size_t)Nq);
    l.C = take(8 * nh * (size_t)Nq * Nt);
    l.scratch = take(scratch ? sizeof(sw_result) * (size_t)Nq * Nt : 0);
    l.err = take(sizeof(int));
    l.total = o;
    return l;
}

}  // namespace

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

// Launch shapes chosen by sw_autotune for one parameter set; 0 = the
// built-in default.  None of them changes what is computed: the FFT radix
// order only changes the rounding.
struct Tune {
    int want = 0;  // target CTA count of the projection's angle split
    int spec = 0;  // signals per FFT batch of the spectra (4, 8, 16)
    int dec = 0;   // decision form: 1 register FFT, else signals per CTA (4, 8, 16)
    int plan = 0;  // FFT radix order (fft_plan variant)
    // output tile width of the tensor-core correlation (columns of D, two per
    // template; 128 or 256, 0 = 256) for batches of at most 64 templates
    // (tile_s) and of more (tile_l)
    int tile_s = 0, tile_l = 0;
    int tile_for(int Nt) const
    {
        const int t = Nt <= 64 ? tile_s : tile_l;
        return t == 128 ? 128 : 256;
    }
};

struct TuneKey {
    int L, n, M, B, prec;
    bool operator==(const TuneKey &o) const
    {
        return L == o.L && n == o.n && M == o.M && B == o.B && prec == o.prec;
    }
};

struct sw_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;
    char *ws = nullptr;
    size_t ws_size = 0;
    size_t limit = 0;
    std::deque<Tables> tables;  // stable addresses
    std::deque<SliceTables> slice_tables;
    float2 *slice_scratch = nullptr;  // grids of the slice projector above L = 128
    size_t slice_scratch_size = 0;
    int64_t launches = 0;
    bool prof = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<TuneKey, Tune>> tunes;
    const Tune *trial = nullptr;  // overrides the lookup (autotuning, banks)
    long long wait_cycles = 0;    // tensor-core pipeline wait limit (0 = default)
    int stall_corr = 0;           // test hook: tensor-core correlations issue no copies
};

struct sw_bank {
    sw_params p{};
    Tune tune{};  // launch shapes at creation, kept for every alignment
    int Nt = 0;
    int device = 0;
    char *mem = nullptr;
    float *spec32 = nullptr;  // [nh][Nt][2M]
    void *lp_t = nullptr;     // [nh][2Nt][2M] (bf16/fp16) or NULL
    float *prof = nullptr;    // [Nt][M]
    double *center = nullptr; // [Nt][2]
    double *norm32 = nullptr, *norm16 = nullptr;
    int32_t *status = nullptr;
};

namespace {

sw_status fail(sw_ctx *c, sw_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
sw_status fail(sw_ctx *c, sw_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define SW_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), SW_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Runs one kernel launch `fn` on `st`, counting it and, when profiling,
// bracketing it with events.
template <typename F>
cudaError_t launch(sw_ctx *c, int stage, cudaStream_t st, F &&fn)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        for (cudaEvent_t *e : {&a, &b}) {
            if (!c->pool.empty()) {
                *e = c->pool.back();
                c->pool.pop_back();
            } else if (cudaEventCreate(e) != cudaSuccess) {
                return cudaGetLastError();
            }
        }
        cudaEventRecord(a, st);
    }
    cudaError_t e = fn();
    ++c->launches;
    if (c->prof) {
        cudaEventRecord(b, st);
        c->recs.push_back({stage, a, b});
    }
    return e;
}

bool smooth235(int n)
{
    for (int q : {2, 3, 5})
        while (n % q == 0) n /= q;
    return n == 1;
}

sw_status check_params(sw_ctx *c, const sw_params *p)
{
    if (!p) return fail(c, SW_ERR_INVALID_ARG, "params is NULL");
    if (p->L < 2 || p->L > 512) return fail(c, SW_ERR_INVALID_ARG, "L=%d outside 2..512", p->L);
    const int n = p->n_theta;
    if (n < 4 || n > 1024 || (n & 1) || !smooth235(n))
        return fail(c, SW_ERR_INVALID_ARG, "n_theta=%d must be even, 4..1024, with factors 2,3,5",
                    n);
    if (p->n_levels < 1 || p->n_levels > 1024)
        return fail(c, SW_ERR_INVALID_ARG, "n_levels=%d outside 1..1024", p->n_levels);
    const int Bd = sw_default_bins(p->L);
    if (p->n_bins != 0 && (p->n_bins < Bd || (p->n_bins & 1) || p->n_bins > 2048))
        return fail(c, SW_ERR_INVALID_ARG, "n_bins=%d must be 0 or even in %d..2048", p->n_bins,
                    Bd);
    if (p->translation != 0 && p->translation != 1)
        return fail(c, SW_ERR_INVALID_ARG, "translation must be 0 or 1");
    if (p->level_rule != 0 && p->level_rule != 1)
        return fail(c, SW_ERR_INVALID_ARG, "level_rule must be 0 or 1");
    if (p->gemm_precision < SW_PREC_FP32 || p->gemm_precision > SW_PREC_FP32_SIMT)
        return fail(c, SW_ERR_INVALID_ARG, "gemm_precision=%d unknown", p->gemm_precision);
    if (p->metric != SW_METRIC_SW2 && p->metric != SW_METRIC_RFSW2 &&
        p->metric != SW_METRIC_MSW2)
        return fail(c, SW_ERR_INVALID_ARG, "metric=%d unknown", p->metric);
    if (p->metric == SW_METRIC_MSW2 && p->shift_grid > 0)
        return fail(c, SW_ERR_INVALID_ARG, "max-sliced W2 takes no translation grid");
    if (p->shift_grid < 0 || p->shift_grid > 4096 ||
        (p->shift_grid > 0 && (p->shift_step_q <= 0 || p->shift_step_q > 65536)))
        return fail(c, SW_ERR_INVALID_ARG, "shift_grid=%d, shift_step_q=%d", p->shift_grid,
                    p->shift_step_q);
    if (p->metric == SW_METRIC_RFSW2) {
        if (p->n_bins != 0 && !smooth235(p->n_bins))
            return fail(c, SW_ERR_INVALID_ARG,
                        "n_bins=%d: the ramp filter needs a 2/3/5-smooth bin count", p->n_bins);
        if (p->n_levels > 512)
            return fail(c, SW_ERR_INVALID_ARG, "n_levels=%d: at most 512 per part", p->n_levels);
    }
    if (p->projector != SW_PROJ_SPLAT && p->projector != SW_PROJ_SLICE)
        return fail(c, SW_ERR_INVALID_ARG, "projector=%d unknown", p->projector);
    if (p->projector == SW_PROJ_SLICE) {
        // the bins are also the oversampled grid: a multiple of 32 (one
        // warp's FFT) and at least 1.5 L (the NUFFT's accuracy)
        const int B = bins_of(p);
        if (p->L > 256)
            return fail(c, SW_ERR_UNSUPPORTED,
                        "L=%d: the Fourier-slice projector is built for L <= 256", p->L);
        if (!swk::slice_bins_supported(p->L, B))
            return fail(c, SW_ERR_INVALID_ARG,
                        "n_bins=%d: the Fourier-slice projector needs a multiple of 32 that is "
                        "at least 1.5 L (32..192 for L <= 128; 256, 320 or 384 above)",
                        p->n_bins);
    }
    return SW_OK;
}

bool aligned16(const void *ptr) { return ((uintptr_t)ptr & 15u) == 0; }

// sw_result holds doubles: an array of them (at any index) is 8-byte aligned.
sw_status check_result_ptr(sw_ctx *c, const void *ptr, const char *name)
{
    if (!ptr) return fail(c, SW_ERR_INVALID_ARG, "%s is NULL", name);
    if ((uintptr_t)ptr & 7u) return fail(c, SW_ERR_INVALID_ARG, "%s is not 8-byte aligned", name);
    return SW_OK;
}

sw_status check_ptr(sw_ctx *c, const void *ptr, const char *name, bool need)
{
    if (!ptr) return need ? fail(c, SW_ERR_INVALID_ARG, "%s is NULL", name) : SW_OK;
    if (!aligned16(ptr)) return fail(c, SW_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
    return SW_OK;
}

sw_status set_device(sw_ctx *c)
{
    SW_CUDA(c, cudaSetDevice(c->device));
    return SW_OK;
}

TuneKey tune_key(const sw_params *p)
{
    return TuneKey{p->L, p->n_theta, p->n_levels, bins_of(p), (int)p->gemm_precision};
}

Tune tune_of(const sw_ctx *c, const sw_params *p)
{
    if (c->trial) return *c->trial;
    const TuneKey k = tune_key(p);
    for (const auto &e : c->tunes)
        if (e.first == k) return e.second;
    return Tune{};
}

sw_status get_tables(sw_ctx *c, int n, const Tables **out, int variant = 0)
{
    for (const Tables &t : c->tables)
        if (t.n == n && t.variant == variant) {
            *out = &t;
            return SW_OK;
        }
    Tables t;
    t.n = n;
    t.variant = variant;
    if (!fft_plan(n, t.plan, variant))
        return fail(c, SW_ERR_INVALID_ARG, "no FFT plan for n=%d", n);
    std::vector<double> co, si;
    swk::angle_table(n, co, si);
    std::vector<float2> cs(n), tw(n);
    std::vector<double2> cs64(n);
    for (int k = 0; k < n; ++k) {
        cs[k] = make_float2((float)co[k], (float)si[k]);
        cs64[k] = make_double2(co[k], si[k]);
        tw[k] = make_float2((float)co[k], (float)-si[k]);  // e^{-i theta_k}
    }
    SW_CUDA(c, cudaMalloc(&t.cs, sizeof(float2) * n));
    SW_CUDA(c, cudaMalloc(&t.cs64, sizeof(double2) * n));
    SW_CUDA(c, cudaMalloc(&t.tw, sizeof(float2) * n));
    SW_CUDA(c, cudaMemcpy(t.cs, cs.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    SW_CUDA(c, cudaMemcpy(t.cs64, cs64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
    SW_CUDA(c, cudaMemcpy(t.tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    c->tables.push_back(t);
    *out = &c->tables.back();
    return SW_OK;
}

sw_status get_slice_tables(sw_ctx *c, const sw_params *p, const SliceTables **out)
{
    const int L = p->L, n = p->n_theta, B = bins_of(p);
    for (const SliceTables &t : c->slice_tables)
        if (t.L == L && t.n == n && t.B == B) {
            *out = &t;
            return SW_OK;
        }
    SliceTables t;
    t.L = L;
    t.n = n;
    t.B = B;
    t.N = B;  // the oversampled grid is the bin count
    const int W = swk::kSliceW;
    // shape for the oversampling sigma = N / L: beta = 0.97 pi (1 - 1/(2 sigma)) W
    const double sigma = (double)t.N / L;
    t.beta = 0.97 * M_PI * (1.0 - 0.5 / sigma) * W;
    swk::slice_fit_weights(t.beta, t.coef);
    std::vector<float> pinv(L);
    for (int cidx = 0; cidx < L; ++cidx)
        pinv[cidx] = (float)(1.0 / swk::slice_kernel_ft(cidx - L / 2, t.N, W, t.beta));
    // per (angle, frequency): sinc(pi t1) sinc(pi t2) (-1)^j e^{i pi j (1 - 2 delta (c + s)) / B}
    const int nh = n / 2, nj = B / 2 + 1;
    const double delta = (L & 1) ? 0.0 : 0.5;
    std::vector<double> co, si;
    swk::angle_table(n, co, si);
    std::vector<float2> fac((size_t)nh * nj);
    auto sinc_pi = [](double x) { return x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x); };
    for (int k = 0; k < nh; ++k)
        for (int j = 0; j < nj; ++j) {
            const double t1 = (double)j / B * co[k], t2 = (double)j / B * si[k];
            const double amp = sinc_pi(t1) * sinc_pi(t2) * ((j & 1) ? -1.0 : 1.0);
            const double ph = M_PI * j * (1.0 - 2.0 * delta * (co[k] + si[k])) / B;
            fac[(size_t)k * nj + j] =
                make_float2((float)(amp * std::cos(ph)), (float)(amp * std::sin(ph)));
        }
    // Half-warp groups of targets (sw_slice_plan.h): for L <= 128 (grid in
    // shared memory) per batch of slice_batch_of(L) angles, with ray-adjacent
    // pairs; addresses follow the kernel's FP32 arithmetic.
    std::vector<uint16_t> gtab;
    std::vector<int> goff(1, 0);
    // L > 128 (grid in global memory, tiles in shared memory): per tile, the
    // targets whose footprint starts in it; entries k << 16 | j; the bank is
    // that of the first tap in the tile's copy (rows kSliceTileRS apart).
    std::vector<uint32_t> ttab;
    std::vector<int> toff(1, 0);
    if (L <= 128) {
        swk::slice_pair_groups(swk::slice_batch_of(L), nh, t.N, nj,
                               [&](int k, int j, int *r, int *cc, bool *l) {
                                   swk::slice_tap_rc(j, (float)co[k], (float)si[k], t.N, r, cc, l);
                               },
                               gtab, goff);
    } else {
        swk::slice_tile_groups(nh, t.N, nj, co, si, ttab, toff);
    }
    // Images of side L/2 upsampled 2 x 2 (128 < L): their own grid of
    // Nu = B/2 points (same oversampling, so the same kernel shape), the
    // factor (1 + e^{-2 pi i t_1}) (1 + e^{-2 pi i t_2}) / 4 folded into fac,
    // and targets j <= Nu in kUpBatch-angle batches.
    const bool up = swk::slice_up_supported(L, B);
    const int Lu = L / 2, Nu = B / 2;
    std::vector<float> upinv;
    std::vector<float2> upfac, uptw;
    std::vector<uint16_t> upgtab;
    std::vector<int> upgoff(1, 0);
    if (up) {
        upinv.resize(Lu);
        for (int cidx = 0; cidx < Lu; ++cidx)
            upinv[cidx] = (float)(1.0 / swk::slice_kernel_ft(cidx - Lu / 2, Nu, W, t.beta));
        upfac.resize((size_t)nh * nj);
        for (int k = 0; k < nh; ++k)
            for (int j = 0; j < nj; ++j) {
                const double t1 = (double)j / B * co[k], t2 = (double)j / B * si[k];
                const std::complex<double> h1(1.0 + std::cos(2.0 * M_PI * t1),
                                              -std::sin(2.0 * M_PI * t1));
                const std::complex<double> h2(1.0 + std::cos(2.0 * M_PI * t2),
                                              -std::sin(2.0 * M_PI * t2));
                const double amp = sinc_pi(t1) * sinc_pi(t2) * ((j & 1) ? -1.0 : 1.0);
                const double ph = M_PI * j * (1.0 - 2.0 * delta * (co[k] + si[k])) / B;
                const std::complex<double> v =
                    std::complex<double>(amp * std::cos(ph), amp * std::sin(ph)) * h1 * h2 * 0.25;
                upfac[(size_t)k * nj + j] = make_float2((float)v.real(), (float)v.imag());
            }
        uptw.resize(Nu);
        for (int q = 0; q < Nu; ++q)
            uptw[q] = make_float2((float)std::cos(2.0 * M_PI * q / Nu),
                                  (float)-std::sin(2.0 * M_PI * q / Nu));
        swk::slice_pair_groups(swk::kUpBatch, nh, Nu, nj,
                               [&](int k, int j, int *r, int *cc, bool *l) {
                                   swk::slice_up_rc(j, (float)co[k], (float)si[k], Nu, r, cc, l);
                               },
                               upgtab, upgoff);
    }
    SW_CUDA(c, cudaMalloc(&t.psi_inv, sizeof(float) * L));
    SW_CUDA(c, cudaMemcpy(t.psi_inv, pinv.data(), sizeof(float) * L, cudaMemcpyHostToDevice));
    cudaError_t e = cudaMalloc(&t.fac, sizeof(float2) * fac.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(t.fac, fac.data(), sizeof(float2) * fac.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !gtab.empty()) e = cudaMalloc(&t.gtab, sizeof(uint16_t) * gtab.size());
    if (e == cudaSuccess && !gtab.empty())
        e = cudaMemcpy(t.gtab, gtab.data(), sizeof(uint16_t) * gtab.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t.goff, sizeof(int) * goff.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(t.goff, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ttab.empty()) e = cudaMalloc(&t.ttab, sizeof(uint32_t) * ttab.size());
    if (e == cudaSuccess && !ttab.empty())
        e = cudaMemcpy(t.ttab, ttab.data(), sizeof(uint32_t) * ttab.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && L > 128) e = cudaMalloc(&t.toff, sizeof(int) * toff.size());
    if (e == cudaSuccess && L > 128)
        e = cudaMemcpy(t.toff, toff.data(), sizeof(int) * toff.size(), cudaMemcpyHostToDevice);
    auto upload = [&](auto **dst, const auto &v) {
        if (e != cudaSuccess || v.empty()) return;
        const size_t bytes = sizeof(v[0]) * v.size();
        e = cudaMalloc(dst, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice);
    };
    if (up) {
        upload(&t.up_psi_inv, upinv);
        upload(&t.up_fac, upfac);
        upload(&t.up_gtab, upgtab);
        upload(&t.up_goff, upgoff);
        upload(&t.up_tw, uptw);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(t.psi_inv);
        cudaFree(t.fac);
        cudaFree(t.gtab);
        cudaFree(t.goff);
        cudaFree(t.ttab);
        cudaFree(t.toff);
        cudaFree(t.up_psi_inv);
        cudaFree(t.up_fac);
        cudaFree(t.up_gtab);
        cudaFree(t.up_goff);
        cudaFree(t.up_tw);
        return fail(c, SW_ERR_CUDA, "slice tables: %s", cudaGetErrorString(e));
    }
    c->slice_tables.push_back(t);
    *out = &c->slice_tables.back();
    return SW_OK;
}

sw_status ensure_ws(sw_ctx *c, size_t bytes)
{
    if (bytes <= c->ws_size) return SW_OK;
    if (c->limit && bytes > c->limit)
        return fail(c, SW_ERR_OOM, "workspace of %zu bytes exceeds the limit of %zu bytes", bytes,
                    c->limit);
    if (c->ws) {
        SW_CUDA(c, cudaFree(c->ws));
        c->ws = nullptr;
        c->ws_size = 0;
    }
    cudaError_t e = cudaMalloc(&c->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->ws = nullptr;
        return fail(c, SW_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->ws_size = bytes;
    return SW_OK;
}

// Scratch of the slice projector above L = 128 (grids of one chunk of images),
// grown on demand and kept for the context's life (sw_reserve sizes it before
// any stream capture).
sw_status ensure_slice_scratch(sw_ctx *c, size_t bytes)
{
    if (bytes <= c->slice_scratch_size) return SW_OK;
    if (c->slice_scratch) {
        SW_CUDA(c, cudaFree(c->slice_scratch));
        c->slice_scratch = nullptr;
        c->slice_scratch_size = 0;
    }
    cudaError_t e = cudaMalloc(&c->slice_scratch, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->slice_scratch = nullptr;
        return fail(c, SW_ERR_OOM, "slice scratch of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    c->slice_scratch_size = bytes;
    return SW_OK;
}

// Per-image stages into a spectrum set.
struct ImageOut {
    int32_t *status;
    float *proj;  // scratch [nb][nh][B]
    float *ramp;  // scratch [nb][2][nh][B] (ramp-filtered parts), or NULL
    float *quant; // scratch [nb][n][M]
    float *spec32;
    size_t fstride;
    int lp_kind;
    void *lp_q;
    size_t lpq_fstride;
    void *lp_t;
    size_t lpt_fstride;
    int Nq;  // images [0, Nq) are queries for the low-precision layout
    float *prof;
    double *center, *norm32, *norm16;
};

// Projections of nb images with the projector of p (one launch; see
// launch_project / launch_project_slice for the layouts).  t: angle tables
// of n_theta.
sw_status project_rows(sw_ctx *c, const sw_params *p, const Tables *t, const float *img,
                       int srcL, int nb, float *out, int full_n, int32_t *status,
                       cudaStream_t st, const float *img2 = nullptr, int nb_first = -1)
{
    const int nh = p->n_theta / 2, B = bins_of(p);
    if (p->projector == SW_PROJ_SLICE) {
        const SliceTables *sl;
        const Tables *tb;
        sw_status s;
        if ((s = get_slice_tables(c, p, &sl)) || (s = get_tables(c, B, &tb))) return s;
        const int clip = p->metric != SW_METRIC_RFSW2;
        if (2 * srcL == p->L && sl->up_gtab) {  // the L/2 image's own grid, one launch
            SW_CUDA(c, launch(c, SW_STAGE_PROJECT, st, [&] {
                        return swk::launch_project_slice_up(img, nb, p->L, nh, B, t->cs,
                                                            sl->up(), sl->coef, tb->tw, clip,
                                                            out, full_n, status, st, img2,
                                                            nb_first);
                    }));
            return SW_OK;
        }
        if ((s = ensure_slice_scratch(c, swk::slice_scratch_bytes(p->L, B, nb, nh)))) return s;
        SW_CUDA(c, launch(c, SW_STAGE_PROJECT, st, [&] {
                    return swk::launch_project_slice(img, nb, p->L, srcL, nh, B, t->cs,
                                                     sl->psi_inv, sl->fac, sl->gtab, sl->goff,
                                                     sl->ttab, sl->toff, sl->coef, tb->tw,
                                                     c->slice_scratch, clip, out, full_n,
                                                     status, st, img2, nb_first);
                }));
        // above L = 128: grid, tile and row kernels per chunk of images
        if (p->L > 128 && nb > 0)
            c->launches += 3 * ((nb + swk::kSliceChunk - 1) / swk::kSliceChunk) - 1;
        return SW_OK;
    }
    SW_CUDA(c, launch(c, SW_STAGE_PROJECT, st, [&] {
                return swk::launch_project(img, nb, p->L, srcL, nh, B, t->cs, out, full_n,
                                           status, st, tune_of(c, p).want, img2, nb_first);
            }));
    return SW_OK;
}

sw_status run_images(sw_ctx *c, const sw_params *p, const Tables *t, const float *img,
                     int srcL, int nb, int img_off, const ImageOut &o, cudaStream_t st)
{
    const int nh = p->n_theta / 2, B = bins_of(p);
    return project_rows(c, p, t, img, srcL, nb, o.proj + (size_t)img_off * nh * B, 0,
                        o.status + img_off, st);
}

sw_status run_after_projection(sw_ctx *c, const sw_params *p, const Tables *t, int nb,
                               const ImageOut &o, cudaStream_t st)
{
    const int L = p->L, n = p->n_theta, M = p->n_levels, B = bins_of(p);
    const float h = 2.0f / (float)L;
    const int parts = parts_of(p);
    if (parts == 2) {
        // ramp filter and split, then the quantiles of both parts (rows
        // 2 img + part, their status folded onto the image)
        const Tables *tb;
        sw_status s = get_tables(c, B, &tb);
        if (s) return s;
        SW_CUDA(c, launch(c, SW_STAGE_RAMP, st, [&] {
                    return swk::launch_ramp(o.proj, nb, n / 2, B, tb->plan, tb->tw, o.ramp, st);
                }));
        SW_CUDA(c, launch(c, SW_STAGE_QUANTILE, st, [&] {
                    return swk::launch_quantiles(o.ramp, 2 * nb, n, B, M, h, p->level_rule, 1,
                                                 o.quant, o.status, st, 1);
                }));
    } else {
        SW_CUDA(c, launch(c, SW_STAGE_QUANTILE, st, [&] {
                    return swk::launch_quantiles(o.proj, nb, n, B, M, h, p->level_rule, 1,
                                                 o.quant, o.status, st);
                }));
    }
    SW_CUDA(c, launch(c, SW_STAGE_SPECTRUM, st, [&] {
                return swk::launch_spectrum(o.quant, nb, n, M * parts, t->plan, t->tw, o.spec32,
                                            o.fstride, o.lp_kind, o.lp_q, o.lpq_fstride, o.lp_t,
                                            o.lpt_fstride, o.Nq, o.prof, o.center, o.norm32,
                                            o.norm16, st, tune_of(c, p).spec, parts);
            }));
    return SW_OK;
}

template <typename T>
T *at(char *base, size_t off)
{
    return reinterpret_cast<T *>(base + off);
}

}  // namespace

extern "C" {

int sw_default_bins(int L)
{
    if (L < 1) return 0;
    return 2 * (int)std::ceil((double)(L - 1) / std::sqrt(2.0)) + 2;
}

sw_status sw_create(int device, sw_ctx **out)
{
    if (!out) return SW_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return SW_ERR_CUDA;
    }
    if (device < 0 || device >= count) return SW_ERR_INVALID_ARG;
    sw_ctx *c = new (std::nothrow) sw_ctx;
    if (!c) return SW_ERR_OOM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SW_ERR_CUDA;
    }
    *out = c;
    return SW_OK;
}

void sw_destroy(sw_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->ws) cudaFree(c->ws);
    for (ProfRec &r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    for (Tables &t : c->tables) {
        cudaFree(t.cs);
        cudaFree(t.cs64);
        cudaFree(t.tw);
    }
    for (SliceTables &t : c->slice_tables) {
        cudaFree(t.psi_inv);
        cudaFree(t.fac);
        cudaFree(t.gtab);
        cudaFree(t.goff);
        cudaFree(t.ttab);
        cudaFree(t.toff);
        cudaFree(t.up_psi_inv);
        cudaFree(t.up_fac);
        cudaFree(t.up_gtab);
        cudaFree(t.up_goff);
        cudaFree(t.up_tw);
    }
    if (c->slice_scratch) cudaFree(c->slice_scratch);
    delete c;
}

const char *sw_last_error(const sw_ctx *c) { return c ? c->err.c_str() : ""; }

sw_status sw_set_wait_limit(sw_ctx *c, int64_t cycles)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    if (cycles < 0) return fail(c, SW_ERR_INVALID_ARG, "cycles=%lld", (long long)cycles);
    c->wait_cycles = (long long)cycles;
    return SW_OK;
}

sw_status sw_set_correlation_stall(sw_ctx *c, int enable)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    c->stall_corr = enable ? 1 : 0;
    return SW_OK;
}

sw_status sw_profile(sw_ctx *c, int enable)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->prof = enable != 0;
    return SW_OK;
}

sw_status sw_profile_read(sw_ctx *c, double *ms, int64_t *launches)
{
    if (!c || !ms || !launches) return SW_ERR_INVALID_ARG;
    for (int i = 0; i < SW_STAGE_COUNT; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    sw_status s = SW_OK;
    for (ProfRec &r : c->recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess ||
            cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            s = fail(c, SW_ERR_CUDA, "profiling event failed");
        }
        ms[r.stage] += t;
        launches[r.stage] += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    return s;
}

int64_t sw_launch_count(const sw_ctx *c) { return c ? c->launches : 0; }

sw_status sw_set_workspace_limit(sw_ctx *c, size_t bytes)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->limit = bytes;
    return SW_OK;
}

size_t sw_batch_workspace_bytes(const sw_params *p, int Nq, int Nt)
{
    if (!p || Nq < 0 || Nt < 0 || check_params(nullptr, p) != SW_OK) return 0;
    return batch_layout(p, Nq, Nt, lp_kind_of(p->gemm_precision), true).total;
}

sw_status sw_reserve(sw_ctx *c, const sw_params *p, int Nq, int Nt)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if (Nq < 0 || Nt < 0) return fail(c, SW_ERR_INVALID_ARG, "negative batch size");
    if ((s = set_device(c))) return s;
    const Tables *t;
    if ((s = get_tables(c, p->n_theta, &t))) return s;
    if (parts_of(p) == 2 && (s = get_tables(c, bins_of(p), &t))) return s;
    if (p->projector == SW_PROJ_SLICE) {  // tables of the projector, built outside any capture
        const SliceTables *sl;
        if ((s = get_slice_tables(c, p, &sl)) || (s = get_tables(c, bins_of(p), &t)) ||
            (s = ensure_slice_scratch(
                 c, swk::slice_scratch_bytes(p->L, bins_of(p), Nq + Nt, p->n_theta / 2))))
            return s;
    }
    return ensure_ws(c, batch_layout(p, Nq, Nt, lp_kind_of(p->gemm_precision), true).total);
}

sw_status sw_project(sw_ctx *c, const sw_params *p, const float *d_img, int nb, float *d_proj,
                     double *d_scale, sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if (nb < 0) return fail(c, SW_ERR_INVALID_ARG, "nb=%d", nb);
    if (nb == 0) return SW_OK;
    if ((s = check_ptr(c, d_img, "d_img", true)) || (s = check_ptr(c, d_proj, "d_proj", true)))
        return s;
    if ((uintptr_t)d_scale & 7u) return fail(c, SW_ERR_INVALID_ARG, "d_scale is not 8-byte aligned");
    if ((s = set_device(c))) return s;
    const Tables *t;
    if ((s = get_tables(c, p->n_theta, &t))) return s;
    const size_t need = align_up(4 * (size_t)nb);
    if ((s = ensure_ws(c, need))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (d_scale)
        SW_CUDA(c, launch(c, SW_STAGE_PROJECT, st, [&] {
                    return swk::launch_image_scale(d_img, nb, p->L, d_scale, st);
                }));
    return project_rows(c, p, t, d_img, p->L, nb, d_proj, 1, at<int32_t>(c->ws, 0), st);
}

sw_status sw_project_upsampled(sw_ctx *c, const sw_params *p, const float *d_img, int nb,
                               float *d_proj, sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if (p->L & 1) return fail(c, SW_ERR_INVALID_ARG, "L=%d is odd: no L/2 images", p->L);
    if (nb < 0) return fail(c, SW_ERR_INVALID_ARG, "nb=%d", nb);
    if (nb == 0) return SW_OK;
    if ((s = check_ptr(c, d_img, "d_img", true)) || (s = check_ptr(c, d_proj, "d_proj", true)))
        return s;
    if ((s = set_device(c))) return s;
    const Tables *t;
    if ((s = get_tables(c, p->n_theta, &t))) return s;
    if ((s = ensure_ws(c, align_up(4 * (size_t)nb)))) return s;
    return project_rows(c, p, t, d_img, p->L / 2, nb, d_proj, 1, at<int32_t>(c->ws, 0),
                        (cudaStream_t)stream);
}

sw_status sw_quantiles(sw_ctx *c, const sw_params *p, const float *d_proj, int nb, float *d_q,
                       double *d_center, double *d_norm, sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if (nb < 0) return fail(c, SW_ERR_INVALID_ARG, "nb=%d", nb);
    if (nb == 0) return SW_OK;
    if ((s = check_ptr(c, d_proj, "d_proj", true)) || (s = check_ptr(c, d_q, "d_q", true)) ||
        (s = check_ptr(c, d_center, "d_center", false)) ||
        (s = check_ptr(c, d_norm, "d_norm", false)))
        return s;
    if ((s = set_device(c))) return s;
    const Tables *t;
    if ((s = get_tables(c, p->n_theta, &t))) return s;
    const int n = p->n_theta, B = bins_of(p), parts = parts_of(p);
    const size_t ramp_bytes = parts == 2 ? 4 * (size_t)nb * 2 * n * B : 0;
    if ((s = ensure_ws(c, align_up(4 * (size_t)nb) + ramp_bytes))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = at<int32_t>(c->ws, 0);
    SW_CUDA(c, cudaMemsetAsync(status, 0, 4 * (size_t)nb, st));
    const float *rows = d_proj;
    if (parts == 2) {  // ramp-filtered parts: rows 2 img + part
        const Tables *tb;
        if ((s = get_tables(c, B, &tb))) return s;
        float *ramp = at<float>(c->ws, align_up(4 * (size_t)nb));
        SW_CUDA(c, launch(c, SW_STAGE_RAMP, st, [&] {
                    return swk::launch_ramp(d_proj, nb, n, B, tb->plan, tb->tw, ramp, st);
                }));
        rows = ramp;
    }
    SW_CUDA(c, launch(c, SW_STAGE_QUANTILE, st, [&] {
                return swk::launch_quantiles(rows, parts * nb, n, B, p->n_levels,
                                             2.0f / (float)p->L, p->level_rule, 0, d_q, status,
                                             st, parts == 2 ? 1 : 0);
            }));
    if (d_center || d_norm)
        SW_CUDA(c, launch(c, SW_STAGE_QUANTILE, st, [&] {
                    return swk::launch_center_norm(d_q, parts * nb, n, p->n_levels, t->cs64,
                                                   d_center, d_norm, st);
                }));
    return SW_OK;
}

}  // extern "C"

namespace {

// Shared body of sw_align_batch / sw_align_all_rotations.
sw_status align_batch_impl(sw_ctx *c, const sw_params *p, const float *dq, int Nq,
                           const float *dt, int Nt, int mode, sw_result *out, double *curve,
                           double *shifts, bool force_fp32, cudaStream_t st)
{
    const int n = p->n_theta, nh = n / 2, M = levels_of(p);
    const int kind = force_fp32 ? 0 : lp_kind_of(p->gemm_precision);
    const bool lp = kind != 0;
    const Tune tu = tune_of(c, p);
    const Tables *t;
    sw_status s = get_tables(c, n, &t, tu.plan);
    if (s) return s;
    const Layout l = batch_layout(p, Nq, Nt, kind, mode == 1);
    if ((s = ensure_ws(c, l.total))) return s;
    char *w = c->ws;
    const int nimg = Nq + Nt;
    const int row = lp ? swk::lp_row_len(M, kind) : 0;
    ImageOut o{};
    o.status = at<int32_t>(w, l.status);
    o.proj = at<float>(w, l.proj);
    o.ramp = at<float>(w, l.ramp);
    o.quant = at<float>(w, l.quant);
    o.spec32 = lp ? nullptr : at<float>(w, l.spec32);
    o.fstride = (size_t)nimg * 2 * M;
    o.lp_kind = kind;
    o.lp_q = lp ? (void *)(w + l.lp_q) : nullptr;
    o.lpq_fstride = (size_t)Nq * row;
    o.lp_t = lp ? (void *)(w + l.lp_t) : nullptr;
    o.lpt_fstride = (size_t)2 * Nt * row;
    o.Nq = Nq;
    o.prof = at<float>(w, l.prof);
    o.center = at<double>(w, l.center);
    o.norm32 = at<double>(w, l.norm32);
    o.norm16 = at<double>(w, l.norm16);
    // queries and templates projected in one launch
    if ((s = project_rows(c, p, t, dq, p->L, nimg, o.proj, 0, o.status, st, dt, Nq))) return s;
    if (p->metric == SW_METRIC_MSW2) {
        // max-sliced: quantiles (and centring vectors), then every column pair
        SW_CUDA(c, launch(c, SW_STAGE_QUANTILE, st, [&] {
                    return swk::launch_quantiles(o.proj, nimg, n, bins_of(p), M,
                                                 2.0f / (float)p->L, p->level_rule, 1, o.quant,
                                                 o.status, st);
                }));
        if (p->translation)
            SW_CUDA(c, launch(c, SW_STAGE_QUANTILE, st, [&] {
                        return swk::launch_center_norm(o.quant, nimg, n, M, t->cs64, o.center,
                                                       nullptr, st);
                    }));
        swk::MswArgs a{};
        a.q = o.quant;
        a.t = o.quant + (size_t)Nq * n * M;
        a.Nq = Nq;
        a.Nt = Nt;
        a.n = n;
        a.M = M;
        a.ctr_q = o.center;
        a.ctr_t = o.center + 2 * (size_t)Nq;
        a.st_q = o.status;
        a.st_t = o.status + Nq;
        a.cs64 = t->cs64;
        a.translation = p->translation;
        a.curve = at<float>(w, l.C);
        a.out = mode == 1 ? (void *)(w + l.scratch) : (void *)out;
        a.full = curve;
        a.shifts = shifts;
        SW_CUDA(c, launch(c, SW_STAGE_DECIDE, st, [&] { return swk::launch_msw(a, st); }));
        if (mode == 1)
            SW_CUDA(c, launch(c, SW_STAGE_BEST, st, [&] {
                        return swk::launch_best_template(w + l.scratch, Nq, Nt, out, st);
                    }));
        return SW_OK;
    }
    if ((s = run_after_projection(c, p, t, nimg, o, st))) return s;
    float2 *C = at<float2>(w, l.C);
    int *err = at<int>(w, l.err);
    SW_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), st));
    if (lp) {
        SW_CUDA(c, launch(c, SW_STAGE_CORR, st, [&] {
                    return swk::launch_corr_tc(o.lp_q, o.lp_t, Nq, Nt, M, nh, kind, C, err,
                                               c->num_sms, st, c->wait_cycles, c->stall_corr,
                                               tu.tile_for(Nt));
                }));
    } else {
        SW_CUDA(c, launch(c, SW_STAGE_CORR, st, [&] {
                    return swk::launch_corr_simt(o.spec32, o.fstride,
                                                 o.spec32 + (size_t)Nq * 2 * M, o.fstride, Nq, Nt,
                                                 M, nh, C, st);
                }));
    }
    swk::DecideArgs a{};
    a.C = C;
    a.Nq = Nq;
    a.Nt = Nt;
    a.n = n;
    a.M = M;
    a.parts = parts_of(p);
    a.prof_q = o.prof;
    a.prof_t = o.prof + (size_t)Nq * M;
    a.ctr_q = o.center;
    a.ctr_t = o.center + 2 * (size_t)a.parts * Nq;
    // the split path approximates the FP32 product: FP32 norms; BF16/FP16: the
    // norms of the rounded spectra, so that self-distances cancel
    const double *nrm = (kind == 1 || kind == 2) ? o.norm16 : o.norm32;
    a.norm_q = nrm;
    a.norm_t = nrm + Nq;
    a.st_q = o.status;
    a.st_t = o.status + Nq;
    a.cs64 = t->cs64;
    a.translation = p->translation;
    a.grid_k = p->translation ? p->shift_grid : 0;
    a.grid_step = (double)p->shift_step_q * (2.0 / p->L) / 16.0;
    a.dev_err = err;
    a.out = mode == 1 ? (void *)(w + l.scratch) : (void *)out;
    a.curve = curve;
    a.shifts = shifts;
    SW_CUDA(c, launch(c, SW_STAGE_DECIDE, st,
                      [&] { return swk::launch_decide(a, t->plan, t->tw, st, tu.dec); }));
    if (mode == 1)
        SW_CUDA(c, launch(c, SW_STAGE_BEST, st, [&] {
                    return swk::launch_best_template(w + l.scratch, Nq, Nt, out, st);
                }));
    return SW_OK;
}

}  // namespace

extern "C" {

sw_status sw_align_all_rotations(sw_ctx *c, const sw_params *p, const float *d_f,
                                 const float *d_g, double *d_D, double *d_shift,
                                 sw_result *d_best, sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if ((s = check_ptr(c, d_f, "d_f", true)) || (s = check_ptr(c, d_g, "d_g", true)) ||
        (s = check_result_ptr(c, d_best, "d_best")))
        return s;
    if (d_D && ((uintptr_t)d_D & 7)) return fail(c, SW_ERR_INVALID_ARG, "d_D misaligned");
    if (d_shift && ((uintptr_t)d_shift & 7))
        return fail(c, SW_ERR_INVALID_ARG, "d_shift misaligned");
    if ((s = set_device(c))) return s;
    return align_batch_impl(c, p, d_f, 1, d_g, 1, 0, d_best, d_D, d_shift, true,
                            (cudaStream_t)stream);
}

sw_status sw_align_batch(sw_ctx *c, const sw_params *p, const float *d_q_img, int Nq,
                         const float *d_t_img, int Nt, int mode, sw_result *d_out,
                         sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if (Nq < 0 || Nt < 0) return fail(c, SW_ERR_INVALID_ARG, "Nq=%d Nt=%d", Nq, Nt);
    if (mode != 0 && mode != 1) return fail(c, SW_ERR_INVALID_ARG, "mode=%d", mode);
    if (Nq == 0) return SW_OK;
    if (Nt == 0 && mode == 0) return SW_OK;
    if ((s = check_ptr(c, d_q_img, "d_q_img", true)) || (s = check_result_ptr(c, d_out, "d_out")))
        return s;
    if (Nt > 0 && (s = check_ptr(c, d_t_img, "d_t_img", true))) return s;
    if ((s = set_device(c))) return s;
    if (Nt == 0) return fail(c, SW_ERR_INVALID_ARG, "mode 1 needs at least one template");
    return align_batch_impl(c, p, d_q_img, Nq, d_t_img, Nt, mode, d_out, nullptr, nullptr,
                            false, (cudaStream_t)stream);
}

sw_status sw_bank_create(sw_ctx *c, const sw_params *p, const float *d_t_img, int Nt,
                         sw_bank **out, sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    if (!out) return fail(c, SW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sw_status s = check_params(c, p);
    if (s) return s;
    if (Nt <= 0) return fail(c, SW_ERR_INVALID_ARG, "Nt=%d", Nt);
    if (p->metric == SW_METRIC_MSW2)
        return fail(c, SW_ERR_UNSUPPORTED, "banks hold spectra; max-sliced W2 needs quantiles");
    if ((s = check_ptr(c, d_t_img, "d_t_img", true))) return s;
    if ((s = set_device(c))) return s;
    const Tune tu = tune_of(c, p);
    const Tables *t;
    if ((s = get_tables(c, p->n_theta, &t, tu.plan))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->n_theta, nh = n / 2, M = levels_of(p), B = bins_of(p);
    const int parts = parts_of(p);
    const int kind = lp_kind_of(p->gemm_precision);
    const bool lp = kind != 0;
    const int row = lp ? swk::lp_row_len(M, kind) : 0;
    // bank memory (owned by the bank)
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at_ = o;
        o = align_up(o + bytes);
        return at_;
    };
    const size_t o_spec = take(lp ? 0 : 4 * (size_t)nh * Nt * 2 * M);
    const size_t o_lp = take(2 * (size_t)nh * 2 * Nt * row);
    const size_t o_prof = take(4 * (size_t)Nt * M);
    const size_t o_ctr = take(16 * (size_t)parts * Nt);
    const size_t o_n32 = take(8 * (size_t)Nt);
    const size_t o_n16 = take(8 * (size_t)Nt);
    const size_t o_st = take(4 * (size_t)Nt);
    sw_bank *b = new (std::nothrow) sw_bank;
    if (!b) return fail(c, SW_ERR_OOM, "bank descriptor");
    b->p = *p;
    b->tune = tu;
    b->Nt = Nt;
    b->device = c->device;
    if (cudaMalloc(&b->mem, o) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(c, SW_ERR_OOM, "bank of %zu bytes does not fit", o);
    }
    b->spec32 = lp ? nullptr : at<float>(b->mem, o_spec);
    b->lp_t = lp ? (void *)(b->mem + o_lp) : nullptr;
    b->prof = at<float>(b->mem, o_prof);
    b->center = at<double>(b->mem, o_ctr);
    b->norm32 = at<double>(b->mem, o_n32);
    b->norm16 = at<double>(b->mem, o_n16);
    b->status = at<int32_t>(b->mem, o_st);
    // projections, ramp-filtered parts and quantiles pass through the
    // context workspace
    const size_t need = align_up(4 * (size_t)Nt * nh * B) + align_up(4 * (size_t)Nt * n * M) +
                        (parts == 2 ? align_up(4 * (size_t)Nt * 2 * nh * B) : 0);
    if ((s = ensure_ws(c, need))) {
        cudaFree(b->mem);
        delete b;
        return s;
    }
    ImageOut io{};
    io.status = b->status;
    io.proj = at<float>(c->ws, 0);
    io.quant = at<float>(c->ws, align_up(4 * (size_t)Nt * nh * B));
    io.ramp = parts == 2 ? at<float>(c->ws, align_up(4 * (size_t)Nt * nh * B) +
                                                align_up(4 * (size_t)Nt * n * M))
                         : nullptr;
    io.spec32 = b->spec32;
    io.fstride = (size_t)Nt * 2 * M;
    io.lp_kind = kind;
    io.lp_q = nullptr;
    io.lpq_fstride = 0;
    io.lp_t = b->lp_t;
    io.lpt_fstride = (size_t)2 * Nt * row;
    io.Nq = 0;  // every image is a template (doubled low-precision rows)
    io.prof = b->prof;
    io.center = b->center;
    io.norm32 = b->norm32;
    io.norm16 = b->norm16;
    const Tune *prev = c->trial;
    c->trial = &b->tune;
    s = run_images(c, p, t, d_t_img, p->L, Nt, 0, io, st);
    if (!s) s = run_after_projection(c, p, t, Nt, io, st);
    c->trial = prev;
    if (s) {
        cudaStreamSynchronize(st);
        cudaFree(b->mem);
        delete b;
        return s;
    }
    *out = b;
    return SW_OK;
}

size_t sw_bank_workspace_bytes(const sw_bank *bank, int Nq, int mode)
{
    if (!bank || Nq < 0) return 0;
    return bank_layout(&bank->p, Nq, bank->Nt, mode == 1).total;
}

static sw_status bank_align_impl(sw_ctx *c, const sw_bank *bank, const float *d_q_img, int Nq,
                                 int q_L, int mode, sw_result *d_out, sw_stream_t stream);

sw_status sw_bank_align(sw_ctx *c, const sw_bank *bank, const float *d_q_img, int Nq, int q_L,
                        int mode, sw_result *d_out, sw_stream_t stream)
{
    if (!c) return SW_ERR_INVALID_ARG;
    if (!bank) {
        c->err = "bank is NULL";
        return SW_ERR_INVALID_ARG;
    }
    // the bank's launch shapes (its template spectra used the same FFT plan)
    const Tune *prev = c->trial;
    c->trial = &bank->tune;
    const sw_status s = bank_align_impl(c, bank, d_q_img, Nq, q_L, mode, d_out, stream);
    c->trial = prev;
    return s;
}

static sw_status bank_align_impl(sw_ctx *c, const sw_bank *bank, const float *d_q_img, int Nq,
                                 int q_L, int mode, sw_result *d_out, sw_stream_t stream)
{
    c->err.clear();
    if (!bank) return fail(c, SW_ERR_INVALID_ARG, "bank is NULL");
    const sw_params *p = &bank->p;
    if (Nq < 0) return fail(c, SW_ERR_INVALID_ARG, "Nq=%d", Nq);
    if (mode != 0 && mode != 1) return fail(c, SW_ERR_INVALID_ARG, "mode=%d", mode);
    if (q_L != p->L && !(2 * q_L == p->L))
        return fail(c, SW_ERR_INVALID_ARG, "q_L=%d must be L=%d or L/2", q_L, p->L);
    if (Nq == 0) return SW_OK;
    sw_status s;
    if ((s = check_ptr(c, d_q_img, "d_q_img", true)) || (s = check_result_ptr(c, d_out, "d_out")))
        return s;
    if (bank->device != c->device)
        return fail(c, SW_ERR_INVALID_ARG, "bank lives on device %d, context on %d", bank->device,
                    c->device);
    if ((s = set_device(c))) return s;
    const Tables *t;
    if ((s = get_tables(c, p->n_theta, &t, bank->tune.plan))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->n_theta, nh = n / 2, M = levels_of(p), Nt = bank->Nt;
    const int kind = lp_kind_of(p->gemm_precision);
    const bool lp = kind != 0;
    const Layout l = bank_layout(p, Nq, Nt, mode == 1);
    if ((s = ensure_ws(c, l.total))) return s;
    char *w = c->ws;
    const int row = lp ? swk::lp_row_len(M, kind) : 0;
    ImageOut o{};
    o.status = at<int32_t>(w, l.status);
    o.proj = at<float>(w, l.proj);
    o.ramp = at<float>(w, l.ramp);
    o.quant = at<float>(w, l.quant);
    o.spec32 = lp ? nullptr : at<float>(w, l.spec32);
    o.fstride = (size_t)Nq * 2 * M;
    o.lp_kind = kind;
    o.lp_q = lp ? (void *)(w + l.lp_q) : nullptr;
    o.lpq_fstride = (size_t)Nq * row;
    o.lp_t = nullptr;
    o.lpt_fstride = 0;
    o.Nq = Nq;  // every image is a query
    o.prof = at<float>(w, l.prof);
    o.center = at<double>(w, l.center);
    o.norm32 = at<double>(w, l.norm32);
    o.norm16 = at<double>(w, l.norm16);
    if ((s = run_images(c, p, t, d_q_img, q_L, Nq, 0, o, st))) return s;
    if ((s = run_after_projection(c, p, t, Nq, o, st))) return s;
    float2 *C = at<float2>(w, l.C);
    int *err = at<int>(w, l.err);
    SW_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), st));
    if (lp) {
        SW_CUDA(c, launch(c, SW_STAGE_CORR, st, [&] {
                    return swk::launch_corr_tc(o.lp_q, bank->lp_t, Nq, Nt, M, nh, kind, C, err,
                                               c->num_sms, st, c->wait_cycles, c->stall_corr,
                                               bank->tune.tile_for(Nt));
                }));
    } else {
        SW_CUDA(c, launch(c, SW_STAGE_CORR, st, [&] {
                    return swk::launch_corr_simt(o.spec32, o.fstride, bank->spec32,
                                                 (size_t)Nt * 2 * M, Nq, Nt, M, nh, C, st);
                }));
    }
    swk::DecideArgs a{};
    a.C = C;
    a.Nq = Nq;
    a.Nt = Nt;
    a.n = n;
    a.M = M;
    a.parts = parts_of(p);
    a.prof_q = o.prof;
    a.prof_t = bank->prof;
    a.ctr_q = o.center;
    a.ctr_t = bank->center;
    const bool n16 = kind == 1 || kind == 2;
    a.norm_q = n16 ? o.norm16 : o.norm32;
    a.norm_t = n16 ? bank->norm16 : bank->norm32;
    a.st_q = o.status;
    a.st_t = bank->status;
    a.cs64 = t->cs64;
    a.translation = p->translation;
    a.grid_k = p->translation ? p->shift_grid : 0;
    a.grid_step = (double)p->shift_step_q * (2.0 / p->L) / 16.0;
    a.dev_err = err;
    a.out = mode == 1 ? (void *)(w + l.scratch) : (void *)d_out;
    SW_CUDA(c, launch(c, SW_STAGE_DECIDE, st, [&] {
                return swk::launch_decide(a, t->plan, t->tw, st, bank->tune.dec);
            }));
    if (mode == 1)
        SW_CUDA(c, launch(c, SW_STAGE_BEST, st, [&] {
                    return swk::launch_best_template(w + l.scratch, Nq, Nt, d_out, st);
                }));
    return SW_OK;
}

int sw_bank_size(const sw_bank *bank) { return bank ? bank->Nt : 0; }

void sw_bank_destroy(sw_bank *bank)
{
    if (!bank) return;
    cudaSetDevice(bank->device);
    cudaDeviceSynchronize();
    cudaFree(bank->mem);
    delete bank;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single-pair alignment (sw_align_all_rotations_noalloc).
//
// Some callers may not allocate device memory once they are running: a
// serving process that has handed all device memory to its own pool, a
// latency-critical loop where the implicit device synchronisation of
// cudaMalloc / cudaFree is not acceptable, or a plugin whose host forbids
// device allocations after start-up.  For them this entry point runs the same
// kernel sequence as sw_align_all_rotations with every intermediate buffer
// and table carved from one file-scope device array of fixed size, and calls
// no cudaMalloc, cudaFree or allocating library routine.  The angle tables
// are computed by a kernel into that array, so a call copies nothing from
// host memory and does not wait on the host.
//
// The array is a __device__ variable: host code cannot use its name as a
// device address, so its address is taken with cudaGetSymbolAddress, once per
// device with that device current, on the first call made on that device
// (make that first call before any stream capture).  Every call on a device
// shares the array and leaves its contents behind; calls that overlap on the
// GPU (different streams, no ordering) race on it.
namespace {

constexpr size_t kNoAllocBytes = (size_t)4 << 20;  // 4 MiB on every device that loads the library
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocState {
    std::mutex mu;
    char *addr[kNoAllocMaxDevices] = {};
    // FFT plans (host values passed by kernel argument), per n
    std::deque<std::pair<int, FftPlan>> plans;
};

NoAllocState &noalloc_state()
{
    static NoAllocState s;
    return s;
}

// The angle tables of one call, computed on the device so that a call copies
// nothing from host memory: cs[k] = (cos, sin) theta_k for k < n/2 (FP32),
// cs64[k] for k < n (FP64), tw[k] = e^{-i theta_k} (FP32), theta_k = 2 pi k / n.
// Each angle is reduced to the first octant by integer arithmetic and
// rebuilt by the symmetries of the square, as the host tables of a context
// are, so quarter turns give the exact axis vectors.  Thread 0 also clears
// the decision's error word, the one scratch value that must start at zero.
__global__ void k_noalloc_tables(int n, float2 *cs, double2 *cs64, float2 *tw, int *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) *err = 0;
    if (k >= n) return;
    const long long num = 8LL * k;  // angle = (num / n) pi / 4
    const int oct = (int)(num / n);
    const long long rem = num - (long long)oct * n;
    const bool from_top = oct & 1;
    double t = (double)rem / n * (M_PI / 4.0);
    if (from_top) t = M_PI / 4.0 - t;
    const double co = cos(t), si = sin(t);
    double cc, ss;
    switch (oct & 7) {
    case 0: cc = co; ss = si; break;
    case 1: cc = si; ss = co; break;
    case 2: cc = -si; ss = co; break;
    case 3: cc = -co; ss = si; break;
    case 4: cc = -co; ss = -si; break;
    case 5: cc = -si; ss = -co; break;
    case 6: cc = si; ss = -co; break;
    default: cc = co; ss = -si; break;
    }
    if (k < n / 2) cs[k] = make_float2((float)cc, (float)ss);
    cs64[k] = make_double2(cc, ss);
    tw[k] = make_float2((float)cc, (float)-ss);
}

}  // namespace

extern "C" sw_status sw_align_all_rotations_noalloc(const sw_params *p, const float *d_f,
                                                    const float *d_g, double *d_D,
                                                    double *d_shift, sw_result *d_best,
                                                    sw_stream_t stream)
{
    const sw_status sp = check_params(nullptr, p);
    if (sp != SW_OK) return sp;
    if (p->metric != SW_METRIC_SW2 || p->projector != SW_PROJ_SPLAT)
        return SW_ERR_UNSUPPORTED;  // sliced W2 on the linear splat only
    if (!d_f || !d_g || !d_best || !aligned16(d_f) || !aligned16(d_g) || !aligned16(d_best) ||
        ((uintptr_t)d_D & 7) || ((uintptr_t)d_shift & 7))
        return SW_ERR_INVALID_ARG;
    const int n = p->n_theta, nh = n / 2, M = p->n_levels, B = bins_of(p);
    // scratch: the FP32 batch layout for one query and one template, then the tables
    const Layout l = batch_layout(p, 1, 1, 0, false);
    const size_t o_cs = align_up(l.total);
    const size_t o_cs64 = align_up(o_cs + sizeof(float2) * nh);
    const size_t o_tw = align_up(o_cs64 + sizeof(double2) * n);
    const size_t need = o_tw + sizeof(float2) * n;
    if (need > kNoAllocBytes) return SW_ERR_OOM;  // beyond the fixed scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SW_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return SW_ERR_UNSUPPORTED;
    NoAllocState &ns = noalloc_state();
    char *w = nullptr;
    FftPlan plan{};
    {
        std::lock_guard<std::mutex> g(ns.mu);
        if (!ns.addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return SW_ERR_CUDA;
            }
            ns.addr[dev] = static_cast<char *>(ptr);
        }
        w = ns.addr[dev];
        const FftPlan *found = nullptr;
        for (const auto &e : ns.plans)
            if (e.first == n) found = &e.second;
        if (!found) {
            FftPlan fp{};
            if (!fft_plan(n, fp)) return SW_ERR_INVALID_ARG;
            ns.plans.emplace_back(n, fp);
            found = &ns.plans.back().second;
        }
        plan = *found;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float2 *cs = reinterpret_cast<float2 *>(w + o_cs);
    double2 *cs64 = reinterpret_cast<double2 *>(w + o_cs64);
    float2 *tw = reinterpret_cast<float2 *>(w + o_tw);
    int *err = reinterpret_cast<int *>(w + l.err);
#define SW_NA(call)                                \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            cudaGetLastError();                    \
            return SW_ERR_CUDA;                    \
        }                                          \
    } while (0)
    k_noalloc_tables<<<(n + 255) / 256, 256, 0, st>>>(n, cs, cs64, tw, err);
    SW_NA(cudaGetLastError());

    int32_t *status = reinterpret_cast<int32_t *>(w + l.status);
    float *proj = reinterpret_cast<float *>(w + l.proj);
    float *quant = reinterpret_cast<float *>(w + l.quant);
    float *spec32 = reinterpret_cast<float *>(w + l.spec32);
    float *prof = reinterpret_cast<float *>(w + l.prof);
    double *center = reinterpret_cast<double *>(w + l.center);
    double *norm32 = reinterpret_cast<double *>(w + l.norm32);
    double *norm16 = reinterpret_cast<double *>(w + l.norm16);
    float2 *C = reinterpret_cast<float2 *>(w + l.C);
    const size_t fstride = (size_t)2 * 2 * M;
    SW_NA(swk::launch_project(d_f, 1, p->L, p->L, nh, B, cs, proj, 0, status, st));
    SW_NA(swk::launch_project(d_g, 1, p->L, p->L, nh, B, cs, proj + (size_t)nh * B, 0,
                              status + 1, st));
    SW_NA(swk::launch_quantiles(proj, 2, n, B, M, 2.0f / (float)p->L, p->level_rule, 1, quant,
                                status, st));
    SW_NA(swk::launch_spectrum(quant, 2, n, M, plan, tw, spec32, fstride, 0, nullptr, 0,
                               nullptr, 0, 1, prof, center, norm32, norm16, st));
    SW_NA(swk::launch_corr_simt(spec32, fstride, spec32 + (size_t)2 * M, fstride, 1, 1, M, nh, C,
                                st));
    swk::DecideArgs a{};
    a.C = C;
    a.Nq = 1;
    a.Nt = 1;
    a.n = n;
    a.M = M;
    a.prof_q = prof;
    a.prof_t = prof + M;
    a.ctr_q = center;
    a.ctr_t = center + 2;
    a.norm_q = norm32;
    a.norm_t = norm32 + 1;
    a.st_q = status;
    a.st_t = status + 1;
    a.cs64 = cs64;
    a.translation = p->translation;
    a.grid_k = p->translation ? p->shift_grid : 0;
    a.grid_step = (double)p->shift_step_q * (2.0 / p->L) / 16.0;
    a.dev_err = err;
    a.out = d_best;
    a.curve = d_D;
    a.shifts = d_shift;
    SW_NA(swk::launch_decide(a, plan, tw, st));
#undef SW_NA
    return SW_OK;
}

// ---------------------------------------------------------------------------
// Autotuning (sw_autotune): per parameter set, the projection's CTA split,
// the FFT batch widths of the spectra and of the decision, and the FFT radix
// order are chosen by timing candidates on a batch of random images with the
// stage events of the profiler.  The stages are separate kernels, so each
// stage's choice is taken from its own time; the radix order is chosen on the time of the
// spectra and decision together (both run the FFT).
namespace {

struct TrialTimes {
    double proj = 1e30, spec = 1e30, dec = 1e30, corr = 1e30;
};

sw_status run_trial(sw_ctx *c, const sw_params *p, const Tune &tu, const float *dq, int Nq,
                    const float *dt, int Nt, sw_result *out, cudaStream_t st, TrialTimes &tt)
{
    c->trial = &tu;
    sw_status s = SW_OK;
    for (int r = 0; r < 4 && s == SW_OK; ++r) {
        s = align_batch_impl(c, p, dq, Nq, dt, Nt, 0, out, nullptr, nullptr, false, st);
        double ms[SW_STAGE_COUNT];
        int64_t cnt[SW_STAGE_COUNT];
        const sw_status sr = sw_profile_read(c, ms, cnt);  // waits for the events
        if (s == SW_OK) s = sr;
        if (s != SW_OK || r == 0) continue;  // the first run warms up
        tt.proj = std::min(tt.proj, ms[SW_STAGE_PROJECT]);
        tt.spec = std::min(tt.spec, ms[SW_STAGE_SPECTRUM]);
        tt.dec = std::min(tt.dec, ms[SW_STAGE_DECIDE]);
        tt.corr = std::min(tt.corr, ms[SW_STAGE_CORR]);
    }
    c->trial = nullptr;
    return s;
}

bool same_plan(const FftPlan &a, const FftPlan &b)
{
    if (a.nst != b.nst) return false;
    for (int i = 0; i < a.nst; ++i)
        if (a.radix[i] != b.radix[i]) return false;
    return true;
}

}  // namespace

extern "C" {

sw_status sw_autotune(sw_ctx *c, const sw_params *p, const char *cache_path)
{
    if (!c) return SW_ERR_INVALID_ARG;
    c->err.clear();
    sw_status s = check_params(c, p);
    if (s) return s;
    if ((s = set_device(c))) return s;
    cudaDeviceProp prop;
    SW_CUDA(c, cudaGetDeviceProperties(&prop, c->device));
    std::string dev = prop.name;
    for (char &ch : dev)
        if (ch == ' ' || ch == '\t') ch = '_';
    char kb[256];
    snprintf(kb, sizeof kb, "swtune2 %s L=%d n=%d M=%d B=%d prec=%d", dev.c_str(), p->L,
             p->n_theta, p->n_levels, bins_of(p), (int)p->gemm_precision);
    const std::string key = kb;
    const TuneKey tk = tune_key(p);
    if (p->metric == SW_METRIC_MSW2) return SW_OK;  // no spectra or FFT: defaults stand
    auto store = [&](const Tune &tu) {
        for (auto &e : c->tunes)
            if (e.first == tk) {
                e.second = tu;
                return;
            }
        c->tunes.push_back({tk, tu});
    };
    if (cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            if (line.size() <= key.size() || line.compare(0, key.size(), key) != 0 ||
                line[key.size()] != ' ')
                continue;
            Tune tu;
            std::istringstream is(line.substr(key.size()));
            if (is >> tu.want >> tu.spec >> tu.dec >> tu.plan >> tu.tile_s >> tu.tile_l &&
                tu.want >= 0 && tu.spec >= 0 && tu.dec >= 0 && tu.plan >= 0 &&
                tu.plan < kPlanVariants && tu.tile_s >= 0 && tu.tile_l >= 0) {
                store(tu);
                return SW_OK;
            }
        }
    }

    // trial batch: up to 1,024 queries x 64 templates of random images,
    // at most ~64 MB of images, within the workspace limit
    const int L = p->L, n = p->n_theta;
    const int Nt = 64;
    int Nq = (int)std::min<size_t>(1024, std::max<size_t>(64, (64u << 20) / (4u * L * L)));
    const int kind = lp_kind_of(p->gemm_precision);
    while (c->limit && Nq > 1 && batch_layout(p, Nq, Nt, kind, false).total > c->limit) Nq /= 2;
    const size_t nimg = (size_t)Nq + Nt;
    std::vector<float> h(nimg * L * L);
    std::mt19937 rng(20250317u);
    std::uniform_real_distribution<float> U(0.f, 1.f);
    for (float &x : h) x = U(rng);
    float *d_img = nullptr;
    sw_result *d_out = nullptr;
    cudaStream_t st = nullptr;
    auto cleanup = [&] {
        if (st) cudaStreamSynchronize(st);
        if (d_img) cudaFree(d_img);
        if (d_out) cudaFree(d_out);
        if (st) cudaStreamDestroy(st);
    };
    if (cudaMalloc(&d_img, sizeof(float) * h.size()) != cudaSuccess ||
        cudaMalloc(&d_out, sizeof(sw_result) * std::max<size_t>((size_t)Nq * Nt,
                                                                 (nimg > 256 ? nimg - 256 : 0) * 256)) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(c, SW_ERR_OOM, "autotune trial buffers");
    }
    if (cudaMemcpy(d_img, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cleanup();
        return fail(c, SW_ERR_CUDA, "autotune upload");
    }
    const float *dq = d_img, *dt = d_img + (size_t)Nq * L * L;

    // the profiler's state is the caller's: set it aside
    const bool was_prof = c->prof;
    std::vector<ProfRec> saved;
    saved.swap(c->recs);
    c->prof = true;

    const int wants[3] = {456, 304, 912};
    const int widths_small[3] = {16, 8, 4}, widths_large[3] = {8, 4, 4};
    const int *specs = n <= 512 ? widths_small : widths_large;
    // decision: 1 = the register form where it exists, else shared-memory widths
    const int dec_reg[3] = {1, 8, 16}, dec_small[3] = {8, 16, 4}, dec_large[3] = {4, 8, 4};
    const int *decs = swk::decide_reg_ok(n) ? dec_reg : (n <= 512 ? dec_small : dec_large);
    TrialTimes t1[3];
    for (int i = 0; i < 3 && s == SW_OK; ++i) {
        Tune tu;
        tu.want = wants[i];
        tu.spec = specs[i];
        tu.dec = decs[i];
        s = run_trial(c, p, tu, dq, Nq, dt, Nt, d_out, st, t1[i]);
    }
    Tune best;
    if (s == SW_OK) {
        int bw = 0, bs = 0, bd = 0;
        for (int i = 1; i < 3; ++i) {
            if (t1[i].proj < t1[bw].proj) bw = i;
            if (t1[i].spec < t1[bs].spec) bs = i;
            if (t1[i].dec < t1[bd].dec) bd = i;
        }
        best.want = wants[bw];
        best.spec = specs[bs];
        best.dec = decs[bd];
        double best_fft = t1[bs].spec + t1[bd].dec;
        FftPlan tried[kPlanVariants];
        fft_plan(n, tried[0], 0);
        for (int v = 1; v < kPlanVariants && s == SW_OK; ++v) {
            fft_plan(n, tried[v], v);
            bool dup = false;
            for (int u = 0; u < v; ++u) dup = dup || same_plan(tried[u], tried[v]);
            if (dup) continue;
            Tune tu = best;
            tu.plan = v;
            TrialTimes tv;
            s = run_trial(c, p, tu, dq, Nq, dt, Nt, d_out, st, tv);
            if (s == SW_OK && tv.spec + tv.dec < best_fft) {
                best_fft = tv.spec + tv.dec;
                best.plan = v;
            }
        }
        // the correlation's output tile on the tensor cores: 256 or 128
        // columns, timed on the trial batch (64 templates) for the small
        // class and on 256 templates (the rest of the trial images as
        // queries) for the large class
        if (kind != 0 && s == SW_OK) {
            double tc[2][2] = {{1e30, 1e30}, {1e30, 1e30}};
            const int tiles[2] = {256, 128};
            const int Nt_l = 256, Nq_l = (int)nimg - Nt_l;
            for (int cls = 0; cls < 2 && s == SW_OK; ++cls) {
                if (cls == 1 && (Nq_l < 64 || (c->limit && batch_layout(p, Nq_l, Nt_l, kind, false)
                                                               .total > c->limit)))
                    break;  // too few trial images, or beyond the workspace limit: default
                for (int v = 0; v < 2 && s == SW_OK; ++v) {
                    Tune tu = best;
                    tu.tile_s = tu.tile_l = tiles[v];
                    TrialTimes tv;
                    s = cls == 0 ? run_trial(c, p, tu, dq, Nq, dt, Nt, d_out, st, tv)
                                 : run_trial(c, p, tu, d_img, Nq_l,
                                             d_img + (size_t)Nq_l * L * L, Nt_l, d_out, st, tv);
                    tc[cls][v] = tv.corr;
                }
            }
            best.tile_s = tc[0][1] < tc[0][0] ? 128 : 256;
            best.tile_l = tc[1][1] < tc[1][0] ? 128 : 256;
        }
    }
    c->trial = nullptr;
    c->prof = was_prof;
    c->recs.swap(saved);
    cleanup();
    if (s != SW_OK) return s;
    store(best);
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (!f) return fail(c, SW_ERR_INVALID_ARG, "cannot append to %s", cache_path);
        f << key << ' ' << best.want << ' ' << best.spec << ' ' << best.dec << ' ' << best.plan
          << ' ' << best.tile_s << ' ' << best.tile_l << '\n';
    }
    return SW_OK;
}

sw_status sw_autotune_get(const sw_ctx *c, const sw_params *p, int *choice)
{
    if (!c || !choice) return SW_ERR_INVALID_ARG;
    if (check_params(nullptr, p) != SW_OK) return SW_ERR_INVALID_ARG;
    const TuneKey k = tune_key(p);
    Tune tu;
    for (const auto &e : c->tunes)
        if (e.first == k) tu = e.second;
    choice[0] = tu.want;
    choice[1] = tu.spec;
    choice[2] = tu.dec;
    choice[3] = tu.plan;
    choice[4] = tu.tile_s;
    choice[5] = tu.tile_l;
    return SW_OK;
}

}  // extern "C"
