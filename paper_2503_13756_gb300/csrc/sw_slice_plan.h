// sw_slice_plan.h -- host-side target tables of the Fourier-slice projector
// (Sec. 2.3 "Computation": the slice samples of the type-2 NUFFT).
//
// The interpolation kernels take their targets from a table of half-warp
// groups of 16 entries: the 16 lanes of a group read distinct shared-memory
// banks at every tap, and, for L <= 128 and for half-size images, ray-adjacent
// samples (j, j + 1) travel as one pair entry over their union footprint.
// These functions build the tables on the host from the same FP32 geometry
// the kernels use (slice_tap_rc, slice_up_rc), beside the host-side numbers
// of the spreading kernel (its Fourier transform, its tap-weight
// polynomials).  Host code only, so that tests can build and check them
// without a device.
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <vector>

#include "sw_internal.cuh"

namespace swk {

// The angles theta_k = 2 pi k / n (k < n): c[k] = cos, s[k] = sin in FP64,
// each reduced to the first octant so that the symmetries of the angle set
// (theta -> pi/2 - theta, quarter turns) hold exactly in the tables.
inline void angle_table(int n, std::vector<double> &c, std::vector<double> &s)
{
    c.assign(n, 0.0);
    s.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        // reduce 8k/n to the first octant
        long long num = 8LL * k;  // angle = (num / n) * (pi / 4)
        int oct = (int)(num / n);
        long long rem = num - (long long)oct * n;  // angle = (oct + rem/n) pi/4
        double cc, ss;
        auto base = [&](long long r, bool from_top, double &co, double &si) {
            // t in [0, pi/4]
            double t = (double)r / n * (M_PI / 4.0);
            if (from_top) t = M_PI / 4.0 - t;
            co = std::cos(t);
            si = std::sin(t);
        };
        double co, si;
        switch (oct & 7) {
        case 0: base(rem, false, co, si); cc = co; ss = si; break;
        case 1: base(rem, true, co, si); cc = si; ss = co; break;
        case 2: base(rem, false, co, si); cc = -si; ss = co; break;
        case 3: base(rem, true, co, si); cc = -co; ss = si; break;
        case 4: base(rem, false, co, si); cc = -co; ss = -si; break;
        case 5: base(rem, true, co, si); cc = -si; ss = -co; break;
        case 6: base(rem, false, co, si); cc = si; ss = -co; break;
        default: base(rem, true, co, si); cc = co; ss = -si; break;
        }
        c[k] = cc;
        s[k] = ss;
    }
}

// The spreading kernel psi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)) on
// |u| <= W/2 (exponential of semicircle), its Fourier transform for the
// deapodisation and its tap weights as polynomials in the target's offset.
// Psi(k) = integral over |u| <= W/2 of psi(u) cos(2 pi k u / N) du.  With
// u = (W/2) sin(phi) the square root becomes cos(phi) and the integrand
// W/2 exp(beta (cos phi - 1)) cos(pi k W sin(phi) / N) cos(phi) is smooth on
// [-pi/2, pi/2]; composite Simpson with 2048 panels in FP64.
inline double slice_kernel_ft(int k, int N, int W, double beta)
{
    const int m = 2048;
    const double a = 0.5 * M_PI, hstep = a / m;  // integrate 2 x [0, pi/2]
    double acc = 0.0;
    for (int i = 0; i <= m; ++i) {
        const double ph = i * hstep;
        const double f = std::exp(beta * (std::cos(ph) - 1.0)) *
                         std::cos(M_PI * k * W * std::sin(ph) / N) * std::cos(ph);
        acc += f * (i == 0 || i == m ? 1.0 : (i & 1) ? 4.0 : 2.0);
    }
    return 2.0 * (0.5 * W) * acc * hstep / 3.0;
}

// Tap weights as polynomials in the target's offset x in (-1/2, 1/2]: for
// tap a, psi(x + W/2 - a) interpolated at the W Chebyshev points of
// [-1/2, 1/2] (degree W - 1 = kSliceDeg), monomial coefficients by Gaussian
// elimination in FP64.  Error below 1e-8 for the kernel shapes used here.
// The nodes are symmetric and psi is even, so the interpolant of tap W-1-a
// is that of tap a at -x: taps 0..W/2 are fitted, the others mirrored
// (c[W-1-a][d] = (-1)^d c[a][d]) and the middle tap's odd terms are zero,
// which is the form slice_tap_weights evaluates.
inline void slice_fit_weights(double beta, SliceCoef &out)
{
    constexpr int W = kSliceW, D = kSliceDeg + 1;
    static_assert(D == W, "one interpolation node per coefficient");
    for (int a = 0; a <= W / 2; ++a) {
        double A[D][D + 1];
        for (int k = 0; k < D; ++k) {
            const double x = 0.5 * std::cos(M_PI * (k + 0.5) / D);
            const double u = x + W / 2 - a, z = 2.0 * u / W;
            const double arg = 1.0 - z * z;
            double xp = 1.0;
            for (int d = 0; d < D; ++d, xp *= x) A[k][d] = xp;
            A[k][D] = arg >= 0.0 ? std::exp(beta * (std::sqrt(arg) - 1.0)) : 0.0;
        }
        for (int col = 0; col < D; ++col) {  // elimination with partial pivoting
            int piv = col;
            for (int r = col + 1; r < D; ++r)
                if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
            for (int q = 0; q <= D; ++q) std::swap(A[col][q], A[piv][q]);
            for (int r = 0; r < D; ++r) {
                if (r == col) continue;
                const double f = A[r][col] / A[col][col];
                for (int q = col; q <= D; ++q) A[r][q] -= f * A[col][q];
            }
        }
        for (int d = 0; d < D; ++d) out.c[a][d] = (float)(A[d][D] / A[d][d]);
    }
    for (int d = 1; d < D; d += 2) out.c[W / 2][d] = 0.f;
    for (int a = W / 2 + 1; a < W; ++a)
        for (int d = 0; d < D; ++d) out.c[a][d] = (d & 1) ? -out.c[W - 1 - a][d] : out.c[W - 1 - a][d];
}

// Half-warp groups from classes of targets.  cls[half][residue] maps a first
// tap address to its targets (residue = address mod 16, per half of the grid:
// taps at increasing or decreasing addresses).  Group g takes the g-th class
// of every residue, so the 16 lanes of a group read distinct banks at every
// tap; targets with the same first address (near the origin the angles meet)
// read the same words, which the hardware broadcasts, so such a class may
// fill several lanes.  Appends whole groups of 16 to tab (idle lanes hold
// `idle`).
template <typename Cls, typename Tab, typename E>
void slice_half_warp_groups(Cls &cls, Tab &tab, E idle)
{
    using T = typename Tab::value_type;
    for (auto &half : cls) {
        std::vector<std::vector<T>> q[16];  // per residue, largest class first
        for (int r = 0; r < 16; ++r) {
            for (auto &kv : half[r]) q[r].push_back(kv.second);
            std::stable_sort(q[r].begin(), q[r].end(),
                             [](const std::vector<T> &a, const std::vector<T> &b) {
                                 return a.size() > b.size();
                             });
            for (auto &v : q[r]) std::reverse(v.begin(), v.end());  // pop from the back
        }
        size_t head[16] = {};
        for (;;) {
            int busy = 0;
            for (int r = 0; r < 16; ++r) busy += head[r] < q[r].size();
            if (!busy) break;
            T lanes[16];
            int used = 0;
            for (int r = 0; r < 16; ++r) {
                if (head[r] >= q[r].size()) continue;
                --busy;  // residues after r that still wait keep one lane each
                std::vector<T> &v = q[r][head[r]];
                int take = std::min<int>((int)v.size(), 16 - used - busy);
                take = std::max(take, 1);
                for (int i = 0; i < take; ++i) {
                    lanes[used++] = v.back();
                    v.pop_back();
                }
                if (v.empty()) ++head[r];
            }
            for (int i = 0; i < 16; ++i) tab.push_back(i < used ? lanes[i] : (T)idle);
        }
    }
}

// Segments per ray of the pairing choice (see slice_pair_groups).
constexpr int kSlicePairSegs = 4;

// Target table of the grid-in-shared-memory kernels (L <= 128, and images of
// side L/2 on their own grid): for each batch of `batch` angles (of nh), the
// half-warp groups of entries kk 256 + j (kk the angle's row in the batch,
// j < njt the frequency index), tab holding the entries and off[b] the first
// group of batch b (off gains one element per batch).
//
// Ray-adjacent targets (j, j + 1) of one half whose first taps are at most a
// row and a column apart form a pair entry (kSlicePairBit), bucketed by the
// first address of their union footprint and by the offsets of the two
// footprints in it: nine patterns, each a compile-time path of the kernel.
// Each pattern's groups are padded to an even count, so both half-warps of a
// warp take one path; pairs come before the single targets.  Which samples
// pair is a free choice: each ray is cut into kSlicePairSegs segments, and a
// segment either pairs from its first sample or leaves it alone and pairs
// from the next.  The choice moves pairs between classes and bank residues,
// and a class needs as many half-warp groups as its fullest residue holds
// entries, so a local search picks, ray by ray, the segment phases that lower
// the sum over classes of the fullest residue.
//
// tap_rc(k, j, &row, &col, &left): the stored row, column and half of the
// first tap of target (k, j) on the N-point grid, as the kernel forms them.
template <typename TapRC>
void slice_pair_groups(int batch, int nh, int N, int njt, TapRC tap_rc, std::vector<uint16_t> &tab,
                       std::vector<int> &off)
{
    struct PairEnt {
        int cls;       // pattern * 2 + half for a pair; 18 + half for a single target
        int base;      // first stored address of the footprint (union for a pair)
        uint16_t ent;  // table entry
    };
    const int S = slice_stride(N);
    // the entries of ray k (batch row kk) with segment phases `mask`
    auto ray_entries = [&](int k, int kk, int mask, std::vector<PairEnt> &out) {
        out.clear();
        int seg = 0;
        for (int j = 0; j < njt;) {
            while (seg + 1 < kSlicePairSegs && j >= (seg + 1) * njt / kSlicePairSegs) ++seg;
            int rA, cA, rB, cB;
            bool lA, lB;
            tap_rc(k, j, &rA, &cA, &lA);
            const uint16_t ent = (uint16_t)(kk * 256 + j);
            const bool alone = ((mask >> seg) & 1) && j == seg * njt / kSlicePairSegs;
            if (!alone && j + 1 < njt) {
                tap_rc(k, j + 1, &rB, &cB, &lB);
                if (lA == lB && std::abs(rA - rB) <= 1 && std::abs(cA - cB) <= 1) {
                    const int r0 = std::min(rA, rB);
                    const int c0 = lA ? std::min(cA, cB) : std::max(cA, cB);
                    const int pr = rA > rB ? 1 : (rB > rA ? 2 : 0);
                    const int pc = cA != c0 ? 1 : (cB != c0 ? 2 : 0);
                    out.push_back({(pr * 3 + pc) * 2 + (lA ? 0 : 1), r0 * S + c0,
                                   (uint16_t)(ent | kSlicePairBit)});
                    j += 2;
                    continue;
                }
            }
            out.push_back({18 + (lA ? 0 : 1), rA * S + cA, ent});
            j += 1;
        }
    };
    for (int k0 = 0; k0 < nh; k0 += batch) {
        const int k1 = std::min(nh, k0 + batch), nk = k1 - k0;
        constexpr int NOPT = 1 << kSlicePairSegs;
        std::vector<std::array<std::vector<PairEnt>, NOPT>> opt(nk);
        for (int kk = 0; kk < nk; ++kk)
            for (int o = 0; o < NOPT; ++o) ray_entries(k0 + kk, kk, o, opt[kk][o]);
        int cnt[20][16] = {};
        auto add = [&](const std::vector<PairEnt> &v, int d) {
            for (const PairEnt &e : v) cnt[e.cls][e.base & 15] += d;
        };
        auto cost = [&]() {
            int c = 0;
            for (int q = 0; q < 20; ++q) c += *std::max_element(cnt[q], cnt[q] + 16);
            return c;
        };
        std::vector<int> mask(nk, 0);
        for (int kk = 0; kk < nk; ++kk) add(opt[kk][0], 1);
        int best = cost();
        for (int pass = 0; pass < 6; ++pass) {
            bool moved = false;
            for (int kk = 0; kk < nk; ++kk)
                for (int o = 0; o < NOPT; ++o) {
                    if (o == mask[kk]) continue;
                    add(opt[kk][mask[kk]], -1);
                    add(opt[kk][o], 1);
                    const int c = cost();
                    if (c < best) {
                        best = c;
                        mask[kk] = o;
                        moved = true;
                    } else {
                        add(opt[kk][o], -1);
                        add(opt[kk][mask[kk]], 1);
                    }
                }
            if (!moved) break;
        }
        std::map<int, std::vector<uint16_t>> cls[2][16], pcls[9][2][16];
        for (int kk = 0; kk < nk; ++kk)
            for (const PairEnt &e : opt[kk][mask[kk]]) {
                if (e.cls < 18) pcls[e.cls / 2][e.cls % 2][e.base & 15][e.base].push_back(e.ent);
                else cls[e.cls - 18][e.base & 15][e.base].push_back(e.ent);
            }
        const size_t g_start = tab.size() / 16;
        for (auto &pc : pcls) {
            slice_half_warp_groups(pc, tab, (uint16_t)0xFFFF);
            if ((tab.size() / 16 - g_start) & 1) tab.insert(tab.end(), 16, (uint16_t)0xFFFF);
        }
        slice_half_warp_groups(cls, tab, (uint16_t)0xFFFF);
        off.push_back((int)(tab.size() / 16));
    }
}

// Target table of the tiled kernels (128 < L, grid in global memory): per
// tile t of slice_tiles_y(N) x slice_tiles_x(N), the half-warp groups of the
// targets whose footprint starts in it (entries k << 16 | j, k < nh, j < nj),
// tab holding the entries and off[t] the first group of tile t (off gains one
// element per tile).  The bank of an entry is that of its first tap in the
// tile's shared-memory copy (rows kSliceTileRS apart).  co, si: the angle
// table (angle_table).
inline void slice_tile_groups(int nh, int N, int nj, const std::vector<double> &co,
                              const std::vector<double> &si, std::vector<uint32_t> &tab,
                              std::vector<int> &off)
{
    const int TY = slice_tiles_y(N), TX = slice_tiles_x(N);
    std::vector<std::array<std::array<std::map<int, std::vector<uint32_t>>, 16>, 2>> cls(
        (size_t)TY * TX);
    for (int k = 0; k < nh; ++k)
        for (int j = 0; j < nj; ++j) {
            int row, col;
            bool left;
            slice_tap_rc(j, (float)co[k], (float)si[k], N, &row, &col, &left);
            const int cmin = left ? col : col - (kSliceW - 1);
            const int ty = row / kSliceTile, tx = cmin / kSliceTile;
            const int local = (row - ty * kSliceTile) * kSliceTileRS + (col - tx * kSliceTile);
            cls[(size_t)ty * TX + tx][left ? 0 : 1][local & 15][local].push_back(
                ((uint32_t)k << 16) | (uint32_t)j);
        }
    for (auto &tc : cls) {
        slice_half_warp_groups(tc, tab, 0xFFFFFFFFu);
        off.push_back((int)(tab.size() / 16));
    }
}

}  // namespace swk
