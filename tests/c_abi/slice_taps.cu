// Host check of the Fourier-slice projector's target geometry (the index
// arithmetic that the kernels and the host grouping share, from
// sw_internal.cuh): for every angle count n the library accepts up to 1024
// and every grid size, each tap of each target lies inside the stored half
// grid, in the half its first tap names; for the L/2 images of the bank
// (slice_up_tap) also that the first tap and offsets put the target at
// y = -j e modulo the grid period, or at -y when folded.  Prints "ok" or the
// first failure; exits non-zero on a failure.  Host code only (no device is
// used).
#include <cmath>
#include <cstdio>
#include <vector>

#include "sw_internal.cuh"

using namespace swk;

static bool smooth(int n)
{
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

static int fail(const char *what, int n, int N, int k, int j)
{
    std::printf("FAIL %s n=%d N=%d k=%d j=%d\n", what, n, N, k, j);
    return 1;
}

// footprint of W x W taps from stored (row, col) in its half: inside the grid
static bool inside(int row, int col, bool left, int N)
{
    if (row < 0 || row + kSliceW > slice_rows(N)) return false;
    const int nl = slice_left(N), nr = slice_right(N);
    if (left) return col >= 0 && col + kSliceW <= nl;
    return col - (kSliceW - 1) >= nl && col < nl + nr;
}

int main()
{
    long targets = 0;
    for (int n = 4; n <= 1024; n += 2) {
        if (!smooth(n)) continue;
        std::vector<float> ex(n / 2), ey(n / 2);
        for (int k = 0; k < n / 2; ++k) {
            ex[k] = (float)std::cos(2.0 * M_PI * k / n);
            ey[k] = (float)std::sin(2.0 * M_PI * k / n);
        }
        // plain targets j <= N/2 on grids of N = B points (L <= 128 in shared
        // memory, 128 < L in global memory)
        for (int N = 32; N <= 384; N += 32) {
            for (int k = 0; k < n / 2; ++k)
                for (int j = 0; j <= N / 2; ++j, ++targets) {
                    int row, col;
                    bool left;
                    slice_tap_rc(j, ex[k], ey[k], N, &row, &col, &left);
                    if (!inside(row, col, left, N)) return fail("plain", n, N, k, j);
                    // the tile holding the footprint's top-left cell exists
                    const int cmin = left ? col : col - (kSliceW - 1);
                    if (row / kSliceTile >= slice_tiles_y(N) || cmin / kSliceTile >= slice_tiles_x(N))
                        return fail("tile", n, N, k, j);
                }
        }
        // images of side L/2 on their own grid of N = B/2 points, j <= N
        for (int N : {128, 160, 192}) {
            for (int k = 0; k < n / 2; ++k)
                for (int j = 0; j <= N; ++j, ++targets) {
                    int i1, i2, row, col;
                    float x1, x2;
                    bool conj, left;
                    slice_up_tap(j, ex[k], ey[k], N, &i1, &i2, &x1, &x2, &conj);
                    slice_up_rc(j, ex[k], ey[k], N, &row, &col, &left);
                    if (!inside(row, col, left, N)) return fail("upsampled", n, N, k, j);
                    if (!(std::fabs(x1) <= 0.50001f && std::fabs(x2) <= 0.50001f))
                        return fail("offset", n, N, k, j);
                    double y1 = -(double)j * ex[k], y2 = -(double)j * ey[k];
                    if (conj) {
                        y1 = -y1;
                        y2 = -y2;
                    }
                    const double d1 = std::remainder(i1 + kSliceW / 2 + x1 - y1, (double)N);
                    const double d2 = std::remainder(i2 + kSliceW / 2 + x2 - y2, (double)N);
                    if (std::fabs(d1) > 1e-3 || std::fabs(d2) > 1e-3)
                        return fail("position", n, N, k, j);
                }
        }
    }
    std::printf("ok %ld\n", targets);
    return 0;
}
