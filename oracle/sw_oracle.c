/*
 * sw_oracle.c -- plain FP64 CPU oracle for rigid alignment in sliced
 * 2-Wasserstein distance (arXiv 2503.13756).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant generator with the CUDA library: every quantity
 * here is computed from its definition, in double precision, with plain
 * loops and no blocking, fusion or reordering.
 *
 * Conventions (readings of the paper, each restated where it is used):
 *   image    F[r][c], r = row, c = column, L x L cells on [-1,1]^2, pitch
 *            h = 2/L, cell centre x = -1 + (c+1/2)h, y = -1 + (r+1/2)h
 *            (App. A.1.2 "Pixel Grid and Discrete Image").
 *   angles   theta_k = 2*pi*k/n, k = 0..n-1 (App. A.1.2, "Discretization
 *            Parameters"); direction e_k = (cos theta_k, sin theta_k).
 *   bins     B bins of width h with centres s_b = (b - (B-1)/2) h; CDF
 *            nodes e_j = (j - B/2) h, j = 0..B.
 *   levels   z_p = (p + 1/2)/M (level_rule 0) or z_p = p/M (level_rule 1,
 *            the left Riemann points of Theorem E3 in App. A).
 *   projector 0 = pixel-driven linear splat (orc_project), 1 = band-limited
 *            Fourier-slice projection (orc_project_slice, Sec. 2.3 and
 *            Theorem proj_nufft).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t best_l;   /* argmin over the rotation grid, lowest index on ties */
    int32_t status;   /* 0 ok, 1 image f unusable, 2 image g unusable        */
    double angle;     /* 2*pi*best_l/n                                        */
    double shift[2];  /* optimal translation at best_l (0 if translation=0)   */
    double d2;        /* squared sliced-W2 distance at best_l                 */
} orc_result;

/* Direction e_k = (cos theta_k, sin theta_k), theta_k = 2 pi k / n
 * (App. A.1.2).  At quarter turns (4k divisible by n) the direction is the
 * exact axis vector: cos(2 pi k / n) evaluated at the rounded pi would put
 * 1e-16 of mass into bins that the exact direction leaves empty, and the
 * z = 0 quantile (the left edge of the first bin with mass) depends on
 * exactly that. */
static void orc_direction(int k, int n, double *c, double *s)
{
    k %= n;
    if (k < 0) k += n;
    if ((4 * k) % n == 0) {
        static const double cq[4] = {1.0, 0.0, -1.0, 0.0};
        static const double sq[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cq[4 * k / n];
        *s = sq[4 * k / n];
        return;
    }
    const double th = 2.0 * ORC_PI * k / n;
    *c = cos(th);
    *s = sin(th);
}

/* Number of bins that holds every pixel-centre projection of an L x L
 * image with at least half a bin to spare on each side:
 * B = 2*ceil((L-1)/sqrt(2)) + 2.  The paper samples L points on [-1,1]
 * (Sec. 2.3 "Computation"); its images live on the unit disk, ours may fill
 * the square, so the projection range is widened to the square's diagonal.
 * Empty bins never change a quantile. */
int orc_default_bins(int L)
{
    return 2 * (int)ceil((double)(L - 1) / sqrt(2.0)) + 2;
}

/* Image preparation, Sec. 5.4 (noisy images are split g = g+ + g- and the
 * positive part is renormalised) and App. A.1.2 (cell averages normalised
 * to sum 1).  Writes out = max(img,0)/mass and returns mass = sum max(img,0);
 * returns 0 if the mass is not positive or any pixel is not finite. */
double orc_prepare(const double *img, int L, double *out)
{
    double mass = 0.0;
    for (int i = 0; i < L * L; ++i) {
        if (!isfinite(img[i])) return 0.0;
        double v = img[i] > 0.0 ? img[i] : 0.0;
        out[i] = v;
        mass += v;
    }
    if (!(mass > 0.0)) return 0.0;
    for (int i = 0; i < L * L; ++i) out[i] /= mass;
    return mass;
}

/* Radon projection (Eq. radon_transform, Sec. 2.1; the appendix form
 * P_theta g(s) = integral of g(s theta + t theta_perp) dt), discretised as a
 * pixel-driven linear splat.  The paper computes projections with a NUFFT
 * and is silent on a direct discretisation; this reading sends each cell's
 * mass to the two bins around s = <(x,y), e_k>, split linearly, which keeps
 * the mass and the first moment of every projection exact.
 * U is [n][B], row k = projection at theta_k. */
void orc_project(const double *F, int L, int n, int B, double *U)
{
    const double h = 2.0 / L;
    memset(U, 0, sizeof(double) * (size_t)n * B);
    for (int k = 0; k < n; ++k) {
        double ct, st;
        orc_direction(k, n, &ct, &st);
        double *Uk = U + (size_t)k * B;
        for (int r = 0; r < L; ++r) {
            const double y = -1.0 + (r + 0.5) * h;
            for (int c = 0; c < L; ++c) {
                const double x = -1.0 + (c + 0.5) * h;
                const double f = F[r * L + c];
                if (f == 0.0) continue;
                const double s = x * ct + y * st;
                const double u = s / h + 0.5 * (B - 1);
                const double fl = floor(u);
                const int b0 = (int)fl;
                const double t = u - fl;
                Uk[b0] += f * (1.0 - t);
                if (t > 0.0) Uk[b0 + 1] += f * t;
            }
        }
    }
}

/* sinc(x) = sin(x)/x, sinc(0) = 1. */
static double orc_sinc(double x)
{
    return x == 0.0 ? 1.0 : sin(x) / x;
}

/* Band-limited Radon projection through the Fourier slice theorem (Sec. 2.1,
 * Eq. 1d_ift; Sec. 2.3 "Computation"; Theorem proj_nufft in App. A).  The
 * image is the piecewise-constant density f_L that puts the mass F[r][c]
 * uniformly on its cell, so its 2-D transform (convention
 * H^(xi) = integral H(x) e^{-i xi.x} dx) is
 *   f_L^(xi) = sinc(xi_1 h/2) sinc(xi_2 h/2) sum_{r,c} F[r][c] e^{-i (xi_1 x_c + xi_2 y_r)}.
 * The projection P_theta f_L is supported on the diagonal of the square, so
 * it is expanded on the period P = B h (the bin grid, B >= sqrt(2) L), with
 * the slice samples at omega_j = 2 pi j / P, j = -B/2 .. B/2-1: the
 * coefficients c_j = f_L^(omega_j e_k) / P (the slice theorem), and
 *   g~(s) = Re sum_j c_j e^{i omega_j s},
 * the trigonometric polynomial of the theorem (whose frequencies k pi,
 * |k| <= L/2 on the period 2, reach the same Nyquist limit pi/h; the real
 * part drops the imaginary contribution of the unpaired j = -B/2 term).
 * Reading: the discrete projection is the bin mass U[k][b] = h g~(s_b) at
 * the bin centres s_b (the piecewise-constant identification of Sec. 2.3).
 * The rows are signed (g~ rings where f_L has edges); sum_b U[k][b] = sum F
 * exactly, since sum_b e^{i omega_j s_b} = 0 for j != 0.
 * Every sum is taken from its definition: f_L^ directly over all cells for
 * every j (negative j included), g~ directly over all j; every angle k of
 * the n is computed (no mirror or symmetry shortcut).  O(n B L^2). */
void orc_project_slice(const double *F, int L, int n, int B, double *U)
{
    const double h = 2.0 / L, P = B * h;
    double *er = (double *)malloc(sizeof(double) * L), *ei = (double *)malloc(sizeof(double) * L);
    double *cr = (double *)malloc(sizeof(double) * B), *ci = (double *)malloc(sizeof(double) * B);
    for (int k = 0; k < n; ++k) {
        double ct, st;
        orc_direction(k, n, &ct, &st);
        for (int jj = 0; jj < B; ++jj) {
            const int j = jj - B / 2;
            const double om = 2.0 * ORC_PI * j / P;
            const double x1 = om * ct, x2 = om * st;  /* xi = omega_j e_k */
            for (int c = 0; c < L; ++c) {             /* e^{-i xi_1 x_c} */
                const double x = -1.0 + (c + 0.5) * h;
                er[c] = cos(x1 * x);
                ei[c] = -sin(x1 * x);
            }
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < L; ++r) {
                const double y = -1.0 + (r + 0.5) * h;
                double rr = 0.0, ri = 0.0;            /* sum_c F[r][c] e^{-i xi_1 x_c} */
                for (int c = 0; c < L; ++c) {
                    rr += F[r * L + c] * er[c];
                    ri += F[r * L + c] * ei[c];
                }
                const double yr = cos(x2 * y), yi = -sin(x2 * y);  /* e^{-i xi_2 y_r} */
                sr += rr * yr - ri * yi;
                si += rr * yi + ri * yr;
            }
            const double w = orc_sinc(0.5 * x1 * h) * orc_sinc(0.5 * x2 * h) / P;
            cr[jj] = w * sr;
            ci[jj] = w * si;
        }
        double *Uk = U + (size_t)k * B;
        for (int b = 0; b < B; ++b) {
            const double s = (b - 0.5 * (B - 1)) * h;
            double g = 0.0;
            for (int jj = 0; jj < B; ++jj) {
                const double ph = 2.0 * ORC_PI * (jj - B / 2) / P * s;
                g += cr[jj] * cos(ph) - ci[jj] * sin(ph);  /* Re(c_j e^{i omega_j s}) */
            }
            Uk[b] = h * g;
        }
    }
    free(er);
    free(ei);
    free(cr);
    free(ci);
}

/* Quantile function of one histogram (Sec. 2.3 "Computation": CDF by
 * cumulative sum, ICDF by linear interpolation; Eq. inv_cdf with the
 * appendix's ">=" reading, App. A.1.1).  The histogram U[0..B) has a
 * piecewise-constant density on bins [e_j, e_{j+1}], so its CDF is the
 * piecewise-linear function through (e_j, F_j), F_0 = 0, F_j = sum_{b<j} U_b.
 * For tau = z_p * F_B the quantile is Q = e_{j-1} + h (tau - F_{j-1}) / U_{j-1}
 * with j = min{ j >= 1 : F_j >= tau }; for tau = 0 (level p = 0 under
 * level_rule 1) the set {t : F(t) >= 0} is the whole domain, whose infimum
 * is its left end e_0 (App. A.1.1 integrates the CDF from the domain's left
 * end).  This value is the same for every image, so it cancels in the
 * distance; the left edge of the first bin with mass would instead depend on
 * whether a vanishing weight rounds to zero.
 * The levels are walked in increasing order against the cumulative mass
 * (a merge of the two sorted sequences).  Returns 0 if the histogram has no
 * positive mass. */
static int orc_quantiles_1d(const double *U, int B, double h, int M,
                            int level_rule, double *Fbuf, double *Q)
{
    Fbuf[0] = 0.0;
    for (int j = 1; j <= B; ++j) Fbuf[j] = Fbuf[j - 1] + U[j - 1];
    const double total = Fbuf[B];
    if (!(total > 0.0)) return 0;
    int j = 1;
    for (int p = 0; p < M; ++p) {
        const double z = level_rule == 0 ? (p + 0.5) / M : (double)p / M;
        const double tau = z * total;
        if (tau == 0.0) {
            /* inf{t : F(t) >= 0} is the left end of the domain, e_0 */
            Q[p] = -0.5 * B * h;
            continue;
        }
        while (j < B && Fbuf[j] < tau) ++j;
        const double mass = Fbuf[j] - Fbuf[j - 1];
        double frac = mass > 0.0 ? (tau - Fbuf[j - 1]) / mass : 0.0;
        if (frac < 0.0) frac = 0.0;
        if (frac > 1.0) frac = 1.0;
        Q[p] = (j - 1 - 0.5 * B) * h + h * frac;
    }
    return 1;
}

/* Quantiles of every projection: Q is [n][M], row k = U_I column k of the
 * paper (Sec. 2.3).  Returns 0 if some projection has no mass. */
int orc_quantiles(const double *U, int n, int B, double h, int M,
                  int level_rule, double *Q)
{
    double *Fbuf = (double *)malloc(sizeof(double) * (B + 1));
    int ok = 1;
    for (int k = 0; k < n; ++k)
        ok &= orc_quantiles_1d(U + (size_t)k * B, B, h, M, level_rule, Fbuf,
                               Q + (size_t)k * M);
    free(Fbuf);
    return ok;
}

/* Squared 1-D W2 distance between two histograms on the same bin grid,
 * computed exactly (App. A.1.1: W2^2 = integral over z in [0,1] of
 * (Q_u(z) - Q_v(z))^2).  Both quantile functions are piecewise linear in z
 * with breakpoints at the normalised cumulative masses; on each interval of
 * the merged breakpoints the integrand is the square of a linear function
 * and is integrated in closed form.  Used only to check the sampled-level
 * sums against the bound of Theorem E3 (App. A). */
double orc_w2_hist_exact(const double *Ua, const double *Ub, int B, double h)
{
    double ta = 0.0, tb = 0.0;
    for (int b = 0; b < B; ++b) { ta += Ua[b]; tb += Ub[b]; }
    if (!(ta > 0.0) || !(tb > 0.0)) return NAN;
    int ia = 0, ib = 0;
    while (ia < B && Ua[ia] <= 0.0) ++ia;
    while (ib < B && Ub[ib] <= 0.0) ++ib;
    double Fa = 0.0, Fb = 0.0;   /* cumulative mass before bin ia / ib  */
    double z = 0.0, acc = 0.0;
    while (ia < B && ib < B && z < 1.0) {
        const double za1 = (Fa + Ua[ia]) / ta;  /* end of bin ia in z     */
        const double zb1 = (Fb + Ub[ib]) / tb;
        double z1 = za1 < zb1 ? za1 : zb1;
        if (z1 > 1.0) z1 = 1.0;
        const double dz = z1 - z;
        if (dz > 0.0) {
            /* Q_a(z) = e_ia + h (z*ta - Fa)/Ua[ia], same for b. */
            const double sa = h * ta / Ua[ia], sb = h * tb / Ub[ib];
            const double qa0 = (ia - 0.5 * B) * h + sa * (z - Fa / ta);
            const double qb0 = (ib - 0.5 * B) * h + sb * (z - Fb / tb);
            const double d0 = qa0 - qb0, slope = sa - sb;
            acc += dz * (d0 * d0 + d0 * slope * dz + slope * slope * dz * dz / 3.0);
        }
        z = z1;
        if (za1 <= z1) {
            Fa += Ua[ia];
            ++ia;
            while (ia < B && Ua[ia] <= 0.0) ++ia;
        }
        if (zb1 <= z1) {
            Fb += Ub[ib];
            ++ib;
            while (ib < B && Ub[ib] <= 0.0) ++ib;
        }
    }
    return acc;
}

/* Translation centring (closed-form optimal translation; derived from the
 * shift lemma in the proof of the translation theorem, App. B, where
 * P_theta(T_s f)(t) = P_theta f(t - <s, theta>)): a translation by s adds
 * <s, e_k> to every quantile of column k.  With ubar_k = mean_p Q[k][p],
 * a = (2/n) sum_k ubar_k e_k and Qc[k][p] = Q[k][p] - <a, e_k>.
 * For n >= 3, sum_k e_k e_k^T = (n/2) I, which makes a the least-squares
 * optimum. */
void orc_center(const double *Q, int n, int M, double *a, double *Qc)
{
    double ax = 0.0, ay = 0.0;
    for (int k = 0; k < n; ++k) {
        double ub = 0.0;
        for (int p = 0; p < M; ++p) ub += Q[(size_t)k * M + p];
        ub /= M;
        double ct, st;
        orc_direction(k, n, &ct, &st);
        ax += ub * ct;
        ay += ub * st;
    }
    ax *= 2.0 / n;
    ay *= 2.0 / n;
    a[0] = ax;
    a[1] = ay;
    if (Qc) {
        for (int k = 0; k < n; ++k) {
            double ct, st;
            orc_direction(k, n, &ct, &st);
            const double off = ax * ct + ay * st;
            for (int p = 0; p < M; ++p)
                Qc[(size_t)k * M + p] = Q[(size_t)k * M + p] - off;
        }
    }
}

/* Squared distance over the rotation grid, computed directly from its
 * definition (Eq. discrete_sw2 and Eq. discrete_rot_sw2, Sec. 2.3):
 *   D[l] = 1/(n M) * sum_k sum_p (Qf[k][p] - Qg[(k-l) mod n][p])^2,
 * which compares f with R_{alpha_l} g, alpha_l = 2 pi l / n, because
 * P_theta(R_alpha g) = P_{theta - alpha} g.  O(n^2 M), no FFT. */
void orc_rotation_curve(const double *Qf, const double *Qg, int n, int M,
                        double *D)
{
    const double inv = 1.0 / ((double)n * M);
    for (int l = 0; l < n; ++l) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) {
            const int kg = ((k - l) % n + n) % n;
            const double *u = Qf + (size_t)k * M;
            const double *v = Qg + (size_t)kg * M;
            for (int p = 0; p < M; ++p) {
                const double d = u[p] - v[p];
                acc += d * d;
            }
        }
        D[l] = acc * inv;
    }
}

/* Per-image transform: prepare, project (splat, or Fourier slice clipped at
 * zero), quantiles and (if translation)
 * centring.  Q receives the quantiles used in the distance (centred when
 * translation != 0), a the centring vector.  Returns 0 for an unusable
 * image. */
typedef struct {
    int L, n, M, B, level_rule, translation, projector;
} orc_cfg;

/* Projection rows of a prepared image for the configured projector.  With
 * the Fourier-slice projector, clip != 0 keeps max(U, 0): reading, the paper
 * normalises the projections to probability measures (Sec. 2.3), which
 * needs nonnegative bins, and the band-limited rows ring slightly below
 * zero; the ramp-filtered path splits signed rows itself (clip = 0). */
static void orc_project_cfg(const orc_cfg *cfg, const double *F, double *U, int clip)
{
    if (!cfg->projector) {
        orc_project(F, cfg->L, cfg->n, cfg->B, U);
        return;
    }
    orc_project_slice(F, cfg->L, cfg->n, cfg->B, U);
    if (clip)
        for (size_t i = 0; i < (size_t)cfg->n * cfg->B; ++i)
            if (U[i] < 0.0) U[i] = 0.0;
}

static int orc_transform(const orc_cfg *cfg, const double *img, double *Q,
                         double *a)
{
    const int L = cfg->L, n = cfg->n, M = cfg->M, B = cfg->B;
    double *F = (double *)malloc(sizeof(double) * (size_t)L * L);
    double *U = (double *)malloc(sizeof(double) * (size_t)n * B);
    double *Qraw = (double *)malloc(sizeof(double) * (size_t)n * M);
    int ok = orc_prepare(img, L, F) > 0.0;
    if (ok) {
        orc_project_cfg(cfg, F, U, 1);
        ok = orc_quantiles(U, n, B, 2.0 / L, M, cfg->level_rule, Qraw);
    }
    if (ok) {
        orc_center(Qraw, n, M, a, cfg->translation ? Q : NULL);
        if (!cfg->translation) memcpy(Q, Qraw, sizeof(double) * (size_t)n * M);
    }
    free(F);
    free(U);
    free(Qraw);
    return ok;
}

/* Decision (Eq. optimal_rotation and Eq. discrete_rot_sw2): l* = argmin D,
 * lowest index on exact ties; shift s*(l) = a_f - R_{alpha_l} a_g when the
 * translation is optimised, 0 otherwise. */
static void orc_decide(const double *D, int n, const double *af,
                       const double *ag, int translation, double *shifts,
                       orc_result *res)
{
    int best = 0;
    for (int l = 1; l < n; ++l)
        if (D[l] < D[best]) best = l;
    for (int l = 0; l < n; ++l) {
        if (!shifts) break;
        double ca, sa;
        orc_direction(l, n, &ca, &sa);
        const double rx = ca * ag[0] - sa * ag[1];
        const double ry = sa * ag[0] + ca * ag[1];
        shifts[2 * l] = translation ? af[0] - rx : 0.0;
        shifts[2 * l + 1] = translation ? af[1] - ry : 0.0;
    }
    double cb, sb;
    orc_direction(best, n, &cb, &sb);
    res->best_l = best;
    res->status = 0;
    res->angle = 2.0 * ORC_PI * best / n;
    if (translation) {
        res->shift[0] = af[0] - (cb * ag[0] - sb * ag[1]);
        res->shift[1] = af[1] - (sb * ag[0] + cb * ag[1]);
    } else {
        res->shift[0] = res->shift[1] = 0.0;
    }
    res->d2 = D[best];
}

static void orc_bad(orc_result *res, int status)
{
    res->best_l = -1;
    res->status = status;
    res->angle = NAN;
    res->shift[0] = res->shift[1] = NAN;
    res->d2 = NAN;
}

/* One pair, full curve: f is the reference, g is rotated (and translated
 * when translation != 0) onto f.  D (may be NULL) receives the n distances,
 * shifts (may be NULL) the n optimal translations. */
void orc_align_pair(const double *f, const double *g, int L, int n, int M,
                    int B, int level_rule, int translation, int projector, double *D,
                    double *shifts, orc_result *res)
{
    orc_cfg cfg = {L, n, M, B, level_rule, translation, projector};
    double *Qf = (double *)malloc(sizeof(double) * (size_t)n * M);
    double *Qg = (double *)malloc(sizeof(double) * (size_t)n * M);
    double *Dl = (double *)malloc(sizeof(double) * (size_t)n);
    double af[2] = {0, 0}, ag[2] = {0, 0};
    const int okf = orc_transform(&cfg, f, Qf, af);
    const int okg = orc_transform(&cfg, g, Qg, ag);
    if (!okf || !okg) {
        orc_bad(res, okf ? 2 : 1);
        if (D) for (int l = 0; l < n; ++l) D[l] = NAN;
        if (shifts) for (int l = 0; l < 2 * n; ++l) shifts[l] = NAN;
    } else {
        orc_rotation_curve(Qf, Qg, n, M, Dl);
        orc_decide(Dl, n, af, ag, translation, shifts, res);
        if (D) memcpy(D, Dl, sizeof(double) * (size_t)n);
    }
    free(Qf);
    free(Qg);
    free(Dl);
}

/* ---- many pairs, parallel over independent work items ------------------ */

typedef struct {
    const orc_cfg *cfg;
    const double *imgs;    /* [nimg][L][L] */
    double *Q;             /* [nimg][n][M] */
    double *A;             /* [nimg][2]    */
    int *ok;               /* [nimg]       */
    int nimg;
    /* pair stage */
    int Nq, Nt;
    orc_result *out;       /* [Nq][Nt]     */
    int next;              /* shared work counter (guarded by mu) */
    pthread_mutex_t mu;
} orc_job;

static int orc_take(orc_job *job, int limit)
{
    pthread_mutex_lock(&job->mu);
    const int i = job->next < limit ? job->next++ : -1;
    pthread_mutex_unlock(&job->mu);
    return i;
}

static void *orc_image_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    const orc_cfg *c = job->cfg;
    for (int i; (i = orc_take(job, job->nimg)) >= 0;)
        job->ok[i] = orc_transform(c, job->imgs + (size_t)i * c->L * c->L,
                                   job->Q + (size_t)i * c->n * c->M,
                                   job->A + 2 * (size_t)i);
    return NULL;
}

static void *orc_pair_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    const orc_cfg *c = job->cfg;
    double *D = (double *)malloc(sizeof(double) * c->n);
    for (int w; (w = orc_take(job, job->Nq * job->Nt)) >= 0;) {
        const int i = w / job->Nt, j = job->Nq + w % job->Nt;
        orc_result *res = job->out + w;
        if (!job->ok[w / job->Nt]) { orc_bad(res, 1); continue; }
        if (!job->ok[j]) { orc_bad(res, 2); continue; }
        orc_rotation_curve(job->Q + (size_t)i * c->n * c->M,
                           job->Q + (size_t)j * c->n * c->M, c->n, c->M, D);
        orc_decide(D, c->n, job->A + 2 * (size_t)i, job->A + 2 * (size_t)j,
                   c->translation, NULL, res);
    }
    free(D);
    return NULL;
}

static void orc_run(orc_job *job, void *(*fn)(void *), int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    job->next = 0;
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, fn, job);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
}

/* The per-image transform of every image, in parallel: Q [nimg][n][M]
 * receives the uncentred quantiles, A [nimg][2] the centring vectors and
 * ok [nimg] 0 for an unusable image (the same steps as orc_align_pair:
 * prepare, project, quantiles, centre).  Returns 0 on allocation failure. */
int orc_transform_images(const double *imgs, int nimg, int L, int n, int M, int B,
                         int level_rule, int projector, int nthreads, double *Q, double *A,
                         int *ok)
{
    orc_cfg cfg = {L, n, M, B, level_rule, 0, projector};
    orc_job job;
    memset(&job, 0, sizeof(job));
    job.cfg = &cfg;
    job.imgs = imgs;
    job.Q = Q;
    job.A = A;
    job.ok = ok;
    job.nimg = nimg;
    pthread_mutex_init(&job.mu, NULL);
    orc_run(&job, orc_image_worker, nthreads);
    pthread_mutex_destroy(&job.mu);
    return 1;
}

/* All pairs (query i, template j): out[i*Nt + j] aligns template j onto
 * query i (query = reference f, template = g).  Queries are [Nq][L][L],
 * templates [Nt][L][L], both double.  Returns 0 on allocation failure. */
int orc_align_all_pairs(const double *queries, int Nq, const double *templates,
                        int Nt, int L, int n, int M, int B, int level_rule,
                        int translation, int projector, int nthreads, orc_result *out)
{
    orc_cfg cfg = {L, n, M, B, level_rule, translation, projector};
    const int nimg = Nq + Nt;
    double *imgs = (double *)malloc(sizeof(double) * (size_t)nimg * L * L);
    double *Q = (double *)malloc(sizeof(double) * (size_t)nimg * n * M);
    double *A = (double *)malloc(sizeof(double) * 2 * (size_t)nimg);
    int *ok = (int *)malloc(sizeof(int) * (size_t)nimg);
    if (!imgs || !Q || !A || !ok) {
        free(imgs); free(Q); free(A); free(ok);
        return 0;
    }
    memcpy(imgs, queries, sizeof(double) * (size_t)Nq * L * L);
    memcpy(imgs + (size_t)Nq * L * L, templates, sizeof(double) * (size_t)Nt * L * L);
    orc_job job;
    memset(&job, 0, sizeof(job));
    job.cfg = &cfg;
    job.imgs = imgs;
    job.Q = Q;
    job.A = A;
    job.ok = ok;
    job.nimg = nimg;
    job.Nq = Nq;
    job.Nt = Nt;
    job.out = out;
    pthread_mutex_init(&job.mu, NULL);
    orc_run(&job, orc_image_worker, nthreads);
    orc_run(&job, orc_pair_worker, nthreads);
    pthread_mutex_destroy(&job.mu);
    free(imgs); free(Q); free(A); free(ok);
    return 1;
}

/* ======================================================================
 * Ramp-filtered sliced W2 (RFSW).  Sec. 2.1 "High-pass filter (optional)"
 * (Eq. 1d_ift_ramp, Eq. line_decomp) and Eq. signed_sliced_wasserstein;
 * the appendix on ramp-filtered distances fixes the negative part as the
 * absolute value max(-mu~, 0) and normalises each part to unit mass.
 * Discrete form (Eq. discrete_ssw2, Eq. discrete_rot_signed_sw2):
 *   D(l) = 1/(n M) (|U+ - T_l V+|^2 + |U- - T_l V-|^2)
 * over the quantiles of the two parts.
 *
 * Reading of the discrete filter (the paper filters NUFFT central slices,
 * which we do not form): each projection row U[0..B) is filtered circularly
 * on its own bin grid,
 *   Ut[b] = (1/B) sum_j |xi_j| Uh[j] e^{+2 pi i j b / B},
 *   Uh[j] = sum_b U[b] e^{-2 pi i j b / B},  |xi_j| = min(j, B - j),
 * the frequency in cycles per B bins (a constant factor would cancel in the
 * normalisation of each part).  Plain DFT sums, O(B^2) per row.
 * ====================================================================== */

/* Ut = ramp-filtered rows of U ([nrows][B] each). */
void orc_ramp_filter(const double *U, int nrows, int B, double *Ut)
{
    double *cs = (double *)malloc(sizeof(double) * B);
    double *sn = (double *)malloc(sizeof(double) * B);
    double *re = (double *)malloc(sizeof(double) * B);
    double *im = (double *)malloc(sizeof(double) * B);
    for (int m = 0; m < B; ++m) {
        cs[m] = cos(2.0 * ORC_PI * m / B);
        sn[m] = sin(2.0 * ORC_PI * m / B);
    }
    for (int r = 0; r < nrows; ++r) {
        const double *u = U + (size_t)r * B;
        for (int j = 0; j < B; ++j) {
            double a = 0.0, c = 0.0;
            for (int b = 0; b < B; ++b) {
                const int m = (int)(((long long)j * b) % B);
                a += u[b] * cs[m];
                c -= u[b] * sn[m];
            }
            re[j] = a;
            im[j] = c;
        }
        double *o = Ut + (size_t)r * B;
        for (int b = 0; b < B; ++b) {
            double acc = 0.0;
            for (int j = 0; j < B; ++j) {
                const int m = (int)(((long long)j * b) % B);
                const double xi = j < B - j ? j : B - j;
                acc += xi * (re[j] * cs[m] - im[j] * sn[m]);  /* Re(Uh e^{+i..}) */
            }
            o[b] = acc / B;
        }
    }
    free(cs);
    free(sn);
    free(re);
    free(im);
}

/* Positive part and absolute negative part of the filtered rows. */
void orc_rfsw_parts(const double *U, int nrows, int B, double *Up, double *Um)
{
    double *Ut = (double *)malloc(sizeof(double) * (size_t)nrows * B);
    orc_ramp_filter(U, nrows, B, Ut);
    for (size_t i = 0; i < (size_t)nrows * B; ++i) {
        Up[i] = Ut[i] > 0.0 ? Ut[i] : 0.0;
        Um[i] = Ut[i] < 0.0 ? -Ut[i] : 0.0;
    }
    free(Ut);
}

/* Per image: prepare, project, filter, split, and the quantiles of both
 * parts (uncentred): Q = [2][n][M] (part 0 positive, part 1 negative).  A
 * part with no mass at some angle (only for an image without mass) makes
 * the image unusable.  Returns 0 then. */
static int orc_rfsw_transform(const orc_cfg *cfg, const double *img, double *Q)
{
    const int L = cfg->L, n = cfg->n, M = cfg->M, B = cfg->B;
    double *F = (double *)malloc(sizeof(double) * (size_t)L * L);
    double *U = (double *)malloc(sizeof(double) * (size_t)n * B);
    double *Up = (double *)malloc(sizeof(double) * (size_t)n * B);
    double *Um = (double *)malloc(sizeof(double) * (size_t)n * B);
    int ok = orc_prepare(img, L, F) > 0.0;
    if (ok) {
        orc_project_cfg(cfg, F, U, 0);
        orc_rfsw_parts(U, n, B, Up, Um);
        ok = orc_quantiles(Up, n, B, 2.0 / L, M, cfg->level_rule, Q);
        ok &= orc_quantiles(Um, n, B, 2.0 / L, M, cfg->level_rule, Q + (size_t)n * M);
    }
    free(F);
    free(U);
    free(Up);
    free(Um);
    return ok;
}

/* RFSW squared distance over the rotation grid from its definition.  With
 * w+-_pk = Qf+-[k][p] - Qg+-[(k-l) mod n][p] (parts + and -):
 *   translation 0:  D(l) = 1/(nM) sum_parts sum_k sum_p w^2;
 *   translation 1:  one translation s of the whole image adds <s, e_k> to
 *     every quantile of column k of both parts, so
 *       D(l) = min_s 1/(nM) sum_parts sum_k sum_p (w_pk - <s, e_k>)^2.
 *     Setting the gradient to zero with sum_k e_k e_k^T = (n/2) I gives
 *     s*(l) = (c+ + c-)/2, c = (2/n) sum_k (mean_p w_pk) e_k per part; D(l)
 *     is then evaluated at s*(l) by the same triple sum.
 * shifts[l] (may be NULL) = s*(l), or 0 without translation. */
void orc_rfsw_curve(const double *Qf, const double *Qg, int n, int M, int translation,
                    double *D, double *shifts)
{
    const double inv = 1.0 / ((double)n * M);
    for (int l = 0; l < n; ++l) {
        double s[2] = {0.0, 0.0};
        if (translation) {
            for (int part = 0; part < 2; ++part) {
                const double *qf = Qf + (size_t)part * n * M, *qg = Qg + (size_t)part * n * M;
                for (int k = 0; k < n; ++k) {
                    const int kg = ((k - l) % n + n) % n;
                    double wbar = 0.0;
                    for (int p = 0; p < M; ++p) wbar += qf[(size_t)k * M + p] - qg[(size_t)kg * M + p];
                    wbar /= M;
                    double ct, st;
                    orc_direction(k, n, &ct, &st);
                    s[0] += wbar * ct;
                    s[1] += wbar * st;
                }
            }
            /* (c+ + c-)/2 with c = (2/n) sum_k wbar_k e_k */
            s[0] *= 1.0 / n;
            s[1] *= 1.0 / n;
        }
        double acc = 0.0;
        for (int part = 0; part < 2; ++part) {
            const double *qf = Qf + (size_t)part * n * M, *qg = Qg + (size_t)part * n * M;
            for (int k = 0; k < n; ++k) {
                const int kg = ((k - l) % n + n) % n;
                double ct, st;
                orc_direction(k, n, &ct, &st);
                const double off = s[0] * ct + s[1] * st;
                for (int p = 0; p < M; ++p) {
                    const double d = qf[(size_t)k * M + p] - qg[(size_t)kg * M + p] - off;
                    acc += d * d;
                }
            }
        }
        D[l] = acc * inv;
        if (shifts) {
            shifts[2 * l] = s[0];
            shifts[2 * l + 1] = s[1];
        }
    }
}

static void orc_rfsw_decide(const double *D, const double *S, int n, orc_result *res)
{
    int best = 0;
    for (int l = 1; l < n; ++l)
        if (D[l] < D[best]) best = l;
    res->best_l = best;
    res->status = 0;
    res->angle = 2.0 * ORC_PI * best / n;
    res->shift[0] = S[2 * best];
    res->shift[1] = S[2 * best + 1];
    res->d2 = D[best];
}

/* One pair under RFSW; arguments as orc_align_pair (B must be the bin count
 * the filter runs on). */
void orc_align_pair_rfsw(const double *f, const double *g, int L, int n, int M, int B,
                         int level_rule, int translation, int projector, double *D,
                         double *shifts, orc_result *res)
{
    orc_cfg cfg = {L, n, M, B, level_rule, translation, projector};
    double *Qf = (double *)malloc(sizeof(double) * 2 * (size_t)n * M);
    double *Qg = (double *)malloc(sizeof(double) * 2 * (size_t)n * M);
    double *Dl = (double *)malloc(sizeof(double) * (size_t)n);
    double *Sl = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    const int okf = orc_rfsw_transform(&cfg, f, Qf);
    const int okg = orc_rfsw_transform(&cfg, g, Qg);
    if (!okf || !okg) {
        orc_bad(res, okf ? 2 : 1);
        if (D) for (int l = 0; l < n; ++l) D[l] = NAN;
        if (shifts) for (int l = 0; l < 2 * n; ++l) shifts[l] = NAN;
    } else {
        orc_rfsw_curve(Qf, Qg, n, M, translation, Dl, Sl);
        orc_rfsw_decide(Dl, Sl, n, res);
        if (D) memcpy(D, Dl, sizeof(double) * (size_t)n);
        if (shifts) memcpy(shifts, Sl, sizeof(double) * 2 * (size_t)n);
    }
    free(Qf);
    free(Qg);
    free(Dl);
    free(Sl);
}

static void *orc_rfsw_image_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    const orc_cfg *c = job->cfg;
    for (int i; (i = orc_take(job, job->nimg)) >= 0;)
        job->ok[i] = orc_rfsw_transform(c, job->imgs + (size_t)i * c->L * c->L,
                                        job->Q + 2 * (size_t)i * c->n * c->M);
    return NULL;
}

static void *orc_rfsw_pair_worker(void *arg)
{
    orc_job *job = (orc_job *)arg;
    const orc_cfg *c = job->cfg;
    double *D = (double *)malloc(sizeof(double) * c->n);
    double *S = (double *)malloc(sizeof(double) * 2 * c->n);
    for (int w; (w = orc_take(job, job->Nq * job->Nt)) >= 0;) {
        const int i = w / job->Nt, j = job->Nq + w % job->Nt;
        orc_result *res = job->out + w;
        if (!job->ok[i]) { orc_bad(res, 1); continue; }
        if (!job->ok[j]) { orc_bad(res, 2); continue; }
        orc_rfsw_curve(job->Q + 2 * (size_t)i * c->n * c->M, job->Q + 2 * (size_t)j * c->n * c->M,
                       c->n, c->M, c->translation, D, S);
        orc_rfsw_decide(D, S, c->n, res);
    }
    free(D);
    free(S);
    return NULL;
}

/* All pairs under RFSW; arguments as orc_align_all_pairs. */
int orc_align_all_pairs_rfsw(const double *queries, int Nq, const double *templates,
                             int Nt, int L, int n, int M, int B, int level_rule,
                             int translation, int projector, int nthreads, orc_result *out)
{
    orc_cfg cfg = {L, n, M, B, level_rule, translation, projector};
    const int nimg = Nq + Nt;
    double *imgs = (double *)malloc(sizeof(double) * (size_t)nimg * L * L);
    double *Q = (double *)malloc(sizeof(double) * 2 * (size_t)nimg * n * M);
    int *ok = (int *)malloc(sizeof(int) * (size_t)nimg);
    if (!imgs || !Q || !ok) {
        free(imgs); free(Q); free(ok);
        return 0;
    }
    memcpy(imgs, queries, sizeof(double) * (size_t)Nq * L * L);
    memcpy(imgs + (size_t)Nq * L * L, templates, sizeof(double) * (size_t)Nt * L * L);
    orc_job job;
    memset(&job, 0, sizeof(job));
    job.cfg = &cfg;
    job.imgs = imgs;
    job.Q = Q;
    job.ok = ok;
    job.nimg = nimg;
    job.Nq = Nq;
    job.Nt = Nt;
    job.out = out;
    pthread_mutex_init(&job.mu, NULL);
    orc_run(&job, orc_rfsw_image_worker, nthreads);
    orc_run(&job, orc_rfsw_pair_worker, nthreads);
    pthread_mutex_destroy(&job.mu);
    free(imgs); free(Q); free(ok);
    return 1;
}

/* ======================================================================
 * Explicit translation sampling (Sec. 1 lists exhaustive search over a
 * grid of translations; Sec. 7 names explicit translation sampling as an
 * extension).  The translation of g is restricted to the grid
 *   s = (i, j) * step,  -K <= i, j <= K,
 * and for every rotation l the distance is the minimum over the grid of
 *   J(l, s) = 1/(n M) sum_parts sum_k sum_p (Qf[k][p] - Qg[(k-l) mod n][p] - <s, e_k>)^2
 * evaluated directly for every grid point (brute force, no closed form).
 * Qf, Qg: [parts][n][M] uncentred quantiles.  shifts[l] = the minimising
 * grid point (lowest (i, j) in row-major order on exact ties). */
void orc_grid_curve(const double *Qf, const double *Qg, int parts, int n, int M, int K,
                    double step, double *D, double *shifts)
{
    const double inv = 1.0 / ((double)n * M);
    for (int l = 0; l < n; ++l) {
        double best = INFINITY, bx = 0.0, by = 0.0;
        for (int i = -K; i <= K; ++i) {
            for (int j = -K; j <= K; ++j) {
                const double sx = i * step, sy = j * step;
                double acc = 0.0;
                for (int part = 0; part < parts; ++part) {
                    const double *qf = Qf + (size_t)part * n * M, *qg = Qg + (size_t)part * n * M;
                    for (int k = 0; k < n; ++k) {
                        const int kg = ((k - l) % n + n) % n;
                        double ct, st;
                        orc_direction(k, n, &ct, &st);
                        const double off = sx * ct + sy * st;
                        for (int p = 0; p < M; ++p) {
                            const double d = qf[(size_t)k * M + p] - qg[(size_t)kg * M + p] - off;
                            acc += d * d;
                        }
                    }
                }
                acc *= inv;
                if (acc < best) {
                    best = acc;
                    bx = sx;
                    by = sy;
                }
            }
        }
        D[l] = best;
        if (shifts) {
            shifts[2 * l] = bx;
            shifts[2 * l + 1] = by;
        }
    }
}

/* One pair with the translation restricted to the grid; metric 0 = sliced
 * W2, 1 = ramp-filtered (B must be the filter's bin count). */
void orc_align_pair_grid(const double *f, const double *g, int L, int n, int M, int B,
                         int level_rule, int metric, int K, double step, int projector,
                         double *D, double *shifts, orc_result *res)
{
    orc_cfg cfg = {L, n, M, B, level_rule, 0, projector};
    const int parts = metric ? 2 : 1;
    double *Qf = (double *)malloc(sizeof(double) * parts * (size_t)n * M);
    double *Qg = (double *)malloc(sizeof(double) * parts * (size_t)n * M);
    double *Dl = (double *)malloc(sizeof(double) * (size_t)n);
    double *Sl = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double af[2], ag[2];
    int okf, okg;
    if (metric) {
        okf = orc_rfsw_transform(&cfg, f, Qf);
        okg = orc_rfsw_transform(&cfg, g, Qg);
    } else {
        okf = orc_transform(&cfg, f, Qf, af);  /* translation 0: uncentred */
        okg = orc_transform(&cfg, g, Qg, ag);
    }
    if (!okf || !okg) {
        orc_bad(res, okf ? 2 : 1);
        if (D) for (int l = 0; l < n; ++l) D[l] = NAN;
        if (shifts) for (int l = 0; l < 2 * n; ++l) shifts[l] = NAN;
    } else {
        orc_grid_curve(Qf, Qg, parts, n, M, K, step, Dl, Sl);
        orc_rfsw_decide(Dl, Sl, n, res);
        if (D) memcpy(D, Dl, sizeof(double) * (size_t)n);
        if (shifts) memcpy(shifts, Sl, sizeof(double) * 2 * (size_t)n);
    }
    free(Qf);
    free(Qg);
    free(Dl);
    free(Sl);
}

/* ======================================================================
 * Max-sliced W2 over rotations (App. "alignment extended", Eq.
 * max_sliced_wasserstein): the squared distance at rotation l is the
 * largest, over the angles, of the squared 1-D W2 between the columns,
 *   D(l) = max_k (1/M) sum_p (Qf[k][p] - Qg[(k-l) mod n][p])^2 ,
 * read with the level average 1/M (the per-angle W2^2 of the sampled
 * quantiles, the normalisation of Eq. discrete_sw2 without the angle
 * average).  No FFT applies; direct O(n^2 M).  With translation the
 * quantiles are centred (the sliced-W2 optimal translation, s*(l) =
 * a_f - R a_g, applied before the maximum). */
void orc_msw_curve(const double *Qf, const double *Qg, int n, int M, double *D)
{
    for (int l = 0; l < n; ++l) {
        double mx = 0.0;
        for (int k = 0; k < n; ++k) {
            const int kg = ((k - l) % n + n) % n;
            double acc = 0.0;
            for (int p = 0; p < M; ++p) {
                const double d = Qf[(size_t)k * M + p] - Qg[(size_t)kg * M + p];
                acc += d * d;
            }
            acc /= M;
            if (acc > mx) mx = acc;
        }
        D[l] = mx;
    }
}

void orc_align_pair_msw(const double *f, const double *g, int L, int n, int M, int B,
                        int level_rule, int translation, int projector, double *D,
                        double *shifts, orc_result *res)
{
    orc_cfg cfg = {L, n, M, B, level_rule, translation, projector};
    double *Qf = (double *)malloc(sizeof(double) * (size_t)n * M);
    double *Qg = (double *)malloc(sizeof(double) * (size_t)n * M);
    double *Dl = (double *)malloc(sizeof(double) * (size_t)n);
    double af[2] = {0, 0}, ag[2] = {0, 0};
    const int okf = orc_transform(&cfg, f, Qf, af);
    const int okg = orc_transform(&cfg, g, Qg, ag);
    if (!okf || !okg) {
        orc_bad(res, okf ? 2 : 1);
        if (D) for (int l = 0; l < n; ++l) D[l] = NAN;
        if (shifts) for (int l = 0; l < 2 * n; ++l) shifts[l] = NAN;
    } else {
        orc_msw_curve(Qf, Qg, n, M, Dl);
        orc_decide(Dl, n, af, ag, translation, shifts, res);
        if (D) memcpy(D, Dl, sizeof(double) * (size_t)n);
    }
    free(Qf);
    free(Qg);
    free(Dl);
}
