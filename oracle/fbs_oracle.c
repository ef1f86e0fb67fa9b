/*
 * Plain FP64 CPU oracle for fast bilateral stereo (FBS).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark have an obviously correct reference to compare
 * the CUDA kernels with.  It shares no code with the CUDA path.
 *
 * Every function is a literal, single-threaded evaluation of the paper's
 * definitions, in the order the paper states them, with no blocking, fusion
 * or reordering:
 *   - matching cost:   Eq. (1)-(3), normalised cross-correlation over a
 *                      (2*varrho+1)^2 block with varrho = 1 (Sec. II-A);
 *   - aggregation:     Eq. (6)-(8), bilateral weights
 *                      w = exp{-((x-u)^2+(y-v)^2)/gamma_d^2} *
 *                          exp{-(i(x,y)-i(u,v))^2/gamma_r^2}   (Sec. II-B);
 *   - optimisation:    winner-take-all over d (Sec. II-C, Sec. III);
 *   - refinement:      parabola fit, Eq. (10) (Sec. II-D).
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes):
 *   R1  the stored cost is C = 1 - c and the winner is its smallest value,
 *       which is the paper's highest correlation;  Eq. (10) is unchanged by
 *       c -> 1 - c.
 *   R2  an optional truncated-absolute-difference cost (TAD) is offered:
 *       C = min(mean_c |I_l - I_r|, tau).  It is not in the paper.
 *   R3  for colour images the intensity used by the NCC is the channel sum
 *       (NCC is scale invariant, so this equals the channel mean), and the
 *       range weight uses the squared Euclidean colour distance.
 *   R4  Gaussians are exp(-r^2/gamma^2) exactly as printed (no factor 2),
 *       gamma_d = sigma_s, gamma_r = sigma_r.
 *   R5  the left image guides the weights of the left cost volume.
 *   R6  NCC blocks are clamped to the image (replicate); the aggregation
 *       window is clipped to the image; when u - d < 0 there is no match and
 *       the cost is the maximum (2 for NCC, tau for TAD).
 *   R7  a block with zero variance makes Eq. (1) undefined; c := 0 there.
 *   R8  Eq. (10) is applied to the aggregated costs; no offset is applied at
 *       d = 0, d = D-1, or when the denominator is not positive.
 *   R9  ties in the winner-take-all go to the smallest d.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCC_RHO 1 /* varrho = 1, so n = 9 (Sec. II-A) */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Intensity of pixel (x, y): the channel sum (reading R3). */
static double intensity(const uint8_t *img, int W, int C, int x, int y)
{
    double s = 0.0;
    for (int c = 0; c < C; ++c) s += (double)img[((size_t)y * W + x) * C + c];
    return s;
}

/*
 * Eq. (1)-(3): correlation c(u, v, d) between the left block centred at
 * (u, v) and the right block centred at (u - d, v).  Both blocks are clamped
 * to their image (reading R6).  Returns 0 for a block of zero variance (R7).
 */
double oracle_ncc(const uint8_t *L, const uint8_t *R, int H, int W, int C, int u, int v, int d)
{
    const int n = (2 * NCC_RHO + 1) * (2 * NCC_RHO + 1);
    double il[9], ir[9];
    int k = 0;
    for (int y = v - NCC_RHO; y <= v + NCC_RHO; ++y) {
        for (int x = u - NCC_RHO; x <= u + NCC_RHO; ++x) {
            int yc = clampi(y, 0, H - 1);
            il[k] = intensity(L, W, C, clampi(x, 0, W - 1), yc);
            ir[k] = intensity(R, W, C, clampi(x - d, 0, W - 1), yc);
            ++k;
        }
    }
    /* zero variance <=> every value of the block is equal */
    int flat_l = 1, flat_r = 1;
    for (k = 1; k < n; ++k) {
        if (il[k] != il[0]) flat_l = 0;
        if (ir[k] != ir[0]) flat_r = 0;
    }
    if (flat_l || flat_r) return 0.0;
    double mu_l = 0.0, mu_r = 0.0;
    for (k = 0; k < n; ++k) { mu_l += il[k]; mu_r += ir[k]; }
    mu_l /= n;
    mu_r /= n;
    double sq_l = 0.0, sq_r = 0.0, dot = 0.0;
    for (k = 0; k < n; ++k) {
        sq_l += il[k] * il[k];
        sq_r += ir[k] * ir[k];
        dot += il[k] * ir[k];
    }
    double sigma_l = sqrt(sq_l / n - mu_l * mu_l);   /* Eq. (2) */
    double sigma_r = sqrt(sq_r / n - mu_r * mu_r);   /* Eq. (3) */
    return (dot - n * mu_l * mu_r) / (n * sigma_l * sigma_r);  /* Eq. (1) */
}

/* Matching cost C(u, v, d).  mode 0: NCC, C = 1 - c (R1); mode 1: TAD (R2). */
double oracle_cost(const uint8_t *L, const uint8_t *R, int H, int W, int C, int u, int v, int d,
                   int mode, double tau)
{
    if (u - d < 0) return mode == 0 ? 2.0 : tau;   /* no match in the image (R6) */
    if (mode == 0) return 1.0 - oracle_ncc(L, R, H, W, C, u, v, d);
    double s = 0.0;
    for (int c = 0; c < C; ++c) {
        double a = (double)L[((size_t)v * W + u) * C + c];
        double b = (double)R[((size_t)v * W + (u - d)) * C + c];
        s += fabs(a - b);
    }
    s /= C;
    return s < tau ? s : tau;
}

/* Full cost volume, layout [H][W][D]. */
void oracle_cost_volume(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D,
                        int mode, double tau, double *cost)
{
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u)
            for (int d = 0; d < D; ++d)
                cost[((size_t)v * W + u) * D + d] = oracle_cost(L, R, H, W, C, u, v, d, mode, tau);
}

/* Eq. (7) times Eq. (8): bilateral weight of neighbour (x, y) for centre (u, v). */
double oracle_weight(const uint8_t *guide, int W, int C, int u, int v, int x, int y,
                     double gamma_d, double gamma_r)
{
    double dist2 = (double)(x - u) * (x - u) + (double)(y - v) * (y - v);
    double omega_d = exp(-dist2 / (gamma_d * gamma_d));
    double col2 = 0.0;
    for (int c = 0; c < C; ++c) {
        double diff = (double)guide[((size_t)y * W + x) * C + c] - (double)guide[((size_t)v * W + u) * C + c];
        col2 += diff * diff;
    }
    double omega_r = exp(-col2 / (gamma_r * gamma_r));
    return omega_d * omega_r;
}

/*
 * Eq. (6) for output rows [y0, y1): agg[(v - y0)][u][d] = sum_q w C(q, d) / sum_q w,
 * where q runs over the (2 rho + 1)^2 window clipped to the image.  ``cost``
 * holds rows [c0, c0 + crows) of the [H][W][D] volume; every row the window
 * reaches must be inside that range.
 */
void oracle_aggregate_rows(const double *cost, int c0, const uint8_t *guide, int H, int W, int C,
                           int D, int rho, double gamma_d, double gamma_r, int y0, int y1,
                           double *agg)
{
    double *num = (double *)malloc(sizeof(double) * (size_t)D);
    for (int v = y0; v < y1; ++v) {
        for (int u = 0; u < W; ++u) {
            for (int d = 0; d < D; ++d) num[d] = 0.0;
            double den = 0.0;
            for (int y = v - rho; y <= v + rho; ++y) {
                if (y < 0 || y >= H) continue;
                for (int x = u - rho; x <= u + rho; ++x) {
                    if (x < 0 || x >= W) continue;
                    double w = oracle_weight(guide, W, C, u, v, x, y, gamma_d, gamma_r);
                    den += w;
                    const double *cq = cost + ((size_t)(y - c0) * W + x) * D;
                    for (int d = 0; d < D; ++d) num[d] += w * cq[d];
                }
            }
            double *out = agg + ((size_t)(v - y0) * W + u) * D;
            for (int d = 0; d < D; ++d) out[d] = num[d] / den;
        }
    }
    free(num);
}

void oracle_aggregate(const double *cost, const uint8_t *guide, int H, int W, int C, int D, int rho,
                      double gamma_d, double gamma_r, double *agg)
{
    oracle_aggregate_rows(cost, 0, guide, H, W, C, D, rho, gamma_d, gamma_r, 0, H, agg);
}

/*
 * Winner-take-all (smallest d on ties, R9) and the parabola refinement of
 * Eq. (10) on one pixel's aggregated costs a[0..D-1].
 */
void oracle_wta_subpixel_pixel(const double *a, int D, int32_t *d_int, double *d_sub)
{
    int best = 0;
    for (int d = 1; d < D; ++d)
        if (a[d] < a[best]) best = d;
    double ds = (double)best;
    if (best > 0 && best < D - 1) {
        double cm = a[best - 1], c0 = a[best], cp = a[best + 1];
        double den = 2.0 * cm + 2.0 * cp - 4.0 * c0;
        if (den > 0.0) ds = best + (cm - cp) / den;
    }
    *d_int = best;
    *d_sub = ds;
}

void oracle_wta_subpixel(const double *agg, int npix, int D, int32_t *d_int, double *d_sub)
{
    for (int p = 0; p < npix; ++p)
        oracle_wta_subpixel_pixel(agg + (size_t)p * D, D, d_int + p, d_sub + p);
}

/*
 * The whole path for output rows [y0, y1): cost rows [y0 - rho, y1 + rho)
 * clipped to the image, aggregation, WTA and subpixel.  agg_out (nullable)
 * receives (y1 - y0) * W * D aggregated costs.
 */
int oracle_fbs_rows(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D, int rho,
                    double gamma_d, double gamma_r, double tau, int mode, int y0, int y1,
                    double *agg_out, int32_t *d_int, double *d_sub)
{
    int c0 = y0 - rho < 0 ? 0 : y0 - rho;
    int c1 = y1 + rho > H ? H : y1 + rho;
    size_t crow = (size_t)W * D;
    double *cost = (double *)malloc(sizeof(double) * crow * (size_t)(c1 - c0));
    double *agg = agg_out ? agg_out : (double *)malloc(sizeof(double) * crow * (size_t)(y1 - y0));
    if (!cost || !agg) { free(cost); if (!agg_out) free(agg); return -1; }
    for (int v = c0; v < c1; ++v)
        for (int u = 0; u < W; ++u)
            for (int d = 0; d < D; ++d)
                cost[((size_t)(v - c0) * W + u) * D + d] = oracle_cost(L, R, H, W, C, u, v, d, mode, tau);
    oracle_aggregate_rows(cost, c0, L, H, W, C, D, rho, gamma_d, gamma_r, y0, y1, agg);
    oracle_wta_subpixel(agg, (y1 - y0) * W, D, d_int, d_sub);
    free(cost);
    if (!agg_out) free(agg);
    return 0;
}

/*
 * The whole path at isolated pixels (xs[i], ys[i]): every cost the window
 * needs is evaluated on the spot, so a few pixels of a large frame can be
 * checked without building its volume.  agg_out (nullable) is n * D.
 */
int oracle_fbs_points(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D, int rho,
                      double gamma_d, double gamma_r, double tau, int mode, int n,
                      const int32_t *xs, const int32_t *ys, double *agg_out, int32_t *d_int,
                      double *d_sub)
{
    double *num = (double *)malloc(sizeof(double) * (size_t)D);
    if (!num) return -1;
    for (int i = 0; i < n; ++i) {
        int u = xs[i], v = ys[i];
        for (int d = 0; d < D; ++d) num[d] = 0.0;
        double den = 0.0;
        for (int y = v - rho; y <= v + rho; ++y) {
            if (y < 0 || y >= H) continue;
            for (int x = u - rho; x <= u + rho; ++x) {
                if (x < 0 || x >= W) continue;
                double w = oracle_weight(L, W, C, u, v, x, y, gamma_d, gamma_r);
                den += w;
                for (int d = 0; d < D; ++d) num[d] += w * oracle_cost(L, R, H, W, C, x, y, d, mode, tau);
            }
        }
        for (int d = 0; d < D; ++d) num[d] /= den;
        if (agg_out) memcpy(agg_out + (size_t)i * D, num, sizeof(double) * (size_t)D);
        oracle_wta_subpixel_pixel(num, D, d_int + i, d_sub + i);
    }
    free(num);
    return 0;
}

/*
 * Right view (Sec. II-A, Sec. III): the right cost volume stores the same costs
 * as the left one, C_r(u_r, v, d) = C_l(u_r + d, v, d); where u_r + d >= W no
 * left pixel exists and the cost is the maximum (2 for NCC, tau for TAD;
 * reading R6).  The right aggregation is guided by the right image (R5), and
 * WTA / Eq. (10) follow as on the left.
 */
double oracle_cost_right(const uint8_t *L, const uint8_t *R, int H, int W, int C, int ur, int v, int d,
                         int mode, double tau)
{
    if (ur + d >= W) return mode == 0 ? 2.0 : tau;
    return oracle_cost(L, R, H, W, C, ur + d, v, d, mode, tau);
}

int oracle_fbs_right_rows(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D, int rho,
                          double gamma_d, double gamma_r, double tau, int mode, int y0, int y1,
                          double *agg_out, int32_t *d_int, double *d_sub)
{
    int c0 = y0 - rho < 0 ? 0 : y0 - rho;
    int c1 = y1 + rho > H ? H : y1 + rho;
    size_t crow = (size_t)W * D;
    double *cost = (double *)malloc(sizeof(double) * crow * (size_t)(c1 - c0));
    double *agg = agg_out ? agg_out : (double *)malloc(sizeof(double) * crow * (size_t)(y1 - y0));
    if (!cost || !agg) { free(cost); if (!agg_out) free(agg); return -1; }
    for (int v = c0; v < c1; ++v)
        for (int u = 0; u < W; ++u)
            for (int d = 0; d < D; ++d)
                cost[((size_t)(v - c0) * W + u) * D + d] = oracle_cost_right(L, R, H, W, C, u, v, d, mode, tau);
    oracle_aggregate_rows(cost, c0, R, H, W, C, D, rho, gamma_d, gamma_r, y0, y1, agg);
    oracle_wta_subpixel(agg, (y1 - y0) * W, D, d_int, d_sub);
    free(cost);
    if (!agg_out) free(agg);
    return 0;
}

/*
 * Left-right consistency, Eq. (9): the left disparity d at (u, v) is kept when
 * u - d >= 0 and the right disparity at (u - d, v) equals d exactly
 * (reading R14); valid[p] = 1 or 0.
 */
void oracle_lrc(const int32_t *d_left, const int32_t *d_right, int H, int W, int32_t *valid)
{
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            const int d = d_left[(size_t)v * W + u];
            valid[(size_t)v * W + u] = (u - d >= 0 && d_right[(size_t)v * W + u - d] == d) ? 1 : 0;
        }
}
