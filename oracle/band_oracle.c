/*
 * Oracle of the learned band proposal (TEST INFRASTRUCTURE ONLY; nothing on
 * the product path links, loads or calls this file, and it shares no code
 * with the CUDA path).
 *
 * The paper names, as future work (Sec. V), restricting the disparity search
 * range of each pixel to cut the aggregation work.  The band form does this:
 * a small network proposes a per-pixel disparity centre and a confidence; a
 * pixel with enough confidence aggregates only the disparities of a band
 * around its centre, every other pixel keeps the full range.  This file
 * holds the plain definitions of the non-network parts:
 *
 *   quarter-resolution input features   oracle_band_features
 *   per-pixel band from centre/conf     oracle_band_limits
 *   Eq. (6)-(10) restricted to a band   oracle_fbs_band_points
 *   training targets from plain FBS     oracle_band_targets
 *
 * The network itself (six 3x3 convolutions, its loss and gradients, Adam)
 * is written in numpy in band_net.py.
 *
 * Readings (also listed in the design notes):
 *   B1  quarter resolution: Hq = ceil(H/4), Wq = ceil(W/4), Dq = ceil(D/4);
 *       the quarter-resolution intensity of block (X, Y) is the integer sum of
 *       the channel sums over the 4x4 block, its pixels clamped to the image.
 *   B2  coarse cost: Eq. (1)-(3) with varrho = 1 on the quarter-resolution
 *       intensity, quarter disparities e in [0, Dq), the same boundary rules
 *       as the full-resolution cost (clamped blocks, cost 2 when X - e < 0,
 *       c = 0 for a flat block); cost K = 1 - c.  Sums are exact integers,
 *       the normalisation is FP64.
 *   B3  coarse aggregation: Kbar(X, Y, e) = the mean of K(X', Y', e) over the
 *       5x5 quarter-resolution window around (X, Y) clipped to the image
 *       (FP64) -- a box-filter counterpart, at quarter resolution, of the
 *       aggregation of Sec. II-B, which makes the coarse winner reliable.
 *       The kernels evaluate B2-B3 in FP32; the tests allow the FP32
 *       rounding bound and compare the integer decisions (the winner, the
 *       feature points of B7) exactly wherever the FP64 values are not
 *       within that bound of a tie or of the threshold.
 *       Features per quarter pixel (FP64):
 *         f0 = G_l / (16 * 255 * C) - 0.5      (left intensity)
 *         f1 = e* / Dq                         (coarse winner of Kbar, smallest e on ties)
 *         f2 = Kbar(e*)                        (its cost)
 *         f3 = min(K2 - Kbar(e*), 1)           (margin to the best e with |e - e*| >= 2;
 *                                               K2 = 2 when there is none)
 *         f4 = Kbar(e* - 1) - Kbar(e*)   (2 - Kbar(e*) at e* = 0)
 *         f5 = Kbar(e* + 1) - Kbar(e*)   (2 - Kbar(e*) at e* = Dq - 1)
 *   B4  band of a full-resolution pixel from its centre c and confidence k:
 *       full range [0, D-1] when !(k >= theta) or c is not finite; otherwise
 *       m = floor(c + 0.5) in FP32, clamped to [0, D-1], band
 *       [max(m - h, 0), min(m + h, D - 1)].
 *   B5  band FBS: Agg(p, d) of Eq. (6) for d in the band only; the winner is
 *       the smallest d of the band with the least Agg; Eq. (10) is applied
 *       only when both neighbours d* - 1 and d* + 1 lie in the band (the band
 *       ends play the role of 0 and D - 1).
 *   B7  feature-point proposal (the paper's future work, Sec. V: reliable
 *       feature points suggest the search range of their neighbours): a
 *       quarter pixel is a feature point when its margin f3 >= theta_m;
 *       a full-resolution pixel in quarter pixel i takes the feature points of
 *       the 5x5 quarter window around i (clipped); with at least 3 of them and
 *       max e* - min e* <= 2 its centre is 2 (max e* + min e*) (= 4 x the
 *       mid-range, exact in FP32) and its confidence 1, otherwise confidence 0
 *       (full range).
 *   B6  targets of quarter pixel i from plain full-range FBS (integer d*,
 *       subpixel ds) over the in-image pixels of its 4x4 block: centre target
 *       t = median of ds (for an even count the mean of the two middle
 *       values), robust to the block's outlier winners; confidence target
 *       y = the fraction of the block's d* that lie in [m - h + 1, m + h - 1],
 *       m being the band centre of B4 for the predicted centre
 *       c_i = 4 (e*_i + o0_i) -- the share of pixels whose winner and both of
 *       its neighbours the band holds (a soft target of the logistic loss).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int bclampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* B1: quarter-resolution intensity plane of one image, Hq x Wq int32. */
void oracle_band_downsample(const uint8_t *img, int H, int W, int C, int32_t *gq)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    for (int Y = 0; Y < Hq; ++Y) {
        for (int X = 0; X < Wq; ++X) {
            int32_t s = 0;
            for (int j = 0; j < 4; ++j) {
                const int y = bclampi(4 * Y + j, 0, H - 1);
                for (int i = 0; i < 4; ++i) {
                    const int x = bclampi(4 * X + i, 0, W - 1);
                    for (int c = 0; c < C; ++c) s += img[((size_t)y * W + x) * C + c];
                }
            }
            gq[(size_t)Y * Wq + X] = s;
        }
    }
}

/* B2: coarse cost K(X, Y, e) from the two quarter-resolution planes. */
static double coarse_cost(const int32_t *gl, const int32_t *gr, int Hq, int Wq, int X, int Y, int e)
{
    if (X - e < 0) return 2.0;
    int64_t Sl = 0, Ql = 0, Sr = 0, Qr = 0, P = 0;
    for (int j = -1; j <= 1; ++j) {
        const int y = bclampi(Y + j, 0, Hq - 1);
        for (int i = -1; i <= 1; ++i) {
            const int64_t a = gl[(size_t)y * Wq + bclampi(X + i, 0, Wq - 1)];
            const int64_t b = gr[(size_t)y * Wq + bclampi(X - e + i, 0, Wq - 1)];
            Sl += a;
            Ql += a * a;
            Sr += b;
            Qr += b * b;
            P += a * b;
        }
    }
    const int64_t Vl = 9 * Ql - Sl * Sl;
    const int64_t Vr = 9 * Qr - Sr * Sr;
    if (Vl == 0 || Vr == 0) return 1.0;
    const int64_t num = 9 * P - Sl * Sr;
    return 1.0 - (double)num / sqrt((double)Vl * (double)Vr);
}

#define BAND_AGG_R 2   /* 5x5 coarse aggregation window */

/*
 * B1-B3: features [Hq][Wq][6] (FP64) and the coarse winner e* [Hq][Wq] of a
 * pair; gap [Hq][Wq] (nullable): second smallest minus smallest Kbar of each
 * quarter pixel (how close its winner is to a tie).  Scratch is allocated
 * here.  Returns 0, or -1 when out of memory.
 */
int oracle_band_features(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D, double *feat,
                         int32_t *estar, double *gap)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4, Dq = (D + 3) / 4;
    const size_t nq = (size_t)Hq * Wq;
    int32_t *gl = (int32_t *)malloc(sizeof(int32_t) * nq);
    int32_t *gr = (int32_t *)malloc(sizeof(int32_t) * nq);
    double *K = (double *)malloc(sizeof(double) * nq * Dq);
    double *Kb = (double *)malloc(sizeof(double) * Dq);
    if (!gl || !gr || !K || !Kb) { free(gl); free(gr); free(K); free(Kb); return -1; }
    oracle_band_downsample(L, H, W, C, gl);
    oracle_band_downsample(R, H, W, C, gr);
    for (int Y = 0; Y < Hq; ++Y)
        for (int X = 0; X < Wq; ++X)
            for (int e = 0; e < Dq; ++e) K[((size_t)Y * Wq + X) * Dq + e] = coarse_cost(gl, gr, Hq, Wq, X, Y, e);
    const double gscale = 16.0 * 255.0 * C;
    for (int Y = 0; Y < Hq; ++Y) {
        for (int X = 0; X < Wq; ++X) {
            /* B3: mean over the clipped 5x5 window */
            for (int e = 0; e < Dq; ++e) {
                double s = 0.0;
                int n = 0;
                for (int y = Y - BAND_AGG_R; y <= Y + BAND_AGG_R; ++y)
                    for (int x = X - BAND_AGG_R; x <= X + BAND_AGG_R; ++x)
                        if (y >= 0 && y < Hq && x >= 0 && x < Wq) {
                            s += K[((size_t)y * Wq + x) * Dq + e];
                            ++n;
                        }
                Kb[e] = s / n;
            }
            int best = 0;
            for (int e = 1; e < Dq; ++e)
                if (Kb[e] < Kb[best]) best = e;
            double k2 = 2.0, second = INFINITY;
            for (int e = 0; e < Dq; ++e) {
                if (abs(e - best) >= 2 && Kb[e] < k2) k2 = Kb[e];
                if (e != best && Kb[e] < second) second = Kb[e];
            }
            const double k1 = Kb[best];
            const double km = best > 0 ? Kb[best - 1] : 2.0;
            const double kp = best < Dq - 1 ? Kb[best + 1] : 2.0;
            double *f = feat + ((size_t)Y * Wq + X) * 6;
            f[0] = gl[(size_t)Y * Wq + X] / gscale - 0.5;
            f[1] = (double)best / Dq;
            f[2] = k1;
            f[3] = k2 - k1 < 1.0 ? k2 - k1 : 1.0;
            f[4] = km - k1;
            f[5] = kp - k1;
            estar[(size_t)Y * Wq + X] = best;
            if (gap) gap[(size_t)Y * Wq + X] = second - k1;
        }
    }
    free(gl);
    free(gr);
    free(K);
    free(Kb);
    return 0;
}

/* B4: band [lo, hi] of every pixel of an H x W centre/confidence pair. */
void oracle_band_limits(const float *centre, const float *conf, int n, int D, int h, float theta, int32_t *lo,
                        int32_t *hi)
{
    for (int p = 0; p < n; ++p) {
        const float c = centre[p], k = conf[p];
        if (!(k >= theta) || !isfinite(c)) {
            lo[p] = 0;
            hi[p] = D - 1;
            continue;
        }
        float m = floorf(c + 0.5f);
        if (m < 0.0f) m = 0.0f;
        if (m > (float)(D - 1)) m = (float)(D - 1);
        const int mi = (int)m;
        lo[p] = mi - h < 0 ? 0 : mi - h;
        hi[p] = mi + h > D - 1 ? D - 1 : mi + h;
    }
}

/* Eq. (1)-(3) cost and Eq. (7)-(8) weight: the pinned definitions of fbs_oracle.c. */
double oracle_cost(const uint8_t *L, const uint8_t *R, int H, int W, int C, int u, int v, int d, int mode,
                   double tau);
double oracle_weight(const uint8_t *guide, int W, int C, int u, int v, int x, int y, double gamma_d,
                     double gamma_r);

/*
 * B5 at isolated pixels (xs[i], ys[i]) with band [lo_i, hi_i] each (NCC cost).
 * agg_out (nullable) receives n x D values, NaN outside each band.
 */
int oracle_fbs_band_points(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D, int rho, double gamma_d,
                           double gamma_r, int n, const int32_t *xs, const int32_t *ys, const int32_t *lo,
                           const int32_t *hi, double *agg_out, int32_t *d_int, double *d_sub)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)D);
    if (!a) return -1;
    for (int i = 0; i < n; ++i) {
        const int u = xs[i], v = ys[i], b0 = lo[i], b1 = hi[i];
        for (int d = 0; d < D; ++d) a[d] = NAN;
        for (int d = b0; d <= b1; ++d) {
            double num = 0.0, den = 0.0;
            for (int y = v - rho; y <= v + rho; ++y) {
                if (y < 0 || y >= H) continue;
                for (int x = u - rho; x <= u + rho; ++x) {
                    if (x < 0 || x >= W) continue;
                    const double w = oracle_weight(L, W, C, u, v, x, y, gamma_d, gamma_r);
                    num += w * oracle_cost(L, R, H, W, C, x, y, d, 0, 0.0);
                    den += w;
                }
            }
            a[d] = num / den;
        }
        int best = b0;
        for (int d = b0 + 1; d <= b1; ++d)
            if (a[d] < a[best]) best = d;
        double ds = (double)best;
        if (best > b0 && best < b1) {
            const double den = 2.0 * a[best - 1] + 2.0 * a[best + 1] - 4.0 * a[best];
            if (den > 0.0) ds = best + (a[best - 1] - a[best + 1]) / den;
        }
        d_int[i] = best;
        d_sub[i] = ds;
        if (agg_out) memcpy(agg_out + (size_t)i * D, a, sizeof(double) * (size_t)D);
    }
    free(a);
    return 0;
}

/*
 * B6: targets of every quarter pixel.  label_int / label_sub are the plain
 * FBS outputs (H x W); centre_q is the predicted centre 4 (e* + o0) per
 * quarter pixel (Hq x Wq).  Writes t and y (both FP64).
 */
static int cmp_double(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void oracle_band_targets(const int32_t *label_int, const float *label_sub, int H, int W, int D, int h,
                         const double *centre_q, double *t, double *y)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    for (int Y = 0; Y < Hq; ++Y) {
        for (int X = 0; X < Wq; ++X) {
            const size_t i = (size_t)Y * Wq + X;
            float m = floorf((float)centre_q[i] + 0.5f);
            if (!(m >= 0.0f)) m = 0.0f;
            if (m > (float)(D - 1)) m = (float)(D - 1);
            const int mi = (int)m;
            double v[16];
            int cnt = 0, in = 0;
            for (int yy = 4 * Y; yy < 4 * Y + 4 && yy < H; ++yy) {
                for (int xx = 4 * X; xx < 4 * X + 4 && xx < W; ++xx) {
                    const size_t p = (size_t)yy * W + xx;
                    v[cnt++] = label_sub[p];
                    if (label_int[p] >= mi - h + 1 && label_int[p] <= mi + h - 1) ++in;
                }
            }
            qsort(v, (size_t)cnt, sizeof(double), cmp_double);
            t[i] = (cnt & 1) ? v[cnt / 2] : 0.5 * (v[cnt / 2 - 1] + v[cnt / 2]);
            y[i] = (double)in / cnt;
        }
    }
}

/*
 * B7: feature-point centre and confidence [H][W] (FP32 outputs) of a pair.
 * ambiguous [H][W] (nullable) is set where the window holds a quarter pixel
 * whose decision is within tol of changing: a margin within tol of theta_m,
 * or a winner within tol of a tie (then its e* and margin may differ under
 * rounding).
 */
int oracle_band_feature_points(const uint8_t *L, const uint8_t *R, int H, int W, int C, int D, double theta_m,
                               float *centre, float *conf, double tol, uint8_t *ambiguous)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    double *feat = (double *)malloc(sizeof(double) * (size_t)Hq * Wq * 6);
    double *gap = (double *)malloc(sizeof(double) * (size_t)Hq * Wq);
    int32_t *est = (int32_t *)malloc(sizeof(int32_t) * (size_t)Hq * Wq);
    if (!feat || !gap || !est || oracle_band_features(L, R, H, W, C, D, feat, est, gap) != 0) {
        free(feat);
        free(gap);
        free(est);
        return -1;
    }
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const int Y = y / 4, X = x / 4;
            int n = 0, emin = 1 << 30, emax = -1, amb = 0;
            for (int j = Y - 2; j <= Y + 2; ++j) {
                if (j < 0 || j >= Hq) continue;
                for (int i = X - 2; i <= X + 2; ++i) {
                    if (i < 0 || i >= Wq) continue;
                    const size_t q = (size_t)j * Wq + i;
                    if (fabs(feat[q * 6 + 3] - theta_m) <= tol || gap[q] <= tol) amb = 1;
                    if (!(feat[q * 6 + 3] >= theta_m)) continue;
                    ++n;
                    if (est[q] < emin) emin = est[q];
                    if (est[q] > emax) emax = est[q];
                }
            }
            const size_t p = (size_t)y * W + x;
            if (n >= 3 && emax - emin <= 2) {
                centre[p] = 2.0f * (float)(emax + emin);
                conf[p] = 1.0f;
            } else {
                centre[p] = 0.0f;
                conf[p] = 0.0f;
            }
            if (ambiguous) ambiguous[p] = (uint8_t)amb;
        }
    }
    free(feat);
    free(gap);
    free(est);
    return 0;
}
