/*
 * CPU oracle for the local stereo method of Chang & Maruyama,
 * "Real-Time High-Quality Stereo Matching System on a GPU" (arXiv 2212.00488).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may call,
 * link or load this file; only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg use it. It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Every function is the plain definition written out with direct loops:
 * aggregation sums each arm element by element (no prefix sums), so this code
 * is independent of the GPU's scan-based design. Each function names the
 * passage of the paper it follows. Where the paper is silent or ambiguous the
 * chosen reading is stated next to the code.
 *
 * Parity status: every stage here is pinned by the CPU tests (hand-worked
 * values, closed forms, invariants, brute force on tiny inputs). The paper
 * prints no intermediate values and its figures are missing, so nothing here
 * is pinned against numbers printed in the paper itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the row loops marked "omp parallel for" below (OpenMP over
 * rows, used only to time the oracle on all host cores). Each output element
 * is still computed by one thread in the same order, so results do not depend
 * on the count. n <= 0 takes every processor. Returns the count in effect
 * (1 when built without OpenMP). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int absi(int v) { return v < 0 ? -v : v; }

/* Sec. III step 1: grey-scale conversion. The paper gives no formula; this
 * reading uses BT.601 luma weights in 8-bit fixed point, rounded:
 * g = (77 R + 150 G + 29 B + 128) >> 8. Input is HWC interleaved RGB. */
void oracle_grey(const uint8_t *rgb, int W, int H, uint8_t *g)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const uint8_t *p = rgb + 3 * ((size_t)y * W + x);
            int v = (77 * p[0] + 150 * p[1] + 29 * p[2] + 128) >> 8;
            g[(size_t)y * W + x] = (uint8_t)v;
        }
}

/* Sec. III-A, Eq. 2 with K = 2 and m = 1 (Step 1 of Sec. IV adds the 3x3
 * neighbourhood of every even-coordinate pixel): the scaled image is the mean
 * of the (2m+1)^2 window centred on (Kx, Ky). The paper does not state the
 * rounding or the border; this reading rounds half up, (sum + 4) / 9, and
 * clamps coordinates to the image. Output is (W/2) x (H/2), floor. */
void oracle_downscale(const uint8_t *g, int W, int H, uint8_t *s)
{
    int X = W / 2, Y = H / 2;
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int sum = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) {
                    int xx = clampi(2 * x + i, 0, W - 1);
                    int yy = clampi(2 * y + j, 0, H - 1);
                    sum += g[(size_t)yy * W + xx];
                }
            s[(size_t)y * X + x] = (uint8_t)((sum + 4) / 9);
        }
}

/* Sec. III-B: mini-census transform, the centre compared with six neighbours
 * giving a six-bit string. The pattern figure (Fig. 3) is missing; Step 3
 * caches three image lines for it, so the six neighbours lie in rows y-1..y+1.
 * This reading takes the mirror-symmetric set below; bit k is set when the
 * neighbour k is strictly darker than the centre. Borders clamp. */
static const int census_dx[6] = {-1, +1, -2, +2, -1, +1};
static const int census_dy[6] = {-1, -1, 0, 0, +1, +1};

void oracle_census(const uint8_t *g, int X, int Y, uint8_t *code)
{
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int c = g[(size_t)y * X + x];
            int bits = 0;
            for (int k = 0; k < 6; ++k) {
                int xx = clampi(x + census_dx[k], 0, X - 1);
                int yy = clampi(y + census_dy[k], 0, Y - 1);
                if (g[(size_t)yy * X + xx] < c) bits |= 1 << k;
            }
            code[(size_t)y * X + x] = (uint8_t)bits;
        }
}

/* Sec. III-C (with Steps 2 and 4 of Sec. IV): the arms of pixel (x, y) count
 * the contiguous pixels on each side whose brightness differs from the centre
 * by less than delta (strict), up to W_x horizontally and W_y vertically per
 * side (Table II footnote: W_+- = 21, W*_+- = 31, TC = 13 taken as delta).
 * Arms never leave the image. */
void oracle_arms(const uint8_t *g, int X, int Y, int wx, int wy, int tc,
                 uint8_t *hm, uint8_t *hp, uint8_t *vm, uint8_t *vp)
{
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int c = g[(size_t)y * X + x];
            int k;
            k = 0;
            while (k < wx && x - (k + 1) >= 0 && absi(g[(size_t)y * X + x - (k + 1)] - c) < tc) ++k;
            hm[(size_t)y * X + x] = (uint8_t)k;
            k = 0;
            while (k < wx && x + (k + 1) < X && absi(g[(size_t)y * X + x + (k + 1)] - c) < tc) ++k;
            hp[(size_t)y * X + x] = (uint8_t)k;
            k = 0;
            while (k < wy && y - (k + 1) >= 0 && absi(g[(size_t)(y - (k + 1)) * X + x] - c) < tc) ++k;
            vm[(size_t)y * X + x] = (uint8_t)k;
            k = 0;
            while (k < wy && y + (k + 1) < Y && absi(g[(size_t)(y + (k + 1)) * X + x] - c) < tc) ++k;
            vp[(size_t)y * X + x] = (uint8_t)k;
        }
}

/* Eqs. 4 and 5. Brightness differences are read on the [0, 1] scale
 * (a / 255), since on raw 0..255 levels lambda_AD = 0.3 would saturate the AD
 * term for any nonzero difference. The integer mode quantises each term to
 * round(scale * value) (half away from zero), evaluated in double with the
 * host C library. */
void oracle_cost_tables(double lambda_ad, double lambda_mc, int scale,
                        int32_t *lut_ad /* 256 */, int32_t *lut_mc /* 7 */)
{
    for (int a = 0; a < 256; ++a)
        lut_ad[a] = (int32_t)lround((double)scale * (1.0 - exp(-((double)a / 255.0) / lambda_ad)));
    for (int h = 0; h <= 6; ++h)
        lut_mc[h] = (int32_t)lround((double)scale * (1.0 - exp(-(double)h / lambda_mc)));
}

static int popcount6(int v)
{
    int n = 0;
    for (int k = 0; k < 6; ++k) n += (v >> k) & 1;
    return n;
}

/* Eq. 3 (C = C_AD + C_MC) for one disparity plane, integer mode.
 * dir = -1: left base, the match is M(x - d, y) (Sec. II).
 * dir = +1: right base, the match is M(x + d, y) (Eq. 6, written directly).
 * A match outside the image costs the maximum P = AD(255) + MC(6) (the paper
 * is silent; P is symmetric for both bases). */
static void cost_plane_int(const uint8_t *gB, const uint8_t *cB, const uint8_t *gM, const uint8_t *cM,
                           int X, int Y, int d, int dir, const int32_t *lut_ad, const int32_t *lut_mc,
                           int64_t *Cp)
{
    int64_t P = (int64_t)lut_ad[255] + lut_mc[6];
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int xm = x + dir * d;
            size_t b = (size_t)y * X + x;
            if (xm < 0 || xm >= X) {
                Cp[b] = P;
            } else {
                size_t m = (size_t)y * X + xm;
                int ad = absi((int)gB[b] - (int)gM[m]);
                int mc = popcount6(cB[b] ^ cM[m]);
                Cp[b] = (int64_t)lut_ad[ad] + lut_mc[mc];
            }
        }
}

/* The same plane in double precision: Eqs. 3-5 without quantisation. */
static void cost_plane_f64(const uint8_t *gB, const uint8_t *cB, const uint8_t *gM, const uint8_t *cM,
                           int X, int Y, int d, int dir, double lambda_ad, double lambda_mc, double *Cp)
{
    double P = (1.0 - exp(-1.0 / lambda_ad)) + (1.0 - exp(-6.0 / lambda_mc));
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int xm = x + dir * d;
            size_t b = (size_t)y * X + x;
            if (xm < 0 || xm >= X) {
                Cp[b] = P;
            } else {
                size_t m = (size_t)y * X + xm;
                int ad = absi((int)gB[b] - (int)gM[m]);
                int mc = popcount6(cB[b] ^ cM[m]);
                Cp[b] = (1.0 - exp(-((double)ad / 255.0) / lambda_ad)) + (1.0 - exp(-(double)mc / lambda_mc));
            }
        }
}

/* Eq. 7: CA_x(x, y) = sum over dx in [-m, n] of C(x + dx, y), with m, n the
 * pixel's own left/right arms; then Eq. 8: CA(x, y) = sum over dy in [-M, N]
 * of CA_x(x, y + dy), with M, N the anchor's up/down arms. Direct loops. */
static void aggregate_plane_int(const int64_t *Cp, const uint8_t *hm, const uint8_t *hp,
                                const uint8_t *vm, const uint8_t *vp, int X, int Y,
                                int64_t *CAx, int64_t *CA)
{
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            size_t i = (size_t)y * X + x;
            int64_t s = 0;
            for (int t = -(int)hm[i]; t <= (int)hp[i]; ++t) s += Cp[i + t];
            CAx[i] = s;
        }
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            size_t i = (size_t)y * X + x;
            int64_t s = 0;
            for (int t = -(int)vm[i]; t <= (int)vp[i]; ++t) s += CAx[(size_t)(y + t) * X + x];
            CA[i] = s;
        }
}

static void aggregate_plane_f64(const double *Cp, const uint8_t *hm, const uint8_t *hp,
                                const uint8_t *vm, const uint8_t *vp, int X, int Y,
                                double *CAx, double *CA)
{
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            size_t i = (size_t)y * X + x;
            double s = 0;
            for (int t = -(int)hm[i]; t <= (int)hp[i]; ++t) s += Cp[i + t];
            CAx[i] = s;
        }
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            size_t i = (size_t)y * X + x;
            double s = 0;
            for (int t = -(int)vm[i]; t <= (int)vp[i]; ++t) s += CAx[(size_t)(y + t) * X + x];
            CA[i] = s;
        }
}

/* Integer-mode aggregated volume of one base, CA[d][y][x] (for small inputs;
 * the brute-force support enumeration in the tests checks it). Also returns
 * the cost volume C[d][y][x] when C is not NULL. */
int oracle_volume_int(const uint8_t *gB, const uint8_t *cB, const uint8_t *gM, const uint8_t *cM,
                      const uint8_t *hm, const uint8_t *hp, const uint8_t *vm, const uint8_t *vp,
                      int X, int Y, int D, int dir, const int32_t *lut_ad, const int32_t *lut_mc,
                      int64_t *C, int64_t *CA)
{
    size_t n = (size_t)X * Y;
    int64_t *Cp = malloc(n * sizeof *Cp), *CAx = malloc(n * sizeof *CAx);
    if (!Cp || !CAx) { free(Cp); free(CAx); return -1; }
    for (int d = 0; d < D; ++d) {
        cost_plane_int(gB, cB, gM, cM, X, Y, d, dir, lut_ad, lut_mc, Cp);
        if (C) memcpy(C + (size_t)d * n, Cp, n * sizeof *Cp);
        aggregate_plane_int(Cp, hm, hp, vm, vp, X, Y, CAx, CA + (size_t)d * n);
    }
    free(Cp); free(CAx);
    return 0;
}

/* Eq. 9 (printed as a min; the text chooses the d that minimises CA), one
 * base, integer mode. Disparities are tried in ascending order and a new d
 * wins only when strictly smaller (Step 5 replaces its running minimum only
 * on a strictly lower value), so the smallest minimising d is chosen.
 * disp is [Y][X]. */
int oracle_wta_int(const uint8_t *gB, const uint8_t *cB, const uint8_t *gM, const uint8_t *cM,
                   const uint8_t *hm, const uint8_t *hp, const uint8_t *vm, const uint8_t *vp,
                   int X, int Y, int D, int dir, const int32_t *lut_ad, const int32_t *lut_mc,
                   uint8_t *disp, int64_t *best_cost)
{
    size_t n = (size_t)X * Y;
    int64_t *Cp = malloc(n * sizeof *Cp), *CAx = malloc(n * sizeof *CAx), *CA = malloc(n * sizeof *CA);
    int64_t *best = malloc(n * sizeof *best);
    if (!Cp || !CAx || !CA || !best) { free(Cp); free(CAx); free(CA); free(best); return -1; }
    for (int d = 0; d < D; ++d) {
        cost_plane_int(gB, cB, gM, cM, X, Y, d, dir, lut_ad, lut_mc, Cp);
        aggregate_plane_int(Cp, hm, hp, vm, vp, X, Y, CAx, CA);
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i)
            if (d == 0 || CA[i] < best[i]) { best[i] = CA[i]; disp[i] = (uint8_t)d; }
    }
    if (best_cost) memcpy(best_cost, best, n * sizeof *best);
    free(Cp); free(CAx); free(CA); free(best);
    return 0;
}

/* The same selection in double precision. best and second return the lowest
 * and second-lowest aggregated cost per pixel (over all d), which the tests use
 * to identify near-ties. */
int oracle_wta_f64(const uint8_t *gB, const uint8_t *cB, const uint8_t *gM, const uint8_t *cM,
                   const uint8_t *hm, const uint8_t *hp, const uint8_t *vm, const uint8_t *vp,
                   int X, int Y, int D, int dir, double lambda_ad, double lambda_mc,
                   uint8_t *disp, double *best, double *second)
{
    size_t n = (size_t)X * Y;
    double *Cp = malloc(n * sizeof *Cp), *CAx = malloc(n * sizeof *CAx), *CA = malloc(n * sizeof *CA);
    if (!Cp || !CAx || !CA) { free(Cp); free(CAx); free(CA); return -1; }
    for (size_t i = 0; i < n; ++i) { best[i] = INFINITY; second[i] = INFINITY; disp[i] = 0; }
    for (int d = 0; d < D; ++d) {
        cost_plane_f64(gB, cB, gM, cM, X, Y, d, dir, lambda_ad, lambda_mc, Cp);
        aggregate_plane_f64(Cp, hm, hp, vm, vp, X, Y, CAx, CA);
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i) {
            if (CA[i] < best[i]) { second[i] = best[i]; best[i] = CA[i]; disp[i] = (uint8_t)d; }
            else if (CA[i] < second[i]) second[i] = CA[i];
        }
    }
    free(Cp); free(CAx); free(CA);
    return 0;
}

/* Eq. 10: (x, y) is a ground control point when D^L(x, y) = k and
 * D^R(x - k, y) = k. A match column x - k < 0 is not a GCP (the paper is
 * silent). gcp is 1 or 0. */
void oracle_crosscheck(const uint8_t *dl, const uint8_t *dr, int X, int Y, uint8_t *gcp)
{
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int k = dl[(size_t)y * X + x];
            int ok = (x - k >= 0) && dr[(size_t)y * X + x - k] == k;
            gcp[(size_t)y * X + x] = (uint8_t)ok;
        }
}

/* Sec. III step 7 / Step 7: median filter of D^L. The window is not given;
 * this reading uses 3x3 with clamped borders. The middle of the nine sorted
 * values is kept. */
void oracle_median3(const uint8_t *dl, int X, int Y, uint8_t *dm)
{
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            int v[9], n = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i)
                    v[n++] = dl[(size_t)clampi(y + j, 0, Y - 1) * X + clampi(x + i, 0, X - 1)];
            for (int a = 1; a < 9; ++a) {           /* insertion sort */
                int t = v[a], b = a - 1;
                while (b >= 0 && v[b] > t) { v[b + 1] = v[b]; --b; }
                v[b + 1] = t;
            }
            dm[(size_t)y * X + x] = (uint8_t)v[4];
        }
}

/* Sec. III-E (bilateral estimation, Eq. 11) and Step 7. For a non-GCP at
 * (x, y), i and j are the distances to the nearest GCPs on its left and right
 * in the same row, with disparities a = Dm(x - i) and b = Dm(x + j).
 *  - |a - b| <= T: linear fill between the two GCPs (Step 7 describes a
 *    linear fill; Eq. 11 as printed has the sign of its correction term
 *    reversed, which would extrapolate away from b). Written as
 *    (a*j + b*i) / (i + j): exact integer numerator, one float division.
 *  - |a - b| > T: a when L(x - i) is strictly closer in brightness to L(x)
 *    than L(x + j), otherwise b.
 *  - One side only: that side's disparity. Neither side: 0 (paper silent).
 * GCP pixels keep Dm. Output is float [Y][X] in processed-resolution units.
 * mode selects the fill between two GCPs: 0 the bilateral estimation above
 * (the paper's method); 1 and 2 the two prior-art approaches Sec. III-E
 * describes before it (Fig. 5): 1 takes the GCP nearer in distance (the left
 * one only when strictly nearer: the paper is silent on a tie), 2 takes the
 * smaller of the two disparities (the occluded side). */
void oracle_fill(const uint8_t *dm, const uint8_t *gcp, const uint8_t *g, int X, int Y, int T,
                 int mode, float *out)
{
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            size_t r = (size_t)y * X;
            if (gcp[r + x]) { out[r + x] = (float)dm[r + x]; continue; }
            int i = 0, j = 0;
            for (int t = 1; x - t >= 0; ++t) if (gcp[r + x - t]) { i = t; break; }
            for (int t = 1; x + t < X; ++t) if (gcp[r + x + t]) { j = t; break; }
            float v;
            if (i && j) {
                int a = dm[r + x - i], b = dm[r + x + j];
                if (mode == 1) {
                    v = (float)(i < j ? a : b);
                } else if (mode == 2) {
                    v = (float)(a < b ? a : b);
                } else if (absi(a - b) <= T) {
                    v = (float)(a * j + b * i) / (float)(i + j);
                } else {
                    int ga = absi((int)g[r + x - i] - (int)g[r + x]);
                    int gb = absi((int)g[r + x + j] - (int)g[r + x]);
                    v = (float)(ga < gb ? a : b);
                }
            } else if (i) {
                v = (float)dm[r + x - i];
            } else if (j) {
                v = (float)dm[r + x + j];
            } else {
                v = 0.0f;
            }
            out[r + x] = v;
        }
}

/* Step 8: scale the filled map up by 2, bilateral estimation along x and
 * linear along y; values are converted to full-resolution disparity units
 * (x2). The paper gives no further detail; this reading:
 *  row pass on low-res row y, output column X':
 *    X' even: 2 Dp(X'/2) (last low-res column when X'/2 is past the end);
 *    X' odd, both neighbours a = Dp(x), b = Dp(x+1) present (x = X'/2):
 *       |a - b| <= T -> a + b; otherwise 2a when the low-res grey at x is
 *       strictly closer than that at x + 1 to the full-res grey G(X', 2y),
 *       else 2b; with no right neighbour: 2 Dp(x).
 *  column pass, output row Y': even -> row Y'/2 (clamped); odd -> the mean of
 *  rows y and y + 1, or row y when y + 1 is past the end.
 * Float operations are single IEEE operations (no fused multiply-add). */
static float rowpass(const float *dp, const uint8_t *gs, const uint8_t *gf, int X, int W, int T,
                     int Xo, int y)
{
    int x = Xo >> 1;
    const float *row = dp + (size_t)y * X;
    if ((Xo & 1) == 0) return 2.0f * row[x < X ? x : X - 1];
    if (x + 1 >= X) return 2.0f * row[x < X ? x : X - 1];
    float a = row[x], b = row[x + 1];
    float diff = a - b;
    if (fabsf(diff) <= (float)T) return a + b;
    int gfull = gf[(size_t)(2 * y) * W + Xo];
    int ga = absi((int)gs[(size_t)y * X + x] - gfull);
    int gb = absi((int)gs[(size_t)y * X + x + 1] - gfull);
    return 2.0f * (ga < gb ? a : b);
}

void oracle_upscale(const float *dp, const uint8_t *gs, const uint8_t *gf, int X, int Y,
                    int W, int H, int T, float *out)
{
    for (int Yo = 0; Yo < H; ++Yo)
        for (int Xo = 0; Xo < W; ++Xo) {
            int y = Yo >> 1;
            float v;
            if ((Yo & 1) == 0 || y + 1 >= Y) {
                v = rowpass(dp, gs, gf, X, W, T, Xo, y < Y ? y : Y - 1);
            } else {
                float r0 = rowpass(dp, gs, gf, X, W, T, Xo, y);
                float r1 = rowpass(dp, gs, gf, X, W, T, Xo, y + 1);
                float s = r0 + r1;
                v = 0.5f * s;
            }
            out[(size_t)Yo * W + Xo] = v;
        }
}

/* ------------------------------------------------------------------------
 * Differentiable form, FP64 (test infrastructure like the rest of the file).
 * Left base only. Intensities gL, gR are grey values on [0, 1]; the census
 * codes and the arms are frozen inputs (computed from the quantised images),
 * so the only non-smooth steps are |.| and the comparisons they freeze.
 *   C(x,y,d)  = w_AD (1 - exp(-|gL(x,y) - gR(x-d,y)| / l_AD))
 *             + w_MC (1 - exp(-MC / l_MC))            (Eqs. 3-5)
 *             = P = w_AD (1 - exp(-1/l_AD)) + w_MC (1 - exp(-6/l_MC)) if x < d
 *   CA        = aggregation of Eqs. 7-8 over the frozen arms, divided by the
 *               support size n(x,y) (constant over d, so the WTA of Eq. 9 is
 *               unchanged; it keeps the soft-argmin's inputs of order one)
 *   p_d       = softmax over d of -CA(x,y,d) / tau
 *   dhat(x,y) = sum_d d p_d
 * theta = (w_AD, w_MC, l_AD, l_MC). With go != NULL the gradient of
 * sum(go * dhat) is returned for gL, gR and theta: the aggregation's adjoint
 * is written as plain scatters over each anchor's support.
 * ------------------------------------------------------------------------ */
int oracle_diff(const double *gL, const double *gR, const uint8_t *cL, const uint8_t *cR,
                const uint8_t *hm, const uint8_t *hp, const uint8_t *vm, const uint8_t *vp,
                int X, int Y, int D, const double *theta, double tau, double *dhat,
                const double *go, double *g_gL, double *g_gR, double *g_theta)
{
    const double wad = theta[0], wmc = theta[1], lad = theta[2], lmc = theta[3];
    const size_t n = (size_t)X * Y, nv = n * (size_t)D;
    double *C = malloc(nv * sizeof *C), *Z = malloc(nv * sizeof *Z), *CAx = malloc(n * sizeof *CAx);
    double *ns = malloc(n * sizeof *ns);
    if (!C || !Z || !CAx || !ns) { free(C); free(Z); free(CAx); free(ns); return -1; }
    const double P = wad * (1.0 - exp(-1.0 / lad)) + wmc * (1.0 - exp(-6.0 / lmc));
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            size_t i = (size_t)y * X + x;
            double s = 0;
            for (int t = -(int)vm[i]; t <= (int)vp[i]; ++t) {
                size_t k = (size_t)(y + t) * X + x;
                s += (double)hm[k] + (double)hp[k] + 1.0;
            }
            ns[i] = s;
        }
    for (int d = 0; d < D; ++d) {
        double *Cd = C + (size_t)d * n, *Zd = Z + (size_t)d * n;
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                size_t i = (size_t)y * X + x;
                if (x - d < 0) { Cd[i] = P; continue; }
                double a = fabs(gL[i] - gR[i - d]);
                int h = popcount6(cL[i] ^ cR[i - d]);
                Cd[i] = wad * (1.0 - exp(-a / lad)) + wmc * (1.0 - exp(-(double)h / lmc));
            }
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                size_t i = (size_t)y * X + x;
                double s = 0;
                for (int t = -(int)hm[i]; t <= (int)hp[i]; ++t) s += Cd[i + t];
                CAx[i] = s;
            }
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                size_t i = (size_t)y * X + x;
                double s = 0;
                for (int t = -(int)vm[i]; t <= (int)vp[i]; ++t) s += CAx[(size_t)(y + t) * X + x];
                Zd[i] = -(s / ns[i]) / tau;
            }
    }
    /* softmax over d and the expected disparity; Z becomes p */
    for (size_t i = 0; i < n; ++i) {
        double m = -INFINITY;
        for (int d = 0; d < D; ++d) if (Z[(size_t)d * n + i] > m) m = Z[(size_t)d * n + i];
        double s = 0;
        for (int d = 0; d < D; ++d) s += exp(Z[(size_t)d * n + i] - m);
        double e = 0;
        for (int d = 0; d < D; ++d) {
            double p = exp(Z[(size_t)d * n + i] - m) / s;
            Z[(size_t)d * n + i] = p;
            e += d * p;
        }
        dhat[i] = e;
    }
    if (go) {
        double *G1 = malloc(n * sizeof *G1), *G2 = malloc(n * sizeof *G2), *Gc = malloc(n * sizeof *Gc);
        if (!G1 || !G2 || !Gc) { free(G1); free(G2); free(Gc); free(C); free(Z); free(CAx); free(ns); return -1; }
        for (size_t i = 0; i < n; ++i) { g_gL[i] = 0; g_gR[i] = 0; }
        for (int k = 0; k < 4; ++k) g_theta[k] = 0;
        for (int d = 0; d < D; ++d) {
            const double *pd = Z + (size_t)d * n;
            /* d dhat / d CA(x,y,d) = p_d (d - dhat) * (-1/tau) / n(x,y) */
            for (size_t i = 0; i < n; ++i) Gc[i] = go[i] * pd[i] * ((double)d - dhat[i]) * (-1.0 / tau) / ns[i];
            /* adjoint of the vertical sum: each anchor sends its value to its span */
            for (size_t i = 0; i < n; ++i) G1[i] = 0;
            for (int y = 0; y < Y; ++y)
                for (int x = 0; x < X; ++x) {
                    size_t i = (size_t)y * X + x;
                    for (int t = -(int)vm[i]; t <= (int)vp[i]; ++t) G1[(size_t)(y + t) * X + x] += Gc[i];
                }
            /* adjoint of the horizontal sum: each pixel sends to its own row window */
            for (size_t i = 0; i < n; ++i) G2[i] = 0;
            for (int y = 0; y < Y; ++y)
                for (int x = 0; x < X; ++x) {
                    size_t i = (size_t)y * X + x;
                    for (int t = -(int)hm[i]; t <= (int)hp[i]; ++t) G2[i + t] += G1[i];
                }
            /* through the cost */
            for (int y = 0; y < Y; ++y)
                for (int x = 0; x < X; ++x) {
                    size_t i = (size_t)y * X + x;
                    double g = G2[i];
                    if (x - d < 0) {
                        double ea = exp(-1.0 / lad), eh = exp(-6.0 / lmc);
                        g_theta[0] += g * (1.0 - ea);
                        g_theta[1] += g * (1.0 - eh);
                        g_theta[2] += g * wad * (-ea * (1.0 / (lad * lad)));
                        g_theta[3] += g * wmc * (-eh * (6.0 / (lmc * lmc)));
                        continue;
                    }
                    double diff = gL[i] - gR[i - d], a = fabs(diff);
                    double h = (double)popcount6(cL[i] ^ cR[i - d]);
                    double ea = exp(-a / lad), eh = exp(-h / lmc);
                    g_theta[0] += g * (1.0 - ea);
                    g_theta[1] += g * (1.0 - eh);
                    g_theta[2] += g * wad * (-ea * (a / (lad * lad)));
                    g_theta[3] += g * wmc * (-eh * (h / (lmc * lmc)));
                    double sgn = diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0);
                    double dCda = wad * ea / lad;
                    g_gL[i] += g * dCda * sgn;
                    g_gR[i - d] -= g * dCda * sgn;
                }
        }
        free(G1); free(G2); free(Gc);
    }
    free(C); free(Z); free(CAx); free(ns);
    return 0;
}
