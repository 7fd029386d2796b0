/*
 * gi_oracle.c -- FP64 CPU oracle for the accumulated-summation 2D Gaussian
 * rasterizer of GaussianImage (arXiv 2403.08551).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header or constant with the CUDA library.
 *
 * Every function is the plain definition written out as loops, in the
 * paper's notation:
 *   Sigma = L L^T with L = [[l1, 0], [l2, l3]]            (Sec. 3.1, Eq. 1)
 *   sigma_n = 1/2 d^T Sigma^-1 d, d = pixel centre - mu     (Sec. 3.2, Eq. 5)
 *   C_i = sum_n c'_n exp(-sigma_n)                          (Sec. 3.2, Eq. 7)
 *   L2 reconstruction loss                                  (Sec. 3.4)
 *   gradients                                               (App. A.1, A.2)
 * The paper is silent on the screen support of a Gaussian; the reading used
 * here (identical on the GPU side) is the tile-granular 3-sigma rectangle
 * evaluated in FP32 by gio_rect_rule below.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared
 * (-ffp-contract=off keeps every float operation of the rect rule a separate
 * correctly rounded IEEE operation.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int gio_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void gio_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static float clampf_(float v, float lo, float hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/*
 * Support rule (reading of the paper; FP32, round-to-nearest, no fused ops).
 *   S11 = l1*l1, S12 = l1*l2, S22 = l2*l2 + l3*l3, det = (l1*l3)*(l1*l3)
 *   conic (A, B, C) = (S22/det, -S12/det, S11/det)     -- used only to cull
 *   rx = 3*|l1|, ry = 3*sqrt(S22)   (exact half-extents of the 3-sigma
 *                                    ellipse d^T Sigma^-1 d <= 9)
 *   tx0 = clamp(floor((mx - rx) / T), 0, tw)
 *   tx1 = clamp(floor((mx + rx) / T) + 1, 0, tw)     (same for y with ry, th)
 * A Gaussian is culled (rect = 0, cnt = 0) if any parameter is non-finite,
 * det == 0, any entry of Sigma^-1 = (A, B, C) or rx, ry is non-finite (Eq. 5
 * needs a finite inverse covariance), or the rectangle is empty.
 * cnt = (tx1 - tx0) * (ty1 - ty0) tiles.
 */
void gio_rect_rule(const float* means, const float* chol, const float* color,
                   int64_t n, int32_t W, int32_t H, int32_t T,
                   int32_t* rect, int32_t* cnt) {
    const int32_t tw = (W + T - 1) / T, th = (H + T - 1) / T;
    const float inv_t = 1.0f / (float)T; /* T is a power of two: exact */
    for (int64_t g = 0; g < n; ++g) {
        const float mx = means[2 * g], my = means[2 * g + 1];
        const float l1 = chol[3 * g], l2 = chol[3 * g + 1], l3 = chol[3 * g + 2];
        int32_t* r = rect + 4 * g;
        r[0] = r[1] = r[2] = r[3] = 0;
        cnt[g] = 0;
        int finite = isfinite(mx) && isfinite(my) && isfinite(l1) && isfinite(l2) &&
                     isfinite(l3) && isfinite(color[3 * g]) &&
                     isfinite(color[3 * g + 1]) && isfinite(color[3 * g + 2]);
        if (!finite) continue;
        float s11 = l1 * l1;
        float s12 = l1 * l2;
        float s22 = l2 * l2 + l3 * l3;
        float d = l1 * l3;
        float det = d * d;
        if (det == 0.0f) continue;
        float ca = s22 / det, cb = -s12 / det, cc = s11 / det;
        if (!isfinite(det) || !isfinite(ca) || !isfinite(cb) || !isfinite(cc)) continue;
        float rx = 3.0f * fabsf(l1);
        float ry = 3.0f * sqrtf(s22);
        if (!isfinite(rx) || !isfinite(ry)) continue;
        float fx0 = clampf_(floorf((mx - rx) * inv_t), 0.0f, (float)tw);
        float fx1 = clampf_(floorf((mx + rx) * inv_t) + 1.0f, 0.0f, (float)tw);
        float fy0 = clampf_(floorf((my - ry) * inv_t), 0.0f, (float)th);
        float fy1 = clampf_(floorf((my + ry) * inv_t) + 1.0f, 0.0f, (float)th);
        int32_t tx0 = (int32_t)fx0, tx1 = (int32_t)fx1;
        int32_t ty0 = (int32_t)fy0, ty1 = (int32_t)fy1;
        if (tx0 >= tx1 || ty0 >= ty1) continue;
        r[0] = tx0; r[1] = ty0; r[2] = tx1; r[3] = ty1;
        cnt[g] = (tx1 - tx0) * (ty1 - ty0);
    }
}

/*
 * Tile binning by definition: the list of tile t (row-major tile index
 * t = ty*tw + tx) is every Gaussian g with t inside rect(g), in ascending g.
 * Lists are concatenated in tile order into ids[]; ranges[2t], ranges[2t+1]
 * are the [begin, end) of tile t (empty tiles: [0, 0)).  pair_off[g] is the
 * exclusive prefix sum of cnt (the index of g's first (tile, g) pair in
 * emission order) and pair_off[n] = K.  Returns K; ids is written only when
 * K <= cap.
 */
int64_t gio_bin(const int32_t* rect, const int32_t* cnt, int64_t n, int32_t tw,
                int32_t th, int64_t cap, uint32_t* ids, int32_t* ranges,
                int64_t* pair_off) {
    const int64_t T_img = (int64_t)tw * th;
    int64_t* count = (int64_t*)calloc((size_t)T_img, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)T_img, sizeof(int64_t));
    int64_t K = 0;
    for (int64_t g = 0; g < n; ++g) {
        pair_off[g] = K;
        K += cnt[g];
        if (cnt[g] == 0) continue;
        const int32_t* r = rect + 4 * g;
        for (int32_t ty = r[1]; ty < r[3]; ++ty)
            for (int32_t tx = r[0]; tx < r[2]; ++tx) count[(int64_t)ty * tw + tx]++;
    }
    pair_off[n] = K;
    int64_t start = 0;
    for (int64_t t = 0; t < T_img; ++t) {
        if (count[t] == 0) {
            ranges[2 * t] = 0;
            ranges[2 * t + 1] = 0;
        } else {
            ranges[2 * t] = (int32_t)start;
            ranges[2 * t + 1] = (int32_t)(start + count[t]);
        }
        fill[t] = start;
        start += count[t];
    }
    if (K <= cap) {
        for (int64_t g = 0; g < n; ++g) {
            if (cnt[g] == 0) continue;
            const int32_t* r = rect + 4 * g;
            for (int32_t ty = r[1]; ty < r[3]; ++ty)
                for (int32_t tx = r[0]; tx < r[2]; ++tx)
                    ids[fill[(int64_t)ty * tw + tx]++] = (uint32_t)g;
        }
    }
    free(count);
    free(fill);
    return K;
}

/* Sigma^-1 = [[A, B], [B, C]] of Sigma = L L^T, by the 2x2 adjugate formula
 * (Eq. 1), in FP64. */
static void conic64(const float* chol, int64_t g, double* A, double* B, double* C) {
    const double l1 = chol[3 * g], l2 = chol[3 * g + 1], l3 = chol[3 * g + 2];
    const double s11 = l1 * l1, s12 = l1 * l2, s22 = l2 * l2 + l3 * l3;
    const double det = s11 * s22 - s12 * s12;
    *A = s22 / det;
    *B = -s12 / det;
    *C = s11 / det;
}

void gio_conic(const float* chol, int64_t n, double* q) {
    for (int64_t g = 0; g < n; ++g) conic64(chol, g, q + 3 * g, q + 3 * g + 1, q + 3 * g + 2);
}

/* exp(-sigma) with sigma = 1/2 d^T Sigma^-1 d (Eq. 5), d = p - mu. */
static double weight64(double A, double B, double C, double dx, double dy) {
    const double sigma = 0.5 * (A * dx * dx + 2.0 * B * dx * dy + C * dy * dy);
    return exp(-sigma);
}

/*
 * Binned render (Eq. 7): for every pixel i of every tile, C_i = sum over the
 * tile's list (ascending g) of c'_g exp(-sigma_g(i)), pixel centre
 * (x + 0.5, y + 0.5).  out is [H][W][3] FP64.
 */
void gio_render(const float* means, const float* chol, const float* color,
                const uint32_t* ids, const int32_t* ranges, int32_t W, int32_t H,
                int32_t T, double* out) {
    const int32_t tw = (W + T - 1) / T, th = (H + T - 1) / T;
    const int64_t T_img = (int64_t)tw * th;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < T_img; ++t) {
        const int32_t tx = (int32_t)(t % tw), ty = (int32_t)(t / tw);
        const int32_t b = ranges[2 * t], e = ranges[2 * t + 1];
        for (int32_t y = ty * T; y < (ty + 1) * T && y < H; ++y) {
            for (int32_t x = tx * T; x < (tx + 1) * T && x < W; ++x) {
                double c[3] = {0.0, 0.0, 0.0};
                const double px = x + 0.5, py = y + 0.5;
                for (int32_t k = b; k < e; ++k) {
                    const int64_t g = ids[k];
                    double A, B, C;
                    conic64(chol, g, &A, &B, &C);
                    const double w = weight64(A, B, C, px - means[2 * g], py - means[2 * g + 1]);
                    c[0] += (double)color[3 * g] * w;
                    c[1] += (double)color[3 * g + 1] * w;
                    c[2] += (double)color[3 * g + 2] * w;
                }
                double* o = out + 3 * ((int64_t)y * W + x);
                o[0] = c[0];
                o[1] = c[1];
                o[2] = c[2];
            }
        }
    }
}

/*
 * Brute-force render: every Gaussian at every pixel, ascending g.  With
 * use_support != 0 a Gaussian contributes to pixel i only when tile(i) lies
 * in its rect (the same support as the binned form); with use_support == 0
 * the sum is untruncated (culled Gaussians still excluded).
 */
void gio_render_brute(const float* means, const float* chol, const float* color,
                      const int32_t* rect, const int32_t* cnt, int64_t n, int32_t W,
                      int32_t H, int32_t T, int32_t use_support, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            const int32_t tx = x / T, ty = y / T;
            double c[3] = {0.0, 0.0, 0.0};
            for (int64_t g = 0; g < n; ++g) {
                if (cnt[g] == 0) continue;
                const int32_t* r = rect + 4 * g;
                if (use_support && !(tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]))
                    continue;
                double A, B, C;
                conic64(chol, g, &A, &B, &C);
                const double w = weight64(A, B, C, x + 0.5 - means[2 * g], y + 0.5 - means[2 * g + 1]);
                c[0] += (double)color[3 * g] * w;
                c[1] += (double)color[3 * g + 1] * w;
                c[2] += (double)color[3 * g + 2] * w;
            }
            double* o = out + 3 * ((int64_t)y * W + x);
            o[0] = c[0];
            o[1] = c[1];
            o[2] = c[2];
        }
    }
}

/*
 * L2 reconstruction loss (Sec. 3.4), read as the mean over the 3*H*W
 * values: L = 1/(3HW) sum (C - x)^2.  Writes dL/dC = 2 (C - x) / (3HW)
 * when dldc is not NULL.  Returns L.
 */
double gio_loss(const double* out, const float* target, int32_t W, int32_t H, double* dldc) {
    const int64_t m = 3 * (int64_t)W * H;
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const double r = out[i] - (double)target[i];
        s += r * r;
        if (dldc) dldc[i] = 2.0 * r / (double)m;
    }
    return s / (double)m;
}

/*
 * Analytic gradients (App. A) of a loss with upstream gradient
 * G_i = dL/dC_i ([H][W][3] FP64) through the binned render.
 * For each supported pair (pixel i, Gaussian g), w = exp(-sigma):
 *   dL/dc'_g        += G_i w                                    (App. A.1)
 *   e               = dL/dsigma = -<G_i, c'_g> w   (the colour factor c'
 *                     that App. A.1's dC/dsigma omits is restored here)
 *   dL/dmu_g        += e * dsigma/dmu = e * (-Sigma^-1 d)   (d = p - mu)
 *   dL/dQ_ab        += e * 1/2 d_a d_b      (Q = Sigma^-1, four entries)
 * Per Gaussian: dL/dSigma = -Q (dL/dQ) Q (matrix calculus; this is App.
 * A.1's dsigma/dSigma = -1/2 Q d d^T Q summed with e), then with
 * G = dL/dSigma = [[g1, g2], [g2, g3]] (App. A.2):
 *   dL/dl1 = 2 g1 l1 + 2 g2 l2
 *   dL/dl2 = 2 g2 l1 + 2 g3 l2     (App. A.2 prints "g2 l2" for the last
 *                                   term; Sigma22 = l2^2 + l3^2 gives 2 g3 l2)
 *   dL/dl3 = 2 g3 l3
 * Each Gaussian loops over its own rect's tiles (row-major) and their
 * in-image pixels (row-major); Gaussians are independent, so the loop over
 * g is parallel.  Outputs (FP64): g_means [n][2], g_chol [n][3],
 * g_color [n][3], g_conic [n][3] = dL/dA, dL/dB, dL/dC of the symmetric
 * conic (B counted once, i.e. dL/dQ12 + dL/dQ21), and, when g_abs is not
 * NULL, g_abs [n][8] = the condition magnitude of each of the 8 parameter
 * gradients as App. A computes them (sums over pixels first, then the
 * per-Gaussian chain): the same formulas with every per-pixel term and every
 * chain coefficient replaced by its absolute value. It bounds |gradient|
 * and scales the rounding error of any floating-point evaluation of those
 * sums; it equals |gradient| when nothing cancels.
 */
void gio_backward(const float* means, const float* chol, const float* color,
                  const int32_t* rect, const int32_t* cnt, int64_t n, int32_t W,
                  int32_t H, int32_t T, const double* dldc, double* g_means,
                  double* g_chol, double* g_color, double* g_conic, double* g_abs) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < n; ++g) {
        double gm[2] = {0, 0}, gc[3] = {0, 0, 0}, gq11 = 0, gq12 = 0, gq22 = 0;
        /* sum over pixels of |per-pixel contribution| to each parameter's
         * gradient (the condition magnitude of each gradient sum) */
        double ab[8] = {0, 0, 0, 0, 0, 0, 0, 0}, am[5] = {0, 0, 0, 0, 0};
        if (cnt[g] > 0) {
            double A, B, C;
            conic64(chol, g, &A, &B, &C);
            const double mx = means[2 * g], my = means[2 * g + 1];
            const double cr = color[3 * g], cg = color[3 * g + 1], cbl = color[3 * g + 2];
            const double l1 = chol[3 * g], l2 = chol[3 * g + 1], l3 = chol[3 * g + 2];
            const int32_t* r = rect + 4 * g;
            for (int32_t ty = r[1]; ty < r[3]; ++ty)
                for (int32_t tx = r[0]; tx < r[2]; ++tx)
                    for (int32_t y = ty * T; y < (ty + 1) * T && y < H; ++y)
                        for (int32_t x = tx * T; x < (tx + 1) * T && x < W; ++x) {
                            const double* G = dldc + 3 * ((int64_t)y * W + x);
                            const double dx = x + 0.5 - mx, dy = y + 0.5 - my;
                            const double w = weight64(A, B, C, dx, dy);
                            gc[0] += G[0] * w;
                            gc[1] += G[1] * w;
                            gc[2] += G[2] * w;
                            const double e = -(G[0] * cr + G[1] * cg + G[2] * cbl) * w;
                            /* dsigma/dmu = -(Q d) */
                            gm[0] += e * -(A * dx + B * dy);
                            gm[1] += e * -(B * dx + C * dy);
                            gq11 += e * 0.5 * dx * dx;
                            gq12 += e * 0.5 * dx * dy;
                            gq22 += e * 0.5 * dy * dy;
                            if (g_abs) {
                                /* absolute per-pixel terms of the sums App. A
                                 * accumulates: e d (for mu), e/2 d d^T (for
                                 * dL/dSigma, chained afterwards), G w (for c') */
                                am[0] += fabs(e * dx);
                                am[1] += fabs(e * dy);
                                am[2] += fabs(0.5 * e * dx * dx);
                                am[3] += fabs(0.5 * e * dx * dy);
                                am[4] += fabs(0.5 * e * dy * dy);
                                ab[5] += fabs(G[0] * w);
                                ab[6] += fabs(G[1] * w);
                                ab[7] += fabs(G[2] * w);
                            }
                        }
            /* dL/dSigma = -Q G_Q Q, G_Q = [[gq11, gq12], [gq12, gq22]] */
            const double QG11 = A * gq11 + B * gq12, QG12 = A * gq12 + B * gq22;
            const double QG21 = B * gq11 + C * gq12, QG22 = B * gq12 + C * gq22;
            const double g1 = -(QG11 * A + QG12 * B);
            const double g2 = -(QG11 * B + QG12 * C);
            const double g3 = -(QG21 * B + QG22 * C);
            g_chol[3 * g] = 2.0 * g1 * l1 + 2.0 * g2 * l2;
            g_chol[3 * g + 1] = 2.0 * g2 * l1 + 2.0 * g3 * l2;
            g_chol[3 * g + 2] = 2.0 * g3 * l3;
            if (g_abs) {
                /* the same linear maps with every coefficient and every sum
                 * replaced by its absolute value */
                ab[0] = fabs(A) * am[0] + fabs(B) * am[1];
                ab[1] = fabs(B) * am[0] + fabs(C) * am[1];
                const double k11a = A * A * l1 + A * B * l2, k12a = 2.0 * A * B * l1 + (A * C + B * B) * l2,
                             k22a = B * B * l1 + B * C * l2;
                const double k11b = A * B * l1 + B * B * l2, k12b = (A * C + B * B) * l1 + 2.0 * B * C * l2,
                             k22b = B * C * l1 + C * C * l2;
                ab[2] = 2.0 * (fabs(k11a) * am[2] + fabs(k12a) * am[3] + fabs(k22a) * am[4]);
                ab[3] = 2.0 * (fabs(k11b) * am[2] + fabs(k12b) * am[3] + fabs(k22b) * am[4]);
                ab[4] = 2.0 * fabs(l3) * (B * B * am[2] + 2.0 * fabs(B * C) * am[3] + C * C * am[4]);
            }
        } else {
            g_chol[3 * g] = g_chol[3 * g + 1] = g_chol[3 * g + 2] = 0.0;
        }
        g_means[2 * g] = gm[0];
        g_means[2 * g + 1] = gm[1];
        g_color[3 * g] = gc[0];
        g_color[3 * g + 1] = gc[1];
        g_color[3 * g + 2] = gc[2];
        if (g_abs)
            for (int j = 0; j < 8; ++j) g_abs[8 * g + j] = ab[j];
        if (g_conic) {
            g_conic[3 * g] = gq11;
            g_conic[3 * g + 1] = 2.0 * gq12;
            g_conic[3 * g + 2] = gq22;
        }
    }
}

/*
 * Sorted alpha-blending render (Sec. 3.2, Eq. 3-4), the rasterisation that
 * accumulated summation replaces (the "w/o AR" ablation, Table 3). Per pixel,
 * front to back over the tile's list in ascending g (the only order a 2D
 * image offers):
 *   alpha = min(a_max, o_g exp(-sigma_g)); skipped when alpha < a_min;
 *   the walk stops before a Gaussian that would take the transmittance
 *   T (1 - alpha) below t_min; otherwise C += c_g alpha T, T *= 1 - alpha.
 * (a_min, a_max, t_min) = (1/255, 0.99, 1e-4) are 3D GS's thresholds.
 * out [H][W][3] FP64; t_final [H][W] the final T; n_last [H][W] the list
 * position (from the tile's first entry) just past the last Gaussian that
 * contributed; ambiguous [H][W] = 1 where some decision lay within a relative
 * amb of its threshold (there an FP32 evaluation may decide otherwise).
 */
void gio_render_blend(const float* means, const float* chol, const float* color, const float* opac,
                      const uint32_t* ids, const int32_t* ranges, int32_t W, int32_t H, int32_t T,
                      double a_min, double a_max, double t_min, double amb, double* out, double* t_final,
                      int32_t* n_last, uint8_t* ambiguous) {
    const int32_t tw = (W + T - 1) / T, th = (H + T - 1) / T;
    const int64_t T_img = (int64_t)tw * th;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < T_img; ++t) {
        const int32_t tx = (int32_t)(t % tw), ty = (int32_t)(t / tw);
        const int32_t b = ranges[2 * t], e = ranges[2 * t + 1];
        for (int32_t y = ty * T; y < (ty + 1) * T && y < H; ++y) {
            for (int32_t x = tx * T; x < (tx + 1) * T && x < W; ++x) {
                double c[3] = {0.0, 0.0, 0.0}, Tr = 1.0;
                int32_t last = 0;
                uint8_t am = 0;
                const double px = x + 0.5, py = y + 0.5;
                for (int32_t k = b; k < e; ++k) {
                    const int64_t g = ids[k];
                    double A, B, C;
                    conic64(chol, g, &A, &B, &C);
                    double a = (double)opac[g] * weight64(A, B, C, px - means[2 * g], py - means[2 * g + 1]);
                    if (fabs(a - a_min) <= amb * a_min || fabs(a - a_max) <= amb * a_max) am = 1;
                    if (a < a_min) continue;
                    if (a > a_max) a = a_max;
                    const double test = Tr * (1.0 - a);
                    if (fabs(test - t_min) <= amb * t_min) am = 1;
                    if (test < t_min) break;
                    c[0] += (double)color[3 * g] * a * Tr;
                    c[1] += (double)color[3 * g + 1] * a * Tr;
                    c[2] += (double)color[3 * g + 2] * a * Tr;
                    Tr = test;
                    last = k - b + 1;
                }
                const int64_t pix = (int64_t)y * W + x;
                out[3 * pix] = c[0];
                out[3 * pix + 1] = c[1];
                out[3 * pix + 2] = c[2];
                t_final[pix] = Tr;
                n_last[pix] = last;
                ambiguous[pix] = am;
            }
        }
    }
}

/*
 * Gradients of the alpha-blending render for upstream dL/dC (dldc [H][W][3])
 * and the final colours out (from gio_render_blend). Per pixel, front to back
 * over the contributing Gaussians (the same decisions as the forward), with
 * the prefix P_n = sum_{m <= n} c_m alpha_m T_m and the suffix S = C - P_n:
 *   dL/dc_n     = sum_px dL/dC alpha_n T_n
 *   dL/dalpha_n = sum_ch dL/dC (c_n T_n - S / (1 - alpha_n))
 * and, unless alpha_n was clamped to a_max, dL/do_n = dL/dalpha_n w and
 * dL/dsigma_n = -dL/dalpha_n alpha_n, chained to mu and the Cholesky vector
 * as in gio_backward. Gradients are summed per Gaussian over all pixels
 * (serial: the sums are in a fixed order). g_opac is dL/do; g_abs [n][9] the
 * condition magnitudes (means 2, chol 3, colour 3, opacity 1); g_abs_amb [n][9]
 * the same magnitudes over the pixels flagged in ambiguous only, where the
 * walk is continued to the end of the list and skipped Gaussians count as
 * contributing (a bound on what a decision taken the other way can change).
 */
static void blend_abs_terms(double* s, double ea, double dx, double dy, double dla_abs, double w,
                            const double* gabs_at) {
    s[0] += ea * fabs(dx);
    s[1] += ea * fabs(dy);
    s[2] += ea * 0.5 * dx * dx;
    s[3] += ea * 0.5 * fabs(dx * dy);
    s[4] += ea * 0.5 * dy * dy;
    s[5] += gabs_at[0];
    s[6] += gabs_at[1];
    s[7] += gabs_at[2];
    s[8] += dla_abs * w;
}

static void chain_abs(const double* am, double A, double B, double C, double l1, double l2, double l3, int live,
                      double* ab) {
    ab[0] = fabs(A) * am[0] + fabs(B) * am[1];
    ab[1] = fabs(B) * am[0] + fabs(C) * am[1];
    const double k11a = A * A * l1 + A * B * l2, k12a = 2.0 * A * B * l1 + (A * C + B * B) * l2,
                 k22a = B * B * l1 + B * C * l2;
    const double k11b = A * B * l1 + B * B * l2, k12b = (A * C + B * B) * l1 + 2.0 * B * C * l2,
                 k22b = B * C * l1 + C * C * l2;
    ab[2] = live ? 2.0 * (fabs(k11a) * am[2] + fabs(k12a) * am[3] + fabs(k22a) * am[4]) : 0.0;
    ab[3] = live ? 2.0 * (fabs(k11b) * am[2] + fabs(k12b) * am[3] + fabs(k22b) * am[4]) : 0.0;
    ab[4] = live ? 2.0 * fabs(l3) * (B * B * am[2] + 2.0 * fabs(B * C) * am[3] + C * C * am[4]) : 0.0;
    ab[5] = am[5];
    ab[6] = am[6];
    ab[7] = am[7];
    ab[8] = am[8];
}

void gio_backward_blend(const float* means, const float* chol, const float* color, const float* opac,
                        const uint32_t* ids, const int32_t* ranges, int64_t n, int32_t W, int32_t H,
                        int32_t T, double a_min, double a_max, const double* out, const int32_t* n_last,
                        const uint8_t* ambiguous, const double* dldc, double* g_means, double* g_chol,
                        double* g_color, double* g_opac, double* g_abs, double* g_abs_amb) {
    const int32_t tw = (W + T - 1) / T, th = (H + T - 1) / T;
    const int64_t T_img = (int64_t)tw * th;
    /* per Gaussian: [0..8] sums e d (2), e/2 d d^T (3), colour (3), opacity (1);
     * [9..17] their absolute counterparts; [18..26] those over ambiguous pixels */
    double* acc = (double*)calloc((size_t)(n > 0 ? n : 1) * 27, sizeof(double));
    for (int64_t t = 0; t < T_img; ++t) {
        const int32_t tx = (int32_t)(t % tw), ty = (int32_t)(t / tw);
        const int32_t b = ranges[2 * t], e_end = ranges[2 * t + 1];
        for (int32_t y = ty * T; y < (ty + 1) * T && y < H; ++y) {
            for (int32_t x = tx * T; x < (tx + 1) * T && x < W; ++x) {
                const int64_t pix = (int64_t)y * W + x;
                const double* G = dldc + 3 * pix;
                const double* Cf = out + 3 * pix;
                const int amb = ambiguous && ambiguous[pix];
                double P[3] = {0.0, 0.0, 0.0}, Tr = 1.0;
                const double px = x + 0.5, py = y + 0.5;
                for (int32_t k = b; k < (amb ? e_end : b + n_last[pix]); ++k) {
                    const int walked = k < b + n_last[pix];
                    const int64_t g = ids[k];
                    double A, B, C;
                    conic64(chol, g, &A, &B, &C);
                    const double dx = px - means[2 * g], dy = py - means[2 * g + 1];
                    const double w = weight64(A, B, C, dx, dy);
                    double a = (double)opac[g] * w;
                    const int skipped = a < a_min;
                    if (skipped && !amb) continue;
                    const int clamped = a > a_max;
                    if (clamped) a = a_max;
                    const double cc[3] = {color[3 * g], color[3 * g + 1], color[3 * g + 2]};
                    double dla = 0.0, dla_abs = 0.0, gat[3];
                    double* s = acc + 27 * g;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double Pn = P[ch] + cc[ch] * a * Tr;
                        const double S = Cf[ch] - Pn;
                        dla += G[ch] * (cc[ch] * Tr - S / (1.0 - a));
                        dla_abs += fabs(G[ch]) * (fabs(cc[ch]) * Tr + (fabs(Cf[ch]) + fabs(Pn)) / (1.0 - a));
                        gat[ch] = fabs(G[ch] * a * Tr);
                        if (walked && !skipped) {
                            P[ch] = Pn;
                            s[5 + ch] += G[ch] * a * Tr;
                        }
                    }
                    const double ea = clamped ? 0.0 : dla_abs * a; /* magnitude of dL/dsigma */
                    if (amb) blend_abs_terms(s + 18, ea, dx, dy, clamped ? 0.0 : dla_abs, w, gat);
                    if (!walked || skipped) continue;
                    blend_abs_terms(s + 9, ea, dx, dy, clamped ? 0.0 : dla_abs, w, gat);
                    if (!clamped) {
                        const double e = -dla * a; /* dL/dsigma */
                        s[0] += e * -(A * dx + B * dy);
                        s[1] += e * -(B * dx + C * dy);
                        s[2] += e * 0.5 * dx * dx;
                        s[3] += e * 0.5 * dx * dy;
                        s[4] += e * 0.5 * dy * dy;
                        s[8] += dla * w;
                    }
                    Tr *= 1.0 - a;
                }
            }
        }
    }
    for (int64_t g = 0; g < n; ++g) {
        const double* s = acc + 27 * g;
        double A, B, C;
        conic64(chol, g, &A, &B, &C);
        const double l1 = chol[3 * g], l2 = chol[3 * g + 1], l3 = chol[3 * g + 2];
        const double gq11 = s[2], gq12 = s[3], gq22 = s[4];
        const double QG11 = A * gq11 + B * gq12, QG12 = A * gq12 + B * gq22;
        const double QG21 = B * gq11 + C * gq12, QG22 = B * gq12 + C * gq22;
        const double g1 = -(QG11 * A + QG12 * B), g2 = -(QG11 * B + QG12 * C), g3 = -(QG21 * B + QG22 * C);
        const int live = s[14] + s[15] + s[16] + s[9] + s[10] + s[18] + s[19] + s[23] > 0.0;
        g_means[2 * g] = s[0];
        g_means[2 * g + 1] = s[1];
        g_chol[3 * g] = live ? 2.0 * g1 * l1 + 2.0 * g2 * l2 : 0.0;
        g_chol[3 * g + 1] = live ? 2.0 * g2 * l1 + 2.0 * g3 * l2 : 0.0;
        g_chol[3 * g + 2] = live ? 2.0 * g3 * l3 : 0.0;
        g_color[3 * g] = s[5];
        g_color[3 * g + 1] = s[6];
        g_color[3 * g + 2] = s[7];
        g_opac[g] = s[8];
        if (g_abs) chain_abs(s + 9, A, B, C, l1, l2, l3, live, g_abs + 9 * g);
        if (g_abs_amb) chain_abs(s + 18, A, B, C, l1, l2, l3, live, g_abs_amb + 9 * g);
    }
    free(acc);
}
