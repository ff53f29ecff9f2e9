/*
 * CPU oracle of the stereo lane-detection path (Fan & Dahnoun, arXiv 1807.02752, Sec. 2.2-2.4).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded restatement of the paper's steps in the
 * paper's order, used to check the CUDA library element by element.  The library never calls it and
 * the two share no source.  Build: gcc -O2 -ffp-contract=off (no fused multiply-add anywhere, so every
 * float expression below is evaluated exactly as written, one IEEE rounding per operation).
 *
 * Where the paper is silent or ambiguous the reading taken is stated at the function that applies it.
 * Integer arithmetic is used wherever the method allows (histograms, DP energies, Sobel, votes, band
 * sums, box filters, lane energies); floating point enters only in the polynomial fits and their
 * evaluation, and in three float32 decisions (vote column, w_g angle, lane track).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

void or_default_params(or_params *p)
{
    memset(p, 0, sizeof(*p));
    p->n_disp = 128;
    p->tau_y = 6;
    p->lambda_y = 1;
    p->tr_y = 4.0f;
    p->eps_num = 99;
    p->eps_den = 100;
    p->varpi = 3.0f;
    p->bilateral = 1;
    p->bf_rho = 5;
    p->sigma_s = 300.0;
    p->sigma_r = 0.3;
    p->edge_thresh = 100;
    p->vote_rho = 1;
    p->chi = 25;
    p->tau_x = 5;
    p->lambda_x = 1;
    p->tr_x = 16.0f;
    p->sigma_g = 3.5;
    p->box_nu = 1;
    p->box_vs = 3;
    p->lambda_g = 1;
    p->xi_num = 1;
    p->xi_den = 2;
    p->thr_num = 1;
    p->thr_den = 32;
    p->near_px = 30;
    p->max_lanes = OR_MAX_LANES;
    p->ransac_hyps = 64;
    p->ransac_rounds = 64;
    p->seed = 0x1807027520ull;
    p->wg_gaussian = 0;
    p->pad0 = 0;
    p->thr_abs = 0;
    p->dp_literal = 0;
    p->band_literal_bottom = 0;
}

/* Sec. 2.4 and Alg. 7: the histogram H spans starts u in [-xi W, (1 + xi) W) (xi = 0.5). */
int32_t or_n_starts(int32_t W, const or_params *p)
{
    int32_t S0 = (int32_t)((int64_t)W * p->xi_num / p->xi_den);
    return W + 2 * S0;
}

/* ------------------------------------------------------------------------------------------------ */
/* Lookup tables.                                                                                    */
/* Eq. 16 spatial and range weights, rounded to Q15: floor(w * 32768 + 0.5).  Intensities enter w_r   */
/* scaled to [0, 1] (I / 255), the only scale at which sigma_r = 0.3 is meaningful.                  */
/* Eq. 23 weight, rounded to Q12, tabulated over sin(dtheta) in steps of 2^-15 up to the cut-off      */
/* dtheta = pi/6 (sin = 1/2); entry i holds the weight at dtheta = asin(i / 32768).                   */
/* ------------------------------------------------------------------------------------------------ */
void or_tables(const or_params *p, int32_t *ws_q, int32_t *wr_q, int32_t *wg_q)
{
    int32_t rho = p->bf_rho, n = 2 * rho + 1;
    if (ws_q) {
        for (int32_t dy = -rho; dy <= rho; dy++)
            for (int32_t dx = -rho; dx <= rho; dx++) {
                double r2 = (double)(dx * dx + dy * dy);
                double w = exp(-r2 / (p->sigma_s * p->sigma_s));
                ws_q[(dy + rho) * n + (dx + rho)] = (int32_t)floor(w * 32768.0 + 0.5);
            }
    }
    if (wr_q) {
        for (int32_t k = 0; k < 256; k++) {
            double t = (double)k / 255.0;
            double w = exp(-(t * t) / (p->sigma_r * p->sigma_r));
            wr_q[k] = (int32_t)floor(w * 32768.0 + 0.5);
        }
    }
    if (wg_q) {
        for (int32_t i = 0; i <= 16384; i++) {
            double dtheta = asin((double)i / 32768.0);
            double pp = dtheta * (36.0 / M_PI);   /* p = dtheta / theta_s, theta_s = pi / 36 */
            double w = p->wg_gaussian ? exp(-(pp * pp) / (p->sigma_g * p->sigma_g))
                                      : exp(-pp / (p->sigma_g * p->sigma_g));
            wg_q[i] = (int32_t)floor(w * 4096.0 + 0.5);
        }
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):  */
/* ten rounds of two 32x32->64 multiplies with the round keys bumped by the Weyl constants.          */
/* ------------------------------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ------------------------------------------------------------------------------------------------ */
/* Sec. 2.2: the v-disparity map m_y(d, v) is the histogram of each row of the disparity map.        */
/* Reading: a pixel is counted when its disparity is finite and > 0 (0 marks invalid pixels after the */
/* left-right check, Eq. 10 / Alg. 3); its bin is floor(l + 0.5) in float32, and bins >= D drop.      */
/* ------------------------------------------------------------------------------------------------ */
void or_vdisparity(const float *disp, int32_t W, int32_t H, int32_t D, int32_t *m_y)
{
    memset(m_y, 0, sizeof(int32_t) * (size_t)H * D);
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            float l = disp[(size_t)v * W + u];
            if (!isfinite(l) || !(l > 0.0f))
                continue;
            float b = floorf(l + 0.5f);
            if (b >= (float)D)
                continue;
            m_y[(size_t)v * D + (int32_t)b] += 1;
        }
}

/* ------------------------------------------------------------------------------------------------ */
/* Eq. 11-12: DP over the v-disparity map, from d = D-1 down to d = 1.                               */
/* Reading (rows run v = 0 at the top, road disparity grows downwards): a path point at (d, v) links  */
/* to (d+1, v + tau) with tau in [0, tau_y] and cost lambda_y * tau; the data term is -m_y(d, v).     */
/*   E_{D-1}(v) = -m_y(D-1, v)                                                                       */
/*   E_d(v)     = -m_y(d, v) + min_{tau, v+tau <= H-1} [ E_{d+1}(v + tau) + lambda_y tau ]           */
/* Ties take the smallest tau; the path starts at the smallest v minimising E_1.  Bin d = 0 (invalid  */
/* and near-zero disparities) is left out of the path.  path_v[d] receives the row at d, d = 1..D-1. */
/* Returns the minimum energy.                                                                       */
/* ------------------------------------------------------------------------------------------------ */
int64_t or_dp_vdisp(const int32_t *m_y, int32_t H, int32_t D, int32_t tau, int32_t lambda, int16_t *path_v)
{
    int64_t *Ep = (int64_t *)malloc(sizeof(int64_t) * H);
    int64_t *Ec = (int64_t *)malloc(sizeof(int64_t) * H);
    uint8_t *bt = (uint8_t *)calloc((size_t)D * H, 1);
    for (int32_t v = 0; v < H; v++)
        Ep[v] = -(int64_t)m_y[(size_t)v * D + (D - 1)];
    for (int32_t d = D - 2; d >= 1; d--) {
        for (int32_t v = 0; v < H; v++) {
            int64_t best = INT64_MAX;
            int32_t arg = 0;
            for (int32_t t = 0; t <= tau; t++) {
                if (v + t > H - 1)
                    break;
                int64_t cand = Ep[v + t] + (int64_t)lambda * t;
                if (cand < best) {
                    best = cand;
                    arg = t;
                }
            }
            Ec[v] = -(int64_t)m_y[(size_t)v * D + d] + best;
            bt[(size_t)d * H + v] = (uint8_t)arg;
        }
        int64_t *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    int32_t vbest = 0;
    for (int32_t v = 1; v < H; v++)
        if (Ep[v] < Ep[vbest])
            vbest = v;
    int64_t emin = Ep[vbest];
    path_v[0] = -1;
    path_v[1] = (int16_t)vbest;
    for (int32_t d = 1; d <= D - 2; d++)
        path_v[d + 1] = (int16_t)(path_v[d] + bt[(size_t)d * H + path_v[d]]);
    free(Ep);
    free(Ec);
    free(bt);
    return emin;
}

/* ------------------------------------------------------------------------------------------------ */
/* Eq. 12 as printed (dp_literal): E(v)_d = -m_y(d, v) + min_{tau in [0, tau_y], v - tau >= 0}          */
/* [E(v - tau)_{d+1} - lambda tau], the link to the row v - tau and a reward for the jump.  Ties take  */
/* the smaller tau; the path starts at the smallest v minimising E_1, then v_{d+1} = v_d - tau.       */
/* ------------------------------------------------------------------------------------------------ */
int64_t or_dp_vdisp_literal(const int32_t *m_y, int32_t H, int32_t D, int32_t tau, int32_t lambda, int16_t *path_v)
{
    int64_t *Ep = (int64_t *)malloc(sizeof(int64_t) * H);
    int64_t *Ec = (int64_t *)malloc(sizeof(int64_t) * H);
    uint8_t *bt = (uint8_t *)calloc((size_t)D * H, 1);
    for (int32_t v = 0; v < H; v++)
        Ep[v] = -(int64_t)m_y[(size_t)v * D + (D - 1)];
    for (int32_t d = D - 2; d >= 1; d--) {
        for (int32_t v = 0; v < H; v++) {
            int64_t best = INT64_MAX;
            int32_t arg = 0;
            for (int32_t t = 0; t <= tau; t++) {
                if (v - t < 0)
                    break;
                int64_t cand = Ep[v - t] - (int64_t)lambda * t;
                if (cand < best) {
                    best = cand;
                    arg = t;
                }
            }
            Ec[v] = -(int64_t)m_y[(size_t)v * D + d] + best;
            bt[(size_t)d * H + v] = (uint8_t)arg;
        }
        int64_t *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    int32_t vbest = 0;
    for (int32_t v = 1; v < H; v++)
        if (Ep[v] < Ep[vbest])
            vbest = v;
    int64_t emin = Ep[vbest];
    path_v[0] = -1;
    path_v[1] = (int16_t)vbest;
    for (int32_t d = 1; d <= D - 2; d++)
        path_v[d + 1] = (int16_t)(path_v[d] - bt[(size_t)d * H + path_v[d]]);
    free(Ep);
    free(Ec);
    free(bt);
    return emin;
}

/* ------------------------------------------------------------------------------------------------ */
/* Least squares fit (Eq. 13, Eq. 19) through the normal equations of Eq. 20.                        */
/* Basis: tau = t / 2^e with t = v - centre (integer).  The sums of t^k and y t^k are exact integers; */
/* each is rounded once to the nearest double and scaled by an exact power of two, which plays the    */
/* role of kappa in Eq. 20 (it keeps v^8 out of overflow).  The m x m system is solved by Gaussian     */
/* elimination with partial pivoting (first row of largest |pivot|); a pivot below 2^-40 counts as     */
/* singular.  coef[k] multiplies tau^k.  Returns 0, or -1 when singular or with fewer than m points.  */
/* ------------------------------------------------------------------------------------------------ */
static int32_t solve_normal(const i128 *Sx, const i128 *Sy, int32_t m, int32_t e, double *coef)
{
    double A[5][6];
    for (int32_t j = 0; j < m; j++) {
        for (int32_t k = 0; k < m; k++)
            A[j][k] = ldexp((double)Sx[j + k], -(j + k) * e);
        A[j][m] = ldexp((double)Sy[j], -j * e);
    }
    for (int32_t k = 0; k < m; k++) {
        int32_t piv = k;
        for (int32_t i = k + 1; i < m; i++)
            if (fabs(A[i][k]) > fabs(A[piv][k]))
                piv = i;
        if (!(fabs(A[piv][k]) >= 0x1p-40))
            return -1;
        if (piv != k)
            for (int32_t j = 0; j <= m; j++) {
                double t = A[k][j];
                A[k][j] = A[piv][j];
                A[piv][j] = t;
            }
        for (int32_t i = k + 1; i < m; i++) {
            double f = A[i][k] / A[k][k];
            for (int32_t j = k; j <= m; j++)
                A[i][j] = A[i][j] - f * A[k][j];
        }
    }
    for (int32_t k = m - 1; k >= 0; k--) {
        double s = A[k][m];
        for (int32_t j = k + 1; j < m; j++)
            s = s - A[k][j] * coef[j];
        coef[k] = s / A[k][k];
    }
    return 0;
}

int32_t or_lsf(const int32_t *x, const int32_t *y, const uint8_t *use, int32_t n, int32_t m,
               int32_t centre, int32_t e, double *coef)
{
    i128 Sx[9], Sy[5];
    memset(Sx, 0, sizeof(Sx));
    memset(Sy, 0, sizeof(Sy));
    int32_t cnt = 0;
    for (int32_t j = 0; j < n; j++) {
        if (use && !use[j])
            continue;
        cnt++;
        i128 t = (i128)(x[j] - centre), pw = 1;
        for (int32_t k = 0; k <= 2 * (m - 1); k++) {
            Sx[k] += pw;
            if (k < m)
                Sy[k] += pw * (i128)y[j];
            pw *= t;
        }
    }
    if (cnt < m)
        return -1;
    return solve_normal(Sx, Sy, m, e, coef);
}

/* The polynomial through m sample points (tau_i, y_i), tau_i = (x_i - centre) / 2^e, in Newton form:     */
/* divided differences c_i computed in float32 in place (c_i = y_i; for k = 1..m-1, i = m-1 down to k:   */
/* c_i = (c_i - c_{i-1}) / (tau_i - tau_{i-k})).  For m points the least squares fit of Eq. 13 / Eq. 19   */
/* is this interpolant; the Newton form computes it without squaring the conditioning of the system.      */
static void newton_fit(const float *tau, const float *y, int32_t m, float *c)
{
    for (int32_t i = 0; i < m; i++)
        c[i] = y[i];
    for (int32_t k = 1; k < m; k++)
        for (int32_t i = m - 1; i >= k; i--)
            c[i] = (c[i] - c[i - 1]) / (tau[i] - tau[i - k]);
}

/* Model value in float32 (nested Newton form, one rounding per operation) and the inlier test of        */
/* Sec. 2.2 and Sec. 2.3.3: r = (y - model)^2 < tr.                                                       */
static int32_t is_inlier(const float *c, const float *nodes, int32_t m, int32_t x, int32_t y, int32_t centre,
                         int32_t e, float tr)
{
    float tau = (float)(x - centre) * ldexpf(1.0f, -e);
    float p = c[m - 1];
    for (int32_t k = m - 2; k >= 0; k--)
        p = p * (tau - nodes[k]) + c[k];
    float r = (float)y - p;
    return r * r < tr;
}

/* ------------------------------------------------------------------------------------------------ */
/* One RANSAC hypothesis (Alg. 4 / Alg. 6: a random sample of the working set and the fit through it).   */
/* Reading: the sample is minimal (m points: 3 for beta, 5 for gamma) and drawn from the current      */
/* working set S (member[j] = 1), listed in increasing j.  Draw j = 0, 1, ... takes word (j & 3) of    */
/* Philox4x32-10 at counter (stage << 24 | round, hyp, j >> 2, 0), key = seed; the word x picks list   */
/* position floor(x * |S| / 2^32).  A draw repeating a chosen point or a chosen x is skipped; after   */
/* 8m draws without m distinct points the hypothesis is void.  The m points, in draw order, are fitted  */
/* exactly (newton_fit: the least squares fit of Eq. 13 / Eq. 19 through m points) and scored by the    */
/* inliers among S.                                                                                    */
/* Returns the inlier count, or -1 for a void hypothesis.  chosen[m] and inliers[n] may be NULL.      */
/* ------------------------------------------------------------------------------------------------ */
int32_t or_hypothesis(const int32_t *x, const int32_t *y, const uint8_t *member, int32_t n, int32_t m,
                      float tr, int32_t stage, int32_t round, int32_t hyp, const or_params *p,
                      int32_t centre, int32_t e, int32_t *chosen, uint8_t *inliers)
{
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t ns = 0;
    for (int32_t j = 0; j < n; j++)
        if (member[j])
            list[ns++] = j;
    int32_t pick[5], got = 0;
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    for (int32_t j = 0; j < 8 * m && got < m && ns > 0; j++) {
        uint32_t ctr[4] = {((uint32_t)stage << 24) | (uint32_t)round, (uint32_t)hyp, (uint32_t)(j >> 2), 0u};
        uint32_t out[4];
        or_philox4x32_10(ctr, key, out);
        uint32_t w = out[j & 3];
        int32_t pos = (int32_t)(((uint64_t)w * (uint64_t)ns) >> 32);
        int32_t pt = list[pos];
        int32_t dup = 0;
        for (int32_t q = 0; q < got; q++)
            if (pick[q] == pt || x[pick[q]] == x[pt])
                dup = 1;
        if (!dup)
            pick[got++] = pt;
    }
    free(list);
    if (chosen)
        for (int32_t q = 0; q < m; q++)
            chosen[q] = q < got ? pick[q] : -1;
    if (got < m)
        return -1;
    float nodes[5], sy[5], c[5];
    for (int32_t q = 0; q < m; q++) {
        nodes[q] = (float)(x[pick[q]] - centre) * ldexpf(1.0f, -e);
        sy[q] = (float)y[pick[q]];
    }
    newton_fit(nodes, sy, m, c);
    int32_t cnt = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t in = member[j] && is_inlier(c, nodes, m, x[j], y[j], centre, e, tr);
        if (inliers)
            inliers[j] = (uint8_t)in;
        cnt += in;
    }
    return cnt;
}

/* ------------------------------------------------------------------------------------------------ */
/* Alg. 4 / Alg. 6: RANSAC that re-partitions inliers and outliers until the inlier fraction reaches  */
/* eps, then fits the remaining set.                                                                 */
/* Reading: each round draws ransac_hyps hypotheses and keeps the one with the most inliers (ties: the */
/* lowest hypothesis index); its outliers leave the working set.  The loop stops after the first round */
/* with eps_den * n_I >= eps_num * n (n = working-set size at the start of the round), or when no      */
/* hypothesis is valid, or at the round cap.  The final fit is the least squares fit of the remaining  */
/* set.  member[n] returns the final set.  Returns flags: 1 = round cap, 2 = degenerate.             */
/* ------------------------------------------------------------------------------------------------ */
int32_t or_ransac(const int32_t *x, const int32_t *y, int32_t n, int32_t m, float tr, int32_t stage,
                  const or_params *p, int32_t centre, int32_t e, uint8_t *member, double *coef,
                  int32_t *rounds)
{
    int32_t flags = 0, r = 0;
    uint8_t *best_in = (uint8_t *)malloc(n > 0 ? n : 1);
    uint8_t *cur_in = (uint8_t *)malloc(n > 0 ? n : 1);
    for (int32_t j = 0; j < n; j++)
        member[j] = 1;
    for (;;) {
        int32_t ns = 0;
        for (int32_t j = 0; j < n; j++)
            ns += member[j];
        if (ns < m) {
            flags |= 2;
            break;
        }
        if (r == p->ransac_rounds) {
            flags |= 1;
            break;
        }
        int32_t best = -1;
        for (int32_t h = 0; h < p->ransac_hyps; h++) {
            int32_t c = or_hypothesis(x, y, member, n, m, tr, stage, r, h, p, centre, e, NULL, cur_in);
            if (c > best) {
                best = c;
                memcpy(best_in, cur_in, n);
            }
        }
        r++;
        if (best < 0) {
            flags |= 2;
            break;
        }
        for (int32_t j = 0; j < n; j++)
            member[j] = member[j] && best_in[j];
        if ((int64_t)p->eps_den * best >= (int64_t)p->eps_num * ns)
            break;
    }
    if (!(flags & 2))
        if (or_lsf(x, y, member, n, m, centre, e, coef) != 0)
            flags |= 2;
    if (rounds)
        *rounds = r;
    free(best_in);
    free(cur_in);
    return flags;
}

/* ------------------------------------------------------------------------------------------------ */
/* Median filter (the pre-filter the paper compares the bilateral with, Sec. 2.3.1): the lower median  */
/* of the window's taps inside the image, i.e. the ((n + 1) / 2)-th smallest of the n taps (n odd for  */
/* every interior pixel, so the middle value there), found by sorting the taps.                     */
/* ------------------------------------------------------------------------------------------------ */
static int cmp_u8(const void *a, const void *b) { return (int)*(const uint8_t *)a - (int)*(const uint8_t *)b; }

void or_median(const uint8_t *img, int32_t W, int32_t H, int32_t rho, uint8_t *out)
{
    uint8_t win[(2 * 16 + 1) * (2 * 16 + 1)];
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            int32_t n = 0;
            for (int32_t y = v - rho; y <= v + rho; y++)
                for (int32_t x = u - rho; x <= u + rho; x++)
                    if (y >= 0 && y < H && x >= 0 && x < W)
                        win[n++] = img[(size_t)y * W + x];
            qsort(win, (size_t)n, 1, cmp_u8);
            out[(size_t)v * W + u] = win[(n + 1) / 2 - 1];
        }
}

/* ------------------------------------------------------------------------------------------------ */
/* Eq. 15-16: bilateral filter over a (2 rho + 1)^2 window, clipped at the image border.            */
/* Weights per tap: w = (ws_q * wr_q[|I(i,j) - I(u,v)|] + 2^14) >> 15 (Q15).  The output is the      */
/* weighted mean rounded half up: (2 sum(w I) + sum(w)) / (2 sum(w)), an exact integer expression.   */
/* ------------------------------------------------------------------------------------------------ */
void or_bilateral(const uint8_t *img, int32_t W, int32_t H, const or_params *p, uint8_t *out)
{
    int32_t rho = p->bf_rho, n = 2 * rho + 1;
    int32_t *ws = (int32_t *)malloc(sizeof(int32_t) * n * n);
    int32_t wr[256];
    or_tables(p, ws, wr, NULL);
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            int32_t c = img[(size_t)v * W + u];
            int64_t num = 0, den = 0;
            for (int32_t j = v - rho; j <= v + rho; j++) {
                if (j < 0 || j >= H)
                    continue;
                for (int32_t i = u - rho; i <= u + rho; i++) {
                    if (i < 0 || i >= W)
                        continue;
                    int32_t q = img[(size_t)j * W + i];
                    int64_t w = ((int64_t)ws[(j - v + rho) * n + (i - u + rho)] * wr[abs(q - c)] + 16384) >> 15;
                    num += w * q;
                    den += w;
                }
            }
            out[(size_t)v * W + u] = (uint8_t)((2 * num + den) / (2 * den));
        }
    free(ws);
}

/* ------------------------------------------------------------------------------------------------ */
/* 3x3 Sobel derivatives (Sec. 2.3.1).  G_x > 0 for a dark-to-light transition from left to right,     */
/* G_y > 0 from top to bottom.  The one-pixel border ring is 0.                                       */
/* ------------------------------------------------------------------------------------------------ */
void or_sobel(const uint8_t *I, int32_t W, int32_t H, int16_t *gx, int16_t *gy)
{
#define PIX(uu, vv) ((int32_t)I[(size_t)(vv) * W + (uu)])
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            int32_t x = 0, y = 0;
            if (u > 0 && u < W - 1 && v > 0 && v < H - 1) {
                x = (PIX(u + 1, v - 1) - PIX(u - 1, v - 1)) + 2 * (PIX(u + 1, v) - PIX(u - 1, v)) +
                    (PIX(u + 1, v + 1) - PIX(u - 1, v + 1));
                y = (PIX(u - 1, v + 1) - PIX(u - 1, v - 1)) + 2 * (PIX(u, v + 1) - PIX(u, v - 1)) +
                    (PIX(u + 1, v + 1) - PIX(u + 1, v - 1));
            }
            gx[(size_t)v * W + u] = (int16_t)x;
            gy[(size_t)v * W + u] = (int16_t)y;
        }
#undef PIX
}

/* ------------------------------------------------------------------------------------------------ */
/* Alg. 5: dense V_px accumulator.  The listing is not self-consistent; the reading follows the text  */
/* around it: row j holds minus rho times the votes of the band of rows [j - chi, j + chi], clipped to */
/* the road rows [v_top, H - 1] (so the band is thinner at both ends).                               */
/* ------------------------------------------------------------------------------------------------ */
void or_band(const int32_t *votes, int32_t W, int32_t H, int32_t v_top, int32_t chi, int32_t rho, int32_t literal_bottom,
             int32_t *m_x)
{
    memset(m_x, 0, sizeof(int32_t) * (size_t)W * H);
    for (int32_t j = v_top; j < H; j++) {
        int32_t lo = j - chi < v_top ? v_top : j - chi;
        /* band_literal_bottom: the bottom rows j > v_max - chi - 1 use the band [j, v_max] of Alg. 5's listing */
        if (literal_bottom && j > H - 1 - chi - 1)
            lo = j;
        int32_t hi = j + chi > H - 1 ? H - 1 : j + chi;
        for (int32_t u = 0; u < W; u++) {
            int32_t s = 0;
            for (int32_t r = lo; r <= hi; r++)
                s += votes[(size_t)r * W + u];
            m_x[(size_t)j * W + u] = -rho * s;
        }
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Eq. 18: DP over the accumulator from row H-1 up to v_top.                                        */
/*   E_{H-1}(u) = m_x(u, H-1)                                                                        */
/*   E_v(u)     = m_x(u, v) + min_{tau in [-tau_x, tau_x], 0 <= u+tau < W} [E_{v+1}(u+tau) + lambda |tau|] */
/* Reading: the smoothness term is lambda_x |tau| (a signed term would reward moving left).  tau is    */
/* scanned 0, -1, +1, -2, +2, ... and only a strictly smaller candidate replaces the best; the path    */
/* starts at the smallest u minimising E_{v_top}.  path_u[v] receives the column at row v.           */
/* ------------------------------------------------------------------------------------------------ */
int64_t or_dp_vpx(const int32_t *m_x, int32_t W, int32_t H, int32_t v_top, int32_t tau, int32_t lambda,
                  int16_t *path_u)
{
    int64_t *Ep = (int64_t *)malloc(sizeof(int64_t) * W);
    int64_t *Ec = (int64_t *)malloc(sizeof(int64_t) * W);
    int8_t *bt = (int8_t *)calloc((size_t)W * H, 1);
    for (int32_t u = 0; u < W; u++)
        Ep[u] = m_x[(size_t)(H - 1) * W + u];
    for (int32_t v = H - 2; v >= v_top; v--) {
        for (int32_t u = 0; u < W; u++) {
            int64_t best = INT64_MAX;
            int32_t arg = 0;
            for (int32_t k = 0; k <= 2 * tau; k++) {
                int32_t t = (k & 1) ? -((k + 1) / 2) : k / 2;
                int32_t uu = u + t;
                if (uu < 0 || uu >= W)
                    continue;
                int64_t cand = Ep[uu] + (int64_t)lambda * (t < 0 ? -t : t);
                if (cand < best) {
                    best = cand;
                    arg = t;
                }
            }
            Ec[u] = (int64_t)m_x[(size_t)v * W + u] + best;
            bt[(size_t)v * W + u] = (int8_t)arg;
        }
        int64_t *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    int32_t ub = 0;
    for (int32_t u = 1; u < W; u++)
        if (Ep[u] < Ep[ub])
            ub = u;
    int64_t emin = Ep[ub];
    path_u[v_top] = (int16_t)ub;
    for (int32_t v = v_top; v < H - 1; v++)
        path_u[v + 1] = (int16_t)(path_u[v] + bt[(size_t)v * W + path_u[v]]);
    free(Ep);
    free(Ec);
    free(bt);
    return emin;
}

/* ------------------------------------------------------------------------------------------------ */
/* Alg. 7: M_0 = box sum of G_x w_g over (2 nu + 1) x (2 varsigma + 1); M_1 = G conv M_0 with the      */
/* Sobel kernel G = [1,2,1]^T [1,0,-1] (as a convolution: M_1 = sum w_dv [M_0(u+1) - M_0(u-1)]).      */
/* Both use zero padding outside the image.                                                          */
/* ------------------------------------------------------------------------------------------------ */
void or_box_sobel(const int32_t *gw, int32_t W, int32_t H, int32_t nu, int32_t vs, int32_t *m0, int32_t *m1)
{
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            int32_t s = 0;
            for (int32_t y = -vs; y <= vs; y++)
                for (int32_t x = -nu; x <= nu; x++) {
                    int32_t uu = u + x, vv = v + y;
                    if (uu >= 0 && uu < W && vv >= 0 && vv < H)
                        s += gw[(size_t)vv * W + uu];
                }
            m0[(size_t)v * W + u] = s;
        }
    static const int32_t wv[3] = {1, 2, 1};
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            int32_t s = 0;
            for (int32_t y = -1; y <= 1; y++) {
                int32_t vv = v + y;
                if (vv < 0 || vv >= H)
                    continue;
                int32_t r = (u + 1 < W) ? m0[(size_t)vv * W + u + 1] : 0;
                int32_t l = (u - 1 >= 0) ? m0[(size_t)vv * W + u - 1] : 0;
                s += wv[y + 1] * (r - l);
            }
            m1[(size_t)v * W + u] = s;
        }
}

/* ------------------------------------------------------------------------------------------------ */
/* Eq. 24-25: energy of the track started at every bottom-row position s = i - S0.                   */
/* u_{H-1} = s; each step up, u_v = (V_px(v+1) + v u_{v+1} - V_py(v+1) u_{v+1}) / (v + 1 - V_py(v+1))   */
/* in float32 with exactly this operation order; the track reads M_1 at column floor(u_v + 0.5) (0 when */
/* off the image) and E = M_1 + lambda_g E from row H-1 up to v_top.                                 */
/* ------------------------------------------------------------------------------------------------ */
void or_energy(const int32_t *m1, int32_t W, int32_t H, int32_t v_top, const float *Vpx, const float *Vpy,
               int32_t S0, int32_t n_starts, int32_t lambda_g, int64_t *he)
{
    for (int32_t i = 0; i < n_starts; i++) {
        float u = (float)(i - S0);
        int64_t E = 0;
        for (int32_t v = H - 1; v >= v_top; v--) {
            if (v < H - 1) {
                float vx = Vpx[v + 1], vy = Vpy[v + 1];
                float num = (vx + (float)v * u) - vy * u;
                float den = (float)(v + 1) - vy;
                u = num / den;
            }
            float col = floorf(u + 0.5f);
            int64_t m = 0;
            if (col >= 0.0f && col < (float)W)
                m = m1[(size_t)v * W + (int32_t)col];
            E = m + (int64_t)lambda_g * E;
        }
        he[i] = E;
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Alg. 7, last step: a selected lane is drawn by iterating Eq. 25 from its start (s, H-1) up to v_top.  */
/* u_out[v] is the track's column at row v in float32 with the operation order of or_energy (the     */
/* positions whose rounded columns the lane's energy summed); rows above v_top get NaN.               */
/* ------------------------------------------------------------------------------------------------ */
void or_track(const float *Vpx, const float *Vpy, int32_t H, int32_t v_top, int32_t start_u, float *u_out)
{
    for (int32_t v = 0; v < H; v++)
        u_out[v] = NAN;
    float u = (float)start_u;
    for (int32_t v = H - 1; v >= v_top && v >= 0; v--) {
        if (v < H - 1) {
            float vx = Vpx[v + 1], vy = Vpy[v + 1];
            float num = (vx + (float)v * u) - vy * u;
            float den = (float)(v + 1) - vy;
            u = num / den;
        }
        u_out[v] = u;
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Alg. 7 selection: strict interior local minima of H whose energy is below t, then suppression of    */
/* nearby minima.  Readings: t = ceil(thr * min H) (a fraction of the deepest minimum, since the       */
/* energy scale depends on image contrast); candidates are taken in increasing (energy, position) and  */
/* one within near_px of an accepted lane is dropped; at most max_lanes lanes, reported by position.   */
/* ------------------------------------------------------------------------------------------------ */
void or_select(const int64_t *he, int32_t n_starts, int32_t S0, const or_params *p, or_lanes *out)
{
    out->n_lanes = 0;
    int64_t mn = 0;
    for (int32_t i = 0; i < n_starts; i++)
        if (i == 0 || he[i] < mn)
            mn = he[i];
    if (n_starts < 3 || mn >= 0) {
        out->flags |= OR_F_NO_LANES;
        return;
    }
    int64_t t = p->thr_abs != 0 ? p->thr_abs : -(((-mn) * p->thr_num) / p->thr_den);
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * n_starts);
    int32_t nc = 0;
    for (int32_t i = 1; i < n_starts - 1; i++)
        if (he[i] < he[i - 1] && he[i] < he[i + 1] && he[i] < t)
            cand[nc++] = i;
    /* insertion sort by (energy, position) */
    for (int32_t a = 1; a < nc; a++) {
        int32_t c = cand[a], b = a - 1;
        while (b >= 0 && (he[cand[b]] > he[c] || (he[cand[b]] == he[c] && cand[b] > c))) {
            cand[b + 1] = cand[b];
            b--;
        }
        cand[b + 1] = c;
    }
    int32_t acc[OR_MAX_LANES], na = 0;
    for (int32_t a = 0; a < nc && na < p->max_lanes; a++) {
        int32_t ok = 1;
        for (int32_t b = 0; b < na; b++)
            if (abs(cand[a] - acc[b]) <= p->near_px)
                ok = 0;
        if (ok)
            acc[na++] = cand[a];
    }
    free(cand);
    for (int32_t a = 1; a < na; a++) {
        int32_t c = acc[a], b = a - 1;
        while (b >= 0 && acc[b] > c) {
            acc[b + 1] = acc[b];
            b--;
        }
        acc[b + 1] = c;
    }
    out->n_lanes = na;
    for (int32_t a = 0; a < na; a++) {
        out->start_u[a] = acc[a] - S0;
        out->energy[a] = he[acc[a]];
    }
    if (na == 0)
        out->flags |= OR_F_NO_LANES;
}

/* ------------------------------------------------------------------------------------------------ */
/* The whole path on one frame, in the paper's order.                                               */
/* ------------------------------------------------------------------------------------------------ */
static double poly_f64(const double *c, int32_t m, double tau)
{
    double p = c[m - 1];
    for (int32_t k = m - 2; k >= 0; k--)
        p = p * tau + c[k];
    return p;
}

int32_t or_detect(const float *disp, const uint8_t *img, int32_t W, int32_t H, const or_params *p,
                  or_lanes *out, or_dumps *dumps)
{
    or_dumps nd;
    memset(&nd, 0, sizeof(nd));
    if (!dumps)
        dumps = &nd;
    memset(out, 0, sizeof(*out));
    int32_t D = p->n_disp;
    if (W < 8 || H < 8 || D < 4 || p->max_lanes > OR_MAX_LANES)
        return -1;
    size_t WH = (size_t)W * H;
    const int32_t vmax = H - 1;
    /* polynomial basis: tau = (v - centre) / 2^e with 2^e >= max |v - centre| */
    int32_t centre = (H - 1) / 2, e = 0;
    while ((1 << e) < (H - 1 - centre > centre ? H - 1 - centre : centre))
        e++;
    out->centre = centre;
    out->scale_exp = e;
    double sc = ldexp(1.0, -e);

    /* ---- Sec. 2.2: v-disparity, DP, RANSAC road fit ---- */
    int32_t *m_y = (int32_t *)malloc(sizeof(int32_t) * (size_t)H * D);
    or_vdisparity(disp, W, H, D, m_y);
    int16_t *path_y = (int16_t *)malloc(sizeof(int16_t) * D);
    if (p->dp_literal)
        or_dp_vdisp_literal(m_y, H, D, p->tau_y, p->lambda_y, path_y);
    else
        or_dp_vdisp(m_y, H, D, p->tau_y, p->lambda_y, path_y);
    /* Reading: a path point whose cell holds no count carries no observation (the path crosses empty */
    /* bins beyond the largest road disparity, for instance); M_y keeps the points with m_y > 0.        */
    int32_t cap = D > H ? D : H, k = 0;
    int32_t *px = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *py = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *pid = (int32_t *)malloc(sizeof(int32_t) * cap);
    uint8_t *mem = (uint8_t *)malloc(cap);
    for (int32_t d = 1; d < D; d++)
        if (m_y[(size_t)path_y[d] * D + d] > 0) {
            px[k] = path_y[d];
            py[k] = d;
            pid[k++] = d;
        }
    int32_t fy = or_ransac(px, py, k, 3, p->tr_y, 0, p, centre, e, mem, out->beta, &out->rounds_y);
    if (dumps->m_y)
        memcpy(dumps->m_y, m_y, sizeof(int32_t) * (size_t)H * D);
    if (dumps->path_y)
        memcpy(dumps->path_y, path_y, sizeof(int16_t) * D);
    if (dumps->inl_y) {
        memset(dumps->inl_y, 0, D);
        for (int32_t j = 0; j < k; j++)
            dumps->inl_y[pid[j]] = mem[j];
    }
    if (fy & 1)
        out->flags |= OR_F_CAP_Y;
    float *F = (float *)calloc(H, sizeof(float));
    float *Vpy = (float *)calloc(H, sizeof(float));
    float *Vpx = (float *)calloc(H, sizeof(float));
    int32_t v_top = H;
    if (fy & 2) {
        out->flags |= OR_F_DEGEN_Y;
    } else {
        /* Sec. 2.3.1 on-road rows: f^-1(0) <= v <= v_max.  Reading: on the row grid, v_top is the first */
        /* row of the bottom run of rows with f(v) > 0 and f'(v) > 0.                                     */
        for (int32_t v = vmax; v >= 0; v--) {
            double tau = (double)(v - centre) * sc;
            double fv = poly_f64(out->beta, 3, tau);
            double dfv = (out->beta[1] + (2.0 * out->beta[2]) * tau) * sc;
            if (!(fv > 0.0 && dfv > 0.0))
                break;
            v_top = v;
            F[v] = (float)fv;
            Vpy[v] = (float)((double)v - fv / dfv); /* Eq. 14 */
        }
        if (v_top > vmax)
            out->flags |= OR_F_NO_ROAD;
    }
    out->v_top = v_top;
    if (dumps->F)
        memcpy(dumps->F, F, sizeof(float) * H);
    if (dumps->Vpy)
        memcpy(dumps->Vpy, Vpy, sizeof(float) * H);

    if (out->flags & (OR_F_DEGEN_Y | OR_F_NO_ROAD)) {
        out->flags |= OR_F_NO_LANES;
        goto done_early;
    }

    /* ---- Sec. 2.3.1: road mask, bilateral filter, Sobel edges, sparse V_px votes ---- */
    {
        uint8_t *Ibf = (uint8_t *)malloc(WH);
        if (p->bilateral == 2)
            or_median(img, W, H, p->bf_rho, Ibf);
        else if (p->bilateral)
            or_bilateral(img, W, H, p, Ibf);
        else
            memcpy(Ibf, img, WH);
        int16_t *gx = (int16_t *)malloc(sizeof(int16_t) * WH);
        int16_t *gy = (int16_t *)malloc(sizeof(int16_t) * WH);
        or_sobel(Ibf, W, H, gx, gy);
        uint8_t *edge = (uint8_t *)calloc(WH, 1);
        int32_t *votes = (int32_t *)calloc(WH, sizeof(int32_t));
        int64_t thr2 = (int64_t)p->edge_thresh * p->edge_thresh;
        for (int32_t v = v_top; v <= vmax; v++)
            for (int32_t u = 0; u < W; u++) {
                size_t o = (size_t)v * W + u;
                float l = disp[o];
                int32_t road = isfinite(l) && l > 0.0f && fabsf(l - F[v]) <= p->varpi;
                int64_t g2 = (int64_t)gx[o] * gx[o] + (int64_t)gy[o] * gy[o];
                if (!road || g2 <= thr2)
                    continue;
                edge[o] = 1;
                if (gx[o] == 0)
                    continue;
                /* Eq. 17, with 1/grad read as G_y / G_x: the edge line through (u, v), perpendicular to */
                /* the gradient, meets row V_py(v) at column u + (v - V_py) G_y / G_x.                    */
                float a = (float)v - Vpy[v];
                float b = a * (float)gy[o];
                float q = b / (float)gx[o];
                float vs = (float)u + q;
                float col = floorf(vs + 0.5f);
                if (col >= 0.0f && col < (float)W)
                    votes[(size_t)v * W + (int32_t)col] += 1;
            }
        if (dumps->Ibf)
            memcpy(dumps->Ibf, Ibf, WH);
        if (dumps->edge)
            memcpy(dumps->edge, edge, WH);
        if (dumps->Gx)
            for (size_t o = 0; o < WH; o++)
                dumps->Gx[o] = edge[o] ? gx[o] : 0;
        if (dumps->Gy)
            for (size_t o = 0; o < WH; o++)
                dumps->Gy[o] = edge[o] ? gy[o] : 0;
        if (dumps->votes)
            memcpy(dumps->votes, votes, sizeof(int32_t) * WH);

        /* ---- Sec. 2.3.2-2.3.3: band accumulator, DP, RANSAC quartic, V_px ---- */
        int32_t *m_x = (int32_t *)malloc(sizeof(int32_t) * WH);
        or_band(votes, W, H, v_top, p->chi, p->vote_rho, p->band_literal_bottom, m_x);
        if (dumps->m_x)
            memcpy(dumps->m_x, m_x, sizeof(int32_t) * WH);
        int16_t *path_x = (int16_t *)calloc(H, sizeof(int16_t));
        or_dp_vpx(m_x, W, H, v_top, p->tau_x, p->lambda_x, path_x);
        if (dumps->path_x)
            memcpy(dumps->path_x, path_x, sizeof(int16_t) * H);
        /* as for M_y, a row whose path cell holds no vote carries no observation */
        int32_t t = 0;
        for (int32_t v = v_top; v <= vmax; v++)
            if (m_x[(size_t)v * W + path_x[v]] != 0) {
                px[t] = v;
                py[t] = path_x[v];
                pid[t++] = v;
            }
        int32_t fx = or_ransac(px, py, t, 5, p->tr_x, 1, p, centre, e, mem, out->gamma, &out->rounds_x);
        if (dumps->inl_x) {
            memset(dumps->inl_x, 0, H);
            for (int32_t j = 0; j < t; j++)
                dumps->inl_x[pid[j]] = mem[j];
        }
        if (fx & 1)
            out->flags |= OR_F_CAP_X;
        int32_t *Gw = NULL, *M0 = NULL, *M1 = NULL;
        int64_t *he = NULL;
        if (fx & 2) {
            out->flags |= OR_F_DEGEN_X | OR_F_NO_LANES;
        } else {
            for (int32_t v = v_top; v <= vmax; v++)
                Vpx[v] = (float)poly_f64(out->gamma, 5, (double)(v - centre) * sc); /* Eq. 22 */

            /* ---- Sec. 2.4: w_g, M_0, M_1, energies, selection ---- */
            int32_t *wg = (int32_t *)malloc(sizeof(int32_t) * 16385);
            or_tables(p, NULL, NULL, wg);
            Gw = (int32_t *)calloc(WH, sizeof(int32_t));
            for (int32_t v = v_top; v <= vmax; v++)
                for (int32_t u = 0; u < W; u++) {
                    size_t o = (size_t)v * W + u;
                    if (!edge[o])
                        continue;
                    /* Eq. 23.  theta_e is the direction of the edge (the gradient turned by 90 degrees), */
                    /* theta_Vp the direction from the pixel to V_p(v); lines are undirected, so the       */
                    /* angle between them is taken in [0, pi/2] through s = sin^2(dtheta).                */
                    float tu = (float)(-gy[o]), tv = (float)gx[o];
                    float ru = Vpx[v] - (float)u, rv = Vpy[v] - (float)v;
                    float cr = tu * rv - tv * ru;
                    float num = cr * cr;
                    float den = (tu * tu + tv * tv) * (ru * ru + rv * rv);
                    int32_t w = 0;
                    if (den > 0.0f) {
                        float s = num / den;
                        if (s <= 0.25f)
                            w = wg[(int32_t)(sqrtf(s) * 32768.0f)];
                    }
                    Gw[o] = (int32_t)gx[o] * w;
                }
            free(wg);
            M0 = (int32_t *)malloc(sizeof(int32_t) * WH);
            M1 = (int32_t *)malloc(sizeof(int32_t) * WH);
            or_box_sobel(Gw, W, H, p->box_nu, p->box_vs, M0, M1);
            int32_t ns = or_n_starts(W, p);
            int32_t S0 = (ns - W) / 2;
            he = (int64_t *)malloc(sizeof(int64_t) * ns);
            or_energy(M1, W, H, v_top, Vpx, Vpy, S0, ns, p->lambda_g, he);
            or_select(he, ns, S0, p, out);
            if (dumps->HE)
                memcpy(dumps->HE, he, sizeof(int64_t) * ns);
        }
        if (dumps->Vpx)
            memcpy(dumps->Vpx, Vpx, sizeof(float) * H);
        if (dumps->Gw) {
            if (Gw)
                memcpy(dumps->Gw, Gw, sizeof(int32_t) * WH);
            else
                memset(dumps->Gw, 0, sizeof(int32_t) * WH);
        }
        if (dumps->M1) {
            if (M1)
                memcpy(dumps->M1, M1, sizeof(int32_t) * WH);
            else
                memset(dumps->M1, 0, sizeof(int32_t) * WH);
        }
        free(Ibf);
        free(gx);
        free(gy);
        free(edge);
        free(votes);
        free(m_x);
        free(path_x);
        free(Gw);
        free(M0);
        free(M1);
        free(he);
    }
done_early:
    free(m_y);
    free(path_y);
    free(px);
    free(py);
    free(pid);
    free(mem);
    free(F);
    free(Vpy);
    free(Vpx);
    return 0;
}

/* ================================================================================================ */
/* Sec. 2.1 stereo matching: block statistics through integral images (Alg. 1, Eq. 4-5), the NCC cost */
/* (Eq. 1-8), search range propagation (Eq. 9, Alg. 2) and the left-right consistency check (Alg. 3). */
/*                                                                                                  */
/* Readings.  Blocks are (2 rho + 1)^2 and must lie inside both images: rows rho .. H-1-rho, columns  */
/* rho .. W-1-rho, and a candidate d only while the other image's block stays inside; pixels with no */
/* candidate get 0.  With s the block sum, Q the sum of squares, P the sum of products and n the     */
/* block size, Eq. 8 is c = (n P - s_l s_r) / sqrt(D_l D_r), D = n Q - s^2 (multiply Eq. 8's numerator */
/* and denominator by n); c = 0 where D_l D_r = 0 (then the numerator is 0 as well).  The best d has  */
/* the largest c, compared exactly in integers (below), ties to the smaller d.  Rows are estimated   */
/* from H-1-rho up to rho; the first over the full range [0, d_max], each later pixel over the union  */
/* of [l - tau, l + tau] for the three estimates below it that exist.  The right map matches the     */
/* right image's block at (u, v) with the left image's at (u + d, v).  LRC keeps l_lf(u, v) when      */
/* |l_lf(u, v) - l_rt(u - l_lf(u, v), v)| <= tr, else 0.                                             */
/* ================================================================================================ */

/* Alg. 1: In(u, v) = sum of I over [0, u] x [0, v], by the serial recurrence; stored with a zero     */
/* first row and column so that In(-1, .) = In(., -1) = 0: entry (v + 1) * (W + 1) + (u + 1).          */
void or_integral(const uint8_t *img, int32_t W, int32_t H, int32_t square, int64_t *In)
{
    const int32_t Wp = W + 1;
    for (int32_t u = 0; u <= W; u++)
        In[u] = 0;
    for (int32_t v = 0; v < H; v++) {
        In[(size_t)(v + 1) * Wp] = 0;
        for (int32_t u = 0; u < W; u++) {
            int64_t x = img[(size_t)v * W + u];
            if (square)
                x *= x;
            In[(size_t)(v + 1) * Wp + u + 1] = x + In[(size_t)(v + 1) * Wp + u] + In[(size_t)v * Wp + u + 1] -
                                               In[(size_t)v * Wp + u];
        }
    }
}

/* Eq. 5: block sums from four references of the integral images; s and D = n Q - s^2 at every pixel */
/* whose block lies inside the image (0 elsewhere).                                                 */
void or_block_stats(const uint8_t *img, int32_t W, int32_t H, int32_t rho, int32_t *s, int64_t *D)
{
    const int32_t Wp = W + 1;
    const int64_t n = (int64_t)(2 * rho + 1) * (2 * rho + 1);
    int64_t *In = (int64_t *)malloc(sizeof(int64_t) * (size_t)(W + 1) * (H + 1));
    int64_t *In2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(W + 1) * (H + 1));
    or_integral(img, W, H, 0, In);
    or_integral(img, W, H, 1, In2);
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            size_t o = (size_t)v * W + u;
            if (v < rho || v > H - 1 - rho || u < rho || u > W - 1 - rho) {
                s[o] = 0;
                D[o] = 0;
                continue;
            }
            /* r1 = In(u + rho, v + rho), r2 = In(u - rho - 1, v - rho - 1), r3 = In(u - rho - 1, v + rho),
               r4 = In(u + rho, v - rho - 1); s = r1 + r2 - r3 - r4 (padded indices are +1) */
            size_t a = (size_t)(v + rho + 1) * Wp + (u + rho + 1), b = (size_t)(v - rho) * Wp + (u - rho);
            size_t c = (size_t)(v + rho + 1) * Wp + (u - rho), d = (size_t)(v - rho) * Wp + (u + rho + 1);
            int64_t s1 = In[a] + In[b] - In[c] - In[d];
            int64_t q1 = In2[a] + In2[b] - In2[c] - In2[d];
            s[o] = (int32_t)s1;
            D[o] = n * q1 - s1 * s1;
        }
    free(In);
    free(In2);
}

/* Sign of c1 - c2 for c = N / sqrt(D_a D_b) with a common D_a > 0: c1 > c2 compared as                */
/* N1 |N1| D2 > N2 |N2| D1 in 128-bit integers (the square root never taken); D = 0 means c = 0.     */
int32_t or_ncc_cmp(int64_t N1, int64_t D1, int64_t N2, int64_t D2)
{
    if (D1 == 0)
        N1 = 0;
    if (D2 == 0)
        N2 = 0;
    __int128 l = (__int128)N1 * (N1 < 0 ? -N1 : N1) * (D2 == 0 ? 1 : D2);
    __int128 r = (__int128)N2 * (N2 < 0 ? -N2 : N2) * (D1 == 0 ? 1 : D1);
    if (N1 == 0 && N2 == 0)
        return 0;
    if (N1 == 0)
        return N2 > 0 ? -1 : 1;
    if (N2 == 0)
        return N1 > 0 ? 1 : -1;
    return l > r ? 1 : (l < r ? -1 : 0);
}

/* Eq. 9, Alg. 2: one disparity map by search range propagation.  dir 0: the left map (blocks of a   */
/* at u against b at u - d); dir 1: the right map (a at u against b at u + d).                        */
void or_srp(const uint8_t *a, const uint8_t *b, int32_t W, int32_t H, int32_t rho, int32_t dmax, int32_t tau,
            int32_t dir, int16_t *out)
{
    const int64_t n = (int64_t)(2 * rho + 1) * (2 * rho + 1);
    int32_t *sa = (int32_t *)malloc(sizeof(int32_t) * (size_t)W * H), *sb = (int32_t *)malloc(sizeof(int32_t) * (size_t)W * H);
    int64_t *Da = (int64_t *)malloc(sizeof(int64_t) * (size_t)W * H), *Db = (int64_t *)malloc(sizeof(int64_t) * (size_t)W * H);
    or_block_stats(a, W, H, rho, sa, Da);
    or_block_stats(b, W, H, rho, sb, Db);
    memset(out, 0, sizeof(int16_t) * (size_t)W * H);
    for (int32_t v = H - 1 - rho; v >= rho; v--) {
        for (int32_t u = rho; u <= W - 1 - rho; u++) {
            /* candidate disparities: d in [0, dmax] with the other block inside */
            int32_t dhi = dir == 0 ? u - rho : W - 1 - rho - u;
            if (dhi > dmax)
                dhi = dmax;
            int32_t best = -1;
            int64_t bN = 0, bD = 0;
            for (int32_t d = 0; d <= dhi; d++) {
                if (v < H - 1 - rho) {
                    int32_t in = 0;
                    for (int32_t k = u - 1; k <= u + 1; k++) {
                        if (k < rho || k > W - 1 - rho)
                            continue;
                        int32_t l = out[(size_t)(v + 1) * W + k];
                        if (d >= l - tau && d <= l + tau)
                            in = 1;
                    }
                    if (!in)
                        continue;
                }
                int32_t ub = dir == 0 ? u - d : u + d;
                int64_t P = 0;
                for (int32_t y = v - rho; y <= v + rho; y++)
                    for (int32_t x = -rho; x <= rho; x++)
                        P += (int64_t)a[(size_t)y * W + u + x] * b[(size_t)y * W + ub + x];
                size_t oa = (size_t)v * W + u, ob = (size_t)v * W + ub;
                int64_t N = n * P - (int64_t)sa[oa] * sb[ob];
                if (Da[oa] == 0)
                    N = 0;
                if (best < 0 || or_ncc_cmp(N, Db[ob], bN, bD) > 0) {
                    best = d;
                    bN = N;
                    bD = Db[ob];
                }
            }
            out[(size_t)v * W + u] = (int16_t)(best < 0 ? 0 : best);
        }
    }
    free(sa);
    free(sb);
    free(Da);
    free(Db);
}

/* Alg. 3: left-right consistency. */
void or_lrc(const int16_t *lf, const int16_t *rt, int32_t W, int32_t H, int32_t tr, int16_t *out)
{
    for (int32_t v = 0; v < H; v++)
        for (int32_t u = 0; u < W; u++) {
            int32_t l = lf[(size_t)v * W + u];
            int32_t x = u - l;
            int32_t ok = x >= 0 && abs(l - rt[(size_t)v * W + x]) <= tr;
            out[(size_t)v * W + u] = (int16_t)(ok ? l : 0);
        }
}

/* The disparity map of a rectified pair: both SRP maps, then LRC. */
void or_stereo(const uint8_t *left, const uint8_t *right, int32_t W, int32_t H, int32_t rho, int32_t dmax,
               int32_t tau, int32_t tr, int16_t *lf, int16_t *rt, int16_t *disp)
{
    or_srp(left, right, W, H, rho, dmax, tau, 0, lf);
    or_srp(right, left, W, H, rho, dmax, tau, 1, rt);
    or_lrc(lf, rt, W, H, tr, disp);
}
