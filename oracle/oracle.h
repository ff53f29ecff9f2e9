/*
 * CPU oracle of the stereo lane-detection path (Fan & Dahnoun, arXiv 1807.02752, Sec. 2.2-2.4).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded restatement of the paper's steps,
 * used to check the CUDA library.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the library never calls it.  It shares no source with the CUDA path.
 *
 * Every function takes host pointers; arrays are row-major [H][W] with row v = 0 at the top.
 */
#ifndef LD_ORACLE_H
#define LD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_LANES 8

/* per-frame flags */
#define OR_F_NO_ROAD 1      /* no row range with f > 0 and f' > 0 at the bottom of the image */
#define OR_F_CAP_Y 2        /* beta RANSAC hit its round cap */
#define OR_F_DEGEN_Y 4      /* beta fit impossible (too few points / singular) */
#define OR_F_CAP_X 8        /* gamma RANSAC hit its round cap */
#define OR_F_DEGEN_X 16     /* gamma fit impossible */
#define OR_F_NO_LANES 32    /* no lane passed validation */

typedef struct or_params {
    int32_t n_disp;          /* D, bins of the v-disparity map */
    int32_t tau_y;           /* Eq. 12: tau_y in [0, tau_y] */
    int32_t lambda_y;        /* Eq. 12 smoothness weight */
    float tr_y;              /* Sec. 2.2: squared-residual tolerance of the road fit (4) */
    int32_t eps_num, eps_den;/* inlier-fraction stop test eps = eps_num/eps_den (0.99) */
    float varpi;             /* Sec. 2.3.1: on-road tolerance (3) */
    int32_t bilateral;       /* 1: bilateral pre-filter (Eq. 15-16); 2: median filter over the same window
                                (the filter of the authors' previous system, Sec. 2.3.1); 0: none */
    int32_t bf_rho;          /* window half-size (5 -> 11x11) */
    double sigma_s, sigma_r; /* Eq. 16 (300, 0.3; intensities scaled to [0,1]) */
    int32_t edge_thresh;     /* Sobel magnitude threshold (100) */
    int32_t vote_rho;        /* Alg. 5 vote weight (1) */
    int32_t chi;             /* Alg. 5 band half-height (25) */
    int32_t tau_x;           /* Eq. 18: tau_x in [-tau_x, tau_x] */
    int32_t lambda_x;        /* Eq. 18 smoothness weight */
    float tr_x;              /* Sec. 2.3.3 tolerance (16) */
    double sigma_g;          /* Eq. 23 (3.5) */
    int32_t box_nu, box_vs;  /* Alg. 7 box half-sizes nu, varsigma (1, 3) */
    int32_t lambda_g;        /* Eq. 24 (1) */
    int32_t xi_num, xi_den;  /* xi = 1/2: starts in [-xi W, (1+xi) W) */
    int32_t thr_num, thr_den;/* lane threshold t = thr * min(H_E) (1/4) */
    int32_t near_px;         /* suppression distance of nearby minima (30) */
    int32_t max_lanes;       /* <= OR_MAX_LANES */
    int32_t ransac_hyps;     /* hypotheses drawn per RANSAC round (64) */
    int32_t ransac_rounds;   /* round cap (64) */
    uint64_t seed;           /* Philox key */
    int32_t wg_gaussian;     /* 0: Eq. 23 as printed, exp(-p / sigma_g^2); 1: the Gaussian the text names,
                                exp(-p^2 / sigma_g^2); p = dtheta / (pi / 36) */
    int32_t pad0;
    int64_t thr_abs;         /* 0: t = ceil(thr * min H); < 0: the absolute threshold t = thr_abs */
    int32_t dp_literal;      /* 1: Eq. 12 as printed (links to row v - tau, reward -lambda tau) */
    int32_t band_literal_bottom; /* 1: Alg. 5's listing for the bottom rows j > v_max - chi - 1: band [j, v_max] */
} or_params;

typedef struct or_lanes {
    int32_t n_lanes, flags;
    int32_t start_u[OR_MAX_LANES];   /* bottom-row start position of each lane, ascending */
    int64_t energy[OR_MAX_LANES];
    int32_t v_top;                   /* first road row, ceil(f^-1(0)) on the row grid */
    int32_t centre, scale_exp;       /* polynomial basis: tau = (v - centre) / 2^scale_exp */
    double beta[3];                  /* f(v) in the tau basis */
    double gamma[5];                 /* g(v) in the tau basis */
    int32_t rounds_y, rounds_x;
} or_lanes;

/* Intermediate results; any pointer may be NULL.  Sizes: H, W, D of the frame. */
typedef struct or_dumps {
    int32_t *m_y;        /* [H][D] v-disparity histogram */
    int16_t *path_y;     /* [D] row of the DP path at each d (entry 0 unused) */
    uint8_t *inl_y;      /* [D] final RANSAC membership of path point d (0 for points without data) */
    float *F;            /* [H] f(v) as float (0 above v_top) */
    float *Vpy;          /* [H] */
    uint8_t *Ibf;        /* [H][W] bilateral output */
    uint8_t *edge;       /* [H][W] 1 on road edge pixels */
    int16_t *Gx, *Gy;    /* [H][W] Sobel derivatives, kept on road edge pixels only */
    int32_t *votes;      /* [H][W] per-row histogram of sparse V_px votes c(u, v) */
    int32_t *m_x;        /* [H][W] dense accumulator */
    int16_t *path_x;     /* [H] column of the DP path at each row (rows v_top..H-1) */
    uint8_t *inl_x;      /* [H] final RANSAC membership of path point at row v */
    float *Vpx;          /* [H] */
    int32_t *Gw;         /* [H][W] G_x * w_g (Q12) */
    int32_t *M1;         /* [H][W] */
    int64_t *HE;         /* [n_starts] energy histogram H */
} or_dumps;

void or_default_params(or_params *p);
int32_t or_n_starts(int32_t W, const or_params *p);

/* LUTs: ws_q[(2rho+1)^2] and wr_q[256] in Q15; wg_q[16385] in Q12, indexed by floor(sin(dtheta) * 2^15). */
void or_tables(const or_params *p, int32_t *ws_q, int32_t *wr_q, int32_t *wg_q);
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

void or_vdisparity(const float *disp, int32_t W, int32_t H, int32_t D, int32_t *m_y);
int64_t or_dp_vdisp(const int32_t *m_y, int32_t H, int32_t D, int32_t tau, int32_t lambda, int16_t *path_v);
int64_t or_dp_vdisp_literal(const int32_t *m_y, int32_t H, int32_t D, int32_t tau, int32_t lambda, int16_t *path_v);
int32_t or_lsf(const int32_t *x, const int32_t *y, const uint8_t *use, int32_t n, int32_t m,
               int32_t centre, int32_t e, double *coef);
int32_t or_hypothesis(const int32_t *x, const int32_t *y, const uint8_t *member, int32_t n, int32_t m,
                      float tr, int32_t stage, int32_t round, int32_t hyp, const or_params *p,
                      int32_t centre, int32_t e, int32_t *chosen, uint8_t *inliers);
int32_t or_ransac(const int32_t *x, const int32_t *y, int32_t n, int32_t m, float tr, int32_t stage,
                  const or_params *p, int32_t centre, int32_t e, uint8_t *member, double *coef,
                  int32_t *rounds);
void or_bilateral(const uint8_t *img, int32_t W, int32_t H, const or_params *p, uint8_t *out);
void or_median(const uint8_t *img, int32_t W, int32_t H, int32_t rho, uint8_t *out);
void or_sobel(const uint8_t *I, int32_t W, int32_t H, int16_t *gx, int16_t *gy);
void or_band(const int32_t *votes, int32_t W, int32_t H, int32_t v_top, int32_t chi, int32_t rho,
             int32_t literal_bottom, int32_t *m_x);
int64_t or_dp_vpx(const int32_t *m_x, int32_t W, int32_t H, int32_t v_top, int32_t tau, int32_t lambda,
                  int16_t *path_u);
void or_box_sobel(const int32_t *gw, int32_t W, int32_t H, int32_t nu, int32_t vs, int32_t *m0, int32_t *m1);
void or_energy(const int32_t *m1, int32_t W, int32_t H, int32_t v_top, const float *Vpx, const float *Vpy,
               int32_t S0, int32_t n_starts, int32_t lambda_g, int64_t *he);
void or_select(const int64_t *he, int32_t n_starts, int32_t S0, const or_params *p, or_lanes *out);
void or_track(const float *Vpx, const float *Vpy, int32_t H, int32_t v_top, int32_t start_u, float *u_out);

/* Sec. 2.1 stereo matching (the disparity the path takes as input).  Integral images are (W+1) x (H+1)
   with a zero first row and column; block statistics s (sum) and D = n Q - s^2 per pixel; maps int16. */
void or_integral(const uint8_t *img, int32_t W, int32_t H, int32_t square, int64_t *In);
void or_block_stats(const uint8_t *img, int32_t W, int32_t H, int32_t rho, int32_t *s, int64_t *D);
int32_t or_ncc_cmp(int64_t N1, int64_t D1, int64_t N2, int64_t D2);
void or_srp(const uint8_t *a, const uint8_t *b, int32_t W, int32_t H, int32_t rho, int32_t dmax, int32_t tau,
            int32_t dir, int16_t *out);
void or_lrc(const int16_t *lf, const int16_t *rt, int32_t W, int32_t H, int32_t tr, int16_t *out);
void or_stereo(const uint8_t *left, const uint8_t *right, int32_t W, int32_t H, int32_t rho, int32_t dmax,
               int32_t tau, int32_t tr, int16_t *lf, int16_t *rt, int16_t *disp);

/* The whole path on one frame.  Returns 0, or -1 on bad arguments / allocation failure. */
int32_t or_detect(const float *disp, const uint8_t *img, int32_t W, int32_t H, const or_params *p,
                  or_lanes *out, or_dumps *dumps);

#ifdef __cplusplus
}
#endif
#endif
