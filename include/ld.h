/*
 * ld.h - C-ABI of the GB300 lane-detection library.
 *
 * The library runs the per-frame dense path of Fan & Dahnoun, "Real-Time Stereo Vision-Based Lane
 * Detection System" (arXiv 1807.02752, Sec. 2.2-2.4) on an NVIDIA GB300 (sm_103a): from a disparity map
 * and the left image of each frame to the validated lane positions (the lane vector Gamma of Alg. 7).
 *
 *   Sec. 2.2  v-disparity histogram, DP (Eq. 11-12), RANSAC road profile (Alg. 4, Eq. 13), V_py (Eq. 14)
 *   Sec. 2.3  road mask, bilateral filter (Eq. 15-16), Sobel, sparse V_px votes (Eq. 17), dense
 *             accumulator (Alg. 5), DP (Eq. 18), RANSAC quartic (Alg. 6, Eq. 19-21), V_px (Eq. 22)
 *   Sec. 2.4  w_g (Eq. 23), M_0 / M_1 and lane energies (Alg. 7, Eq. 24-25), local-minimum selection
 *
 * Conventions for every entry point:
 *   - images are row-major [n_frames][h][w], contiguous (pitch = w), row v = 0 at the top;
 *   - disparity is float32 (0 or non-finite = invalid), the image is uint8 grey;
 *   - return value LD_OK (0) or a negative LD_E_* code; ld_last_error() then describes it;
 *   - per-frame algorithmic outcomes (no road, degenerate fit, no lanes) are flags in ld_lanes, not errors;
 *   - nothing aborts, traps or waits without bound; a handle is not thread-safe (one handle per stream).
 */
#ifndef LD_H
#define LD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LD_MAX_LANES 8
#define LD_MAX_W 4096      /* widest frame */
#define LD_MAX_H 1088      /* tallest frame: keeps the exact quartic normal-equation sums below 2^85 */
#define LD_MAX_D 256       /* most disparity bins */

/* return codes */
#define LD_OK 0
#define LD_E_ARG (-1)      /* bad argument (null pointer, size out of range, invalid parameter) */
#define LD_E_CUDA (-2)     /* a CUDA runtime call failed; the message names it */
#define LD_E_NOMEM (-3)    /* device or pinned-host allocation failed (the *_create calls, ld_server_set_learned) */
#define LD_E_STATE (-4)    /* call not valid in the handle's current state (e.g. no detect yet) */
#define LD_E_BUSY (-5)     /* serving: no slot of the frame's size class can take it now (admission) */
#define LD_E_TIMEOUT (-6)  /* a bounded device-side wait ran out; the kernel stopped and released what it held */

/* per-frame flags (ld_lanes.flags) */
#define LD_F_NO_ROAD 1     /* no bottom run of rows with f(v) > 0 and f'(v) > 0 */
#define LD_F_CAP_Y 2       /* road-profile RANSAC stopped at its round cap */
#define LD_F_DEGEN_Y 4     /* road-profile fit impossible (too few points or singular system) */
#define LD_F_CAP_X 8       /* V_px RANSAC stopped at its round cap */
#define LD_F_DEGEN_X 16    /* V_px fit impossible */
#define LD_F_NO_LANES 32   /* no lane passed validation */
#define LD_F_FALLBACK 64   /* learned proposal: no lane among the proposed starts; the exhaustive search ran */

/*
 * Parameters: every constant of the method, named after the paper's symbols.  ld_params_default() fills
 * the paper's values (Sec. 2.2-2.4) and the readings of the points the paper leaves open.
 */
typedef struct ld_params {
    int32_t n_disp;           /* D, bins of the v-disparity map (<= LD_MAX_D) */
    int32_t tau_y;            /* Eq. 12: row step tau_y in [0, tau_y] (6) */
    int32_t lambda_y;         /* Eq. 12 smoothness weight (not given in the paper; 1) */
    float tr_y;               /* Sec. 2.2 squared-residual tolerance (4) */
    int32_t eps_num, eps_den; /* Alg. 4 / Alg. 6 stop fraction eps = 99/100 */
    float varpi;              /* Sec. 2.3.1 on-road tolerance |l - f(v)| <= varpi (3) */
    int32_t bilateral;        /* 1: Eq. 15-16 pre-filter before Sobel; 2: median filter over the same
                                 window (the pre-filter of the authors' previous system, Sec. 2.3.1: lower
                                 median of the in-image taps); 0: Sobel on the raw image */
    int32_t bf_rho;           /* bilateral window half-size rho, 1..5 (5 -> 11x11) */
    double sigma_s, sigma_r;  /* Eq. 16 (300, 0.3 with intensities scaled to [0,1]) */
    int32_t edge_thresh;      /* Sobel magnitude threshold (100) */
    int32_t vote_rho;         /* Alg. 5 vote weight varrho (1) */
    int32_t chi;              /* Alg. 5 band half-height chi (25) */
    int32_t tau_x;            /* Eq. 18 column step tau_x in [-tau_x, tau_x] (5, at most 7) */
    int32_t lambda_x;         /* Eq. 18 smoothness weight (not given; 1) */
    float tr_x;               /* Sec. 2.3.3 squared-residual tolerance (16) */
    double sigma_g;           /* Eq. 23 (3.5) */
    int32_t box_nu, box_vs;   /* Alg. 7 box half-sizes nu = 1, varsigma = 3 */
    int32_t lambda_g;         /* Eq. 24 recursion weight (1) */
    int32_t xi_num, xi_den;   /* xi = 1/2: lane starts s in [-floor(xi W), W + floor(xi W)) */
    int32_t thr_num, thr_den; /* lane threshold t = ceil(thr * min H) (not given; 1/32) */
    int32_t near_px;          /* minima closer than this are suppressed (not given; 30) */
    int32_t max_lanes;        /* <= LD_MAX_LANES */
    int32_t ransac_hyps;      /* hypotheses per RANSAC round (64, at most 256) */
    int32_t ransac_rounds;    /* RANSAC round cap (64) */
    uint64_t seed;            /* Philox4x32-10 key of the RANSAC draws */
    int32_t wg_gaussian;      /* 0: Eq. 23 as printed, w_g = exp(-p / sigma_g^2); 1: the Gaussian the
                                 Sec. 2.4 text names, exp(-p^2 / sigma_g^2); p = dtheta / (pi / 36) */
    int32_t pad0;             /* 0 */
    int64_t thr_abs;          /* 0: relative lane threshold (thr_num / thr_den); < 0: absolute, H < thr_abs */
    int32_t dp_literal;       /* 1: Eq. 12 as printed (the row v - tau, a -lambda_y tau reward); 0: the reading */
    int32_t band_literal_bottom; /* 1: Alg. 5's listing for the bottom rows j > v_max - chi - 1 (band [j, v_max]) */
} ld_params;

/* Result of one frame (caller-allocated; device memory for ld_detect, host memory for ld_detect_host). */
typedef struct ld_lanes {
    int32_t n_lanes, flags;
    int32_t start_u[LD_MAX_LANES];  /* bottom-row start of each lane (u at v = h-1), ascending */
    int64_t energy[LD_MAX_LANES];   /* its energy H(start) (Eq. 24), negative */
    int32_t v_top;                  /* first road row, f^-1(0) on the row grid (h if no road) */
    int32_t centre, scale_exp;      /* polynomial basis tau = (v - centre) / 2^scale_exp */
    int32_t rounds_y, rounds_x;     /* RANSAC rounds run for beta and gamma */
    int32_t reserved;
    double beta[3];                 /* f(v) = sum beta_k tau^k, the road profile (Eq. 13) */
    double gamma[5];                /* V_px(v) = sum gamma_k tau^k (Eq. 19, Eq. 22) */
} ld_lanes;

typedef struct ld_handle ld_handle;

/* Fill p with the paper's constants and the library's readings of the unstated ones. */
void ld_params_default(ld_params *p);

/* Number of lane start positions per frame for width w: w + 2 floor(xi w) (Alg. 7, xi = 1/2). */
int32_t ld_n_starts(const ld_params *p, int32_t w);

/*
 * Create a handle.  All device workspace for frames up to max_w x max_h and batches up to max_batch is
 * allocated here once; ld_detect never allocates.  cuda_stream (a cudaStream_t, may be NULL for the
 * default stream) is the stream every later call enqueues on.  *out receives the handle, or NULL on error.
 * Errors: LD_E_ARG (sizes out of range, invalid params), LD_E_NOMEM, LD_E_CUDA.
 */
int ld_create(const ld_params *p, int32_t max_w, int32_t max_h, int32_t max_batch, void *cuda_stream,
              ld_handle **out);

/*
 * Detect lanes in n_frames frames.  disp (float32) and img (uint8) are DEVICE pointers to
 * [n_frames][h][w]; out_lanes is a DEVICE array of n_frames ld_lanes.  The call only enqueues work on the
 * handle's stream (it returns before the GPU finishes); results are valid after the caller synchronises
 * that stream.  The caller owns all three buffers and must keep them alive until then.
 * Repeated calls with the same pointers and sizes replay a captured CUDA graph.
 * Errors: LD_E_ARG (null pointer, w/h/n_frames out of the handle's range, w < 16, h < 16), LD_E_CUDA.
 */
int ld_detect(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t h_px, int32_t n_frames,
              ld_lanes *out_lanes);

/*
 * Tune the launch shapes for frames of w x h_px: rows per CTA of the v-disparity, gradient and M_1 kernels
 * (the tiled, shared-memory-bound ones), each chosen among a few candidates by timing eager detections of
 * the caller's frames (DEVICE pointers, as ld_detect; out_lanes receives their results).  The choice is
 * kept in the handle and used by every later call with the same w and h_px; results never depend on it
 * (tiles only partition the same work).  The paper has no counterpart.  chosen (may be NULL) receives the
 * three row counts.  The call synchronises the handle's stream.  Errors as ld_detect.
 */
int ld_tune(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t h_px, int32_t n_frames,
            ld_lanes *out_lanes, int32_t *chosen);

/*
 * Frames of several sizes in one call.  A group is n_frames frames of one size, [n_frames][h][w] contiguous
 * in DEVICE memory (disp float32, img uint8), with its own DEVICE array of n_frames ld_lanes.  The groups
 * together hold at most max_batch frames, each size within [16, max_w] x [16, max_h].  Every frame gets the
 * result ld_detect gives it.  Group g works in the handle's workspace from frame F_g on, F_g being the
 * frames of the groups before it, counted in frames of the largest size; the groups run on two streams
 * forked from the handle's stream (larger groups first, each to the stream with fewer pixels so far), so
 * that one group's per-frame serial kernels overlap another group's dense ones.  On a stream of the
 * handle's own the call is captured as one CUDA graph and replayed when the same group list (pointers and
 * sizes) comes back; on the legacy default stream, or inside the caller's capture, the groups are enqueued
 * one after another.  ld_debug_get reports on no group of it.  The paper processes one frame at a time and
 * has no counterpart.  Errors: LD_E_ARG (groups NULL, n_groups outside [1, LD_MAX_GROUPS], a group as
 * ld_detect's arguments, more than max_batch frames in all), LD_E_CUDA.
 */
#define LD_MAX_GROUPS 16
typedef struct ld_group {
    const float *disp;      /* DEVICE [n_frames][h][w] */
    const uint8_t *img;     /* DEVICE [n_frames][h][w] */
    ld_lanes *out_lanes;    /* DEVICE [n_frames] */
    int32_t w, h, n_frames, pad;
} ld_group;
int ld_detect_groups(ld_handle *h, const ld_group *groups, int32_t n_groups);

/*
 * Frames of several sizes in one launch per stage and half.  The same group list, workspace views and
 * results as ld_detect_groups, but the groups are split into two halves (by pixel count, largest first,
 * each to the half with fewer pixels so far; a single group by alternate frames) that run on two streams
 * forked from the handle's, and each of the nine stages is one kernel launch over every frame of a half,
 * whatever the sizes of its groups: a CTA
 * reads its frame's descriptor (the frame's size, start range and polynomial basis, its workspace view
 * and its buffers; built on the host and kept on the device with the captured graph) and returns when its
 * tile lies outside that frame, the grids and shared memory being sized for the list's largest frame.  The
 * tile shapes are the built-in ones (ld_tune tunes one size).  On a stream of the handle's own the call is
 * captured as one CUDA graph per group list (the descriptors are uploaded, with a wait for the stream,
 * when a list is first seen) and replayed when the list comes back; on the legacy default stream, or
 * inside the caller's capture, the groups are enqueued one after another as ld_detect_groups does, with
 * the same results.  ld_debug_get reports on no frame of it.  The paper processes one frame at a time and
 * has no counterpart.  Errors as ld_detect_groups.
 */
int ld_detect_mixed(ld_handle *h, const ld_group *groups, int32_t n_groups);

/*
 * Same as ld_detect with HOST buffers: copies the inputs to device staging owned by the handle, runs the
 * path, copies the results to out_lanes (host, n_frames entries) and waits for the stream.  Page-locked
 * (pinned) inputs give the fastest copies.  Errors as ld_detect.
 */
int ld_detect_host(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t h_px,
                   int32_t n_frames, ld_lanes *out_lanes);

/* Intermediate results of the last ld_detect / ld_detect_host call, for checking against a reference. */
enum ld_stage {
    LD_STAGE_VDISP = 1,    /* int32 [h][D]  v-disparity histogram m_y(d, v) */
    LD_STAGE_PATH_Y = 2,   /* int16 [D]     DP row v_d at each d (entry 0 unused) */
    LD_STAGE_INL_Y = 3,    /* uint8 [D]     final RANSAC membership of path point d */
    LD_STAGE_ROWS = 4,     /* float [3][h]  f(v), V_py(v), V_px(v) on rows >= v_top, 0 above */
    LD_STAGE_EDGES = 5,    /* int32 [h] counts, then int16 [h][w][4] entries (u, vote column or -1, G_x, G_y) */
    LD_STAGE_PATH_X = 6,   /* int16 [h]     DP column u_v at each row v >= v_top */
    LD_STAGE_INL_X = 7,    /* uint8 [h]     final RANSAC membership of the path point at row v */
    LD_STAGE_M1 = 8,       /* int32 [h][w]  M_1 on rows >= v_top (0 above) */
    LD_STAGE_HE = 9,       /* int64 [n_starts] energy histogram H */
    LD_STAGE_MX = 10,      /* int32 [h][w]  dense V_px accumulator m_x of Alg. 5 on rows >= v_top (0 above), the
                              values the V_px DP kernel forms in registers (needs ld_debug_capture) */
    LD_STAGE_IBF = 11,     /* int16 [h][w]  bilateral output I^bf (Eq. 15-16; the median or raw image when
                              bilateral is 2 or 0) at the pixels the gradient kernel filters, -1 at the others:
                              every pixel of the 3x3 neighbourhood of a road pixel that may be an edge (see
                              ld_flat_range), so every pixel the Sobel of an edge reads (needs ld_debug_capture) */
};
/*
 * Copy stage `stage` of frame `frame` (host buffer host_dst of `bytes` bytes, which must equal the
 * stage's size) after synchronising the handle's stream.  Errors: LD_E_ARG, LD_E_STATE (no single-size
 * detection yet, ld_detect_groups ran after the last one, or LD_STAGE_MX / LD_STAGE_IBF of a call made
 * without ld_debug_capture), LD_E_CUDA.
 */
int ld_debug_get(ld_handle *h, int32_t frame, int32_t stage, void *host_dst, size_t bytes);

/* Size in bytes of stage `stage` for the last call's frame size (0 if unknown). */
size_t ld_debug_size(ld_handle *h, int32_t stage);

/*
 * Lane drawing (Alg. 7, last step; Sec. 2.4): each selected lane traced by iterating Eq. 25 from its start
 * (start_u, h-1) up to v_top, with the V_px and V_py rows of the handle's last single-size call, in the
 * float32 operation order of the energy search (the rounded columns floor(u + 0.5) are the ones whose M_1
 * the lane's energy summed).  lanes: DEVICE array of that call's results for its first n_frames frames
 * (out_lanes of ld_detect, or of the learned form); tracks_out: DEVICE float32
 * [n_frames][LD_MAX_LANES][h]: column u of lane k at row v, NaN above v_top and for k >= n_lanes (and for
 * frames without a road or V_p fit).  The caller owns both; enqueued on the handle's stream.  The paper
 * draws these curves on the image; here they are returned, headless.  Errors: LD_E_ARG (null buffer,
 * n_frames outside [1, frames of the last call]), LD_E_STATE (no single-size call yet, or
 * ld_detect_groups since), LD_E_CUDA.
 */
int ld_lane_tracks(ld_handle *h, const ld_lanes *lanes, int32_t n_frames, float *tracks_out);

/*
 * Stage capture of the two intermediates the kernels keep on chip: m_x (Alg. 5, formed inside the V_px
 * DP kernel) and I^bf (Eq. 15-16, formed inside the gradient kernel).  With on != 0 the handle allocates
 * a capture buffer for max_batch frames (6 bytes per pixel) and every later call also writes both there,
 * from the same registers the path uses, so that LD_STAGE_MX and LD_STAGE_IBF report on the last call;
 * on = 0 frees it.  Switching drops the captured CUDA graphs (their launches hold the workspace
 * pointers) and synchronises the handle's stream.  It costs time and memory: for checking, not for
 * production.  Errors: LD_E_ARG (h NULL), LD_E_NOMEM, LD_E_CUDA.
 */
int ld_debug_capture(ld_handle *h, int32_t on);

/*
 * Host-only: the lookup tables the kernels use, built from p exactly as ld_create builds them.
 * ws_q[(2 rho + 1)^2] and wr_q[256] are Eq. 16 weights in Q15; wg_q[16385] is Eq. 23 in Q12 indexed by
 * floor(sin(dtheta) 2^15).  Any pointer may be NULL.  Errors: LD_E_ARG.
 */
int ld_tables(const ld_params *p, int32_t *ws_q, int32_t *wr_q, int32_t *wg_q);

/*
 * Host-only: the exact pruning bound of the gradient kernel.  A road pixel whose neighbourhood (the
 * windows of its 3x3 neighbours, all inside the frame) spans an image range of at most the returned value
 * cannot pass the edge test of Sec. 2.3.1, whatever its values: every Q15 weight of those windows lies in
 * [a, b] (a at the range, b at zero difference), so each bilateral output is within
 * (b - a) r / (4 a) + 1/2 of its window mean; means of windows two pixels apart differ by at most
 * 2 r / (2 rho + 1); the Sobel components are then at most 4 (2 r / (2 rho + 1) + 2 e) each, and the
 * bound is the largest range r for which twice its square stays at most edge_thresh^2.  The kernel leaves
 * such pixels (and the bilateral outputs only they would read) out; every edge, G and vote is unchanged.
 * The paper filters the whole image and has no counterpart.  Returns -1 when nothing is pruned
 * (bilateral != 1, or no range qualifies) or when p is invalid.
 */
int32_t ld_flat_range(const ld_params *p);

/*
 * Bounds-checked build.  lib/libld_checked.so is this library compiled with LD_CHECKED (build.py
 * --checked).  Before each access its kernels test, against the buffer's extent, every index they
 * compute from data: histogram bins, vote and edge columns, decoded backtrack steps, path cells,
 * point-list and sample indices, track columns and list decodes.  They also test every append to a
 * fixed-capacity list and each tile against its frame.  A failing access is skipped (loads read 0) and
 * counted; the first failure's site, index and bound are kept.  Nothing traps.  In the regular library
 * the tests compile away and the calls below report a clean state.
 *   ld_checked_build   1 in the checked library, 0 otherwise.
 *   ld_check_status    waits for the device, then out[0] = failures since the last reset (all kernels),
 *                      out[1..3] = site, index and bound of a first one: the first failure recorded by the
 *                      first translation unit, in link order, that recorded any (0 when none).  LD_E_CUDA
 *                      on a device error.
 *   ld_check_reset     clears the counts (waits for the device first).
 *   ld_check_site_name the name of a site ("?" for an unknown one).
 *   ld_check_selftest  checked library only: one thread evaluates a test with index = bound (no access
 *                      follows), so the status then shows one failure at site "selftest".  LD_E_STATE
 *                      in the regular library.
 */
int32_t ld_checked_build(void);
int ld_check_status(int64_t out[4]);
int ld_check_reset(void);
const char *ld_check_site_name(int32_t site);
int ld_check_selftest(void);

/* Number of kernel launches one ld_detect call enqueues, and the name of launch k (0-based). */
int32_t ld_launches_per_detect(void);
const char *ld_launch_name(int32_t k);

/*
 * Profiling form of ld_detect (DEVICE buffers as ld_detect): enqueues the same kernels without graph
 * capture, with a CUDA event recorded on the handle's stream before the first kernel and after each one,
 * waits for the stream, and writes the duration of launch k in milliseconds to ms_out[k]
 * (ld_launches_per_detect() entries).  The stream is held at a host function (at most one second) until
 * every launch is enqueued, so the kernels run back to back and no interval holds host enqueue time; the
 * buffer resets of the later stages are made before the first event.  Errors as ld_detect.
 */
int ld_detect_timed(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t h_px,
                    int32_t n_frames, ld_lanes *out_lanes, float *ms_out);

/*
 * Allocation-free road-profile path.  The paper has no counterpart: this entry point exists for callers
 * that may not allocate device memory where they need the result, for example software whose memory is
 * all reserved at start-up (safety-certified driving stacks forbid allocation in the per-frame path) or a
 * plugin whose host application hands it only its input and output buffers.
 *
 * For n_frames frames it computes the v-disparity histogram and the road DP path over it, with the same
 * tie rules as ld_detect, and writes the path row of each disparity bin d to path_out[frame][d] (int16,
 * n_disp entries per frame, entry 0 = -1): the values ld_debug_get returns for LD_STAGE_PATH_Y after
 * ld_detect with the same parameters.  disp is a DEVICE pointer to float32 [n_frames][h][w], path_out a
 * DEVICE pointer; the caller owns both.  Only p->n_disp, p->tau_y, p->lambda_y and p->dp_literal are
 * read; the literal form of the DP (dp_literal = 1) is not offered here and returns LD_E_ARG.  The work
 * is enqueued on cuda_stream (NULL = default stream) and the call returns without waiting.
 *
 * No cudaMalloc, cudaFree or allocating library routine is called.  The histogram scratch is a static
 * device array of LD_STATIC_SCRATCH_BYTES bytes inside the library, which every GPU that loads the library
 * keeps until the process exits; a request needing more (n_frames * n_disp * h * 4 bytes) returns LD_E_ARG.
 * The first call on each device, with that device current, looks up the array's device address and
 * configures the kernel; make that first call before any stream capture.  Every call shares the one array:
 * calls that overlap on the GPU (other streams, other host threads) race on it, so serialise them.  Each
 * call overwrites every scratch entry it reads, so no stale contents leak between calls.
 * Errors (message in ld_last_error(NULL)): LD_E_ARG, LD_E_CUDA.
 */
#define LD_STATIC_SCRATCH_BYTES (8u << 20)
int ld_road_path_static(const ld_params *p, const float *disp, int32_t w, int32_t h_px, int32_t n_frames,
                        int16_t *path_out, void *cuda_stream);

/*
 * Serving: frames of several sizes from several camera streams, batched continuously.  The paper runs one
 * camera at a time and has no counterpart; its closing remarks suggest carrying the road profile and the
 * vanishing point from frame to frame, for which the server keeps each stream's latest result in device
 * memory (ld_server_stream_state).
 *
 * A server owns, for every size class, `slots_per_size` slots: a library handle, a CUDA stream, pinned
 * staging for `max_batch` frames and their device buffers, all allocated in ld_server_create (the HBM a
 * server may use is fixed there; admission is by free slot).  ld_server_submit copies a frame into the
 * slot that is filling for its size class (opening a free one if needed); a full slot is launched at once
 * and a partial one when its oldest frame has waited `max_wait_us` (a scheduler thread of the server).
 * Each batch is one detection of its frames (the same kernels as ld_detect, launched without a graph),
 * and every frame's result is the one it would get alone.  Results come back through ld_server_poll in
 * completion order, each with the caller's tag, its stream, its per-stream sequence number and its
 * latency from submit to the result being in host memory.  A server is thread-safe.
 */
#define LD_MAX_SIZE_CLASSES 8
typedef struct ld_server ld_server;

typedef struct ld_server_config {
    int32_t n_sizes;                          /* size classes, 1 .. LD_MAX_SIZE_CLASSES */
    int32_t sizes[LD_MAX_SIZE_CLASSES][2];    /* (w, h) of each class; a frame must match one exactly */
    int32_t slots_per_size;                   /* batches of a class filling or in flight at once, >= 1 */
    int32_t max_batch;                        /* frames per batch, >= 1 */
    int32_t max_wait_us;                      /* a partial batch launches once its oldest frame waited this */
    int32_t n_streams;                        /* camera streams: ids 0 .. n_streams-1 */
    int32_t reserved;                         /* 0 */
    int64_t hbm_budget_bytes;                 /* 0: the slots_per_size slots of each class only.  > 0: when
                                               * every slot of a class is full or in flight, a submit adds
                                               * one more slot while the slots' device bytes stay within
                                               * this budget and the device keeps 256 MiB free; slots are
                                               * kept until ld_server_destroy */
} ld_server_config;

typedef struct ld_result {
    uint64_t tag;                             /* the caller's tag from ld_server_submit */
    int32_t stream_id, w, h;
    int64_t seq;                              /* 0, 1, 2 ... per stream, in submission order */
    double latency_ms;                        /* submit -> result in host memory */
    ld_lanes lanes;
} ld_result;

typedef struct ld_server_stats {
    int64_t submitted, completed, rejected, batches;
    double mean_batch;                        /* frames per launched batch */
    double p50_ms, p99_ms;                    /* latency percentiles of the completed frames */
    int64_t slots;                            /* slots allocated (initial and added under the budget) */
    int64_t device_bytes;                     /* device bytes of the slots' buffers and handle workspaces */
} ld_server_stats;

/* Create a server (all memory allocated here).  Errors: LD_E_ARG (bad config or params), LD_E_NOMEM,
 * LD_E_CUDA; *out is NULL on error and ld_server_last_error(NULL) describes it. */
int ld_server_create(const ld_params *p, const ld_server_config *cfg, ld_server **out);

/* Submit one frame (HOST pointers, [h][w]; copied into the slot's page-locked staging before the call
 * returns, so the caller may reuse them; the copy to the device is enqueued at once on the slot's stream).
 * Errors: LD_E_ARG (unknown size or stream id, null pointer), LD_E_BUSY (every slot of the class is full
 * or in flight and the HBM budget admits no further slot: poll and retry), LD_E_NOMEM or LD_E_CUDA (a slot
 * the budget admitted could not be allocated, or a copy failed; ld_server_last_error says which). */
int ld_server_submit(ld_server *s, int32_t stream_id, const float *disp, const uint8_t *img, int32_t w, int32_t h,
                     uint64_t tag);

/* As ld_server_submit, for frames in PAGE-LOCKED host memory (cudaMallocHost, cudaHostRegister, a pinned
 * torch tensor): the device reads them directly (no host copy), so the caller must leave both buffers
 * unchanged until the frame's result has come out of ld_server_poll.  Pageable pointers still work, at the
 * cost of a copy the driver stages.  Errors as ld_server_submit. */
int ld_server_submit_pinned(ld_server *s, int32_t stream_id, const float *disp, const uint8_t *img, int32_t w,
                            int32_t h, uint64_t tag);

/* Submit n_frames frames of one size at once: disp [n_frames][h][w] and img [n_frames][h][w] contiguous
 * HOST arrays, stream_ids and tags [n_frames]; pinned != 0 as ld_server_submit_pinned, else as
 * ld_server_submit.  Frames are placed in order, a run per slot with one device copy per buffer and run.
 * Several threads may submit at once: the copies are made outside the server's lock.  Returns the number
 * of frames accepted (the first ones; fewer than n_frames when the slots filled up: poll and resubmit the
 * rest) or, when none was, LD_E_BUSY; LD_E_ARG, LD_E_CUDA as ld_server_submit. */
int ld_server_submit_batch(ld_server *s, int32_t n_frames, const int32_t *stream_ids, const float *disp,
                           const uint8_t *img, int32_t w, int32_t h, const uint64_t *tags, int32_t pinned);

/* Switch the server's batches to the learned form (ld_detect_learned below, with the network run and the
 * given top_k) or, with top_k = 0, back to the plain form.  params: DEVICE pointer to LD_NET_PARAMS floats,
 * copied into an inference network on every slot's handle before the call returns (networks are created on
 * the first call and kept; 168 bytes per 4 x 4 pixel block of a slot's batch).  Only while no frame
 * is in the server.  Errors: LD_E_ARG (top_k outside [0, LD_NET_TOPK_MAX], null params with top_k > 0),
 * LD_E_STATE (frames filling or in flight: drain first), LD_E_NOMEM, LD_E_CUDA. */
int ld_server_set_learned(ld_server *s, const float *params, int32_t top_k);

/* Move up to max_out completed results into out (host array); waits up to timeout_ms for the first one.
 * Returns the number moved (>= 0) or a negative LD_E_* code. */
int ld_server_poll(ld_server *s, ld_result *out, int32_t max_out, int32_t timeout_ms);

/* Launch every partial batch now and wait until all submitted frames have completed (results stay queued
 * for ld_server_poll).  Errors: LD_E_CUDA. */
int ld_server_drain(ld_server *s);

/* The latest result of a stream (highest sequence number completed so far), read from the device copy the
 * server keeps.  Errors: LD_E_ARG, LD_E_STATE (no frame of that stream completed yet), LD_E_CUDA. */
int ld_server_stream_state(ld_server *s, int32_t stream_id, ld_lanes *out);

/* Counters and latency percentiles since creation. */
int ld_server_stats_get(ld_server *s, ld_server_stats *out);

/* Message of the last error on s (or of the last failed ld_server_create when s is NULL). */
const char *ld_server_last_error(const ld_server *s);

/* Wait for the work in flight and release everything.  NULL is ignored. */
void ld_server_destroy(ld_server *s);

/*
 * Learned lane-position proposal.  The paper evaluates the energy (Eq. 24-25) of the track started at
 * every bottom-row position and selects lanes among its minima (Alg. 7); it has no learned component.
 * This form ranks the starts first with a small convolutional network and evaluates exact energies only
 * on the best-ranked ones; the exhaustive search remains the fallback.
 *
 *   input    x(i, j) = sum of |G_x w_g| (the Q12 weighted gradient of Eq. 23) over the 4x4 pixel block at
 *            rows 4i.., columns 4j.. (mh = ceil(h/4) by mw = ceil(w/4) cells), fed as bf16(x 2^-22);
 *   network  four 3x3 convolutions (zero padding, channels 1-16-32-32-16, bias, ReLU) and a 1x1 head
 *            16 -> 1 giving a logit z per cell: sigmoid(z) is the chance that a lane crosses the cell, its
 *            rows the per-row lane-position heatmap.  Products in bf16, sums in FP32, activations stored
 *            as bf16; trained with a weighted logistic loss (positive weight 10) and Adam;
 *   ranking  coarse start c covers the starts 4c .. 4c+3; its score sums the heatmap sigmoid(z) along the
 *            Eq. 25 track taken in steps of four rows from u = (4c - S0) + 1.5 on the bottom row;
 *   search   the top_k coarse starts give candidate starts; each candidate and its neighbours get the
 *            exact energy; lanes are the Alg. 7 minima among the candidates (threshold from the smallest
 *            evaluated energy).  A frame where that finds no lane runs the exhaustive search and is
 *            flagged LD_F_FALLBACK.
 *
 * Parameters are a flat float32 vector of LD_NET_PARAMS values: for each convolution W[co][ci][3][3] then
 * b[co]; then the head's w[16] and b.  A network is created for a detector handle and uses its stream and
 * its largest frame and batch; it owns its activations (168 bytes per cell of the largest batch, 330
 * while training), its master weights and Adam state.  All buffer arguments are DEVICE
 * pointers owned by the caller; calls enqueue on the handle's stream and return without waiting.
 * Errors: LD_E_ARG, LD_E_NOMEM, LD_E_STATE (training call on an inference network), LD_E_CUDA.
 */
#define LD_NET_PARAMS 18689
#define LD_NET_TOPK_MAX 256
typedef struct ld_net ld_net;

enum {
    LD_NET_STAGE_XSUM = 1,     /* int32 [mh][mw]  block sums x of the last learned detection */
    LD_NET_STAGE_HEATMAP = 2,  /* float [mh][mw]  heatmap the last learned detection ranked with; rows
                                  * i >= v_top / 4 (the network runs on the road rows only) */
    LD_NET_STAGE_SCORES = 3,   /* float [ceil(n_starts / 4)] coarse-start scores */
    LD_NET_STAGE_CFLAG = 4,    /* uint8 [n_starts] bit 0 candidate, bit 1 energy evaluated */
};

int32_t ld_net_param_count(void);
/* training != 0 also allocates what the backward pass needs. */
int ld_net_create(ld_handle *h, int32_t training, ld_net **out);
/* Copy LD_NET_PARAMS floats in as the master weights; resets the Adam moments and step count. */
int ld_net_set_params(ld_net *net, const float *params);
int ld_net_get_params(ld_net *net, float *params);
/* Form of the inference forward (ld_net_forward, ld_detect_learned): on != 0 runs all four layers and the
 * head in one kernel per 32 x 16-cell tile with the activations kept on chip; 0 (the default, the faster
 * form on GB300) runs one kernel per layer through device memory.  The logits and heatmap values are identical on every cell the road
 * rows need (the two forms issue the same MMAs); the per-layer form also computes rows above them.  Waits
 * for the handle's stream; drops the captured learned calls.  Training always runs per layer. */
int ld_net_set_fused(ld_net *net, int32_t on);
/* logits[n][mh][mw] of the block sums xsum[n][mh][mw] of frames of w x h pixels. */
int ld_net_forward(ld_net *net, const int32_t *xsum, int32_t w, int32_t h_px, int32_t n_frames, float *logits);
/* Gradient of the mean loss over n frames (grad: LD_NET_PARAMS floats) and the loss (1 float); labels are
 * uint8 [n][mh][mw] (nonzero = lane cell).  Training networks only. */
int ld_net_grad(ld_net *net, const int32_t *xsum, const uint8_t *labels, int32_t w, int32_t h_px, int32_t n_frames,
                float *grad, float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) with the given gradient. */
int ld_net_apply_grad(ld_net *net, const float *grad, float lr);
/* ld_net_grad followed by ld_net_apply_grad; loss may be NULL. */
int ld_net_train_step(ld_net *net, const int32_t *xsum, const uint8_t *labels, int32_t w, int32_t h_px,
                      int32_t n_frames, float lr, float *loss);
/* Training pairs from frames: the plain method's lanes (lanes_out, may be NULL), the block sums
 * (xsum_out [n][mh][mw]) and the labels (labels_out [n][mh][mw]: cells crossed by the Eq. 25 tracks of the
 * selected lanes on the road rows). */
int ld_make_training_pairs(ld_net *net, const float *disp, const uint8_t *img, int32_t w, int32_t h_px,
                           int32_t n_frames, int32_t *xsum_out, uint8_t *labels_out, ld_lanes *lanes_out);
/* The learned form of ld_detect.  heatmap == NULL runs the network (heatmap sigmoid(z)); otherwise
 * heatmap[n][mh][mw] is ranked with as given.  top_k in [1, LD_NET_TOPK_MAX]. */
int ld_detect_learned(ld_net *net, const float *heatmap, const float *disp, const uint8_t *img, int32_t w,
                      int32_t h_px, int32_t n_frames, int32_t top_k, ld_lanes *out_lanes);
/* Intermediate results of the last learned detection (synchronises the stream), as ld_debug_get. */
size_t ld_net_debug_size(ld_net *net, int32_t stage);
int ld_net_debug_get(ld_net *net, int32_t frame, int32_t stage, void *host_dst, size_t bytes);
/* LD_OK, or LD_E_TIMEOUT when a tensor-core wait of a network kernel ran out since the last call (the
 * kernel then stopped issuing work and released its tensor memory; results of that call are invalid).
 * Synchronises the device. */
int ld_net_status(ld_net *net);
const char *ld_net_last_error(const ld_net *net);
void ld_net_destroy(ld_net *net);

/*
 * Stereo matching (Sec. 2.1): the disparity map of a rectified grey pair, the input the lane path takes.
 * For each pixel the NCC of its (2 rho + 1)^2 block with the other image's blocks on the same row
 * (Eq. 1-8, from block sums and sums of squares, the quantities the paper gets from integral images,
 * Alg. 1 and Eq. 5), searched by search range propagation (Eq. 9, Alg. 2): rows from the bottom up, the
 * first over [0, d_max], every later pixel over [l - tau, l + tau] around the three estimates below it.
 * Both the left map (left block at u against right at u - d) and the right map (right at u against left
 * at u + d) are estimated, then the left-right consistency check (Alg. 3) keeps l_lf(u, v) where
 * |l_lf(u, v) - l_rt(u - l_lf(u, v), v)| <= tr_lrc and writes 0 elsewhere.
 *
 * Readings: blocks lie inside both images (border pixels and candidates whose other block would leave
 * the image are skipped; a pixel without a candidate gets 0); the best candidate has the largest NCC,
 * compared exactly in integers (ties to the smaller disparity); a block of constant intensity has NCC 0.
 * A stereo object belongs to a handle (its stream, largest frame and batch) and owns its two int16 maps
 * and a float disparity buffer.  Images are DEVICE uint8 [n][h][w]; outputs DEVICE float [n][h][w] with
 * integer values (0 = no disparity).  Errors: LD_E_ARG, LD_E_NOMEM, LD_E_STATE, LD_E_CUDA.
 */
typedef struct ld_stereo ld_stereo;
typedef struct ld_stereo_params {
    int32_t rho;     /* block half-size, 1..3 (3: 7 x 7 blocks, the paper's setting) */
    int32_t tau;     /* search range bound of Eq. 9 (1) */
    int32_t d_max;   /* largest disparity searched; -1: n_disp - 1 of the handle */
    int32_t tr_lrc;  /* LRC threshold of Alg. 3 (3) */
} ld_stereo_params;

void ld_stereo_params_default(ld_stereo_params *sp);
int ld_stereo_create(ld_handle *h, const ld_stereo_params *sp, ld_stereo **out);
/* Disparity of n frames into disp_out (enqueued on the handle's stream). */
int ld_stereo_run(ld_stereo *st, const uint8_t *left, const uint8_t *right, int32_t w, int32_t h_px, int32_t n_frames,
                  float *disp_out);
/* ld_stereo_run with CUDA events: ms_out[0] = both search-range-propagation maps, ms_out[1] = the check
 * (waits for the stream). */
int ld_stereo_run_timed(ld_stereo *st, const uint8_t *left, const uint8_t *right, int32_t w, int32_t h_px,
                        int32_t n_frames, float *disp_out, float *ms_out);
/* The whole path from stereo pairs: the disparity into the object's buffer, then ld_detect on it with the
 * left image. */
int ld_detect_stereo(ld_stereo *st, const uint8_t *left, const uint8_t *right, int32_t w, int32_t h_px,
                     int32_t n_frames, ld_lanes *out_lanes);
/* Host copies of frame `frame` of the last call: left map, right map (int16 [h][w]) and the checked
 * disparity (float [h][w], the object's buffer: valid after ld_detect_stereo); any pointer may be NULL. */
int ld_stereo_maps(ld_stereo *st, int32_t frame, int16_t *lf_host, int16_t *rt_host, float *disp_host);
const char *ld_stereo_last_error(const ld_stereo *st);
void ld_stereo_destroy(ld_stereo *st);

/* Message of the last error on h (or of the last failed ld_create when h is NULL). */
const char *ld_last_error(const ld_handle *h);

/* Release the handle and its workspace (synchronises its stream first).  NULL is ignored. */
void ld_destroy(ld_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* LD_H */
