// Internal definitions shared by the lane-detection kernels and the host runtime.
//
// Exactness: every floating-point decision of the path (vote column, w_g angle, lane track, polynomial
// evaluation and solves) is written with explicit round-to-nearest intrinsics (__fadd_rn, __fmul_rn,
// __fdiv_rn, __dadd_rn, ...), one IEEE rounding per operation and no contraction, so the results are
// fixed by the expression alone.  The library is also compiled with --fmad=false as a safety net.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "ld.h"

namespace ld {

constexpr int kMaxHyps = 256;
constexpr int kWgEntries = 16385;     // Eq. 23 table: sin(dtheta) in [0, 1/2] in steps of 2^-15
constexpr int kWrEntries = 768;       // Q15 range weight of dI at index 256 + dI (symmetric; entries >= 512 are 0)
constexpr int kSentinel = 511;        // image value marking taps outside the frame
constexpr int kClsTables = 24;        // distance classes of the largest bilateral window (rho = 5: 20 used)

// Bounds-checked build (-DLD_CHECKED, lib/libld_checked.so).  LD_IN(i, n, site) holds when 0 <= i < n.
// Otherwise it counts a failure in this translation unit's error word, records the first one (site,
// index, bound) and is false, so the guarded access is skipped: a checked kernel never reads or writes
// outside its buffers and never traps.  In the regular build LD_IN is the constant true and the guards
// compile away.  Checked: every index computed from data (histogram bins, vote and edge columns, decoded
// backtrack steps, path cells, point-list and sample indices, track columns, list decodes), every append
// to a fixed-capacity list, and each kernel's tile against its frame and buffers.
enum CkSite : int {
    CK_NONE = 0,
    CK_SELFTEST,
    CK_VDISP_BIN, CK_VDISP_RUN, CK_VDISP_LOAD, CK_VDISP_OUT,
    CK_ROAD_PATH, CK_ROAD_PTS,
    CK_FIT_NPTS, CK_FIT_SAMPLE, CK_FIT_ROW,
    CK_GRAD_TILE, CK_GRAD_GLIST, CK_GRAD_GROUP, CK_GRAD_TAP, CK_GRAD_EDGE, CK_GRAD_VOTE,
    CK_VPX_TILE, CK_VPX_VOTE, CK_VPX_VOFF, CK_VPX_STAGE, CK_VPX_PATH, CK_VPX_PTS,
    CK_M1_EDGE, CK_M1_COL, CK_M1_CHUNK,
    CK_EN_START, CK_EN_COL, CK_EN_ROW,
    CK_SEL_START, CK_SEL_LANES, CK_TRACK_COL,
    CK_MED_TILE,
    CK_N_SITES
};
}  // namespace ld

#ifdef LD_CHECKED
namespace ld {
using CkRead = cudaError_t (*)(unsigned long long *out4);
using CkReset = cudaError_t (*)();
int ck_register(CkRead read, CkReset reset);   // ld_api.cu: collects every translation unit's error word
}  // namespace ld
namespace {
__device__ unsigned long long g_ld_ck[4];      // failures, first site, first index, first bound
__device__ __noinline__ bool ld_ck_fail(long long i, long long n, int site)
{
    if (atomicAdd(&g_ld_ck[0], 1ull) == 0ull) {
        g_ld_ck[1] = (unsigned long long)site;
        g_ld_ck[2] = (unsigned long long)i;
        g_ld_ck[3] = (unsigned long long)n;
    }
    return false;
}
__device__ __forceinline__ bool ld_ck_in(long long i, long long n, int site)
{
    return (i >= 0 && i < n) ? true : ld_ck_fail(i, n, site);
}
cudaError_t ld_ck_read(unsigned long long *out4) { return cudaMemcpyFromSymbol(out4, g_ld_ck, sizeof(g_ld_ck)); }
cudaError_t ld_ck_reset()
{
    static const unsigned long long zero[4] = {0, 0, 0, 0};
    return cudaMemcpyToSymbol(g_ld_ck, zero, sizeof(zero));
}
[[maybe_unused]] const int ld_ck_registered = ld::ck_register(ld_ck_read, ld_ck_reset);
}  // namespace
#define LD_IN(i, n, site) ld_ck_in((long long)(i), (long long)(n), (int)(::ld::site))
#else
#define LD_IN(i, n, site) true
#endif

namespace ld {

// Per-launch constants, passed by value (they live in the kernel-parameter constant bank).
struct KParams {
    int32_t W, H, D, n_frames;
    int32_t tau_y, lambda_y;
    float tr_y;
    int32_t eps_num, eps_den;
    float varpi;
    int32_t bilateral, rho;
    int32_t edge_thresh2;
    int32_t vote_rho, chi, tau_x, lambda_x;
    float tr_x;
    int32_t box_nu, box_vs, lambda_g;
    int32_t S0, n_starts;
    int32_t thr_num, thr_den, near_px, max_lanes;
    long long thr_abs;                 // 0: relative threshold; < 0: lanes need H < thr_abs
    int32_t dp_literal;                // 1: Eq. 12 as printed (k_road_dp_lit)
    int32_t band_literal;              // 1: Alg. 5's bottom rows j > vmax - chi - 1 use the band [j, vmax]
    int32_t hyps, rounds;
    uint32_t key0, key1;
    int32_t centre, e;                 // polynomial basis tau = (v - centre) / 2^e
    int32_t seg_rows;                  // rows of DP backtrack held in shared memory by the V_px kernel
    int32_t tile_vdisp, tile_grad, tile_m1;  // rows per CTA chosen by ld_tune (0: the built-in rule)
    int32_t vote_cap;                  // votes per frame the V_px kernel stages in shared memory
    uint16_t ws[121];                  // Eq. 16 spatial weights, Q15 (up to 32768), (2 rho + 1)^2 used
    // Taps at equal distance share one weight table in the gradient kernel.  Classes are the ranks of
    // dx^2 + dy^2 among the distinct values of the window (the kernel derives a tap's class at compile
    // time in the same way); cls_ws[c] = the spatial weight of class c.
    int32_t n_cls;
    uint16_t cls_ws[24];
    // Largest image range (max - min over a group's (4 + 2 rho + 6) x (2 rho + 3) neighbourhood) for which no
    // pixel of the group can pass the edge test, or -1 (pruning off: bilateral != 1).  See flat_range().
    int32_t flat_range;
    int32_t pmax_hint;                 // the workspace's path-point capacity (Work::pmax), for launch shapes
};

// Per-frame state written by the fit kernels and read downstream.
struct FrameState {
    int32_t flags, v_top, rounds_y, rounds_x;
    double beta[3];
    double gamma[5];
};

// Device workspace (all pointers device memory, sized for max_w x max_h x max_batch).
struct Work {
    int32_t *myT;        // [n][D][H] v-disparity, transposed so a DP step reads a contiguous row
    FrameState *fs;      // [n]
    float *rows;         // [n][3][H]: f(v), V_py(v), V_px(v)
    int16_t *path_y;     // [n][D]
    uint8_t *inl_y;      // [n][D]
    int32_t *ecount;     // [n][H] road edge pixels per row
    int16_t *edges;      // [n][H][W][4]: u, vote column (-1 none), G_x, G_y
    int32_t *vcount;     // [n][H] votes per row
    int16_t *vbins;      // [n][H][W] vote columns of each row
    int16_t *path_x;     // [n][H]
    uint8_t *inl_x;      // [n][H]
    int16_t *pts;        // [n][2][3][pmax] DP path points with data (x, y, index) for the beta / gamma fits
    int32_t *npts;       // [n][2]
    uint8_t *gbt;        // [n][max_h][vpx_row_bytes(max_w)] V_px backtrack rows below the shared-memory block
    int32_t *M1;         // [n][H][W]
    int32_t *xsum;       // [n][ceil(H/4)][ceil(W/4)] block sums of |G_x w_g| for the learned proposal, or null
    uint8_t *med;        // [n][H][W] median-filtered image (bilateral = 2), or null
    int64_t *HE;         // [n][n_starts]
    int32_t *dbg_mx;     // [n][H][W] the Alg. 5 accumulator m_x as the V_px DP kernel forms it, or null (capture off)
    int16_t *dbg_ibf;    // [n][H][W] bilateral output where the gradient kernel computes it, -1 elsewhere, or null
    const int32_t *wr;   // [kWrEntries] Q15
    const int32_t *wg;   // [kWgEntries] Q12
    const uint16_t *cls_tab;  // [kClsTables][512] Q15 bilateral weights by distance class and |dI| (zero from 256 on)
    int32_t max_w, max_h, pmax;
};

// One frame of a call over frames of several sizes (ld_detect_mixed): its own parameters (W, H, start
// range, polynomial basis), the workspace seen from its slot (frame index 0 inside the view) and its
// buffers.  The per-frame launches below run one CTA grid over all frames, sized for the largest; each
// CTA reads its frame's descriptor and returns when its tile lies outside that frame.
struct FrameDesc {
    KParams kp;
    Work w;
    const float *disp;   // [H][W]
    const uint8_t *img;  // [H][W]
    ld_lanes *out;       // [1]
};

// ---------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, multipliers 0xD2511F53 / 0xCD9E8D57,
// Weyl key increments 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Correctly rounded conversion of an exact integer sum to double.  Valid for |x| < 2^85: the high part
// x >> 32 is then exact in a double, and the final addition is the only rounding.
__device__ __forceinline__ double i128_to_f64(__int128 x)
{
    const long long q = (long long)(x >> 32);
    const unsigned int r = (unsigned int)(x & (__int128)0xffffffffu);
    return __dadd_rn(__dmul_rn((double)q, 4294967296.0), (double)r);
}

// Bytes of one V_px backtrack row: one byte per pair of cells (two 4-bit entries), padded to 16 bytes.
__host__ __device__ inline int vpx_pairs(int W) { return (W + 1) >> 1; }
__host__ __device__ inline int vpx_row_bytes(int W) { return (vpx_pairs(W) + 15) & ~15; }

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// Allow a kernel the largest dynamic shared memory the device offers next to its static shared memory.
template <typename K>
inline cudaError_t allow_max_smem(K kernel, int smem_optin)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)a.sharedSizeBytes);
}

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount), queried once per
// device; grids that stop at a whole number of waves are sized from it.
inline int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// f64 Horner without contraction.
template <int M>
__device__ __forceinline__ double poly_f64(const double *c, double tau)
{
    double p = c[M - 1];
#pragma unroll
    for (int k = M - 2; k >= 0; --k)
        p = __dadd_rn(__dmul_rn(p, tau), c[k]);
    return p;
}

}  // namespace ld

// Kernel launch helpers implemented in the kernel translation units.
namespace ld {
cudaError_t launch_vdisp(const KParams &kp, const Work &w, const float *disp, cudaStream_t s);
cudaError_t launch_road(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_fit_y(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_fit_x(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_grad(const KParams &kp, const Work &w, const float *disp, const uint8_t *img, cudaStream_t s);
cudaError_t launch_median(const KParams &kp, const Work &w, const uint8_t *img, cudaStream_t s);
cudaError_t launch_vpx(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_m1(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_energy(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_select(const KParams &kp, const Work &w, ld_lanes *out, cudaStream_t s);
cudaError_t launch_tracks(const KParams &kp, const Work &w, const ld_lanes *lanes, float *out, cudaStream_t s);
// learned proposal: energies of the listed starts / selection among the candidates (frames without a lane
// are flagged LD_F_FALLBACK), then the exhaustive energies and selection of the flagged frames only
cudaError_t launch_energy_list(const KParams &kp, const Work &w, const int32_t *elist, const int32_t *ecnt, int ecap,
                               cudaStream_t s);
cudaError_t launch_select_set(const KParams &kp, const Work &w, const uint8_t *cflag, ld_lanes *out, cudaStream_t s);
cudaError_t launch_energy_fallback(const KParams &kp, const Work &w, cudaStream_t s);
cudaError_t launch_select_fallback(const KParams &kp, const Work &w, ld_lanes *out, cudaStream_t s);
// the same stages over a descriptor array (kmax: parameters of the call's largest frame, which size the
// grids and shared memory; n: frames)
cudaError_t launch_vdisp_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_road_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_fit_y_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_fit_x_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_grad_fd(const KParams &kmax, const FrameDesc *fd, int n, bool median_input, cudaStream_t s);
cudaError_t launch_median_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_vpx_fd(const KParams &kmax, const FrameDesc *fd, int n, size_t smem, cudaStream_t s);
cudaError_t launch_m1_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_energy_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
cudaError_t launch_select_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s);
size_t road_smem_bytes(const KParams &kp);
size_t vpx_smem_bytes(const KParams &kp);
int vpx_seg_rows(const KParams &kp, size_t budget);
cudaError_t setup_dp(int smem_optin);
cudaError_t setup_ransac(int smem_optin);
cudaError_t setup_grad(int smem_optin);
cudaError_t setup_lpv(int smem_optin);
int detect_eager(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                 ld_lanes *out_lanes);
int detect_learned_eager(ld_net *net, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                         int32_t top_k, ld_lanes *out_lanes);
// device bytes of a handle's workspace (its buffers for max_batch frames of the largest size)
size_t handle_device_bytes(const ld_handle *h);
}  // namespace ld
