// Host runtime behind include/ld.h: parameter checks, lookup tables, workspace, the launch sequence of
// one ld_detect call (replayed from a captured CUDA graph when the same buffers come back; a call of at
// least kSplitMin frames is captured as two concurrent half-batches, so one half's per-frame serial kernels
// overlap the other half's dense kernels), calls over groups of frames of several sizes, the host-buffer
// path and the debug getters.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ld_internal.cuh"

static_assert(sizeof(ld_group) == 40, "C-ABI group layout");

namespace {

constexpr int kLaunches = 9;
const char *const kLaunchNames[kLaunches] = {"k_vdisp", "k_road_dp", "k_fit_y", "k_grad", "k_vpx_dp",
                                             "k_fit_x", "k_m1", "k_energy", "k_select"};
constexpr int kGraphSlots = 4;
constexpr int kSplitMin = 16;  // captured calls of at least this many frames run as two concurrent halves
constexpr int kVoteCap = 12288;

std::string g_create_error;

struct GraphSlot {
    const void *disp = nullptr, *img = nullptr;
    void *out = nullptr;
    int w = 0, h = 0, n = 0;
    cudaGraphExec_t exec = nullptr;
};

// a captured ld_detect_groups call, replayed when the same group list comes back
struct GroupGraph {
    std::vector<ld_group> groups;
    cudaGraphExec_t exec = nullptr;
};

// A captured ld_detect_mixed call: its group list and the device descriptors its launches read.
struct MixedGraph {
    std::vector<ld_group> groups;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

#ifdef LD_CHECKED
namespace {
std::vector<std::pair<ld::CkRead, ld::CkReset>> &ck_registry()
{
    static std::vector<std::pair<ld::CkRead, ld::CkReset>> r;   // filled during static initialisation
    return r;
}
// index == bound: the test fails and is recorded; nothing is accessed
__global__ void k_ck_selftest(int n)
{
    if (!LD_IN(n, n, CK_SELFTEST))
        return;
}
}  // namespace
int ld::ck_register(ld::CkRead read, ld::CkReset reset)
{
    ck_registry().emplace_back(read, reset);
    return (int)ck_registry().size();
}
#endif

struct ld_handle {
    ld_params p{};
    int max_w = 0, max_h = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    int smem_optin = 0;
    void *ws = nullptr;          // device workspace
    size_t ws_bytes = 0;
    ld::Work w{};
    int32_t *d_tables = nullptr; // wr, wg
    int32_t ws_q[121]{};
    // host-buffer path
    float *d_disp = nullptr;
    uint8_t *d_img = nullptr;
    ld_lanes *d_lanes = nullptr;
    // last call
    int last_w = 0, last_h = 0, last_n = 0;
    bool have_last = false;
    GraphSlot graphs[kGraphSlots];
    int next_slot = 0;
    GroupGraph group_graphs[kGraphSlots];
    int next_group_slot = 0;
    MixedGraph mixed_graphs[kGraphSlots];
    int next_mixed_slot = 0;
    ld::FrameDesc *d_fdesc = nullptr;   // [kGraphSlots][max_batch] descriptors of the captured mixed calls
    ld::FrameDesc *h_fdesc = nullptr;   // pinned host staging of one list
    cudaEvent_t ev[kLaunches + 1] = {};
    // two half-batches forked onto their own streams inside a captured call (joined before it ends)
    cudaStream_t sub[2] = {};
    cudaEvent_t fork = nullptr, join[2] = {};
    // tile sizes chosen by ld_tune for frames of tile_w x tile_h (0: the built-in rules)
    int tile_w = 0, tile_h = 0, tile[3] = {0, 0, 0};
    // stage capture (ld_debug_capture): device buffer of m_x and I^bf for max_batch frames, or null
    void *dbg = nullptr;
    bool dbg_valid = false;      // the last single-size call ran with the capture on
    std::string err;
};

namespace {

int fail(ld_handle *h, int code, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(ld_handle *h, cudaError_t e, const char *what)
{
    return fail(h, LD_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Eq. 16 in Q15 and Eq. 23 in Q12, built in double from the definitions.
void build_tables(const ld_params &p, int32_t *ws_q, int32_t *wr_q, int32_t *wg_q)
{
    const int rho = p.bf_rho, n = 2 * rho + 1;
    if (ws_q)
        for (int dy = -rho; dy <= rho; ++dy)
            for (int dx = -rho; dx <= rho; ++dx) {
                const double d2 = (double)(dx * dx + dy * dy);
                ws_q[(dy + rho) * n + dx + rho] = (int32_t)std::floor(std::exp(-d2 / (p.sigma_s * p.sigma_s)) * 32768.0 + 0.5);
            }
    if (wr_q)
        for (int k = 0; k < 256; ++k) {
            const double x = (double)k / 255.0;
            wr_q[k] = (int32_t)std::floor(std::exp(-(x * x) / (p.sigma_r * p.sigma_r)) * 32768.0 + 0.5);
        }
    if (wg_q)
        for (int i = 0; i < ld::kWgEntries; ++i) {
            const double pp = std::asin((double)i / 32768.0) * (36.0 / M_PI);   // p = dtheta / (pi / 36)
            const double e = p.wg_gaussian ? pp * pp : pp;
            wg_q[i] = (int32_t)std::floor(std::exp(-e / (p.sigma_g * p.sigma_g)) * 4096.0 + 0.5);
        }
}

// The largest image range r for which a road pixel provably fails the edge test, whatever the values
// inside its neighbourhood (the exact pruning of the gradient kernel); -1 when none or when the pre-filter
// is not the bilateral.  Let every pixel of the (2 rho + 3)^2 neighbourhood of a pixel s lie in [m, m + r].
//  1. Every tap weight of Eq. 16 in Q15, w = (ws * wr(|dI|) + 2^14) >> 15, of every window centred in the
//     3x3 neighbourhood of s lies in [a, b], a = min over classes at |dI| = r (wr is non-increasing),
//     b = max over classes at |dI| = 0.
//  2. For a window of n taps with mean mu, sum(w q) / sum(w) - mu = sum((w - (a+b)/2)(q - mu)) / sum(w), and
//     sum|q - mu| <= n r / 2 for values in an interval of length r, so the weighted mean is within
//     (b - a) r / (4 a) of mu; the rounded output (2 sum(wq) + sum(w)) / (2 sum(w)) adds at most 1/2: e.
//  3. Windows two columns (or rows) apart share all but 2 (2 rho + 1) taps, so their means differ by at
//     most 2 r / (2 rho + 1).
//  4. Each Sobel component sums weights 1, 2, 1 of such differences: |G_x|, |G_y| <= 4 (2r / (2 rho + 1) + 2e),
//     and G_x^2 + G_y^2 <= 2 * that^2.  When that is at most thr^2 the pixel is not an edge.
// The windows must lie inside the frame (n = (2 rho + 1)^2); the kernel never prunes near the border.
int32_t flat_range(const ld_params &p)
{
    if (p.bilateral != 1)
        return -1;
    const int rho = p.bf_rho, N = 2 * rho + 1;
    int32_t ws_q[121], wr_q[256];
    build_tables(p, ws_q, wr_q, nullptr);
    int64_t b = 0;
    for (int i = 0; i < N * N; ++i)
        b = std::max<int64_t>(b, ((int64_t)ws_q[i] * wr_q[0] + 16384) >> 15);
    const double thr2 = (double)p.edge_thresh * p.edge_thresh;
    int32_t best = -1;
    for (int r = 0; r < 255; ++r) {
        int64_t a = INT64_MAX;
        for (int i = 0; i < N * N; ++i)
            a = std::min<int64_t>(a, ((int64_t)ws_q[i] * wr_q[r] + 16384) >> 15);
        if (a <= 0)
            break;
        const double e = (double)(b - a) * r / (4.0 * a) + 0.5;
        const double g = 4.0 * (2.0 * r / N + 2.0 * e);
        if (2.0 * g * g * (1.0 + 1e-9) > thr2)   // margin against the rounding of this evaluation
            break;
        best = r;
    }
    return best;
}

const char *check_params(const ld_params *p)
{
    if (!p)
        return "params is NULL";
    if (p->n_disp < 4 || p->n_disp > LD_MAX_D)
        return "n_disp must be in [4, 256]";
    if (p->tau_y < 0 || p->tau_y > 15)
        return "tau_y must be in [0, 15]";
    if (p->tau_x < 0 || p->tau_x > 7)
        return "tau_x must be in [0, 7]";
    if (p->lambda_y < 0 || p->lambda_x < 0 || p->lambda_y > 1000 || p->lambda_x > 1000)
        return "lambda_y / lambda_x must be in [0, 1000]";
    if (!(p->tr_y > 0.0f) || !(p->tr_x > 0.0f))
        return "tr_y / tr_x must be > 0";
    if (p->eps_den <= 0 || p->eps_num < 0 || p->eps_num > p->eps_den)
        return "eps must be a fraction in [0, 1]";
    if (!(p->varpi >= 0.0f))
        return "varpi must be >= 0";
    if (p->bf_rho < 1 || p->bf_rho > 5)
        return "bf_rho must be in [1, 5]";
    if (!(p->sigma_s > 0.0) || !(p->sigma_r > 0.0) || !(p->sigma_g > 0.0))
        return "sigma_s, sigma_r, sigma_g must be > 0";
    if (p->edge_thresh < 0 || p->edge_thresh > 4 * 255 * 2)
        return "edge_thresh must be in [0, 2040]";
    if (p->vote_rho < 1 || p->vote_rho > 16)
        return "vote_rho must be in [1, 16]";
    if (p->chi < 0 || p->chi > 256)
        return "chi must be in [0, 256]";
    if (p->box_nu < 0 || p->box_nu > 8 || p->box_vs < 0 || p->box_vs > 8)
        return "box_nu / box_vs must be in [0, 8]";
    if (p->lambda_g < 0 || p->lambda_g > 1)
        return "lambda_g must be 0 or 1";
    if (p->xi_den <= 0 || p->xi_num < 0 || p->xi_num > p->xi_den)
        return "xi must be a fraction in [0, 1]";
    if (p->thr_den <= 0 || p->thr_num < 0 || p->thr_num > p->thr_den)
        return "thr must be a fraction in [0, 1]";
    if (p->near_px < 0 || p->max_lanes < 1 || p->max_lanes > LD_MAX_LANES)
        return "near_px must be >= 0 and max_lanes in [1, 8]";
    if (p->ransac_hyps < 1 || p->ransac_hyps > ld::kMaxHyps || p->ransac_rounds < 1 || p->ransac_rounds > 1 << 20)
        return "ransac_hyps must be in [1, 256] and ransac_rounds >= 1";
    if (p->bilateral < 0 || p->bilateral > 2)
        return "bilateral must be 0 (none), 1 (bilateral) or 2 (median)";
    if (p->wg_gaussian < 0 || p->wg_gaussian > 1 || p->thr_abs > 0 || p->dp_literal < 0 || p->dp_literal > 1 ||
        p->band_literal_bottom < 0 || p->band_literal_bottom > 1)
        return "wg_gaussian, dp_literal and band_literal_bottom must be 0 or 1 and thr_abs <= 0";
    return nullptr;
}

ld::KParams make_kparams(const ld_handle *h, int W, int H, int n)
{
    const ld_params &p = h->p;
    ld::KParams k{};
    k.W = W;
    k.H = H;
    k.D = p.n_disp;
    k.n_frames = n;
    k.tau_y = p.tau_y;
    k.lambda_y = p.lambda_y;
    k.tr_y = p.tr_y;
    k.eps_num = p.eps_num;
    k.eps_den = p.eps_den;
    k.varpi = p.varpi;
    k.bilateral = p.bilateral;
    k.rho = p.bf_rho;
    k.edge_thresh2 = p.edge_thresh * p.edge_thresh;
    k.vote_rho = p.vote_rho;
    k.chi = p.chi;
    k.tau_x = p.tau_x;
    k.lambda_x = p.lambda_x;
    k.tr_x = p.tr_x;
    k.box_nu = p.box_nu;
    k.box_vs = p.box_vs;
    k.lambda_g = p.lambda_g;
    k.S0 = (int32_t)((int64_t)W * p.xi_num / p.xi_den);
    k.n_starts = W + 2 * k.S0;
    k.thr_num = p.thr_num;
    k.thr_den = p.thr_den;
    k.near_px = p.near_px;
    k.max_lanes = p.max_lanes;
    k.thr_abs = p.thr_abs;
    k.dp_literal = p.dp_literal;
    k.band_literal = p.band_literal_bottom;
    k.hyps = p.ransac_hyps;
    k.rounds = p.ransac_rounds;
    k.key0 = (uint32_t)p.seed;
    k.key1 = (uint32_t)(p.seed >> 32);
    k.centre = (H - 1) / 2;
    int e = 0;
    const int half = (H - 1 - k.centre) > k.centre ? (H - 1 - k.centre) : k.centre;
    while ((1 << e) < half)
        ++e;
    k.e = e;
    k.vote_cap = kVoteCap;
    const int n_ws = (2 * p.bf_rho + 1) * (2 * p.bf_rho + 1);
    for (int i = 0; i < n_ws; ++i)
        k.ws[i] = (uint16_t)h->ws_q[i];
    // distance classes of the bilateral taps: rank of dx^2 + dy^2 among the distinct values
    {
        const int rho = p.bf_rho, nn = 2 * rho + 1;
        bool seen[2 * 5 * 5 + 1] = {};
        for (int dy = -rho; dy <= rho; ++dy)
            for (int dx = -rho; dx <= rho; ++dx)
                seen[dx * dx + dy * dy] = true;
        int rank[2 * 5 * 5 + 1] = {}, nc = 0;
        for (int r2 = 0; r2 <= 2 * rho * rho; ++r2)
            if (seen[r2])
                rank[r2] = nc++;
        k.n_cls = nc;
        for (int dy = -rho; dy <= rho; ++dy)
            for (int dx = -rho; dx <= rho; ++dx) {
                const int c = rank[dx * dx + dy * dy];
                k.cls_ws[c] = (uint16_t)h->ws_q[(dy + rho) * nn + dx + rho];
            }
    }
    k.flat_range = flat_range(p);
    k.pmax_hint = h->w.pmax;
    k.seg_rows = ld::vpx_seg_rows(k, (size_t)h->smem_optin - 1024);
    const bool tuned = W == h->tile_w && H == h->tile_h;
    k.tile_vdisp = tuned ? h->tile[0] : 0;
    k.tile_grad = tuned ? h->tile[1] : 0;
    k.tile_m1 = tuned ? h->tile[2] : 0;
    return k;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Launches [first, last) of the sequence of one detection of kp.n_frames frames on stream s, on the
// workspace view w; with `timed`, an event is recorded before and after every kernel.
int enqueue_range(ld_handle *h, const ld::KParams &kp, const ld::Work &w, const float *disp, const uint8_t *img,
                  ld_lanes *out, cudaStream_t s, bool timed, int first, int last)
{
    cudaError_t e = cudaSuccess;
    const size_t npx = (size_t)kp.n_frames * kp.H * kp.W;
    // buffer resets before stage k: stage capture (I^bf starts at -1, not computed; m_x at 0, rows above
    // v_top) and the per-row lists the gradient kernel's tiles append their edges and votes to.  No earlier
    // stage touches these buffers, so the timed form makes them before its first event, which keeps them
    // out of the per-kernel times.
    auto resets = [&](int k) -> int {
        if (k == 3 && w.dbg_ibf && (e = cudaMemsetAsync(w.dbg_ibf, 0xff, npx * 2, s)) != cudaSuccess)
            return cuda_fail(h, e, "capture reset");
        if (k == 3 && ((e = cudaMemsetAsync(w.ecount, 0, (size_t)kp.n_frames * kp.H * 4, s)) != cudaSuccess ||
                       (e = cudaMemsetAsync(w.vcount, 0, (size_t)kp.n_frames * kp.H * 4, s)) != cudaSuccess))
            return cuda_fail(h, e, "edge count reset");
        if (k == 4 && w.dbg_mx && (e = cudaMemsetAsync(w.dbg_mx, 0, npx * 4, s)) != cudaSuccess)
            return cuda_fail(h, e, "capture reset");
        return LD_OK;
    };
    if (timed)
        for (int k = first; k < last; ++k)
            if (resets(k) != LD_OK)
                return LD_E_CUDA;
    if (timed && (e = cudaEventRecord(h->ev[first], s)) != cudaSuccess)
        return cuda_fail(h, e, "event record");
    for (int k = first; k < last; ++k) {
        if (!timed && resets(k) != LD_OK)
            return LD_E_CUDA;
        nvtxRangePushA(kLaunchNames[k]);   // a profiler timeline shows each stage's enqueue by name
        switch (k) {
        case 0: e = ld::launch_vdisp(kp, w, disp, s); break;
        case 1: e = ld::launch_road(kp, w, s); break;
        case 2: e = ld::launch_fit_y(kp, w, s); break;
        case 3:
            if (kp.bilateral == 2) {   // median pre-filter into the workspace, then Sobel on its output
                ld::KParams kg = kp;
                kg.bilateral = 0;
                e = ld::launch_median(kp, w, img, s);
                if (e == cudaSuccess)
                    e = ld::launch_grad(kg, w, disp, w.med, s);
            } else {
                e = ld::launch_grad(kp, w, disp, img, s);
            }
            break;
        case 4: e = ld::launch_vpx(kp, w, s); break;
        case 5: e = ld::launch_fit_x(kp, w, s); break;
        case 6: e = ld::launch_m1(kp, w, s); break;
        case 7: e = ld::launch_energy(kp, w, s); break;
        default: e = ld::launch_select(kp, w, out, s); break;
        }
        nvtxRangePop();
        if (e != cudaSuccess)
            return cuda_fail(h, e, kLaunchNames[k]);
        if (timed && (e = cudaEventRecord(h->ev[k + 1], s)) != cudaSuccess)
            return cuda_fail(h, e, "event record");
    }
    return LD_OK;
}

// The nine launches of one detection.
int enqueue_on(ld_handle *h, const ld::KParams &kp, const ld::Work &w, const float *disp, const uint8_t *img,
               ld_lanes *out, cudaStream_t s, bool timed)
{
    return enqueue_range(h, kp, w, disp, img, out, s, timed, 0, kLaunches);
}

int enqueue(ld_handle *h, const ld::KParams &kp, const float *disp, const uint8_t *img, ld_lanes *out,
            bool timed = false)
{
    return enqueue_on(h, kp, h->w, disp, img, out, h->stream, timed);
}

// The workspace seen from frame f0 on: every per-frame array advanced by f0 frames of this call's size.
ld::Work work_from(const ld::Work &w, const ld::KParams &kp, int f0)
{
    const size_t f = f0, W = kp.W, H = kp.H, D = kp.D;
    ld::Work v = w;
    v.myT += f * D * H;
    v.fs += f;
    v.rows += f * 3 * H;
    v.path_y += f * D;
    v.inl_y += f * D;
    v.ecount += f * H;
    v.edges += f * H * W * 4;
    v.vcount += f * H;
    v.vbins += f * H * W;
    v.path_x += f * H;
    v.inl_x += f * H;
    v.pts += f * 2 * 3 * (size_t)w.pmax;
    v.npts += f * 2;
    v.gbt += f * (size_t)w.max_h * ld::vpx_row_bytes(w.max_w);
    v.M1 += f * H * W;
    if (v.med)
        v.med += f * H * W;
    if (v.xsum)
        v.xsum += f * (size_t)((H + 3) / 4) * ((W + 3) / 4);
    v.HE += f * (size_t)kp.n_starts;
    if (v.dbg_mx)
        v.dbg_mx += f * H * W;
    if (v.dbg_ibf)
        v.dbg_ibf += f * H * W;
    return v;
}

// Two half-batches on the handle's two sub-streams, forked from and joined back to the handle's stream
// (inside a capture, two concurrent branches of the graph that the GPU interleaves).  Staggering the
// halves (the second half's gradient kernel after the first's) was slower: a gradient CTA holds 213 KB of
// shared memory, so the first half's serial kernels waited for SMs.
int enqueue_split(ld_handle *h, int w, int hh, int n, const float *disp, const uint8_t *img, ld_lanes *out)
{
    cudaError_t e = cudaEventRecord(h->fork, h->stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "fork");
    const int n0 = (n + 1) / 2;
    for (int k = 0; k < 2; ++k) {
        const int f0 = k ? n0 : 0, nk = k ? n - n0 : n0;
        const ld::KParams kp = make_kparams(h, w, hh, nk);
        const ld::KParams kfull = make_kparams(h, w, hh, n);
        if ((e = cudaStreamWaitEvent(h->sub[k], h->fork, 0)) != cudaSuccess)
            return cuda_fail(h, e, "fork wait");
        const size_t px = (size_t)f0 * w * hh;
        const int rc = enqueue_on(h, kp, work_from(h->w, kfull, f0), disp + px, img + px, out + f0, h->sub[k], false);
        if (rc != LD_OK)
            return rc;
        if ((e = cudaEventRecord(h->join[k], h->sub[k])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->stream, h->join[k], 0)) != cudaSuccess)
            return cuda_fail(h, e, "join");
    }
    return LD_OK;
}

// The groups of one ld_detect_groups call.  Group g runs on the workspace seen from frame F_g on, counted
// in frames of the handle's largest size: each per-frame array's stride for a smaller frame is at most
// its stride for the largest one, so the group's frames stay inside [F_g, F_g + n_g) of those frames.
// With `fork`, the groups go to the handle's two sub-streams (forked from and joined back to its stream),
// largest first, each to the sub-stream with fewer pixels so far; otherwise they follow one another on the
// handle's stream.
int enqueue_groups(ld_handle *h, const ld_group *g, int ng, bool fork)
{
    const ld::KParams kmax = make_kparams(h, h->max_w, h->max_h, h->max_batch);
    std::vector<int> first(ng), order(ng);
    for (int i = 0, f = 0; i < ng; f += g[i].n_frames, ++i) {
        first[i] = f;
        order[i] = i;
    }
    auto px = [&](int i) { return (size_t)g[i].w * g[i].h * g[i].n_frames; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return px(a) > px(b); });
    cudaError_t e = cudaSuccess;
    if (fork) {
        if ((e = cudaEventRecord(h->fork, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "fork");
        for (int k = 0; k < 2; ++k)
            if ((e = cudaStreamWaitEvent(h->sub[k], h->fork, 0)) != cudaSuccess)
                return cuda_fail(h, e, "fork wait");
    }
    size_t load[2] = {0, 0};
    for (int i : order) {
        const int k = load[0] <= load[1] ? 0 : 1;
        load[k] += px(i);
        const ld::KParams kp = make_kparams(h, g[i].w, g[i].h, g[i].n_frames);
        const int rc = enqueue_on(h, kp, work_from(h->w, kmax, first[i]), g[i].disp, g[i].img, g[i].out_lanes,
                                  fork ? h->sub[k] : h->stream, false);
        if (rc != LD_OK)
            return rc;
    }
    if (fork)
        for (int k = 0; k < 2; ++k)
            if ((e = cudaEventRecord(h->join[k], h->sub[k])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(h->stream, h->join[k], 0)) != cudaSuccess)
                return cuda_fail(h, e, "join");
    return LD_OK;
}

// The frames of a group list as descriptors (h->h_fdesc): each frame's own parameters and the workspace
// seen from its slot (frames counted in the largest size, as enqueue_groups views them).  Returns the
// launch parameters of the list's largest frame (grid and shared-memory shapes) and the V_px kernel's
// shared memory (the largest over the frames).
struct MixedHalf {
    ld::KParams kl;      // launch shapes: the half's largest frame
    int first, n;        // descriptors [first, first + n)
    size_t vpx_smem;
};

// The list is split into two halves that run concurrently: the groups by pixel count, largest first, each
// to the half with fewer pixels so far (a group of one size whose frames outweigh the rest gets a half of
// its own, and its long serial stages overlap the other half's frames; a half holding several groups
// mixes their sizes in each launch); one group alone is split by frames.  Each half's descriptors are
// contiguous.
int fill_descriptors(ld_handle *h, const ld_group *g, int ng, MixedHalf half[2])
{
    const ld::KParams kmax = make_kparams(h, h->max_w, h->max_h, h->max_batch);
    struct Fr { int grp, k, F; size_t px; };
    std::vector<Fr> fr;
    for (int i = 0, F = 0; i < ng; F += g[i].n_frames, ++i)
        for (int k = 0; k < g[i].n_frames; ++k)
            fr.push_back({i, k, F + k, (size_t)g[i].w * g[i].h});
    const int n = (int)fr.size();
    std::vector<int> gside(ng, 0), order(ng);
    for (int i = 0; i < ng; ++i)
        order[i] = i;
    auto gpx = [&](int i) { return (size_t)g[i].w * g[i].h * g[i].n_frames; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gpx(a) > gpx(b); });
    size_t load[2] = {0, 0};
    for (int i : order) {
        const int s = load[0] <= load[1] ? 0 : 1;
        gside[i] = s;
        load[s] += gpx(i);
    }
    std::vector<int> side(n);
    int cnt[2] = {0, 0};
    for (int j = 0; j < n; ++j) {
        // one group alone: its frames alternate between the halves
        const int s = ng == 1 ? (fr[j].k & 1) : gside[fr[j].grp];
        side[j] = s;
        ++cnt[s];
    }
    int pos[2] = {0, cnt[0]};
    int Wm[2] = {16, 16}, Hm[2] = {16, 16};
    size_t vs[2] = {0, 0};
    for (int j = 0; j < n; ++j) {
        const ld_group &gg = g[fr[j].grp];
        ld::KParams kp = make_kparams(h, gg.w, gg.h, 1);
        kp.tile_vdisp = kp.tile_grad = kp.tile_m1 = 0;   // one launch shape for all sizes: the built-in rules
        const int s = side[j];
        Wm[s] = std::max(Wm[s], (int)gg.w);
        Hm[s] = std::max(Hm[s], (int)gg.h);
        vs[s] = std::max(vs[s], ld::vpx_smem_bytes(kp));
        const size_t px = (size_t)gg.w * gg.h;
        ld::FrameDesc &d = h->h_fdesc[pos[s]++];
        d.kp = kp;
        d.w = work_from(h->w, kmax, fr[j].F);
        d.disp = gg.disp + fr[j].k * px;
        d.img = gg.img + fr[j].k * px;
        d.out = gg.out_lanes + fr[j].k;
    }
    for (int s = 0; s < 2; ++s) {
        half[s].kl = make_kparams(h, Wm[s], Hm[s], cnt[s]);
        half[s].kl.tile_vdisp = half[s].kl.tile_grad = half[s].kl.tile_m1 = 0;
        half[s].first = s ? cnt[0] : 0;
        half[s].n = cnt[s];
        half[s].vpx_smem = vs[s];
    }
    return n;
}

// The nine stages of a mixed call, one launch each over all frames (descriptors at fd, already on the
// device), on the handle's stream.
int enqueue_mixed_half(ld_handle *h, const ld::KParams &kl, const ld::FrameDesc *fd, int n, size_t vpx_smem,
                       cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kLaunches; ++k) {
        nvtxRangePushA(kLaunchNames[k]);
        switch (k) {
        case 0: e = ld::launch_vdisp_fd(kl, fd, n, s); break;
        case 1: e = ld::launch_road_fd(kl, fd, n, s); break;
        case 2: e = ld::launch_fit_y_fd(kl, fd, n, s); break;
        case 3:
            if (kl.bilateral == 2) {
                e = ld::launch_median_fd(kl, fd, n, s);
                if (e == cudaSuccess)
                    e = ld::launch_grad_fd(kl, fd, n, true, s);
            } else {
                e = ld::launch_grad_fd(kl, fd, n, false, s);
            }
            break;
        case 4: e = ld::launch_vpx_fd(kl, fd, n, vpx_smem, s); break;
        case 5: e = ld::launch_fit_x_fd(kl, fd, n, s); break;
        case 6: e = ld::launch_m1_fd(kl, fd, n, s); break;
        case 7: e = ld::launch_energy_fd(kl, fd, n, s); break;
        default: e = ld::launch_select_fd(kl, fd, n, s); break;
        }
        nvtxRangePop();
        if (e != cudaSuccess)
            return cuda_fail(h, e, kLaunchNames[k]);
    }
    return LD_OK;
}

// The two halves of a mixed call on the handle's sub-streams, forked from and joined back to its stream;
// the per-row edge counts (and the stage capture) of every frame slot are reset first.
int enqueue_mixed(ld_handle *h, const MixedHalf half[2], const ld::FrameDesc *fd, int n)
{
    cudaStream_t s = h->stream;
    const size_t rows = (size_t)n * h->max_h, px = rows * h->max_w;   // the frames' slots, largest-size strides
    cudaError_t e = cudaSuccess;
    if (h->w.dbg_ibf && (e = cudaMemsetAsync(h->w.dbg_ibf, 0xff, px * 2, s)) != cudaSuccess)
        return cuda_fail(h, e, "capture reset");
    if (h->w.dbg_mx && (e = cudaMemsetAsync(h->w.dbg_mx, 0, px * 4, s)) != cudaSuccess)
        return cuda_fail(h, e, "capture reset");
    if ((e = cudaMemsetAsync(h->w.ecount, 0, rows * 4, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->w.vcount, 0, rows * 4, s)) != cudaSuccess)
        return cuda_fail(h, e, "edge count reset");
    if ((e = cudaEventRecord(h->fork, s)) != cudaSuccess)
        return cuda_fail(h, e, "fork");
    for (int k = 0; k < 2; ++k) {
        if (half[k].n == 0)
            continue;
        if ((e = cudaStreamWaitEvent(h->sub[k], h->fork, 0)) != cudaSuccess)
            return cuda_fail(h, e, "fork wait");
        const int rc = enqueue_mixed_half(h, half[k].kl, fd + half[k].first, half[k].n, half[k].vpx_smem, h->sub[k]);
        if (rc != LD_OK)
            return rc;
        if ((e = cudaEventRecord(h->join[k], h->sub[k])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, h->join[k], 0)) != cudaSuccess)
            return cuda_fail(h, e, "join");
    }
    return LD_OK;
}

bool same_groups(const std::vector<ld_group> &a, const ld_group *b, int n)
{
    if ((int)a.size() != n)
        return false;
    for (int i = 0; i < n; ++i)
        if (a[i].disp != b[i].disp || a[i].img != b[i].img || a[i].out_lanes != b[i].out_lanes || a[i].w != b[i].w ||
            a[i].h != b[i].h || a[i].n_frames != b[i].n_frames)
            return false;
    return true;
}

void drop_graphs(ld_handle *h)
{
    for (GraphSlot &g : h->graphs)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g = GraphSlot();
        }
    for (GroupGraph &g : h->group_graphs)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g = GroupGraph();
        }
    for (MixedGraph &g : h->mixed_graphs)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g = MixedGraph();
        }
}

void release_sync_objects(ld_handle *h)
{
    for (int k = 0; k <= kLaunches; ++k)
        if (h->ev[k])
            cudaEventDestroy(h->ev[k]);
    if (h->fork)
        cudaEventDestroy(h->fork);

    for (int k = 0; k < 2; ++k) {
        if (h->join[k])
            cudaEventDestroy(h->join[k]);
        if (h->sub[k])
            cudaStreamDestroy(h->sub[k]);
    }
}

int check_call(ld_handle *h, const void *disp, const void *img, int w, int hh, int n, const void *out)
{
    if (!h)
        return LD_E_ARG;
    if (!disp || !img || !out)
        return fail(h, LD_E_ARG, "null buffer");
    if (w < 16 || hh < 16 || w > h->max_w || hh > h->max_h)
        return fail(h, LD_E_ARG, "frame size outside [16, max_w] x [16, max_h]");
    if (n < 1 || n > h->max_batch)
        return fail(h, LD_E_ARG, "n_frames outside [1, max_batch]");
    return LD_OK;
}

}  // namespace

namespace ld {
void set_global_error(const char *msg) { g_create_error = msg; }

// Access for the learned proposal's runtime (ld_net.cu), which drives a handle's plain stages.
int handle_fail(ld_handle *h, int code, const char *msg) { return fail(h, code, msg); }
int handle_cuda_fail(ld_handle *h, cudaError_t e, const char *what) { return cuda_fail(h, e, what); }
int handle_check(ld_handle *h, const void *disp, const void *img, int w, int hh, int n, const void *out)
{
    return check_call(h, disp, img, w, hh, n, out);
}
void handle_dims(const ld_handle *h, int *max_w, int *max_h, int *max_batch)
{
    *max_w = h->max_w;
    *max_h = h->max_h;
    *max_batch = h->max_batch;
}
const ld_params &handle_params(const ld_handle *h) { return h->p; }
cudaStream_t handle_stream(const ld_handle *h) { return h->stream; }
Work handle_work(const ld_handle *h) { return h->w; }
// parameters of a call on w x hh x n frames; the call becomes the one ld_debug_get reports on
KParams handle_call(ld_handle *h, int w, int hh, int n)
{
    h->last_w = w;
    h->last_h = hh;
    h->last_n = n;
    h->have_last = true;
    h->dbg_valid = h->dbg != nullptr;
    return make_kparams(h, w, hh, n);
}
KParams handle_kparams(const ld_handle *h, int w, int hh, int n) { return make_kparams(h, w, hh, n); }
// launches [first, last) of the plain sequence (0 k_vdisp ... 6 k_m1, 7 k_energy, 8 k_select) on stream s
// (null: the handle's stream)
int handle_enqueue(ld_handle *h, const KParams &kp, const Work &w, const float *disp, const uint8_t *img,
                   ld_lanes *out, int first, int last, cudaStream_t s)
{
    return enqueue_range(h, kp, w, disp, img, out, s ? s : h->stream, false, first, last);
}
// the workspace seen from frame f0 of a call on frames of kp's size
Work work_view(const Work &w, const KParams &kp, int f0) { return work_from(w, kp, f0); }
}  // namespace ld

extern "C" {

void ld_params_default(ld_params *p)
{
    if (!p)
        return;
    std::memset(p, 0, sizeof(*p));
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
    p->max_lanes = LD_MAX_LANES;
    p->ransac_hyps = 64;
    p->ransac_rounds = 64;
    p->seed = 0x1807027520ull;
}

int32_t ld_n_starts(const ld_params *p, int32_t w)
{
    if (!p || p->xi_den <= 0 || w < 0)
        return 0;
    return w + 2 * (int32_t)((int64_t)w * p->xi_num / p->xi_den);
}

int ld_tables(const ld_params *p, int32_t *ws_q, int32_t *wr_q, int32_t *wg_q)
{
    if (check_params(p))
        return LD_E_ARG;
    build_tables(*p, ws_q, wr_q, wg_q);
    return LD_OK;
}

int32_t ld_flat_range(const ld_params *p)
{
    if (check_params(p))
        return -1;
    return flat_range(*p);
}

int32_t ld_launches_per_detect(void) { return kLaunches; }

const char *ld_launch_name(int32_t k) { return k >= 0 && k < kLaunches ? kLaunchNames[k] : ""; }

int ld_create(const ld_params *p, int32_t max_w, int32_t max_h, int32_t max_batch, void *cuda_stream, ld_handle **out)
{
    if (!out)
        return fail(nullptr, LD_E_ARG, "out is NULL");
    *out = nullptr;
    if (const char *why = check_params(p))
        return fail(nullptr, LD_E_ARG, why);
    if (max_w < 16 || max_w > LD_MAX_W || max_h < 16 || max_h > LD_MAX_H || max_batch < 1 || max_batch > 65535)
        return fail(nullptr, LD_E_ARG, "max_w / max_h / max_batch out of range");
    ld_handle *h = new ld_handle();
    h->p = *p;
    h->max_w = max_w;
    h->max_h = max_h;
    h->max_batch = max_batch;
    h->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "device query");
        delete h;
        return LD_E_CUDA;
    }
    build_tables(h->p, h->ws_q, nullptr, nullptr);

    // the V_px DP needs shared memory for a block of backtrack rows and the vote bitmaps of the largest frame
    ld::KParams kmax = make_kparams(h, max_w, max_h, max_batch);
    if (kmax.seg_rows < 1 || ld::road_smem_bytes(kmax) > (size_t)h->smem_optin - 1024) {
        delete h;
        return fail(nullptr, LD_E_ARG, "frame too large for the shared-memory budget");
    }
    // DP energies stay far below the int32 sentinel of the DP kernels
    const double e_x = ((double)p->vote_rho * (2.0 * p->chi + 1.0) * max_w + (double)p->lambda_x * p->tau_x) * max_h;
    const double e_y = ((double)max_w + (double)p->lambda_y * p->tau_y) * p->n_disp;
    if (e_x >= 1073741824.0 || e_y >= 1073741824.0) {
        delete h;
        return fail(nullptr, LD_E_ARG, "vote_rho, chi, lambda and the frame size allow DP energies beyond 2^30");
    }
    const size_t n = max_batch, W = max_w, H = max_h, D = p->n_disp;
    const size_t pmax = D > H ? D : H;
    const size_t n_starts = (size_t)ld_n_starts(p, max_w);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t o_my = take(n * D * H * 4), o_fs = take(n * sizeof(ld::FrameState)), o_rows = take(n * 3 * H * 4);
    const size_t o_py = take(n * D * 2), o_iy = take(n * D), o_ec = take(n * H * 4), o_ed = take(n * H * W * 8);
    const size_t o_vc = take(n * H * 4), o_vb = take(n * H * W * 2), o_px = take(n * H * 2), o_ix = take(n * H);
    const size_t o_bt = take(n * H * (size_t)ld::vpx_row_bytes(max_w)), o_m1 = take(n * H * W * 4), o_he = take(n * n_starts * 8);
    const size_t o_pts = take(n * 2 * 3 * pmax * 2), o_np = take(n * 2 * 4);
    const size_t o_tab = take(sizeof(int32_t) * (ld::kWrEntries + ld::kWgEntries));
    const size_t o_cls = take(sizeof(uint16_t) * ld::kClsTables * 512);
    const size_t o_d = take(n * H * W * 4), o_i = take(n * H * W), o_l = take(n * sizeof(ld_lanes));
    const size_t o_med = take(p->bilateral == 2 ? n * H * W : 0);
    const size_t o_fd = take(sizeof(ld::FrameDesc) * kGraphSlots * n);
    e = cudaMalloc(&h->ws, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, LD_E_NOMEM, std::string("workspace allocation: ") + cudaGetErrorString(e));
    }
    h->ws_bytes = off;
    char *b = (char *)h->ws;
    ld::Work &w = h->w;
    w.myT = (int32_t *)(b + o_my);
    w.fs = (ld::FrameState *)(b + o_fs);
    w.rows = (float *)(b + o_rows);
    w.path_y = (int16_t *)(b + o_py);
    w.inl_y = (uint8_t *)(b + o_iy);
    w.ecount = (int32_t *)(b + o_ec);
    w.edges = (int16_t *)(b + o_ed);
    w.vcount = (int32_t *)(b + o_vc);
    w.vbins = (int16_t *)(b + o_vb);
    w.path_x = (int16_t *)(b + o_px);
    w.inl_x = (uint8_t *)(b + o_ix);
    w.gbt = (uint8_t *)(b + o_bt);
    w.M1 = (int32_t *)(b + o_m1);
    w.med = p->bilateral == 2 ? (uint8_t *)(b + o_med) : nullptr;
    w.HE = (int64_t *)(b + o_he);
    w.pts = (int16_t *)(b + o_pts);
    w.npts = (int32_t *)(b + o_np);
    w.pmax = (int32_t)pmax;
    h->d_tables = (int32_t *)(b + o_tab);
    w.wr = h->d_tables;
    w.wg = h->d_tables + ld::kWrEntries;
    w.cls_tab = (const uint16_t *)(b + o_cls);
    h->d_fdesc = (ld::FrameDesc *)(b + o_fd);
    w.max_w = max_w;
    w.max_h = max_h;
    h->d_disp = (float *)(b + o_d);
    h->d_img = (uint8_t *)(b + o_i);
    h->d_lanes = (ld_lanes *)(b + o_l);

    std::vector<int32_t> tab(ld::kWrEntries + ld::kWgEntries, 0);
    build_tables(h->p, nullptr, tab.data() + 256, tab.data() + ld::kWrEntries);
    // range weights indexed by q - c + 256: entry 256 + k and 256 - k hold wr(|k|); entries >= 512 stay 0
    for (int k = 1; k < 256; ++k)
        tab[256 - k] = tab[256 + k];
    tab[0] = 0;
    for (int k = 512; k < ld::kWrEntries; ++k)
        tab[k] = 0;
    e = cudaMemcpy(h->d_tables, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice);
    // the gradient kernel's per-class tables T_c[a] = (ws_c * wr(a) + 2^14) >> 15, a = |dI| < 256, zero above
    // (the sentinel outside the frame lands there); classes as in make_kparams
    if (e == cudaSuccess) {
        std::vector<uint16_t> cls((size_t)ld::kClsTables * 512, 0);
        for (int c = 0; c < kmax.n_cls; ++c)
            for (int a = 0; a < 256; ++a)
                cls[(size_t)c * 512 + a] = (uint16_t)(((uint32_t)kmax.cls_ws[c] * (uint32_t)tab[256 + a] + 16384u) >> 15);
        e = cudaMemcpy((void *)w.cls_tab, cls.data(), sizeof(uint16_t) * cls.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = ld::setup_dp(h->smem_optin);
    if (e == cudaSuccess)
        e = ld::setup_ransac(h->smem_optin);
    if (e == cudaSuccess)
        e = ld::setup_grad(h->smem_optin);
    if (e == cudaSuccess)
        e = ld::setup_lpv(h->smem_optin);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "workspace set-up");
        cudaFree(h->ws);
        delete h;
        return LD_E_CUDA;
    }
    for (int k = 0; k <= kLaunches && e == cudaSuccess; ++k)
        e = cudaEventCreate(&h->ev[k]);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);

    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&h->sub[k], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&h->join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h->h_fdesc, sizeof(ld::FrameDesc) * (size_t)max_batch);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "stream and event creation");
        release_sync_objects(h);
        cudaFree(h->ws);
        delete h;
        return LD_E_CUDA;
    }
    *out = h;
    return LD_OK;
}

}  // extern "C"
namespace {
int detect_call(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                ld_lanes *out_lanes);
}
extern "C" {

int ld_detect(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
              ld_lanes *out_lanes)
{
    nvtxRangePushA("ld_detect");
    const int rc = detect_call(h, disp, img, w, hh, n_frames, out_lanes);
    nvtxRangePop();
    return rc;
}

}  // extern "C"

namespace {
int detect_call(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                ld_lanes *out_lanes)
{
    int rc = check_call(h, disp, img, w, hh, n_frames, out_lanes);
    if (rc != LD_OK)
        return rc;
    const ld::KParams kp = make_kparams(h, w, hh, n_frames);
    h->last_w = w;
    h->last_h = hh;
    h->last_n = n_frames;
    h->have_last = true;
    h->dbg_valid = h->dbg != nullptr;
    // replay a captured graph when the same buffers and sizes come back
    for (GraphSlot &g : h->graphs)
        if (g.exec && g.disp == disp && g.img == img && g.out == out_lanes && g.w == w && g.h == hh && g.n == n_frames) {
            cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
            return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "graph launch");
        }
    // capture this call's launch sequence, then replay it
    cudaStreamCaptureStatus st;
    cudaError_t e = cudaStreamIsCapturing(h->stream, &st);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "stream query");
    if (st != cudaStreamCaptureStatusNone || h->stream == nullptr)  // caller captures, or legacy stream
        return enqueue(h, kp, disp, img, out_lanes);
    e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "begin capture");
    rc = n_frames >= kSplitMin ? enqueue_split(h, w, hh, n_frames, disp, img, out_lanes)
                               : enqueue(h, kp, disp, img, out_lanes);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (rc != LD_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess)
        return cuda_fail(h, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "graph instantiate");
    GraphSlot &g = h->graphs[h->next_slot];
    h->next_slot = (h->next_slot + 1) % kGraphSlots;
    if (g.exec)
        cudaGraphExecDestroy(g.exec);
    g.exec = exec;
    g.disp = disp;
    g.img = img;
    g.out = out_lanes;
    g.w = w;
    g.h = hh;
    g.n = n_frames;
    e = cudaGraphLaunch(exec, h->stream);
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "graph launch");
}
}  // namespace

extern "C" {

int ld_detect_groups(ld_handle *h, const ld_group *groups, int32_t n_groups)
{
    if (!h)
        return LD_E_ARG;
    if (!groups || n_groups < 1 || n_groups > LD_MAX_GROUPS)
        return fail(h, LD_E_ARG, "groups is NULL or n_groups outside [1, LD_MAX_GROUPS]");
    int64_t total = 0;
    for (int i = 0; i < n_groups; ++i) {
        const ld_group &g = groups[i];
        const int rc = check_call(h, g.disp, g.img, g.w, g.h, g.n_frames, g.out_lanes);
        if (rc != LD_OK)
            return rc;
        total += g.n_frames;
    }
    if (total > h->max_batch)
        return fail(h, LD_E_ARG, "the groups hold more than max_batch frames");
    h->have_last = false;   // the workspace now holds frames of several sizes
    for (GroupGraph &g : h->group_graphs)
        if (g.exec && same_groups(g.groups, groups, n_groups)) {
            cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
            return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "graph launch");
        }
    cudaStreamCaptureStatus st;
    cudaError_t e = cudaStreamIsCapturing(h->stream, &st);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "stream query");
    if (st != cudaStreamCaptureStatusNone || h->stream == nullptr)  // caller captures, or legacy stream
        return enqueue_groups(h, groups, n_groups, false);
    if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(h, e, "begin capture");
    const int rc = enqueue_groups(h, groups, n_groups, true);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (rc != LD_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess)
        return cuda_fail(h, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "graph instantiate");
    GroupGraph &g = h->group_graphs[h->next_group_slot];
    h->next_group_slot = (h->next_group_slot + 1) % kGraphSlots;
    if (g.exec)
        cudaGraphExecDestroy(g.exec);
    g.exec = exec;
    g.groups.assign(groups, groups + n_groups);
    e = cudaGraphLaunch(exec, h->stream);
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "graph launch");
}

int ld_detect_mixed(ld_handle *h, const ld_group *groups, int32_t n_groups)
{
    if (!h)
        return LD_E_ARG;
    if (!groups || n_groups < 1 || n_groups > LD_MAX_GROUPS)
        return fail(h, LD_E_ARG, "groups is NULL or n_groups outside [1, LD_MAX_GROUPS]");
    int64_t total = 0;
    for (int i = 0; i < n_groups; ++i) {
        const ld_group &g = groups[i];
        const int rc = check_call(h, g.disp, g.img, g.w, g.h, g.n_frames, g.out_lanes);
        if (rc != LD_OK)
            return rc;
        total += g.n_frames;
    }
    if (total > h->max_batch)
        return fail(h, LD_E_ARG, "the groups hold more than max_batch frames");
    h->have_last = false;   // the workspace now holds frames of several sizes
    for (MixedGraph &g : h->mixed_graphs)
        if (g.exec && same_groups(g.groups, groups, n_groups)) {
            cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
            return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "graph launch");
        }
    cudaStreamCaptureStatus st;
    cudaError_t e = cudaStreamIsCapturing(h->stream, &st);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "stream query");
    if (st != cudaStreamCaptureStatusNone || h->stream == nullptr)  // caller captures, or legacy stream
        return enqueue_groups(h, groups, n_groups, false);          // the same results, one group at a time
    // descriptors of this list into the next slot's device region (uploaded before the capture: the
    // graph's launches read them there on every replay)
    const int slot = h->next_mixed_slot;
    MixedHalf half[2];
    const int n = fill_descriptors(h, groups, n_groups, half);
    ld::FrameDesc *fd = h->d_fdesc + (size_t)slot * h->max_batch;
    MixedGraph &g = h->mixed_graphs[slot];
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g = MixedGraph();
    }
    if ((e = cudaMemcpyAsync(fd, h->h_fdesc, sizeof(ld::FrameDesc) * n, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "descriptor upload");
    if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(h, e, "begin capture");
    const int rc = enqueue_mixed(h, half, fd, n);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (rc != LD_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess)
        return cuda_fail(h, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "graph instantiate");
    h->next_mixed_slot = (slot + 1) % kGraphSlots;
    g.exec = exec;
    g.groups.assign(groups, groups + n_groups);
    e = cudaGraphLaunch(exec, h->stream);
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "graph launch");
}

}  // extern "C"

namespace {
// Holds a stream at a host function until the enqueueing thread opens it (at most one second).
struct StartGate {
    std::mutex m;
    std::condition_variable cv;
    bool is_open = false;
    void open()
    {
        {
            std::lock_guard<std::mutex> g(m);
            is_open = true;
        }
        cv.notify_all();
    }
};
void CUDART_CB start_gate_wait(void *arg)
{
    StartGate *g = static_cast<StartGate *>(arg);
    std::unique_lock<std::mutex> lk(g->m);
    g->cv.wait_for(lk, std::chrono::seconds(1), [&] { return g->is_open; });
}
}  // namespace

extern "C" {

int ld_detect_timed(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                    ld_lanes *out_lanes, float *ms_out)
{
    int rc = check_call(h, disp, img, w, hh, n_frames, out_lanes);
    if (rc != LD_OK)
        return rc;
    if (!ms_out)
        return fail(h, LD_E_ARG, "ms_out is NULL");
    const ld::KParams kp = make_kparams(h, w, hh, n_frames);
    h->last_w = w;
    h->last_h = hh;
    h->last_n = n_frames;
    h->have_last = true;
    h->dbg_valid = h->dbg != nullptr;
    // the stream waits at a host gate until every launch is enqueued, so the kernels run back to back as
    // in a captured call and no interval holds host enqueue time
    StartGate gate;
    cudaError_t e = cudaLaunchHostFunc(h->stream, start_gate_wait, &gate);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "start gate");
    rc = enqueue(h, kp, disp, img, out_lanes, true);
    gate.open();
    if (rc != LD_OK) {
        cudaStreamSynchronize(h->stream);   // the gate's host function has returned before it goes
        return rc;
    }
    e = cudaEventSynchronize(h->ev[kLaunches]);
    for (int k = 0; k < kLaunches && e == cudaSuccess; ++k)
        e = cudaEventElapsedTime(&ms_out[k], h->ev[k], h->ev[k + 1]);
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "event timing");
}

int ld_tune(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
            ld_lanes *out_lanes, int32_t *chosen)
{
    int rc = check_call(h, disp, img, w, hh, n_frames, out_lanes);
    if (rc != LD_OK)
        return rc;
    // candidates per tuned kernel (launch index in the sequence, rows per CTA); the launchers reduce a
    // value that does not fit their shared-memory budget
    static const int kTuned[3] = {0, 3, 6};  // k_vdisp, k_grad, k_m1
    static const std::vector<int> kCand[3] = {{8, 16, 32}, {8, 12, 16, 24, 32}, {8, 12, 14, 16}};
    constexpr int kReps = 3;
    h->tile_w = w;
    h->tile_h = hh;
    for (int t = 0; t < 3; ++t)
        h->tile[t] = 0;
    float ms[kLaunches];
    for (int t = 0; t < 3; ++t) {
        int best = 0;
        float best_ms = 1e30f;
        for (int c : kCand[t]) {
            h->tile[t] = c;
            float m = 1e30f;
            for (int r = 0; r < kReps; ++r) {
                rc = ld_detect_timed(h, disp, img, w, hh, n_frames, out_lanes, ms);
                if (rc != LD_OK) {
                    h->tile_w = h->tile_h = 0;
                    return rc;
                }
                m = ms[kTuned[t]] < m ? ms[kTuned[t]] : m;
            }
            if (m < best_ms) {
                best_ms = m;
                best = c;
            }
        }
        h->tile[t] = best;
    }
    // launch shapes changed: drop the captured graphs
    cudaError_t e = cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    if (chosen)
        for (int t = 0; t < 3; ++t)
            chosen[t] = h->tile[t];
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "tune sync");
}

int ld_detect_host(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                   ld_lanes *out_lanes)
{
    int rc = check_call(h, disp, img, w, hh, n_frames, out_lanes);
    if (rc != LD_OK)
        return rc;
    const size_t npx = (size_t)n_frames * hh * w;
    cudaError_t e = cudaMemcpyAsync(h->d_disp, disp, npx * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_img, img, npx, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "input copy");
    rc = ld_detect(h, h->d_disp, h->d_img, w, hh, n_frames, h->d_lanes);
    if (rc != LD_OK)
        return rc;
    e = cudaMemcpyAsync(out_lanes, h->d_lanes, sizeof(ld_lanes) * n_frames, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "result copy");
}

size_t ld_debug_size(ld_handle *h, int32_t stage)
{
    if (!h || !h->have_last)
        return 0;
    const size_t W = h->last_w, H = h->last_h, D = h->p.n_disp;
    switch (stage) {
    case LD_STAGE_VDISP: return H * D * 4;
    case LD_STAGE_PATH_Y: return D * 2;
    case LD_STAGE_INL_Y: return D;
    case LD_STAGE_ROWS: return 3 * H * 4;
    case LD_STAGE_EDGES: return H * 4 + H * W * 8;
    case LD_STAGE_PATH_X: return H * 2;
    case LD_STAGE_INL_X: return H;
    case LD_STAGE_M1: return H * W * 4;
    case LD_STAGE_HE: return (size_t)ld_n_starts(&h->p, (int32_t)W) * 8;
    case LD_STAGE_MX: return H * W * 4;
    case LD_STAGE_IBF: return H * W * 2;
    default: return 0;
    }
}

int ld_debug_get(ld_handle *h, int32_t frame, int32_t stage, void *host_dst, size_t bytes)
{
    if (!h)
        return LD_E_ARG;
    if (!h->have_last)
        return fail(h, LD_E_STATE, "no single-size detect call to report on (none yet, or ld_detect_groups since)");
    if (frame < 0 || frame >= h->last_n || !host_dst)
        return fail(h, LD_E_ARG, "frame out of range or null destination");
    const size_t want = ld_debug_size(h, stage);
    if (want == 0 || bytes != want)
        return fail(h, LD_E_ARG, "unknown stage or wrong byte count");
    if ((stage == LD_STAGE_MX || stage == LD_STAGE_IBF) && !h->dbg_valid)
        return fail(h, LD_E_STATE, "m_x and I^bf are recorded only while ld_debug_capture is on");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "stream sync");
    const size_t W = h->last_w, H = h->last_h, D = h->p.n_disp, f = frame;
    ld::FrameState fs;
    e = cudaMemcpy(&fs, h->w.fs + f, sizeof(fs), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "debug copy");
    const bool no_road = fs.flags & (LD_F_DEGEN_Y | LD_F_NO_ROAD);
    const bool no_vp = no_road || (fs.flags & LD_F_DEGEN_X);
    char *dst = (char *)host_dst;
    switch (stage) {
    case LD_STAGE_VDISP: {
        std::vector<int32_t> t(D * H);
        e = cudaMemcpy(t.data(), h->w.myT + f * D * H, D * H * 4, cudaMemcpyDeviceToHost);
        int32_t *o = (int32_t *)dst;
        for (size_t v = 0; v < H; ++v)
            for (size_t d = 0; d < D; ++d)
                o[v * D + d] = t[d * H + v];
        break;
    }
    case LD_STAGE_PATH_Y: e = cudaMemcpy(dst, h->w.path_y + f * D, D * 2, cudaMemcpyDeviceToHost); break;
    case LD_STAGE_INL_Y: e = cudaMemcpy(dst, h->w.inl_y + f * D, D, cudaMemcpyDeviceToHost); break;
    case LD_STAGE_ROWS: e = cudaMemcpy(dst, h->w.rows + f * 3 * H, 3 * H * 4, cudaMemcpyDeviceToHost); break;
    case LD_STAGE_EDGES: {
        e = cudaMemcpy(dst, h->w.ecount + f * H, H * 4, cudaMemcpyDeviceToHost);
        std::memset(dst + H * 4, 0, H * W * 8);
        if (e == cudaSuccess && !no_road) {
            const int32_t *cnt = (const int32_t *)dst;
            for (size_t v = 0; v < H && e == cudaSuccess; ++v)
                if (cnt[v] > 0)
                    e = cudaMemcpy(dst + H * 4 + v * W * 8, h->w.edges + (f * H + v) * W * 4, (size_t)cnt[v] * 8,
                                   cudaMemcpyDeviceToHost);
        }
        break;
    }
    case LD_STAGE_PATH_X:
    case LD_STAGE_INL_X: {
        const size_t el = stage == LD_STAGE_PATH_X ? 2 : 1;
        std::memset(dst, 0, H * el);
        if (!no_road)
            e = stage == LD_STAGE_PATH_X ? cudaMemcpy(dst, h->w.path_x + f * H, H * 2, cudaMemcpyDeviceToHost)
                                         : cudaMemcpy(dst, h->w.inl_x + f * H, H, cudaMemcpyDeviceToHost);
        break;
    }
    case LD_STAGE_M1: {
        std::memset(dst, 0, H * W * 4);
        const size_t vt = (size_t)fs.v_top;
        if (!no_vp && vt < H)
            e = cudaMemcpy(dst + vt * W * 4, h->w.M1 + (f * H + vt) * W, (H - vt) * W * 4, cudaMemcpyDeviceToHost);
        break;
    }
    case LD_STAGE_HE: {
        const size_t ns = (size_t)ld_n_starts(&h->p, (int32_t)W);
        std::memset(dst, 0, ns * 8);
        if (!no_vp)
            e = cudaMemcpy(dst, h->w.HE + f * ns, ns * 8, cudaMemcpyDeviceToHost);
        break;
    }
    case LD_STAGE_MX: e = cudaMemcpy(dst, h->w.dbg_mx + f * H * W, H * W * 4, cudaMemcpyDeviceToHost); break;
    case LD_STAGE_IBF: e = cudaMemcpy(dst, h->w.dbg_ibf + f * H * W, H * W * 2, cudaMemcpyDeviceToHost); break;
    default: return fail(h, LD_E_ARG, "unknown stage");
    }
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "debug copy");
}

int ld_lane_tracks(ld_handle *h, const ld_lanes *lanes, int32_t n_frames, float *tracks_out)
{
    if (!h)
        return LD_E_ARG;
    if (!lanes || !tracks_out)
        return fail(h, LD_E_ARG, "null buffer");
    if (!h->have_last)
        return fail(h, LD_E_STATE, "no single-size detection to trace (none yet, or ld_detect_groups since)");
    if (n_frames < 1 || n_frames > h->last_n)
        return fail(h, LD_E_ARG, "n_frames outside [1, frames of the last call]");
    const ld::KParams kp = make_kparams(h, h->last_w, h->last_h, n_frames);
    cudaError_t e = ld::launch_tracks(kp, h->w, lanes, tracks_out, h->stream);
    return e == cudaSuccess ? LD_OK : cuda_fail(h, e, "lane tracks");
}

int ld_debug_capture(ld_handle *h, int32_t on)
{
    if (!h)
        return LD_E_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "stream sync");
    if ((on != 0) == (h->dbg != nullptr))
        return LD_OK;
    drop_graphs(h);   // the captured launches hold the workspace pointers
    h->dbg_valid = false;
    if (!on) {
        cudaFree(h->dbg);
        h->dbg = nullptr;
        h->w.dbg_mx = nullptr;
        h->w.dbg_ibf = nullptr;
        return LD_OK;
    }
    const size_t npx = (size_t)h->max_batch * h->max_w * h->max_h;
    e = cudaMalloc(&h->dbg, align_up(npx * 4) + npx * 2);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->dbg = nullptr;
        return fail(h, LD_E_NOMEM, std::string("capture buffer: ") + cudaGetErrorString(e));
    }
    h->w.dbg_mx = (int32_t *)h->dbg;
    h->w.dbg_ibf = (int16_t *)((char *)h->dbg + align_up(npx * 4));
    return LD_OK;
}

const char *ld_last_error(const ld_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int32_t ld_checked_build(void)
{
#ifdef LD_CHECKED
    return 1;
#else
    return 0;
#endif
}

int ld_check_status(int64_t out[4])
{
    if (!out)
        return LD_E_ARG;
    out[0] = out[1] = out[2] = out[3] = 0;
#ifdef LD_CHECKED
    cudaError_t e = cudaDeviceSynchronize();
    for (const auto &fns : ck_registry()) {
        unsigned long long w[4] = {0, 0, 0, 0};
        if (e == cudaSuccess)
            e = fns.first(w);
        if (e != cudaSuccess)
            break;
        if (w[0] && !out[0]) {
            out[1] = (int64_t)w[1];
            out[2] = (int64_t)w[2];
            out[3] = (int64_t)w[3];
        }
        out[0] += (int64_t)w[0];
    }
    if (e != cudaSuccess)
        return cuda_fail(nullptr, e, "check status");
#endif
    return LD_OK;
}

int ld_check_reset(void)
{
#ifdef LD_CHECKED
    cudaError_t e = cudaDeviceSynchronize();
    for (const auto &fns : ck_registry())
        if (e == cudaSuccess)
            e = fns.second();
    if (e != cudaSuccess)
        return cuda_fail(nullptr, e, "check reset");
#endif
    return LD_OK;
}

const char *ld_check_site_name(int32_t site)
{
    static const char *const names[ld::CK_N_SITES] = {
        "none", "selftest",
        "vdisp_bin", "vdisp_run", "vdisp_load", "vdisp_out",
        "road_path", "road_pts",
        "fit_npts", "fit_sample", "fit_row",
        "grad_tile", "grad_glist", "grad_group", "grad_tap", "grad_edge", "grad_vote",
        "vpx_tile", "vpx_vote", "vpx_voff", "vpx_stage", "vpx_path", "vpx_pts",
        "m1_edge", "m1_col", "m1_chunk",
        "energy_start", "energy_col", "energy_row",
        "select_start", "select_lanes", "track_col",
        "median_tile",
    };
    return site >= 0 && site < ld::CK_N_SITES ? names[site] : "?";
}

int ld_check_selftest(void)
{
#ifdef LD_CHECKED
    k_ck_selftest<<<1, 1>>>(7);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LD_OK : cuda_fail(nullptr, e, "check self-test");
#else
    return fail(nullptr, LD_E_STATE, "not the bounds-checked library (LD_CHECKED)");
#endif
}

void ld_destroy(ld_handle *h)
{
    if (!h)
        return;
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    release_sync_objects(h);
    cudaFree(h->ws);
    cudaFree(h->dbg);
    cudaFreeHost(h->h_fdesc);
    delete h;
}

}  // extern "C"

namespace ld {
size_t handle_device_bytes(const ld_handle *h) { return h ? h->ws_bytes : 0; }

// ld_detect without the graph cache: the nine launches are enqueued directly on the handle's stream (the
// serving path, whose batch sizes vary from call to call).
int detect_eager(ld_handle *h, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                 ld_lanes *out_lanes)
{
    int rc = check_call(h, disp, img, w, hh, n_frames, out_lanes);
    if (rc != LD_OK)
        return rc;
    const ld::KParams kp = make_kparams(h, w, hh, n_frames);
    h->last_w = w;
    h->last_h = hh;
    h->last_n = n_frames;
    h->have_last = true;
    h->dbg_valid = h->dbg != nullptr;
    return enqueue(h, kp, disp, img, out_lanes);
}
}  // namespace ld
