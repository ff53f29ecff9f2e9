// Host runtime of the learned lane-position proposal (the ld_net_* and ld_detect_learned entry points of
// include/ld.h): memory of a network, its training calls, and the learned form of the detection, which
// runs the handle's plain stages up to M_1 (with the block sums of |G_x w_g| accumulated on the way), the
// network, the ranking of the starts, exact energies of the proposed starts, the selection among them and
// the exhaustive fallback for the frames where that found no lane.
#include <cmath>
#include <cstring>
#include <string>

#include "ld_net.cuh"

namespace {
constexpr int kLearnedGraphs = 4;
constexpr int kLearnedSplitMin = 16;   // captured calls of at least this many frames run as two halves

struct LearnedGraph {
    const void *disp = nullptr, *img = nullptr, *heat = nullptr;
    void *out = nullptr;
    int w = 0, h = 0, n = 0, k = 0;
    cudaGraphExec_t exec = nullptr;
};
}  // namespace

struct ld_net {
    ld_handle *h = nullptr;
    LearnedGraph graphs[kLearnedGraphs];
    int next_graph = 0;
    cudaStream_t sub[2] = {};
    cudaEvent_t fork = nullptr, join[2] = {};
    int training = 0;
    int max_mh = 0, max_mw = 0, max_n = 0, max_ns = 0;
    void *mem = nullptr;
    ld::NetArgs a{};
    int32_t *xsum = nullptr;     // [n][mh][mw]
    float *z = nullptr;          // [n][mh][mw]
    float *scores = nullptr;     // [n][ceil(n_starts / 4)]
    uint8_t *cflag = nullptr;    // [n][n_starts]
    int32_t *elist = nullptr;    // [n][ecap]
    int32_t *ecnt = nullptr;     // [n]
    ld_lanes *lanes = nullptr;   // [n] scratch results of ld_make_training_pairs
    float *grad = nullptr;       // [kNetParams]
    float *loss = nullptr;       // [1]
    int step = 0;
    int last_w = 0, last_h = 0, last_n = 0;
    bool have_last = false;
    std::string err;
};

namespace {

std::string g_net_error;

int nfail(ld_net *net, int code, const std::string &msg)
{
    if (net)
        net->err = msg;
    else
        g_net_error = msg;
    return code;
}

int ncuda(ld_net *net, cudaError_t e, const char *what)
{
    return nfail(net, LD_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int check_map(ld_net *net, int w, int hh, int n)
{
    int mw, mh, mb;
    ld::handle_dims(net->h, &mw, &mh, &mb);
    if (w < 16 || hh < 16 || w > mw || hh > mh)
        return nfail(net, LD_E_ARG, "frame size outside [16, max_w] x [16, max_h]");
    if (n < 1 || n > mb)
        return nfail(net, LD_E_ARG, "n_frames outside [1, max_batch]");
    return LD_OK;
}

// the argument block for frames of w x hh pixels
ld::NetArgs args_for(const ld_net *net, int w, int hh)
{
    ld::NetArgs a = net->a;
    a.mh = (hh + 3) / 4;
    a.mw = (w + 3) / 4;
    return a;
}

// Frames [f0, f0 + nk) of a learned detection of n frames on stream s: block sums and the plain stages up
// to M_1, the network on the road rows (or the given heatmap), ranking, energies of the proposed starts,
// selection among them, and the exhaustive search of the frames where that found no lane.
int enqueue_learned(ld_net *net, const float *heatmap, const float *disp, const uint8_t *img, int w, int hh, int f0,
                    int nk, int n, int top_k, ld_lanes *out, cudaStream_t s)
{
    ld_handle *h = net->h;
    const ld::KParams kfull = ld::handle_kparams(h, w, hh, n);
    const ld::KParams kp = ld::handle_kparams(h, w, hh, nk);
    ld::Work base = ld::handle_work(h);
    base.xsum = net->xsum;
    const ld::Work wk = ld::work_view(base, kfull, f0);
    ld::NetArgs a = args_for(net, w, hh);
    const size_t cells = (size_t)a.mh * a.mw, fo = f0;
    for (int l = 0; l < 3; ++l)
        a.act[l] += fo * cells * ld::net_ch(l + 1);
    const int ecap = ld::kEvalPerTop * top_k;
    const int nc = (kp.n_starts + 3) / 4;
    float *z = net->z + fo * cells;
    const size_t px = fo * w * hh;
    cudaError_t e = cudaMemsetAsync(wk.xsum, 0, sizeof(int32_t) * nk * cells, s);
    if (e != cudaSuccess)
        return ncuda(net, e, "block sums");
    int rc = ld::handle_enqueue(h, kp, wk, disp + px, img + px, out + f0, 0, 7, s);   // k_vdisp .. k_m1
    if (rc != LD_OK)
        return nfail(net, rc, ld_last_error(h));
    if (!heatmap)
        e = ld::net_forward(a, wk.xsum, nk, z, false, true, s, wk.fs);
    else
        e = cudaMemcpyAsync(z, heatmap + fo * cells, sizeof(float) * nk * cells, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return ncuda(net, e, "network forward");
    uint8_t *cflag = net->cflag + fo * kp.n_starts;
    int32_t *elist = net->elist + fo * ecap, *ecnt = net->ecnt + fo;
    e = ld::net_propose(kp, wk, z, a.mh, a.mw, top_k, net->scores + fo * nc, cflag, elist, ecnt, ecap, s);
    if (e == cudaSuccess)
        e = ld::launch_energy_list(kp, wk, elist, ecnt, ecap, s);
    if (e == cudaSuccess)
        e = ld::launch_select_set(kp, wk, cflag, out + f0, s);
    if (e == cudaSuccess)
        e = ld::launch_energy_fallback(kp, wk, s);
    if (e == cudaSuccess)
        e = ld::launch_select_fallback(kp, wk, out + f0, s);
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "proposal");
}

// Argument checks and the bookkeeping of a learned detection, shared by the captured and the eager call.
int start_learned(ld_net *net, const float *disp, const uint8_t *img, int w, int hh, int n, int top_k, ld_lanes *out)
{
    if (top_k < 1 || top_k > ld::kTopKMax)
        return nfail(net, LD_E_ARG, "top_k outside [1, 256]");
    ld_handle *h = net->h;
    const int rc = ld::handle_check(h, disp, img, w, hh, n, out);
    if (rc != LD_OK)
        return nfail(net, rc, ld_last_error(h));
    ld::handle_call(h, w, hh, n);
    net->last_w = w;
    net->last_h = hh;
    net->last_n = n;
    net->have_last = true;
    return LD_OK;
}

}  // namespace

extern "C" {

int32_t ld_net_param_count(void) { return ld::kNetParams; }

int ld_net_create(ld_handle *h, int32_t training, ld_net **out)
{
    if (!out)
        return nfail(nullptr, LD_E_ARG, "out is NULL");
    *out = nullptr;
    if (!h)
        return nfail(nullptr, LD_E_ARG, "handle is NULL");
    ld_net *net = new ld_net();
    net->h = h;
    net->training = training != 0;
    int mw, mh, mb;
    ld::handle_dims(h, &mw, &mh, &mb);
    net->max_mh = (mh + 3) / 4;
    net->max_mw = (mw + 3) / 4;
    net->max_n = mb;
    net->max_ns = ld_n_starts(&ld::handle_params(h), mw);
    const size_t cells = (size_t)mb * net->max_mh * net->max_mw, P = ld::kNetParams;
    const size_t ncs = (size_t)(net->max_ns + 3) / 4, ecap = (size_t)ld::kEvalPerTop * ld::kTopKMax;
    const size_t nparts = (size_t)ld::sm_count() * ld::kWgradCtasPerSm;  // the weight-gradient grid's CTAs
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const bool tr = net->training;
    const size_t o_x = take(cells * 4), o_z = take(cells * 4), o_sc = take(mb * ncs * 4), o_cf = take((size_t)mb * net->max_ns);
    const size_t o_el = take(mb * ecap * 4), o_ec = take(mb * 4), o_ln = take(mb * sizeof(ld_lanes));
    const size_t o_a0 = take(cells * 16 * 2), o_a1 = take(cells * 32 * 2), o_a2 = take(cells * 32 * 2);
    const size_t o_a3 = tr ? take(cells * 16 * 2) : 0, o_in = tr ? take(cells * 2) : 0;
    const size_t o_d0 = tr ? take(cells * 32 * 2) : 0, o_d1 = tr ? take(cells * 32 * 2) : 0;
    size_t o_wf[4], o_wb[4];
    for (int l = 0; l < 4; ++l) {
        o_wf[l] = take((size_t)ld::net_ch(l) * ld::net_ch(l + 1) * 9 * 2);
        o_wb[l] = take((size_t)ld::net_ch(l) * ld::net_ch(l + 1) * 9 * 2);
    }
    const size_t o_wh = take(16 * 2), o_th = take(P * 4), o_m = take(P * 4), o_v = take(P * 4), o_g = take(P * 4);
    const size_t o_loss = take(4);
    const size_t o_pt = tr ? take(nparts * 32 * 289 * 4) : 0, o_ph = tr ? take(608 * 18 * 4) : 0;
    cudaError_t e = cudaMalloc(&net->mem, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete net;
        return nfail(nullptr, LD_E_NOMEM, std::string("network memory: ") + cudaGetErrorString(e));
    }
    char *b = (char *)net->mem;
    net->xsum = (int32_t *)(b + o_x);
    net->z = (float *)(b + o_z);
    net->scores = (float *)(b + o_sc);
    net->cflag = (uint8_t *)(b + o_cf);
    net->elist = (int32_t *)(b + o_el);
    net->ecnt = (int32_t *)(b + o_ec);
    net->lanes = (ld_lanes *)(b + o_ln);
    ld::NetArgs &a = net->a;
    a.act[0] = (__nv_bfloat16 *)(b + o_a0);
    a.act[1] = (__nv_bfloat16 *)(b + o_a1);
    a.act[2] = (__nv_bfloat16 *)(b + o_a2);
    a.act[3] = tr ? (__nv_bfloat16 *)(b + o_a3) : nullptr;
    a.X = tr ? (__nv_bfloat16 *)(b + o_in) : nullptr;
    a.dS[0] = tr ? (__nv_bfloat16 *)(b + o_d0) : nullptr;
    a.dS[1] = tr ? (__nv_bfloat16 *)(b + o_d1) : nullptr;
    int poff = 0;
    a.theta = (float *)(b + o_th);
    for (int l = 0; l < 4; ++l) {
        a.wf[l] = (__nv_bfloat16 *)(b + o_wf[l]);
        a.wb[l] = (__nv_bfloat16 *)(b + o_wb[l]);
        const int nw = ld::net_ch(l) * ld::net_ch(l + 1) * 9;
        a.bias[l] = a.theta + poff + nw;
        poff += nw + ld::net_ch(l + 1);
    }
    a.whb = (__nv_bfloat16 *)(b + o_wh);
    a.bh = a.theta + ld::kNetParams - 1;
    a.m = (float *)(b + o_m);
    a.v = (float *)(b + o_v);
    net->grad = (float *)(b + o_g);
    net->loss = (float *)(b + o_loss);
    a.part = tr ? (float *)(b + o_pt) : nullptr;
    a.part_head = tr ? (float *)(b + o_ph) : nullptr;
    // zero parameters until ld_net_set_params
    e = cudaMemsetAsync(net->mem, 0, off, ld::handle_stream(h));
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ld::handle_stream(h));
    if (e != cudaSuccess) {
        ncuda(nullptr, e, "network set-up");
        cudaFree(net->mem);
        delete net;
        return LD_E_CUDA;
    }
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&net->fork, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&net->sub[k], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&net->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        ncuda(nullptr, e, "stream and event creation");
        ld_net_destroy(net);
        return LD_E_CUDA;
    }
    *out = net;
    return LD_OK;
}

int ld_net_set_params(ld_net *net, const float *params)
{
    if (!net || !params)
        return nfail(net, LD_E_ARG, "null argument");
    cudaStream_t s = ld::handle_stream(net->h);
    const size_t bytes = sizeof(float) * ld::kNetParams;
    cudaError_t e = cudaMemcpyAsync(net->a.theta, params, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(net->a.m, 0, bytes, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(net->a.v, 0, bytes, s);
    if (e == cudaSuccess)
        e = ld::net_pack(net->a, s);
    net->step = 0;
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "set params");
}

int ld_net_get_params(ld_net *net, float *params)
{
    if (!net || !params)
        return nfail(net, LD_E_ARG, "null argument");
    cudaError_t e = cudaMemcpyAsync(params, net->a.theta, sizeof(float) * ld::kNetParams, cudaMemcpyDeviceToDevice,
                                    ld::handle_stream(net->h));
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "get params");
}

int ld_net_forward(ld_net *net, const int32_t *xsum, int32_t w, int32_t hh, int32_t n, float *logits)
{
    if (!net || !xsum || !logits)
        return nfail(net, LD_E_ARG, "null argument");
    int rc = check_map(net, w, hh, n);
    if (rc != LD_OK)
        return rc;
    cudaError_t e = ld::net_forward(args_for(net, w, hh), xsum, n, logits, false, false, ld::handle_stream(net->h));
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "network forward");
}

int ld_net_grad(ld_net *net, const int32_t *xsum, const uint8_t *labels, int32_t w, int32_t hh, int32_t n, float *grad,
                float *loss)
{
    if (!net || !xsum || !labels || !grad)
        return nfail(net, LD_E_ARG, "null argument");
    if (!net->training)
        return nfail(net, LD_E_STATE, "the network was created without training memory");
    int rc = check_map(net, w, hh, n);
    if (rc != LD_OK)
        return rc;
    const ld::NetArgs a = args_for(net, w, hh);
    cudaStream_t s = ld::handle_stream(net->h);
    cudaError_t e = ld::net_forward(a, xsum, n, net->z, true, false, s);
    if (e == cudaSuccess)
        e = ld::net_backward(a, labels, n, ld::kPosWeight, grad, loss, s);
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "network gradient");
}

int ld_net_apply_grad(ld_net *net, const float *grad, float lr)
{
    if (!net || !grad)
        return nfail(net, LD_E_ARG, "null argument");
    if (!(lr > 0.0f))
        return nfail(net, LD_E_ARG, "lr must be > 0");
    const double b1 = 0.9, b2 = 0.999;
    const int t = ++net->step;
    const float c1 = (float)(1.0 - std::pow(b1, t)), c2 = (float)(1.0 - std::pow(b2, t));
    cudaError_t e = ld::net_adam(net->a, grad, lr, (float)b1, (float)b2, 1e-8f, c1, c2, ld::handle_stream(net->h));
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "adam step");
}

int ld_net_train_step(ld_net *net, const int32_t *xsum, const uint8_t *labels, int32_t w, int32_t hh, int32_t n, float lr,
                      float *loss)
{
    if (!net)
        return LD_E_ARG;
    int rc = ld_net_grad(net, xsum, labels, w, hh, n, net->grad, loss ? loss : net->loss);
    return rc == LD_OK ? ld_net_apply_grad(net, net->grad, lr) : rc;
}

int ld_make_training_pairs(ld_net *net, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n,
                           int32_t *xsum_out, uint8_t *labels_out, ld_lanes *lanes_out)
{
    if (!net || !xsum_out || !labels_out)
        return nfail(net, LD_E_ARG, "null argument");
    ld_handle *h = net->h;
    ld_lanes *lanes = lanes_out ? lanes_out : net->lanes;
    int rc = ld::handle_check(h, disp, img, w, hh, n, lanes);
    if (rc != LD_OK)
        return nfail(net, rc, ld_last_error(h));
    const ld::KParams kp = ld::handle_call(h, w, hh, n);
    ld::Work wk = ld::handle_work(h);
    wk.xsum = xsum_out;
    const int mh = (hh + 3) / 4, mw = (w + 3) / 4;
    cudaStream_t s = ld::handle_stream(h);
    cudaError_t e = cudaMemsetAsync(xsum_out, 0, sizeof(int32_t) * (size_t)n * mh * mw, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(labels_out, 0, (size_t)n * mh * mw, s);
    if (e != cudaSuccess)
        return ncuda(net, e, "training pairs");
    rc = ld::handle_enqueue(h, kp, wk, disp, img, lanes, 0, 9);
    if (rc != LD_OK)
        return nfail(net, rc, ld_last_error(h));
    e = ld::net_labels(kp, wk, lanes, labels_out, mh, mw, s);
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "labels");
}

int ld_detect_learned(ld_net *net, const float *heatmap, const float *disp, const uint8_t *img, int32_t w, int32_t hh,
                      int32_t n, int32_t top_k, ld_lanes *out)
{
    if (!net)
        return LD_E_ARG;
    int rc = start_learned(net, disp, img, w, hh, n, top_k, out);
    if (rc != LD_OK)
        return rc;
    cudaStream_t s = ld::handle_stream(net->h);
    for (LearnedGraph &g : net->graphs)
        if (g.exec && g.disp == disp && g.img == img && g.heat == heatmap && g.out == out && g.w == w && g.h == hh &&
            g.n == n && g.k == top_k) {
            cudaError_t e = cudaGraphLaunch(g.exec, s);
            return e == cudaSuccess ? LD_OK : ncuda(net, e, "graph launch");
        }
    cudaStreamCaptureStatus st;
    cudaError_t e = cudaStreamIsCapturing(s, &st);
    if (e != cudaSuccess)
        return ncuda(net, e, "stream query");
    if (st != cudaStreamCaptureStatusNone || s == nullptr)   // the caller captures, or the legacy stream
        return enqueue_learned(net, heatmap, disp, img, w, hh, 0, n, n, top_k, out, s);
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return ncuda(net, e, "begin capture");
    if (n >= kLearnedSplitMin) {
        // two half-batches on the network's sub-streams, forked from and joined back to the handle's stream
        rc = (e = cudaEventRecord(net->fork, s)) == cudaSuccess ? LD_OK : ncuda(net, e, "fork");
        const int n0 = (n + 1) / 2;
        for (int k = 0; k < 2 && rc == LD_OK; ++k) {
            if ((e = cudaStreamWaitEvent(net->sub[k], net->fork, 0)) != cudaSuccess) {
                rc = ncuda(net, e, "fork wait");
                break;
            }
            rc = enqueue_learned(net, heatmap, disp, img, w, hh, k ? n0 : 0, k ? n - n0 : n0, n, top_k, out, net->sub[k]);
            if (rc == LD_OK && ((e = cudaEventRecord(net->join[k], net->sub[k])) != cudaSuccess ||
                                (e = cudaStreamWaitEvent(s, net->join[k], 0)) != cudaSuccess))
                rc = ncuda(net, e, "join");
        }
    } else {
        rc = enqueue_learned(net, heatmap, disp, img, w, hh, 0, n, n, top_k, out, s);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (rc != LD_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess)
        return ncuda(net, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return ncuda(net, e, "graph instantiate");
    LearnedGraph &g = net->graphs[net->next_graph];
    net->next_graph = (net->next_graph + 1) % kLearnedGraphs;
    if (g.exec)
        cudaGraphExecDestroy(g.exec);
    g = LearnedGraph{disp, img, heatmap, out, w, hh, n, top_k, exec};
    e = cudaGraphLaunch(exec, s);
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "graph launch");
}

size_t ld_net_debug_size(ld_net *net, int32_t stage)
{
    if (!net || !net->have_last)
        return 0;
    const size_t cells = (size_t)((net->last_h + 3) / 4) * ((net->last_w + 3) / 4);
    const size_t ns = (size_t)ld_n_starts(&ld::handle_params(net->h), net->last_w);
    switch (stage) {
    case LD_NET_STAGE_XSUM: return cells * 4;
    case LD_NET_STAGE_HEATMAP: return cells * 4;
    case LD_NET_STAGE_SCORES: return (ns + 3) / 4 * 4;
    case LD_NET_STAGE_CFLAG: return ns;
    default: return 0;
    }
}

int ld_net_debug_get(ld_net *net, int32_t frame, int32_t stage, void *host_dst, size_t bytes)
{
    if (!net)
        return LD_E_ARG;
    if (!net->have_last)
        return nfail(net, LD_E_STATE, "no learned detection yet");
    if (frame < 0 || frame >= net->last_n || !host_dst)
        return nfail(net, LD_E_ARG, "frame out of range or null destination");
    const size_t want = ld_net_debug_size(net, stage);
    if (want == 0 || bytes != want)
        return nfail(net, LD_E_ARG, "unknown stage or wrong byte count");
    cudaError_t e = cudaStreamSynchronize(ld::handle_stream(net->h));
    if (e != cudaSuccess)
        return ncuda(net, e, "sync");
    const size_t f = frame;
    const void *src = nullptr;
    switch (stage) {
    case LD_NET_STAGE_XSUM: src = net->xsum + f * (want / 4); break;
    case LD_NET_STAGE_HEATMAP: src = net->z + f * (want / 4); break;
    case LD_NET_STAGE_SCORES: src = net->scores + f * (want / 4); break;
    default: src = net->cflag + f * want; break;
    }
    e = cudaMemcpy(host_dst, src, want, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LD_OK : ncuda(net, e, "debug copy");
}

int ld_net_set_fused(ld_net *net, int32_t on)
{
    if (!net)
        return LD_E_ARG;
    const cudaError_t e = cudaStreamSynchronize(ld::handle_stream(net->h));
    if (e != cudaSuccess)
        return ncuda(net, e, "sync");
    net->a.fused = on ? 1 : 0;
    for (LearnedGraph &g : net->graphs)   // the captured calls hold the other form's kernels
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g = LearnedGraph{};
        }
    return LD_OK;
}

int ld_net_status(ld_net *net)
{
    if (!net)
        return LD_E_ARG;
    cudaError_t e = cudaStreamSynchronize(ld::handle_stream(net->h));
    if (e != cudaSuccess)
        return ncuda(net, e, "sync");
    const int v = ld::net_tc_status();
    if (v < 0)
        return nfail(net, LD_E_CUDA, "status read");
    return v ? nfail(net, LD_E_TIMEOUT, "a tensor-core wait ran out") : LD_OK;
}

const char *ld_net_last_error(const ld_net *net) { return net ? net->err.c_str() : g_net_error.c_str(); }

void ld_net_destroy(ld_net *net)
{
    if (!net)
        return;
    cudaStreamSynchronize(ld::handle_stream(net->h));
    for (LearnedGraph &g : net->graphs)
        if (g.exec)
            cudaGraphExecDestroy(g.exec);
    if (net->fork)
        cudaEventDestroy(net->fork);
    for (int k = 0; k < 2; ++k) {
        if (net->join[k])
            cudaEventDestroy(net->join[k]);
        if (net->sub[k])
            cudaStreamDestroy(net->sub[k]);
    }
    cudaFree(net->mem);
    delete net;
}

}  // extern "C"

namespace ld {
// ld_detect_learned without the graph cache: the launches are enqueued directly on the handle's stream
// (the serving path, whose batch sizes vary from call to call).
int detect_learned_eager(ld_net *net, const float *disp, const uint8_t *img, int32_t w, int32_t hh, int32_t n_frames,
                         int32_t top_k, ld_lanes *out_lanes)
{
    if (!net)
        return LD_E_ARG;
    const int rc = start_learned(net, disp, img, w, hh, n_frames, top_k, out_lanes);
    if (rc != LD_OK)
        return rc;
    return enqueue_learned(net, nullptr, disp, img, w, hh, 0, n_frames, n_frames, top_k, out_lanes,
                           handle_stream(net->h));
}
}  // namespace ld
