// Serving runtime behind the ld_server_* entry points of include/ld.h: continuous batching of frames of
// several sizes from several camera streams over a set of slots (fixed, or grown within an HBM budget).
//
// A slot is one library handle with its own CUDA stream, pinned host staging for max_batch frames and the
// device buffers the batch runs from (plus, once the learned form is switched on, an inference network on
// that handle).  Slots cycle FREE -> FILLING (frames copied in by submit) ->
// IN_FLIGHT (copies, the nine kernels, the result copy and a host callback enqueued on the slot's stream)
// -> FINISHED (its host callback has run) -> FREE (its results moved to the completion queue).  A scheduler
// thread launches a filling slot whose oldest frame has waited max_wait_us.  After each batch the slot's
// stream also updates the per-stream state in device memory (the latest result of each camera stream),
// ordered on one state stream so that two batches never race on an entry.
//
// Locks: the server lock guards the slots and queues, and CUDA calls are made under it (the launches and
// copies of a batch; a slot the HBM budget adds is allocated with the lock released).  The host callback, which CUDA runs on its own thread,
// never takes it: it only appends the slot to a finished list under a second lock that no thread holds
// across a CUDA call, so a CUDA call that waits for the device (or for the callback thread) can never wait
// on a thread that waits for the server lock.  Finished slots are reaped under the server lock by the
// next submit, poll, drain or stats call.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ld_internal.cuh"

static_assert(sizeof(ld_lanes) == 192 && sizeof(ld_result) == 232, "C-ABI result layouts");

namespace {

using Clock = std::chrono::steady_clock;
std::string g_server_create_error;

enum class SlotState { Free, Filling, InFlight };

struct ReqInfo {
    uint64_t tag;
    int32_t stream_id;
    int64_t seq;
    Clock::time_point t_submit;
};

struct Slot {
    ld_server *server = nullptr;
    int cls = 0;
    ld_handle *h = nullptr;
    ld_net *net = nullptr;            // the learned form's network on h (created by ld_server_set_learned)
    cudaStream_t stream = nullptr;
    float *h_disp = nullptr;          // pinned [max_batch][h][w]
    uint8_t *h_img = nullptr;
    ld_lanes *h_lanes = nullptr;      // pinned [max_batch]
    int32_t *h_meta = nullptr;        // pinned [max_batch][3]: stream id, seq low, seq high
    float *d_disp = nullptr;
    uint8_t *d_img = nullptr;
    ld_lanes *d_lanes = nullptr;
    int32_t *d_meta = nullptr;
    cudaEvent_t done = nullptr;        // the batch's result copy has completed
    cudaEvent_t state_done = nullptr;  // the state update that reads this slot's buffers has completed
    SlotState state = SlotState::Free;
    int n = 0;                        // frames placed in the slot
    int pending = 0;                  // submitters still making their copies into it (launch waits for 0)
    std::vector<ReqInfo> reqs;
};

// Latest result per stream, applied in batch order by one thread: a frame replaces the entry when its
// sequence number is higher than the entry's.
__global__ void k_keep_state(const ld_lanes *lanes, const int32_t *meta, int n, ld_lanes *state, long long *state_seq)
{
    if (threadIdx.x != 0)
        return;
    for (int i = 0; i < n; ++i) {
        const int sid = meta[3 * i];
        const long long seq = (long long)(uint32_t)meta[3 * i + 1] | ((long long)meta[3 * i + 2] << 32);
        if (seq > state_seq[sid]) {
            state_seq[sid] = seq;
            state[sid] = lanes[i];
        }
    }
}

void CUDART_CB on_batch_done(void *arg);

struct Finished {
    Slot *sl;
    Clock::time_point t;   // when the batch's result copy had completed
};

}  // namespace

struct ld_server {
    ld_params p{};
    ld_server_config cfg{};
    std::deque<Slot> slots;            // stable addresses: callbacks hold a slot's address; slots may be added
    int64_t device_bytes = 0;          // device memory of the slots (buffers and handle workspaces)
    int64_t cls_bytes[LD_MAX_SIZE_CLASSES] = {};  // device bytes of one slot of each size class
    bool growing = false;              // a submitter is adding a slot (outside the lock)
    cudaStream_t state_stream = nullptr;
    ld_lanes *d_state = nullptr;
    long long *d_state_seq = nullptr;
    std::vector<int64_t> next_seq;     // per stream
    std::vector<int64_t> done_seq;     // highest completed sequence number per stream (-1: none)
    std::mutex mu;
    std::condition_variable cv_done;   // (with mu) a slot freed or a submit's copies made
    std::condition_variable cv_sched;  // (with mu) the scheduler's wake-up
    std::mutex cb_mu;                  // guards finished only; never held across a CUDA call
    std::condition_variable cv_cb;     // (with cb_mu) a batch finished
    std::vector<Finished> finished;    // slots whose callbacks have run, not yet reaped
    int64_t reaped = 0;                // (with cb_mu) reap calls that freed a slot: wakes the other waiters
    std::deque<ld_result> results;
    std::vector<double> latencies;
    int top_k = 0;                     // > 0: batches run the learned form with this top_k
    float *d_params = nullptr;         // device copy of the learned form's parameters (for slots added later)
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched_frames = 0;
    int in_flight = 0;
    std::atomic<bool> stop{false};     // also read under cb_mu alone
    std::thread scheduler;
    std::string err;
};

namespace {

int sfail(ld_server *s, int code, const std::string &msg)
{
    if (s)
        s->err = msg;
    else
        g_server_create_error = msg;
    return code;
}

size_t frame_px(const ld_server *s, int cls) { return (size_t)s->cfg.sizes[cls][0] * s->cfg.sizes[cls][1]; }

// Enqueue a filling slot's batch (called with the lock held; only asynchronous CUDA calls).  The frames'
// inputs are already on their way: each submit enqueued its own copy on the slot's stream.
int launch_slot(ld_server *s, Slot &sl)
{
    const int w = s->cfg.sizes[sl.cls][0], hh = s->cfg.sizes[sl.cls][1], n = sl.n;
    for (int i = 0; i < n; ++i) {
        sl.h_meta[3 * i] = sl.reqs[i].stream_id;
        sl.h_meta[3 * i + 1] = (int32_t)(uint32_t)(sl.reqs[i].seq & 0xffffffffu);
        sl.h_meta[3 * i + 2] = (int32_t)(sl.reqs[i].seq >> 32);
    }
    // the previous batch's state update reads d_lanes and d_meta: wait for it before overwriting them
    cudaError_t e = cudaStreamWaitEvent(sl.stream, sl.state_done, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.d_meta, sl.h_meta, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess)
        return sfail(s, LD_E_CUDA, std::string("batch input copy: ") + cudaGetErrorString(e));
    if (s->top_k > 0) {
        const int rc = ld::detect_learned_eager(sl.net, sl.d_disp, sl.d_img, w, hh, n, s->top_k, sl.d_lanes);
        if (rc != LD_OK)
            return sfail(s, rc, std::string("batch detect (learned): ") + ld_net_last_error(sl.net));
    } else {
        const int rc = ld::detect_eager(sl.h, sl.d_disp, sl.d_img, w, hh, n, sl.d_lanes);
        if (rc != LD_OK)
            return sfail(s, rc, std::string("batch detect: ") + ld_last_error(sl.h));
    }
    e = cudaMemcpyAsync(sl.h_lanes, sl.d_lanes, sizeof(ld_lanes) * n, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.done, sl.stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s->state_stream, sl.done, 0);
    if (e == cudaSuccess) {
        k_keep_state<<<1, 32, 0, s->state_stream>>>(sl.d_lanes, sl.d_meta, n, s->d_state, s->d_state_seq);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(sl.state_done, s->state_stream);
    if (e == cudaSuccess)
        e = cudaLaunchHostFunc(sl.stream, on_batch_done, &sl);
    if (e != cudaSuccess)
        return sfail(s, LD_E_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    sl.state = SlotState::InFlight;
    ++s->in_flight;
    ++s->batches;
    s->batched_frames += n;
    return LD_OK;
}

// Runs on a CUDA-owned thread once the slot's result copy has completed: host work under cb_mu only.
void CUDART_CB on_batch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    ld_server *s = sl->server;
    {
        std::lock_guard<std::mutex> g(s->cb_mu);
        s->finished.push_back(Finished{sl, Clock::now()});
    }
    s->cv_cb.notify_all();
}

// Move the finished slots' results to the completion queue and free the slots (server lock held).
size_t reap(ld_server *s)
{
    std::vector<Finished> fin;
    {
        std::lock_guard<std::mutex> g(s->cb_mu);
        fin.swap(s->finished);
    }
    for (const Finished &f : fin) {
        Slot &sl = *f.sl;
        const int w = s->cfg.sizes[sl.cls][0], hh = s->cfg.sizes[sl.cls][1];
        for (int i = 0; i < sl.n; ++i) {
            ld_result r;
            r.tag = sl.reqs[i].tag;
            r.stream_id = sl.reqs[i].stream_id;
            r.w = w;
            r.h = hh;
            r.seq = sl.reqs[i].seq;
            r.latency_ms = std::chrono::duration<double, std::milli>(f.t - sl.reqs[i].t_submit).count();
            r.lanes = sl.h_lanes[i];
            s->results.push_back(r);
            s->latencies.push_back(r.latency_ms);
            s->done_seq[r.stream_id] = std::max(s->done_seq[r.stream_id], r.seq);
        }
        s->completed += sl.n;
        sl.n = 0;
        sl.reqs.clear();
        sl.state = SlotState::Free;
        --s->in_flight;
    }
    if (!fin.empty()) {
        {
            std::lock_guard<std::mutex> g(s->cb_mu);
            ++s->reaped;
        }
        s->cv_cb.notify_all();     // another thread waiting for results: they are in the queue now
        s->cv_done.notify_all();
    }
    return fin.size();
}

// Wait (server lock released) until a batch finishes or the deadline passes, then reap.
void wait_finished(ld_server *s, std::unique_lock<std::mutex> &lk, Clock::time_point deadline)
{
    lk.unlock();
    {
        std::unique_lock<std::mutex> g(s->cb_mu);
        const int64_t r0 = s->reaped;
        s->cv_cb.wait_until(g, deadline, [&] { return !s->finished.empty() || s->reaped != r0 || s->stop; });
    }
    lk.lock();
    reap(s);
}

void scheduler_loop(ld_server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    const auto wait = std::chrono::microseconds(std::max(1, s->cfg.max_wait_us));
    while (!s->stop) {
        auto next = Clock::now() + std::chrono::milliseconds(50);
        const auto now = Clock::now();
        for (Slot &sl : s->slots)
            if (sl.state == SlotState::Filling && !sl.reqs.empty() && sl.pending == 0) {
                const auto due = sl.reqs.front().t_submit + wait;
                if (due <= now)
                    launch_slot(s, sl);  // an error stays in s->err; the frames stay queued in the slot
                else
                    next = std::min(next, due);
            }
        s->cv_sched.wait_until(lk, next);
    }
}

void free_slot(Slot &sl)
{
    if (sl.net)
        ld_net_destroy(sl.net);
    if (sl.h)
        ld_destroy(sl.h);
    if (sl.stream)
        cudaStreamDestroy(sl.stream);
    if (sl.done)
        cudaEventDestroy(sl.done);
    if (sl.state_done)
        cudaEventDestroy(sl.state_done);
    cudaFreeHost(sl.h_disp);
    cudaFreeHost(sl.h_img);
    cudaFreeHost(sl.h_lanes);
    cudaFreeHost(sl.h_meta);
    cudaFree(sl.d_disp);
    cudaFree(sl.d_img);
    cudaFree(sl.d_lanes);
    cudaFree(sl.d_meta);
    sl = Slot();
}

// Allocate one slot of size class cls (called without the lock).  Returns its device bytes, or -1 with
// the CUDA error in *err.
int64_t create_slot(ld_server *s, int cls, Slot &sl, std::string *err)
{
    sl.server = s;
    sl.cls = cls;
    const int w = s->cfg.sizes[cls][0], hh = s->cfg.sizes[cls][1], n = s->cfg.max_batch;
    const size_t px = (size_t)n * w * hh;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&sl.state_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMallocHost(&sl.h_disp, px * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMallocHost(&sl.h_img, px);
    if (e == cudaSuccess)
        e = cudaMallocHost(&sl.h_lanes, sizeof(ld_lanes) * n);
    if (e == cudaSuccess)
        e = cudaMallocHost(&sl.h_meta, sizeof(int32_t) * 3 * n);
    if (e == cudaSuccess)
        e = cudaMalloc(&sl.d_disp, px * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&sl.d_img, px);
    if (e == cudaSuccess)
        e = cudaMalloc(&sl.d_lanes, sizeof(ld_lanes) * n);
    if (e == cudaSuccess)
        e = cudaMalloc(&sl.d_meta, sizeof(int32_t) * 3 * n);
    if (e != cudaSuccess) {
        *err = std::string("slot allocation: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return -1;
    }
    const int rc = ld_create(&s->p, w, hh, n, sl.stream, &sl.h);
    if (rc != LD_OK) {
        *err = std::string("slot handle: ") + ld_last_error(nullptr);
        return -1;
    }
    if (s->top_k > 0) {   // a slot added while the learned form is on gets its network too
        int rc2 = ld_net_create(sl.h, 0, &sl.net);
        if (rc2 == LD_OK)
            rc2 = ld_net_set_params(sl.net, s->d_params);
        if (rc2 == LD_OK && cudaStreamSynchronize(sl.stream) != cudaSuccess)
            rc2 = LD_E_CUDA;
        if (rc2 != LD_OK) {
            *err = std::string("slot network: ") + ld_net_last_error(sl.net);
            return -1;
        }
    }
    sl.reqs.reserve(n);
    return (int64_t)(px * 5 + (sizeof(ld_lanes) + 12) * n) + (int64_t)ld::handle_device_bytes(sl.h);
}

void release(ld_server *s)
{
    for (Slot &sl : s->slots)
        free_slot(sl);
    if (s->state_stream)
        cudaStreamDestroy(s->state_stream);
    cudaFree(s->d_state);
    cudaFree(s->d_state_seq);
    cudaFree(s->d_params);
}

}  // namespace

extern "C" {

int ld_server_create(const ld_params *p, const ld_server_config *cfg, ld_server **out)
{
    if (!out)
        return sfail(nullptr, LD_E_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !cfg)
        return sfail(nullptr, LD_E_ARG, "params or config is NULL");
    if (cfg->n_sizes < 1 || cfg->n_sizes > LD_MAX_SIZE_CLASSES || cfg->slots_per_size < 1 || cfg->max_batch < 1 ||
        cfg->n_streams < 1 || cfg->max_wait_us < 0)
        return sfail(nullptr, LD_E_ARG, "n_sizes, slots_per_size, max_batch, n_streams or max_wait_us out of range");
    for (int c = 0; c < cfg->n_sizes; ++c) {
        const int w = cfg->sizes[c][0], hh = cfg->sizes[c][1];
        if (w < 16 || hh < 16 || w > LD_MAX_W || hh > LD_MAX_H)
            return sfail(nullptr, LD_E_ARG, "size class out of range");
        for (int d = 0; d < c; ++d)
            if (cfg->sizes[d][0] == w && cfg->sizes[d][1] == hh)
                return sfail(nullptr, LD_E_ARG, "duplicate size class");
    }
    ld_server *s = new ld_server();
    s->p = *p;
    s->cfg = *cfg;
    s->next_seq.assign(cfg->n_streams, 0);
    s->done_seq.assign(cfg->n_streams, -1);
    s->slots.resize((size_t)cfg->n_sizes * cfg->slots_per_size);
    if (cfg->hbm_budget_bytes < 0)
        return sfail(nullptr, LD_E_ARG, "hbm_budget_bytes must be >= 0");
    cudaError_t e = cudaStreamCreateWithFlags(&s->state_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&s->d_state, sizeof(ld_lanes) * cfg->n_streams);
    if (e == cudaSuccess)
        e = cudaMalloc(&s->d_state_seq, sizeof(long long) * cfg->n_streams);
    if (e == cudaSuccess)
        e = cudaMemset(s->d_state_seq, 0xff, sizeof(long long) * cfg->n_streams);  // -1: nothing yet
    if (e != cudaSuccess) {
        const std::string msg = std::string("server allocation: ") + cudaGetErrorString(e);
        cudaGetLastError();
        release(s);
        delete s;
        return sfail(nullptr, e == cudaErrorMemoryAllocation ? LD_E_NOMEM : LD_E_CUDA, msg);
    }
    for (size_t k = 0; k < s->slots.size(); ++k) {
        std::string why;
        const int64_t bytes = create_slot(s, (int)(k / cfg->slots_per_size), s->slots[k], &why);
        if (bytes < 0) {
            release(s);
            delete s;
            return sfail(nullptr, why.find("out of memory") != std::string::npos ? LD_E_NOMEM : LD_E_CUDA, why);
        }
        s->cls_bytes[s->slots[k].cls] = bytes;
        s->device_bytes += bytes;
    }
    if (cfg->hbm_budget_bytes > 0 && s->device_bytes > cfg->hbm_budget_bytes) {
        release(s);
        delete s;
        return sfail(nullptr, LD_E_ARG, "the initial slots need more device memory than hbm_budget_bytes");
    }
    s->scheduler = std::thread(scheduler_loop, s);
    *out = s;
    return LD_OK;
}

}  // extern "C"

namespace {

// A slot of class cls that can take one more frame (lock held).  With an HBM budget, when every slot of the
// class is full or in flight a new one is allocated, outside the lock, if the budget and the device's free
// memory allow it; the lock is held again on return.  Null when no slot can take the frame; *alloc_error is
// then set when allocating a slot failed (s->err says why) rather than every slot being busy.
Slot *admit(ld_server *s, int cls, std::unique_lock<std::mutex> &lk, bool *alloc_error)
{
    *alloc_error = false;
    reap(s);
    for (Slot &sl : s->slots)
        if (sl.cls == cls && sl.state == SlotState::Filling && sl.n < s->cfg.max_batch)
            return &sl;
    for (Slot &sl : s->slots)
        if (sl.cls == cls && sl.state == SlotState::Free) {
            sl.state = SlotState::Filling;
            return &sl;
        }
    const int64_t need = s->cls_bytes[cls];
    if (s->cfg.hbm_budget_bytes <= 0 || s->growing || s->device_bytes + need > s->cfg.hbm_budget_bytes)
        return nullptr;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || (int64_t)free_b < need + (int64_t)(256u << 20))
        return nullptr;
    s->growing = true;
    lk.unlock();
    Slot fresh;
    std::string why;
    const int64_t bytes = create_slot(s, cls, fresh, &why);
    if (bytes < 0)
        free_slot(fresh);   // before the lock: freeing device memory waits for the device
    lk.lock();
    s->growing = false;
    if (bytes < 0) {
        s->err = why;
        *alloc_error = true;
        return nullptr;
    }
    s->slots.push_back(std::move(fresh));
    s->device_bytes += bytes;
    Slot &sl = s->slots.back();
    sl.state = SlotState::Filling;
    return &sl;
}

// Submit n frames of one size class ([n][h][w] contiguous; stream_ids and tags per frame).  Frames go into
// slots in runs: a run's place in a slot is reserved under the lock, its copies (the host copy into the
// staging for staged frames, then one host-to-device copy per buffer on the slot's stream) are made
// without it, and the last of a slot's concurrent submitters to finish launches the slot when it is full.
// Returns the number of frames accepted (in order) or a negative LD_E_* code.
int submit_frames(ld_server *s, int32_t n, const int32_t *stream_ids, const float *disp, const uint8_t *img,
                  int32_t w, int32_t h, const uint64_t *tags, bool pinned)
{
    if (!s)
        return LD_E_ARG;
    if (n < 0 || (n > 0 && (!disp || !img || !stream_ids || !tags)))
        return sfail(s, LD_E_ARG, "null frame, stream id or tag array");
    for (int i = 0; i < n; ++i)
        if (stream_ids[i] < 0 || stream_ids[i] >= s->cfg.n_streams)
            return sfail(s, LD_E_ARG, "stream id out of range");
    int cls = -1;
    for (int c = 0; c < s->cfg.n_sizes; ++c)
        if (s->cfg.sizes[c][0] == w && s->cfg.sizes[c][1] == h)
            cls = c;
    if (cls < 0)
        return sfail(s, LD_E_ARG, "frame size matches no size class");
    const size_t px = frame_px(s, cls);
    int done = 0;
    while (done < n) {
        std::unique_lock<std::mutex> lk(s->mu);
        bool alloc_error = false;
        Slot *sl = admit(s, cls, lk, &alloc_error);
        if (!sl) {
            s->rejected += n - done;
            if (alloc_error)   // s->err holds the allocation's error
                return done > 0 ? done : (s->err.find("out of memory") != std::string::npos ? LD_E_NOMEM : LD_E_CUDA);
            if (done == 0)
                return sfail(s, LD_E_BUSY, "every slot of the size class is full or in flight and the HBM budget "
                                           "admits no further slot");
            return done;
        }
        const int k = std::min(n - done, s->cfg.max_batch - sl->n);
        const size_t at = (size_t)sl->n * px;
        const auto now = Clock::now();
        for (int i = 0; i < k; ++i) {
            const int32_t sid = stream_ids[done + i];
            sl->reqs.push_back(ReqInfo{tags[done + i], sid, s->next_seq[sid]++, now});
        }
        sl->n += k;
        ++sl->pending;
        s->submitted += k;
        lk.unlock();

        const float *dsrc = disp + (size_t)done * px;
        const uint8_t *isrc = img + (size_t)done * px;
        if (!pinned) {   // staged: copied into the slot's page-locked buffers first
            std::memcpy(sl->h_disp + at, dsrc, (size_t)k * px * sizeof(float));
            std::memcpy(sl->h_img + at, isrc, (size_t)k * px);
            dsrc = sl->h_disp + at;
            isrc = sl->h_img + at;
        }
        cudaError_t e = cudaMemcpyAsync(sl->d_disp + at, dsrc, (size_t)k * px * sizeof(float), cudaMemcpyHostToDevice,
                                        sl->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl->d_img + at, isrc, (size_t)k * px, cudaMemcpyHostToDevice, sl->stream);

        lk.lock();
        if (--sl->pending == 0)
            s->cv_done.notify_all();    // ld_server_drain may be waiting for the copies
        if (e != cudaSuccess)
            return sfail(s, LD_E_CUDA, std::string("frame copy: ") + cudaGetErrorString(e));
        if (sl->pending == 0 && sl->n == s->cfg.max_batch) {
            const int rc = launch_slot(s, *sl);
            if (rc != LD_OK)
                return rc;
        } else {
            s->cv_sched.notify_one();   // a new deadline, or a slot the scheduler skipped while copies were open
        }
        done += k;
    }
    return done;
}

}  // namespace

extern "C" {

int ld_server_submit(ld_server *s, int32_t stream_id, const float *disp, const uint8_t *img, int32_t w, int32_t h,
                     uint64_t tag)
{
    const int rc = submit_frames(s, 1, &stream_id, disp, img, w, h, &tag, false);
    return rc == 1 ? LD_OK : rc;
}

int ld_server_submit_pinned(ld_server *s, int32_t stream_id, const float *disp, const uint8_t *img, int32_t w,
                            int32_t h, uint64_t tag)
{
    const int rc = submit_frames(s, 1, &stream_id, disp, img, w, h, &tag, true);
    return rc == 1 ? LD_OK : rc;
}

int ld_server_submit_batch(ld_server *s, int32_t n_frames, const int32_t *stream_ids, const float *disp,
                           const uint8_t *img, int32_t w, int32_t h, const uint64_t *tags, int32_t pinned)
{
    return submit_frames(s, n_frames, stream_ids, disp, img, w, h, tags, pinned != 0);
}

int ld_server_set_learned(ld_server *s, const float *params, int32_t top_k)
{
    if (!s)
        return LD_E_ARG;
    if (top_k < 0 || top_k > LD_NET_TOPK_MAX || (top_k > 0 && !params))
        return sfail(s, LD_E_ARG, "top_k outside [0, LD_NET_TOPK_MAX] or null parameters");
    std::unique_lock<std::mutex> lk(s->mu);
    reap(s);
    if (s->in_flight > 0 || s->submitted != s->completed || s->growing)
        return sfail(s, LD_E_STATE, "frames are in the server: drain it first");
    if (top_k > 0) {   // kept for slots the HBM budget adds later
        cudaError_t e = s->d_params ? cudaSuccess : cudaMalloc(&s->d_params, sizeof(float) * LD_NET_PARAMS);
        if (e == cudaSuccess)
            e = cudaMemcpy(s->d_params, params, sizeof(float) * LD_NET_PARAMS, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess)
            return sfail(s, LD_E_CUDA, std::string("parameter copy: ") + cudaGetErrorString(e));
    }
    // nothing is filling or in flight, so no callback needs the lock while the slots are set up
    if (top_k > 0)
        for (Slot &sl : s->slots) {
            if (!sl.net) {
                const int rc = ld_net_create(sl.h, 0, &sl.net);
                if (rc != LD_OK)
                    return sfail(s, rc, std::string("slot network: ") + ld_net_last_error(nullptr));
            }
            int rc = ld_net_set_params(sl.net, params);
            if (rc != LD_OK)
                return sfail(s, rc, std::string("slot network parameters: ") + ld_net_last_error(sl.net));
            const cudaError_t e = cudaStreamSynchronize(sl.stream);   // the caller may release params now
            if (e != cudaSuccess)
                return sfail(s, LD_E_CUDA, std::string("slot network parameters: ") + cudaGetErrorString(e));
        }
    s->top_k = top_k;
    return LD_OK;
}

int ld_server_poll(ld_server *s, ld_result *out, int32_t max_out, int32_t timeout_ms)
{
    if (!s || (!out && max_out > 0) || max_out < 0)
        return LD_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    reap(s);
    if (s->results.empty() && timeout_ms > 0) {
        const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
        while (s->results.empty() && Clock::now() < deadline && !s->stop)
            wait_finished(s, lk, deadline);
    }
    int k = 0;
    while (k < max_out && !s->results.empty()) {
        out[k++] = s->results.front();
        s->results.pop_front();
    }
    return k;
}

int ld_server_drain(ld_server *s)
{
    if (!s)
        return LD_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    reap(s);
    for (Slot &sl : s->slots)
        if (sl.state == SlotState::Filling) {
            // a submitter on another thread may still be copying into the slot (bounded wait)
            if (!s->cv_done.wait_for(lk, std::chrono::seconds(10), [&] { return sl.pending == 0; }))
                return sfail(s, LD_E_CUDA, "a submit's copies did not finish within 10 s");
            if (sl.state != SlotState::Filling)
                continue;   // the submitter launched it
            const int rc = launch_slot(s, sl);
            if (rc != LD_OK)
                return rc;
        }
    // bounded wait: a batch that has not finished after a minute is reported, not waited for forever
    const auto deadline = Clock::now() + std::chrono::seconds(60);
    while (s->in_flight > 0 && Clock::now() < deadline)
        wait_finished(s, lk, deadline);
    return s->in_flight == 0 ? LD_OK : sfail(s, LD_E_CUDA, "batches still in flight after 60 s");
}

int ld_server_stream_state(ld_server *s, int32_t stream_id, ld_lanes *out)
{
    if (!s || !out || stream_id < 0 || stream_id >= s->cfg.n_streams)
        return s ? sfail(s, LD_E_ARG, "stream id out of range or null output") : LD_E_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        reap(s);
        if (s->done_seq[stream_id] < 0)
            return sfail(s, LD_E_STATE, "no frame of this stream has completed");
    }
    cudaError_t e = cudaStreamSynchronize(s->state_stream);  // without the lock: callbacks may need it
    if (e == cudaSuccess)
        e = cudaMemcpy(out, s->d_state + stream_id, sizeof(ld_lanes), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LD_OK : sfail(s, LD_E_CUDA, std::string("state copy: ") + cudaGetErrorString(e));
}

int ld_server_stats_get(ld_server *s, ld_server_stats *out)
{
    if (!s || !out)
        return LD_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    reap(s);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->batches = s->batches;
    out->mean_batch = s->batches ? (double)s->batched_frames / (double)s->batches : 0.0;
    out->slots = (int64_t)s->slots.size();
    out->device_bytes = s->device_bytes;
    out->p50_ms = out->p99_ms = 0.0;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        auto pct = [&](double q) {
            const size_t k = (size_t)std::min<double>((double)v.size() - 1, q * (double)(v.size() - 1) + 0.5);
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    return LD_OK;
}

const char *ld_server_last_error(const ld_server *s) { return s ? s->err.c_str() : g_server_create_error.c_str(); }

void ld_server_destroy(ld_server *s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    {
        std::lock_guard<std::mutex> g(s->cb_mu);   // pairs with the predicate check in wait_finished
    }
    s->cv_cb.notify_all();
    if (s->scheduler.joinable())
        s->scheduler.join();
    for (Slot &sl : s->slots)
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);  // runs the last callbacks (they take the lock, now free)
    if (s->state_stream)
        cudaStreamSynchronize(s->state_stream);
    release(s);
    delete s;
}

}  // extern "C"
