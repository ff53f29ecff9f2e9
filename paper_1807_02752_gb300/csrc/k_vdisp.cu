// Sec. 2.2: the v-disparity map m_y(d, v), the histogram of every row of the disparity map.
//
// A pixel counts when its disparity l is finite and > 0 (0 marks pixels invalidated by the left-right
// check, Eq. 10); its bin is floor(l + 0.5) in float32 and bins >= D are dropped.
//
// One CTA covers kRows consecutive rows of one frame (16 unless ld_tune chose another count).  Those
// rows are one contiguous range of memory, so the CTA streams it as 16-byte loads of the aligned chunks
// inside it (several in flight per thread) plus single loads of its head and tail; each warp streams one
// contiguous span.  Counts go to a shared-memory
// histogram per row.  Disparity is locally smooth (a road row holds one or two bins, an obstacle one), so
// each thread counts a run of equal (row, bin) keys in registers and adds the run with one shared-memory
// atomic when the key changes: fewer atomics than pixels, and few 32-way conflicts on the dominant bin.
// The run update is branch-free (the flush is a predicated add; invalid pixels keep the run going), so
// warps do not diverge on the data.  The bin takes two float adds instead of a float-to-integer
// conversion (packed: one instruction adds two pixels): for 0 <= x < 2^23, x + 2^23 rounded toward -infinity is 2^23 + floor(x) exactly (the
// float spacing there is 1), so its bit pattern minus that of 2^23 is floor(x); any other x leaves a
// difference >= D (as unsigned), which the bin test rejects.  The shared histogram rows are D + 1 words
// apart, so the transposed write-out ([D][H] per frame, so that each step of the road DP (Eq. 12) reads
// one contiguous row) reads it without bank conflicts.
#include "ld_internal.cuh"

namespace ld {

namespace {
constexpr int kRowsDefault = 16;  // rows per CTA unless tuned
constexpr int kThreads = 256;
constexpr int kUnroll = 4;  // 16-byte loads in flight per thread
constexpr uint32_t kTwo23Bits = 0x4B000000u;  // bit pattern of 2^23 in float32

// Shared-memory add of v at address a when p holds, as one predicated instruction (no branch).
__device__ __forceinline__ void red_add_if(bool p, uint32_t a, int v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q red.shared.add.s32 [%0], %1;\n\t}" ::"r"(a), "r"(v),
                 "r"((int)p));
}

// One pixel of a run, as one predicated block: when key differs from run_key, add the run's count cnt at
// address a; cnt becomes 1 (a new key comes from a counted pixel) or else inc (cnt plus the pixel's count).
__device__ __forceinline__ void flush_step(int key, int run_key, uint32_t a, int &cnt, int inc)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, %2;\n\t@q red.shared.add.s32 [%3], %4;\n\t"
                 "selp.s32 %0, 1, %5, q;\n\t}"
                 : "=r"(cnt) : "r"(key), "r"(run_key), "r"(a), "r"(cnt), "r"(inc));
}

// 16-byte load of the disparity, which this kernel reads once, under an L2 evict_first policy: its lines
// go first when the L2 needs room, ahead of the lines (often dirty) that earlier kernels left there.
__device__ __forceinline__ float4 ld_stream(const float4 *p, uint64_t pol)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
}

// Rows [tile * kRows, ..) of frame f.
__device__ __forceinline__ void vdisp_body(const KParams &kp, int32_t *__restrict__ myT, const float *__restrict__ disp,
                                           int kRows, int f, int tile)
{
    extern __shared__ int32_t hist[];  // [kRows][D + 1]
    const int W = kp.W, H = kp.H, D = kp.D, Dp = D + 1;
    const int r0 = tile * kRows;
    const int nr = min(kRows, H - r0);
    const int tid = threadIdx.x;
    for (int i = tid; i < kRows * Dp; i += kThreads)
        hist[i] = 0;
    __syncthreads();

    const float *src = disp + ((size_t)f * H + r0) * W;
    const int n = nr * W;
    // bin of a pixel: floor(l + 0.5) when l > 0 and the bin is below D, else -1.  A NaN fails l > 0, and
    // +inf (or any l past the last bin) converts to a value >= D, so one compare covers finiteness too.
    auto bin_of = [&](float l) {
        const int b = __float2int_rd(__fadd_rn(l, 0.5f));
        return (l > 0.0f && b < D) ? b : -1;
    };
    const int head = min((int)(((16u - ((uint32_t)(uintptr_t)src & 15u)) & 15u) >> 2), n);
    const int nb = (n - head) >> 2, tail0 = head + 4 * nb;
    if (tid < head + n - tail0) {
        const int off = tid < head ? tid : tail0 + (tid - head);
        const int b = LD_IN(off, n, CK_VDISP_LOAD) ? bin_of(__ldg(src + off)) : -1;
        if (b >= 0 && LD_IN((off / W) * Dp + b, nr * Dp, CK_VDISP_BIN))
            atomicAdd(&hist[(off / W) * Dp + b], 1);
    }
    // each warp takes one contiguous span of the 16-byte chunks (about one row), so a lane's successive
    // loads (128 pixels apart) mostly stay in one row and its run key changes only with the bin
    const float4 *body = reinterpret_cast<const float4 *>(src + head);
    constexpr int kWarps = kThreads / 32;
    const int lane = tid & 31, span = (nb + kWarps - 1) / kWarps;
    const int w0 = (tid >> 5) * span, w1 = min(nb, w0 + span);
    // row and column of the lane's first pixel, then advanced by 128 pixels per step (no division)
    int off0 = head + 4 * (w0 + lane);
    int row = off0 / W, col = off0 - row * W;
    // one run per lane, updated without branches: an invalid pixel takes the run's key (it neither breaks nor
    // extends the count); a new key flushes the run with a predicated shared-memory add (an empty run adds 0)
    const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(hist);
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    int run_key = 0, run_cnt = 0;
    for (int base = w0; base < w1; base += 32 * kUnroll) {
        float4 x[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int i = base + 32 * k + lane;
            x[k] = i < w1 && LD_IN(head + 4 * i + 3, n, CK_VDISP_LOAD) ? ld_stream(body + i, pol)
                                                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // 0 does not count
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const float l[4] = {x[k].x, x[k].y, x[k].z, x[k].w};
            // both adds of the bin for two pixels at a time (packed FP32, each element rounded as the scalar add)
            const float2 h2 = make_float2(0.5f, 0.5f), t2 = make_float2(8388608.0f, 8388608.0f);
            const float2 p01 = __fadd2_rd(__fadd2_rn(make_float2(l[0], l[1]), h2), t2);
            const float2 p23 = __fadd2_rd(__fadd2_rn(make_float2(l[2], l[3]), h2), t2);
            const float pb[4] = {p01.x, p01.y, p23.x, p23.y};
            const int rb = row * Dp, rw = W - col;  // pixels e >= rw of this chunk are on the next row
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t b = __float_as_uint(pb[e]) - kTwo23Bits;
                const bool ok = l[e] > 0.0f && b < (uint32_t)D;
                const int key = ok ? (e < rw ? rb : rb + Dp) + (int)b : run_key;
#ifdef LD_CHECKED
                const bool nk = key != run_key;
                red_add_if(nk && LD_IN(run_key, nr * Dp, CK_VDISP_RUN), hbase + 4u * (uint32_t)run_key, run_cnt);
                run_cnt = (nk ? 0 : run_cnt) + (int)ok;
#else
                flush_step(key, run_key, hbase + 4u * (uint32_t)run_key, run_cnt, run_cnt + (int)ok);
#endif
                run_key = key;
            }
            col += 128;
            while (col >= W) {
                col -= W;
                ++row;
            }
        }
    }
    red_add_if(run_cnt != 0 && LD_IN(run_key, nr * Dp, CK_VDISP_RUN), hbase + 4u * (uint32_t)run_key, run_cnt);
    __syncthreads();
    // thread t writes row r = t mod nr of bins d = t / nr, t / nr + step, ... (one division per thread)
    int32_t *dst = myT + (size_t)f * D * H;
    const int step = kThreads / nr, r = tid % nr;
    if (tid < step * nr)
        for (int d = tid / nr; d < D; d += step)
            if (LD_IN(r0 + r, H, CK_VDISP_OUT))
                dst[(size_t)d * H + r0 + r] = hist[r * Dp + d];
}

__global__ void __launch_bounds__(kThreads) k_vdisp(const KParams kp, int32_t *__restrict__ myT,
                                                    const float *__restrict__ disp, int kRows)
{
    vdisp_body(kp, myT, disp, kRows, blockIdx.y, blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_vdisp_fd(const FrameDesc *__restrict__ fd, int kRows)
{
    const FrameDesc &d = fd[blockIdx.y];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    if ((int)blockIdx.x * kRows >= kp.H)
        return;
    vdisp_body(kp, w.myT, d.disp, kRows, 0, blockIdx.x);
}
}  // namespace

// Rows per CTA: the tuned value when set, at most one per thread (the write-out gives each row at least
// one thread), kept within 48 KB of histogram shared memory.
int vdisp_rows(const KParams &kp)
{
    int r = kp.tile_vdisp > 0 ? min(kp.tile_vdisp, kThreads) : kRowsDefault;
    while (r > 1 && sizeof(int32_t) * (size_t)r * (kp.D + 1) > 48 * 1024)
        r >>= 1;
    return r;
}

cudaError_t launch_vdisp(const KParams &kp, const Work &w, const float *disp, cudaStream_t s)
{
    const int kRows = vdisp_rows(kp);
    dim3 grid((kp.H + kRows - 1) / kRows, kp.n_frames);
    const size_t smem = sizeof(int32_t) * kRows * (kp.D + 1);
    k_vdisp<<<grid, kThreads, smem, s>>>(kp, w.myT, disp, kRows);
    return cudaGetLastError();
}

cudaError_t launch_vdisp_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    const int kRows = vdisp_rows(kmax);
    dim3 grid((kmax.H + kRows - 1) / kRows, n);
    k_vdisp_fd<<<grid, kThreads, sizeof(int32_t) * kRows * (kmax.D + 1), s>>>(fd, kRows);
    return cudaGetLastError();
}

}  // namespace ld
