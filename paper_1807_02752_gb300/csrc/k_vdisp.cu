// Sec. 2.2: the v-disparity map m_y(d, v), the histogram of every row of the disparity map.
//
// A pixel counts when its disparity l is finite and > 0 (0 marks pixels invalidated by the left-right
// check, Eq. 10); its bin is floor(l + 0.5) in float32 and bins >= D are dropped.
//
// One CTA covers kRows consecutive rows of one frame.  Those rows are contiguous in memory, so the CTA
// streams them as one flat range (coalesced 128-byte warp loads, several loads in flight per thread).
// Counts go to a shared-memory histogram per row with warp-aggregated atomics: lanes holding the same
// (row, bin) key elect one leader that adds the group's size.  On road rows most pixels of a warp share
// one bin, so this turns up to 32 conflicting atomics into one.  The histogram is written transposed,
// [D][H] per frame, so that each step of the road DP (Eq. 12) reads one contiguous row.
#include "ld_internal.cuh"

namespace ld {

namespace {
constexpr int kRows = 8;
constexpr int kThreads = 256;
constexpr int kUnroll = 4;

__global__ void __launch_bounds__(kThreads) k_vdisp(const KParams kp, int32_t *__restrict__ myT,
                                                    const float *__restrict__ disp)
{
    extern __shared__ int32_t hist[];  // [kRows][D]
    const int W = kp.W, H = kp.H, D = kp.D;
    const int f = blockIdx.y;
    const int r0 = blockIdx.x * kRows;
    const int nr = min(kRows, H - r0);
    for (int i = threadIdx.x; i < kRows * D; i += kThreads)
        hist[i] = 0;
    __syncthreads();

    const float *src = disp + ((size_t)f * H + r0) * W;
    const int n = nr * W;
    const float fD = (float)D;
    for (int base = 0; base < n; base += kThreads * kUnroll) {
        float val[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int i = base + k * kThreads + threadIdx.x;
            val[k] = i < n ? __ldg(src + i) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int i = base + k * kThreads + threadIdx.x;
            int key = -1;
            const float l = val[k];
            if (i < n && l > 0.0f && l < __int_as_float(0x7f800000)) {
                const float b = floorf(__fadd_rn(l, 0.5f));
                if (b < fD)
                    key = (i / W) * D + (int)b;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&hist[key], __popc(peers));
        }
    }
    __syncthreads();
    int32_t *dst = myT + (size_t)f * D * H;
    for (int i = threadIdx.x; i < D * nr; i += kThreads) {
        const int d = i / nr, r = i - d * nr;
        dst[(size_t)d * H + r0 + r] = hist[r * D + d];
    }
}
}  // namespace

cudaError_t launch_vdisp(const KParams &kp, const Work &w, const float *disp, cudaStream_t s)
{
    dim3 grid((kp.H + kRows - 1) / kRows, kp.n_frames);
    const size_t smem = sizeof(int32_t) * kRows * kp.D;
    k_vdisp<<<grid, kThreads, smem, s>>>(kp, w.myT, disp);
    return cudaGetLastError();
}

}  // namespace ld
