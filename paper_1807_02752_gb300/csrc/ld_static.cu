// ld_road_path_static: the road-profile DP path (v-disparity histogram and the road DP over it, with the
// tie rules of the handle-based road kernel) for callers that must not allocate device memory.  It is a
// separate variant of the library's two road kernels, fused into one kernel whose v-disparity scratch
// lives in a file-scope static device array instead of a handle's workspace.  No other code path uses it.
//
// The array is LD_STATIC_SCRATCH_BYTES bytes of device memory that every GPU which loads the library
// keeps until the process exits.  Host code cannot use the array's name as a device address (on the host
// it names a stand-in object): the first call on each device, with that device current, looks the address
// up with cudaGetSymbolAddress and caches it; later calls on that device reuse it.
#include <mutex>

#include "ld_internal.cuh"

namespace ld {
void set_global_error(const char *msg);
}

namespace {

constexpr int kThreads = 512;
constexpr int kRows = 8;
constexpr int kPad = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int32_t g_road_scratch[LD_STATIC_SCRATCH_BYTES / sizeof(int32_t)];

std::mutex g_setup_mutex;
int32_t *g_scratch_ptr[kMaxDevices] = {};

// One CTA per frame: the frame's v-disparity map m_y is written transposed ([D][H]) to the scratch, then
// the DP of Eq. 12 runs over it exactly as the handle-based road kernels do (same tie rules) and the path
// row v_d of every d is written to path_out[frame][d] (entry 0 is -1).
__global__ void __launch_bounds__(kThreads) k_road_path_static(const ld::KParams kp, int32_t *__restrict__ scratch,
                                                               const float *__restrict__ disp,
                                                               int16_t *__restrict__ path_out)
{
    extern __shared__ __align__(16) int32_t sm[];
    const int f = blockIdx.x, W = kp.W, H = kp.H, D = kp.D, Hp = (H + 1) >> 1;
    const int tid = threadIdx.x;
    int32_t *my = scratch + (size_t)f * D * H;
    const float *src = disp + (size_t)f * H * W;

    // ---- v-disparity rows, kRows at a time ----
    int32_t *hist = sm;  // [kRows][D]
    const float fD = (float)D;
    for (int r0 = 0; r0 < H; r0 += kRows) {
        const int nr = min(kRows, H - r0);
        for (int i = tid; i < kRows * D; i += kThreads)
            hist[i] = 0;
        __syncthreads();
        const int n = nr * W;
        for (int i0 = 0; i0 < n; i0 += kThreads) {
            const int i = i0 + tid;
            int key = -1;
            if (i < n) {
                const float l = __ldg(src + (size_t)r0 * W + i);
                if (l > 0.0f && l < __int_as_float(0x7f800000)) {
                    const float b = floorf(__fadd_rn(l, 0.5f));
                    if (b < fD)
                        key = (i / W) * D + (int)b;
                }
            }
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && (tid & 31) == __ffs(peers) - 1)
                atomicAdd(&hist[key], __popc(peers));
        }
        __syncthreads();
        for (int i = tid; i < D * nr; i += kThreads) {
            const int d = i / nr, r = i - d * nr;
            my[(size_t)d * H + r0 + r] = hist[r * D + d];
        }
        __syncthreads();
    }
    __threadfence_block();
    __syncthreads();

    // ---- Eq. 12 DP from d = D-1 down to 1 ----
    int32_t *E0 = sm;
    int32_t *E1 = E0 + H + kPad;
    int32_t *scr = E1 + H + kPad;                  // 2 ints
    uint8_t *bt = reinterpret_cast<uint8_t *>(scr + 4);
    for (int v = tid; v < H + kPad; v += kThreads) {
        E0[v] = v < H ? -my[(size_t)(D - 1) * H + v] : 0x3fffffff;
        E1[v] = 0x3fffffff;
    }
    __syncthreads();
    int32_t *Ep = E0, *Ec = E1;
    const int tau = kp.tau_y, lam = kp.lambda_y;
    for (int d = D - 2; d >= 1; --d) {
        const int32_t *row = my + (size_t)d * H;
        for (int i = tid; i < Hp; i += kThreads) {
            uint8_t nib = 0;
            for (int h = 0; h < 2; ++h) {
                const int v = 2 * i + h;
                int best = Ep[v], arg = 0;
                for (int t = 1; t <= tau; ++t) {
                    const int cand = Ep[v + t] + lam * t;
                    if (cand < best) {
                        best = cand;
                        arg = t;
                    }
                }
                if (v < H)
                    Ec[v] = -row[v] + best;
                nib |= (uint8_t)(arg << (4 * h));
            }
            bt[(size_t)d * Hp + i] = nib;
        }
        __syncthreads();
        int32_t *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    if (tid < 32) {
        int bv = 0x7fffffff, bi = 0x7fffffff;
        for (int v = tid; v < H; v += 32)
            if (Ep[v] < bv) {
                bv = Ep[v];
                bi = v;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const int ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (tid == 0) {
            int16_t *out = path_out + (size_t)f * D;
            out[0] = -1;
            int v = bi;
            out[1] = (int16_t)v;
            for (int d = 1; d <= D - 2; ++d) {
                const uint8_t b = bt[(size_t)d * Hp + (v >> 1)];
                v += (v & 1) ? (b >> 4) : (b & 15);
                out[d + 1] = (int16_t)v;
            }
        }
    }
}

size_t static_smem_bytes(int H, int D)
{
    const size_t hist = sizeof(int32_t) * kRows * D;
    const size_t dp = sizeof(int32_t) * (2 * (size_t)(H + kPad) + 4) + (size_t)D * ((H + 1) / 2);
    return (hist > dp ? hist : dp) + 16;
}

}  // namespace

extern "C" int ld_road_path_static(const ld_params *p, const float *disp, int32_t w, int32_t h_px, int32_t n_frames,
                                   int16_t *path_out, void *cuda_stream)
{
    if (!p || !disp || !path_out) {
        ld::set_global_error("ld_road_path_static: null argument");
        return LD_E_ARG;
    }
    if (p->n_disp < 4 || p->n_disp > LD_MAX_D || p->tau_y < 0 || p->tau_y > 15 || p->lambda_y < 0 ||
        p->lambda_y > 1000 || w < 16 || w > LD_MAX_W || h_px < 16 || h_px > LD_MAX_H || n_frames < 1) {
        ld::set_global_error("ld_road_path_static: parameter or size out of range");
        return LD_E_ARG;
    }
    if (p->dp_literal != 0) {
        ld::set_global_error("ld_road_path_static: dp_literal = 1 (the DP as printed) is not offered by this entry point");
        return LD_E_ARG;
    }
    const size_t need = (size_t)n_frames * p->n_disp * h_px * sizeof(int32_t);
    if (need > LD_STATIC_SCRATCH_BYTES) {
        ld::set_global_error("ld_road_path_static: n_frames * n_disp * h * 4 exceeds LD_STATIC_SCRATCH_BYTES");
        return LD_E_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        ld::set_global_error("ld_road_path_static: no usable current device");
        return LD_E_CUDA;
    }
    const size_t smem = static_smem_bytes(h_px, p->n_disp);
    int32_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_road_scratch);
            if (e != cudaSuccess) {
                ld::set_global_error("ld_road_path_static: cudaGetSymbolAddress failed");
                return LD_E_CUDA;
            }
            e = cudaFuncSetAttribute(k_road_path_static, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)static_smem_bytes(LD_MAX_H, LD_MAX_D));
            if (e != cudaSuccess) {
                ld::set_global_error("ld_road_path_static: shared-memory set-up failed");
                return LD_E_CUDA;
            }
            g_scratch_ptr[dev] = (int32_t *)ptr;
        }
        scratch = g_scratch_ptr[dev];
    }
    ld::KParams kp{};
    kp.W = w;
    kp.H = h_px;
    kp.D = p->n_disp;
    kp.n_frames = n_frames;
    kp.tau_y = p->tau_y;
    kp.lambda_y = p->lambda_y;
    k_road_path_static<<<n_frames, kThreads, smem, (cudaStream_t)cuda_stream>>>(kp, scratch, disp, path_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        ld::set_global_error("ld_road_path_static: kernel launch failed");
        return LD_E_CUDA;
    }
    return LD_OK;
}
