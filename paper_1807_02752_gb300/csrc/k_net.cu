// Learned lane-position proposal: a small BF16 convolutional network on the 4x-downsampled map of
// |G_x w_g| (Eq. 23) ranks the bottom-row starts of Eq. 24-25, and exact energies are evaluated only on
// the best-ranked ones (the exhaustive search of Alg. 7 stays as the fallback).  The paper has no such
// network; the form follows a stated configuration: 3x3 convolutions with 1-16-32-32-16 channels, BF16
// operands with FP32 accumulation, a per-cell logit z (the per-row heatmap is sigmoid(z)), top-k = 32.
//
//   k_conv1     layer 1 (one input channel) from the integer block sums; writes the bf16 input and A1
//   k_conv_tc   layers 2-4 as implicit GEMMs on the tcgen05 tensor cores (bf16 -> f32 in tensor memory):
//               a 16 x 8-cell output tile per MMA (M 128), K = 9 taps x C_in straight from the halo in
//               shared memory; epilogues: bias + ReLU (+ the 1x1 head), or the backward data pass
//               (transposed, flipped weights) times the ReLU mask of the layer below
//   k_wgrad     weight and bias gradients of a layer (mma.sync m16n8k16): M = C_out, N = 9 C_in + 1 (a
//               column of ones gives the bias), K = cells; per-CTA partial sums, then k_wreduce adds them
//               in a fixed order
//   k_loss      head, weighted logistic loss, dz, dS_4 and the head's gradient partials
//   k_adam      Adam (Kingma & Ba, Algorithm 1) on the FP32 master weights, then the bf16 operand copies
//   k_labels    training targets: cells crossed by the Eq. 25 tracks of the selected lanes
//   k_score     coarse-start scores: the heatmap summed along the Eq. 25 track taken in steps of four rows
//   k_topk      the k best coarse starts of a frame -> candidate and evaluated starts
//
// Data layout: cell maps are [n][mh][mw] with mh = ceil(H/4), mw = ceil(W/4); activations are bf16
// [n][mh][mw][C] (channels innermost, 32 or 64 bytes per cell).  Weights: W_l[co][tap][ci] (k = tap C_in
// + ci) for the forward pass and W_l^T[ci][8 - tap][co] for the backward data pass.
#include <cuda_bf16.h>

#include "ld_internal.cuh"
#include "ld_net.cuh"

namespace ld {

namespace {

constexpr int kTileR = 8, kTileC = 16;              // output cells per CTA tile
constexpr int kHaloR = kTileR + 2, kHaloC = kTileC + 2;
constexpr int kConvThreads = 128;                   // 4 warps, two tile rows (two m16 tiles) each
constexpr int kCellThreads = 256;
constexpr float kInScale = 2.384185791015625e-07f;  // 2^-22

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// first cell row a layer must produce for frame f, or INT_MAX when the frame needs nothing
__device__ __forceinline__ int first_needed_row(const FrameState *fs, int f, int depth)
{
    if (!fs)
        return 0;
    const FrameState &s = fs[f];
    if (s.flags & (LD_F_NO_ROAD | LD_F_DEGEN_Y | LD_F_DEGEN_X))
        return 0x7fffffff;
    return (s.v_top >> 2) - depth;
}

// network input of one cell: bf16(f32(sum) 2^-22), as a float
__device__ __forceinline__ float cell_input(int32_t s)
{
    return __bfloat162float(__float2bfloat16_rn(__fmul_rn(__int2float_rn(s), kInScale)));
}

// ---------------------------------------------------------------------------------------------------
// layer 1: one input channel, K = 9, direct FMA per cell
// ---------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kCellThreads) k_conv1(const NetArgs a, const int32_t *xsum, int n,
                                                        const FrameState *fs)
{
    __shared__ float wsm[16 * 9 + 16];
    for (int i = threadIdx.x; i < 16 * 9; i += kCellThreads)
        wsm[i] = __bfloat162float(a.wf[0][i]);   // [co][tap]
    for (int i = threadIdx.x; i < 16; i += kCellThreads)
        wsm[144 + i] = a.bias[0][i];
    __syncthreads();
    const int mh = a.mh, mw = a.mw;
    const long long cells = (long long)n * mh * mw;
    for (long long p = blockIdx.x * (long long)kCellThreads + threadIdx.x; p < cells;
         p += (long long)gridDim.x * kCellThreads) {
        const int x = (int)(p % mw);
        const int y = (int)((p / mw) % mh);
        const long long fb = p - (long long)y * mw - x;   // first cell of the frame
        if (y < first_needed_row(fs, (int)(p / ((long long)mh * mw)), 3))
            continue;
        float in[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
            in[t] = (yy >= 0 && yy < mh && xx >= 0 && xx < mw) ? cell_input(__ldg(xsum + fb + (long long)yy * mw + xx)) : 0.0f;
        }
        if (a.X)
            a.X[p] = __float2bfloat16_rn(in[4]);
        uint32_t o[8];
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            float s0 = wsm[144 + c], s1 = wsm[144 + c + 1];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                s0 = __fmaf_rn(wsm[c * 9 + t], in[t], s0);
                s1 = __fmaf_rn(wsm[(c + 1) * 9 + t], in[t], s1);
            }
            o[c >> 1] = pack2(fmaxf(s0, 0.0f), fmaxf(s1, 0.0f));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(a.act[0] + p * 16);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
}

// ---------------------------------------------------------------------------------------------------
// layers 2-4 (and the backward data pass) on the tensor cores
// ---------------------------------------------------------------------------------------------------
enum Epi { kEpiRelu = 0, kEpiHead = 1, kEpiMask = 2 };

struct ConvIO {
    const __nv_bfloat16 *in;     // [n][mh][mw][CIN]
    const __nv_bfloat16 *wt;     // [COUT][9 CIN]
    const float *bias;           // [COUT] (kEpiRelu, kEpiHead)
    __nv_bfloat16 *out;          // [n][mh][mw][COUT] (kEpiHead: may be null)
    const __nv_bfloat16 *mask;   // [n][mh][mw][COUT] activations whose sign gates the result (kEpiMask)
    const __nv_bfloat16 *wh;     // [16] head weights (kEpiHead)
    const float *bh;             // [1]
    float *z;                    // [n][mh][mw] logits, or the heatmap sigmoid(z) when heat (kEpiHead)
    int n, mh, mw, tiles_r, tiles_c;
    int heat;
    // road rows only (learned detection): frame f needs this layer's output rows >= (v_top >> 2) - depth;
    // tiles entirely above, and frames without a road fit, are skipped (null: every tile)
    const FrameState *fs;
    int depth;
};


// ---------------------------------------------------------------------------------------------------
// layers 2-4 and the backward data pass on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory)
//
// Tile: 16 x 8 output cells = the 128 rows (M) of one MMA.  The tile's 18 x 10-cell halo sits in shared
// memory as planes of 8 channels, 16 bytes per cell (plane stride 2880 B, halo row 160 B), which is the
// no-swizzle K-major operand layout for every tap at once: for tap (dy, dx) and 16 input channels the A
// operand starts at the tap's cell of the first plane, its two K halves are one plane apart (leading byte
// offset 2880) and its 16 groups of 8 rows are the tile rows, one halo row apart (stride byte offset 160).
// The weights sit in the matching layout for B (N = C_out rows): per K step of 16 channels, K halves
// C_out x 16 B apart, groups of 8 output channels 128 B apart.  One thread issues the 9 C_in / 16 MMAs of a
// tile (M 128, N C_out, K 16, bf16 -> f32) into one of two accumulators in tensor memory and commits them to
// an mbarrier; meanwhile the CTA reads the other accumulator (tcgen05.ld, one tensor-memory lane quarter per
// warp: a thread gets all C_out channels of one cell) for the previous tile's epilogue and copies the next
// tile's halo in with cp.async (zero-filled outside the map).  Waits are bounded: on a timeout the kernel
// records it in err and stops issuing work.
// ---------------------------------------------------------------------------------------------------
constexpr int kTcRows = 16, kTcCols = 8;                       // output tile (cells)
constexpr int kTcHR = kTcRows + 2, kTcHC = kTcCols + 2;         // halo
constexpr int kTcPlane = kTcHR * kTcHC * 16;                    // bytes of one 8-channel plane of the halo
constexpr unsigned kTcSpin = 1u << 26;                           // wait limit (iterations)

template <int CIN, int COUT>
struct TcSmem {
    static constexpr int halo = (CIN / 8) * kTcPlane;            // one halo buffer
    static constexpr int wts = 9 * CIN * COUT * 2;               // B operand, all taps
    static constexpr size_t bytes = 2 * (size_t)halo + wts + 128;
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);   // no swizzle, base offset 0
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    for (unsigned it = 0; it < kTcSpin; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done)
            return true;
    }
    return false;
}

template <int N>
__device__ __forceinline__ void tc_load(uint32_t taddr, uint32_t (&r)[N]);

template <>
__device__ __forceinline__ void tc_load<16>(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <>
__device__ __forceinline__ void tc_load<32>(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kConvThreads) k_conv_tc(const ConvIO io, int *err)
{
    using S = TcSmem<CIN, COUT>;
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    __shared__ uint32_t taddr_s;
    __shared__ __align__(8) uint64_t mbar[2];
    unsigned char *halo[2] = {tsm_raw, tsm_raw + S::halo};
    unsigned char *wsm = tsm_raw + 2 * S::halo;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mh = io.mh, mw = io.mw;
    const int per_frame = io.tiles_r * io.tiles_c, total = io.n * per_frame;
    // weights -> B layout: K step kk = tap (CIN/16) + c16, half h: 16-byte row n at
    // kk (COUT 32) + h (COUT 16) + (n / 8) 128 + (n % 8) 16; a row holds the 8 input channels c16 16 + 8 h ..
    for (int i = tid; i < COUT * 9 * (CIN / 8); i += kConvThreads) {
        const int n = i / (9 * CIN / 8), rem = i % (9 * CIN / 8), tap = rem / (CIN / 8), c8 = rem % (CIN / 8);
        const int kk = tap * (CIN / 16) + (c8 >> 1), h = c8 & 1;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(io.wt + (size_t)n * 9 * CIN + tap * CIN + c8 * 8));
        *reinterpret_cast<uint4 *>(wsm + kk * COUT * 32 + h * COUT * 16 + (n >> 3) * 128 + (n & 7) * 16) = v;
    }
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]), mb1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&taddr_s);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(dst));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = taddr_s;
    // the tiles this CTA owns: blockIdx.x, + gridDim.x, ...; those above the road rows are skipped
    auto next_tile = [&](int t) {
        for (; t < total; t += gridDim.x) {
            const int f = t / per_frame, rem = t % per_frame;
            if ((rem / io.tiles_c) * kTcRows + kTcRows - 1 >= first_needed_row(io.fs, f, io.depth))
                return t;
        }
        return total;
    };
    auto load_halo = [&](int t, unsigned char *buf) {
        const int f = t / per_frame, rem = t % per_frame;
        const int y0 = (rem / io.tiles_c) * kTcRows - 1, x0 = (rem % io.tiles_c) * kTcCols - 1;
        for (int i = tid; i < kTcHR * kTcHC * (CIN / 8); i += kConvThreads) {
            const int p = i / (kTcHR * kTcHC), cell = i % (kTcHR * kTcHC);
            const int yy = y0 + cell / kTcHC, xx = x0 + cell % kTcHC;
            const bool in = yy >= 0 && yy < mh && xx >= 0 && xx < mw;
            const __nv_bfloat16 *src = io.in + (((size_t)f * mh + (in ? yy : 0)) * mw + (in ? xx : 0)) * CIN + p * 8;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf + p * kTcPlane + cell * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float hw[16], bias[COUT];
    if (EPI == kEpiHead) {
#pragma unroll
        for (int c = 0; c < 16; ++c)
            hw[c] = __bfloat162float(io.wh[c]);
    }
    if (EPI != kEpiMask) {
#pragma unroll
        for (int c = 0; c < COUT; ++c)
            bias[c] = io.bias[c];
    }
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COUT >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(wsm);
    bool ok = true;
    int cur = next_tile(blockIdx.x), prev = total, it = 0;
    uint32_t phase[2] = {0u, 0u};
    if (cur < total)
        load_halo(cur, halo[0]);
    while (cur < total || prev < total) {
        const int b = it & 1;
        if (cur < total) {
            // the halo of `cur` has landed: make it visible to the tensor cores and issue its MMAs
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (tid == 0 && ok) {
                const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(halo[b]);
                const uint32_t dacc = tbase + (uint32_t)(b * 32);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                    for (int c16 = 0; c16 < CIN / 16; ++c16) {
                        const int kk = tap * (CIN / 16) + c16;
                        const uint64_t ad = tc_desc(hbase + (2 * c16) * kTcPlane + ((tap / 3) * kTcHC + tap % 3) * 16,
                                                    kTcPlane, kTcHC * 16);
                        const uint64_t bd = tc_desc(wbase + kk * COUT * 32, COUT * 16, 128);
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     ::"r"(dacc), "l"(ad), "l"(bd), "r"(kIdesc), "r"(kk));
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(b ? mb1 : mb0) : "memory");
            }
        }
        if (prev < total) {
            // the previous tile: wait for its MMAs, then read its accumulator and store the cells
            const int pb = b ^ 1;
            if (ok && !__all_sync(0xffffffffu, tc_wait(pb ? mb1 : mb0, phase[pb]))) {
                ok = false;   // uniform over the warp (tcgen05.ld is a warp-wide instruction)
                if (lane == 0)
                    atomicExch(err, 1);
            }
            phase[pb] ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int f = prev / per_frame, rem = prev % per_frame;
            const int y = (rem / io.tiles_c) * kTcRows + warp * 4 + (lane >> 3), x = (rem % io.tiles_c) * kTcCols + (lane & 7);
            uint32_t r[COUT];
            if (ok)
                tc_load<COUT>(tbase + (uint32_t)(pb * 32) + ((uint32_t)(warp * 32) << 16), r);
            if (ok && y < mh && x < mw) {
                const size_t cell = ((size_t)f * mh + y) * mw + x;
                if (EPI == kEpiMask) {
                    const uint4 *mk = reinterpret_cast<const uint4 *>(io.mask + cell * COUT);
                    uint4 *dst = reinterpret_cast<uint4 *>(io.out + cell * COUT);
#pragma unroll
                    for (int q = 0; q < COUT / 8; ++q) {
                        const uint4 m4 = __ldg(mk + q);
                        const uint32_t mw4[4] = {m4.x, m4.y, m4.z, m4.w};
                        uint32_t o[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float v0 = bf_lo(mw4[k]) > 0.0f ? __uint_as_float(r[q * 8 + 2 * k]) : 0.0f;
                            const float v1 = bf_hi(mw4[k]) > 0.0f ? __uint_as_float(r[q * 8 + 2 * k + 1]) : 0.0f;
                            o[k] = pack2(v0, v1);
                        }
                        dst[q] = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                } else {
                    float zc = 0.0f;
                    uint4 *dst = io.out ? reinterpret_cast<uint4 *>(io.out + cell * COUT) : nullptr;
#pragma unroll
                    for (int q = 0; q < COUT / 8; ++q) {
                        uint32_t o[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int c = q * 8 + 2 * k;
                            const float v0 = fmaxf(__fadd_rn(__uint_as_float(r[c]), bias[c]), 0.0f);
                            const float v1 = fmaxf(__fadd_rn(__uint_as_float(r[c + 1]), bias[c + 1]), 0.0f);
                            o[k] = pack2(v0, v1);
                            if (EPI == kEpiHead)
                                zc = __fmaf_rn(hw[c + 1], bf_hi(o[k]), __fmaf_rn(hw[c], bf_lo(o[k]), zc));
                        }
                        if (dst)
                            dst[q] = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                    if (EPI == kEpiHead) {
                        zc = __fadd_rn(zc, io.bh[0]);
                        io.z[cell] = io.heat ? __frcp_rn(__fadd_rn(1.0f, expf(-zc))) : zc;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
        // the next tile's halo goes into the buffer the previous tile's MMAs have finished with
        prev = cur;
        if (cur < total) {
            cur = next_tile(cur + gridDim.x);
            if (cur < total && ok)
                load_halo(cur, halo[b ^ 1]);
        }
        ++it;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tbase));
}

// ---------------------------------------------------------------------------------------------------
// The inference forward in one kernel: layers 1-4 and the head for a 32 x 16-cell output tile, the
// activations kept in shared memory between the layers and the accumulators in tensor memory.
//
// A layer-4 output tile of kFR x kFC cells needs layer 3 on a one-cell border around it, layer 2 on two
// cells, layer 1 on three and the input on four.  Layers 2 and 3 run as 3 x 3 MMA blocks of 16 x 8 cells
// (M 128) over a 48 x 24 region, layer 4 as 2 x 2 blocks; every block is the per-layer kernel's MMA
// sequence (taps in order, then 16-channel K steps, bf16 x bf16 -> f32) on operands in the same plane
// layout (8 channels per plane, 16 bytes per cell; K halves one plane apart, 8-row groups one region row
// apart), so every accumulator, and therefore every activation and logit of the road rows, equals the
// per-layer kernels' bit for bit.  Cells outside the map are stored as zero (the zero padding of the
// next layer); cells a block computes beyond the region the next layer reads are dropped.  One thread
// issues a layer's MMAs into up to nine accumulators (32 tensor-memory columns each) and commits them to
// an mbarrier; the whole CTA waits (bounded), reads the accumulators back (tcgen05.ld, one lane quarter per
// warp, warps w and w + 4 taking the two column halves) and writes the next layer's input.  Layer 1 (one
// input channel) runs on the CUDA cores in the per-layer kernel's operation order.  The next tile's input
// arrives by cp.async while the current tile runs.
//
// Measured on the 64-frame 1242x375 learned detection (top_k 96): 1.26 ms per call against 1.13 ms with one
// kernel per layer.  With about 170 KB of shared memory a CTA is alone on its SM and a tile's phases run
// one after another (issue 21 % active, tensor pipe 12 %), where the per-layer kernels keep four CTAs per
// SM and overlap one tile's MMAs with the next tile's copies; so the per-layer form is the default.
// ---------------------------------------------------------------------------------------------------
constexpr int kFR = 32, kFC = 16;                                // layer-4 output tile (cells)
constexpr int kF1R = kFR + 18, kF1C = kFC + 10;                  // layer-1 region (layer-2 input), origin (-3, -3)
constexpr int kF2R = kF1R, kF2C = kF1C;                          // layer-2 region (layer-3 input), origin (-2, -2)
constexpr int kF3R = kFR + 2, kF3C = kFC + 2;                    // layer-3 region (layer-4 input), origin (-1, -1)
constexpr int kFXR = kF1R + 2, kFXC = kF1C + 2;                  // input region, origin (-4, -4)
constexpr int kFusedThreads = 256;
constexpr int kFP1 = kF1R * kF1C * 16, kFP2 = kF2R * kF2C * 16, kFP3 = kF3R * kF3C * 16;   // plane bytes
constexpr int kFBufA = 2 * kFP1 > 4 * kFP3 ? 2 * kFP1 : 4 * kFP3;                       // layer 1 / layer 3 out
constexpr int kFBufB = 4 * kFP2;                                                         // layer 2 out
constexpr int kFW2 = 9 * 16 * 32 * 2, kFW3 = 9 * 32 * 32 * 2, kFW4 = 9 * 32 * 16 * 2;
constexpr int kFX = kFXR * kFXC * 4;   // one input buffer (raw block sums); two are kept
constexpr size_t kFusedSmem = (size_t)kFBufA + kFBufB + kFW2 + kFW3 + kFW4 + 2 * kFX;
static_assert(kFBufA % 16 == 0 && kFBufB % 16 == 0 && kFX % 16 == 0, "16-byte aligned regions");
// the MMA operands stay inside their regions: block rows x 16 + 15 + 2 and block cols x 8 + 7 + 2
static_assert(2 * 16 + 15 + 2 < kF1R && 2 * 8 + 7 + 2 < kF1C && 16 + 15 + 2 < kF3R && 8 + 7 + 2 < kF3C, "operands in bounds");

struct FusedIO {
    const int32_t *xsum;                 // [n][mh][mw] block sums
    const __nv_bfloat16 *w1;             // [16][9]
    const __nv_bfloat16 *wt[3];          // layers 2-4: [COUT][9 CIN]
    const float *bias[4];
    const __nv_bfloat16 *wh;             // [16]
    const float *bh;                     // [1]
    float *z;                            // [n][mh][mw]
    int n, mh, mw, tiles_r, tiles_c, heat;
    const FrameState *fs;                // road rows only (null: every tile)
};

// weights of one layer -> the B layout of k_conv_tc (per K step kk: K halves COUT x 16 B apart, groups of 8
// output channels 128 B apart)
template <int CIN, int COUT>
__device__ __forceinline__ void fused_load_w(const __nv_bfloat16 *wt, unsigned char *wsm)
{
    for (int i = threadIdx.x; i < COUT * 9 * (CIN / 8); i += kFusedThreads) {
        const int n = i / (9 * CIN / 8), rem = i % (9 * CIN / 8), tap = rem / (CIN / 8), c8 = rem % (CIN / 8);
        const int kk = tap * (CIN / 16) + (c8 >> 1), h = c8 & 1;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(wt + (size_t)n * 9 * CIN + tap * CIN + c8 * 8));
        *reinterpret_cast<uint4 *>(wsm + kk * COUT * 32 + h * COUT * 16 + (n >> 3) * 128 + (n & 7) * 16) = v;
    }
}

// One thread issues the MMAs of a layer: NBR x NBC blocks of 16 x 8 output cells over an input region of
// RC cells per row (planes of PB bytes), accumulator of block b at column b * COUT.
template <int CIN, int COUT, int NBR, int NBC, int RC, int PB>
__device__ __forceinline__ void fused_mma(uint32_t in_base, uint32_t w_base, uint32_t tbase)
{
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COUT >> 3) << 17) | ((128u >> 4) << 24);
#pragma unroll 1
    for (int b = 0; b < NBR * NBC; ++b) {
        const int by = b / NBC, bx = b % NBC;
        const uint32_t dacc = tbase + (uint32_t)(b * COUT);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
#pragma unroll
            for (int c16 = 0; c16 < CIN / 16; ++c16) {
                const int kk = tap * (CIN / 16) + c16;
                const uint32_t cell = (uint32_t)((by * 16 + tap / 3) * RC + bx * 8 + tap % 3);
                const uint64_t ad = tc_desc(in_base + (uint32_t)(2 * c16 * PB) + cell * 16u, PB, RC * 16);
                const uint64_t bd = tc_desc(w_base + (uint32_t)(kk * COUT * 32), COUT * 16, 128);
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(dacc), "l"(ad), "l"(bd), "r"(kIdesc), "r"(kk));
            }
    }
}

// Epilogue of layer 2 or 3: bias + ReLU -> bf16 into the next layer's input region (ORR x ORC cells,
// planes of PB bytes) whose origin is (oy, ox) in the map; zero outside the map.
template <int NBR, int NBC, int ORR, int ORC, int PB>
__device__ __forceinline__ void fused_epi32(uint32_t tbase, const float *bias, unsigned char *out, int oy, int ox,
                                            int mh, int mw)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
#pragma unroll 1
    for (int b = 0; b < NBR * NBC; ++b) {
        const int Y = (b / NBC) * 16 + q * 4 + (lane >> 3), X = (b % NBC) * 8 + (lane & 7);
        uint32_t r[16];
        tc_load<16>(tbase + (uint32_t)(b * 32 + 16 * h) + ((uint32_t)(q * 32) << 16), r);
        if (Y < ORR && X < ORC) {
            const int y = oy + Y, x = ox + X;
            const bool in = y >= 0 && y < mh && x >= 0 && x < mw;
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                uint32_t o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = 16 * h + 8 * pl + 2 * k;
                    const float v0 = fmaxf(__fadd_rn(__uint_as_float(r[8 * pl + 2 * k]), bias[c]), 0.0f);
                    const float v1 = fmaxf(__fadd_rn(__uint_as_float(r[8 * pl + 2 * k + 1]), bias[c + 1]), 0.0f);
                    o[k] = in ? pack2(v0, v1) : 0u;
                }
                *reinterpret_cast<uint4 *>(out + (2 * h + pl) * PB + (Y * ORC + X) * 16) = make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

// wait for the layer's MMAs (bounded; false on a timeout)
__device__ __forceinline__ bool fused_wait(uint32_t mbar, uint32_t &phase)
{
    const bool ok = tc_wait(mbar, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return ok;
}

__device__ __forceinline__ void fused_sync_for_mma()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor-core reads
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_net_fused(const FusedIO io, int *err)
{
    extern __shared__ __align__(1024) unsigned char fsm[];
    __shared__ uint32_t taddr_s;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ float w1s[16 * 9], b1s[16], b2s[32], b3s[32], b4s[16], hws[16];
    __shared__ int fail_s;
    unsigned char *bufA = fsm, *bufB = fsm + kFBufA;
    unsigned char *w2 = bufB + kFBufB, *w3 = w2 + kFW2, *w4 = w3 + kFW3;
    int32_t *xbuf[2] = {reinterpret_cast<int32_t *>(w4 + kFW4), reinterpret_cast<int32_t *>(w4 + kFW4 + kFX)};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mh = io.mh, mw = io.mw;
    fused_load_w<16, 32>(io.wt[0], w2);
    fused_load_w<32, 32>(io.wt[1], w3);
    fused_load_w<32, 16>(io.wt[2], w4);
    for (int i = tid; i < 16 * 9; i += kFusedThreads)
        w1s[i] = __bfloat162float(io.w1[i]);
    if (tid < 16) {
        b1s[tid] = io.bias[0][tid];
        b4s[tid] = io.bias[3][tid];
        hws[tid] = __bfloat162float(io.wh[tid]);
    }
    if (tid < 32) {
        b2s[tid] = io.bias[1][tid];
        b3s[tid] = io.bias[2][tid];
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (tid == 0) {
        fail_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&taddr_s);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(dst));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fused_sync_for_mma();   // weights (generic stores) visible to the tensor cores, tensor memory allocated
    const uint32_t tbase = taddr_s;
    const uint32_t aA = (uint32_t)__cvta_generic_to_shared(bufA), aB = (uint32_t)__cvta_generic_to_shared(bufB);
    const uint32_t aw2 = (uint32_t)__cvta_generic_to_shared(w2), aw3 = (uint32_t)__cvta_generic_to_shared(w3),
                   aw4 = (uint32_t)__cvta_generic_to_shared(w4);
    const float bh = io.bh[0];
    uint32_t phase = 0u;
    const int per_frame = io.tiles_r * io.tiles_c, total = io.n * per_frame;
    // the tiles this CTA owns that reach a road row: blockIdx.x, + gridDim.x, ...
    auto next_tile = [&](int t) {
        for (; t < total; t += gridDim.x) {
            const int f = t / per_frame, rem = t % per_frame;
            if ((rem / io.tiles_c) * kFR + kFR - 1 >= first_needed_row(io.fs, f, 0))
                return t;
        }
        return total;
    };
    // the raw block sums of tile t's input region (origin y0 - 4, x0 - 4) into buf by cp.async, zero
    // outside the map
    auto load_x = [&](int t, int32_t *buf) {
        const int f = t / per_frame, rem = t % per_frame;
        const int y0 = (rem / io.tiles_c) * kFR, x0 = (rem % io.tiles_c) * kFC;
        const int32_t *xf = io.xsum + (size_t)f * mh * mw;
        for (int i = tid; i < kFXR * kFXC; i += kFusedThreads) {
            const int y = y0 - 4 + i / kFXC, x = x0 - 4 + i % kFXC;
            const bool in = y >= 0 && y < mh && x >= 0 && x < mw;
            const int32_t *src = xf + (size_t)(in ? y : 0) * mw + (in ? x : 0);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(buf + i)),
                         "l"(src), "r"(in ? 4 : 0) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int t = next_tile(blockIdx.x), it = 0;
    if (t < total)
        load_x(t, xbuf[0]);
    for (; t < total; ++it) {
        const int f = t / per_frame, rem = t % per_frame;
        const int y0 = (rem / io.tiles_c) * kFR, x0 = (rem % io.tiles_c) * kFC;
        const int32_t *xs = xbuf[it & 1];
        const int tn = next_tile(t + gridDim.x);
        asm volatile("cp.async.wait_group 0;" ::: "memory");   // this tile's input
        __syncthreads();
        if (tn < total)
            load_x(tn, xbuf[(it + 1) & 1]);   // the next tile's input arrives during this tile
        // layer 1 on the CUDA cores (origin y0 - 3, x0 - 3): the per-layer kernel's FMA order
        for (int i = tid; i < kF1R * kF1C; i += kFusedThreads) {
            const int Y = i / kF1C, X = i % kF1C, y = y0 - 3 + Y, x = x0 - 3 + X;
            float in[9];
#pragma unroll
            for (int tp = 0; tp < 9; ++tp)
                in[tp] = cell_input(xs[(Y + tp / 3) * kFXC + X + tp % 3]);
            const bool inmap = y >= 0 && y < mh && x >= 0 && x < mw;
            uint32_t o[8];
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                float s0 = b1s[c], s1 = b1s[c + 1];
#pragma unroll
                for (int tp = 0; tp < 9; ++tp) {
                    s0 = __fmaf_rn(w1s[c * 9 + tp], in[tp], s0);
                    s1 = __fmaf_rn(w1s[(c + 1) * 9 + tp], in[tp], s1);
                }
                o[c >> 1] = inmap ? pack2(fmaxf(s0, 0.0f), fmaxf(s1, 0.0f)) : 0u;
            }
            *reinterpret_cast<uint4 *>(bufA + i * 16) = make_uint4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<uint4 *>(bufA + kFP1 + i * 16) = make_uint4(o[4], o[5], o[6], o[7]);
        }
        fused_sync_for_mma();
        // layer 2: 3 x 3 blocks over the layer-1 region -> layer-2 region (origin y0 - 2, x0 - 2)
        if (tid == 0) {
            fused_mma<16, 32, 3, 3, kF1C, kFP1>(aA, aw2, tbase);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
        }
        if (!fused_wait(mb, phase))
            atomicExch(&fail_s, 1);
        __syncthreads();
        if (fail_s)
            break;
        fused_epi32<3, 3, kF2R, kF2C, kFP2>(tbase, b2s, bufB, y0 - 2, x0 - 2, mh, mw);
        fused_sync_for_mma();
        // layer 3 -> layer-3 region (origin y0 - 1, x0 - 1), into the buffer layer 1 used
        if (tid == 0) {
            fused_mma<32, 32, 3, 3, kF2C, kFP2>(aB, aw3, tbase);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
        }
        if (!fused_wait(mb, phase))
            atomicExch(&fail_s, 1);
        __syncthreads();
        if (fail_s)
            break;
        fused_epi32<3, 3, kF3R, kF3C, kFP3>(tbase, b3s, bufA, y0 - 1, x0 - 1, mh, mw);
        fused_sync_for_mma();
        // layer 4: 2 x 2 blocks -> bias + ReLU, the 1x1 head, the logit or the heatmap
        if (tid == 0) {
            fused_mma<32, 16, 2, 2, kF3C, kFP3>(aA, aw4, tbase);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
        }
        if (!fused_wait(mb, phase))
            atomicExch(&fail_s, 1);
        __syncthreads();
        if (fail_s)
            break;
        {
            const int q = warp & 3;
#pragma unroll 1
            for (int b = (warp >> 2) * 2; b < (warp >> 2) * 2 + 2; ++b) {
                const int Y = (b >> 1) * 16 + q * 4 + (lane >> 3), X = (b & 1) * 8 + (lane & 7);
                uint32_t r[16];
                tc_load<16>(tbase + (uint32_t)(b * 16) + ((uint32_t)(q * 32) << 16), r);
                const int y = y0 + Y, x = x0 + X;
                if (y < mh && x < mw) {
                    float zc = 0.0f;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int c = 2 * k;
                        const float v0 = fmaxf(__fadd_rn(__uint_as_float(r[c]), b4s[c]), 0.0f);
                        const float v1 = fmaxf(__fadd_rn(__uint_as_float(r[c + 1]), b4s[c + 1]), 0.0f);
                        const uint32_t o = pack2(v0, v1);
                        zc = __fmaf_rn(hws[c + 1], bf_hi(o), __fmaf_rn(hws[c], bf_lo(o), zc));
                    }
                    zc = __fadd_rn(zc, bh);
                    io.z[((size_t)f * mh + y) * mw + x] = io.heat ? __frcp_rn(__fadd_rn(1.0f, expf(-zc))) : zc;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();   // the next tile overwrites both buffers and the accumulators
        asm volatile("tcgen05.fence::after_thread_sync;");
        t = tn;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (tid == 0 && fail_s)
        atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

// ---------------------------------------------------------------------------------------------------
// weight gradients: dW[co][tap][ci] = sum_cells dS[co] A[cell + (tap)][ci]; column 9 CIN holds the bias
// ---------------------------------------------------------------------------------------------------
struct WgradIO {
    const __nv_bfloat16 *dS;     // [n][mh][mw][COUT]
    const __nv_bfloat16 *A;      // [n][mh][mw][CIN]
    float *part;                 // [gridDim.x][COUT][9 CIN + 1]
    int n, mh, mw, tiles_r, tiles_c;
};

template <int CIN, int COUT>
struct WgradShape {
    static constexpr int NCOL = 9 * CIN + 1;
    static constexpr int NTT = (NCOL + 7) / 8;          // n8 tiles
    static constexpr int NPW = (NTT + 3) / 4;           // per warp
    static constexpr int MT = COUT / 16;
    static constexpr int CINP = CIN == 1 ? 2 : CIN + 8; // halo cell stride (elements)
    static constexpr int PXP = kTileR * kTileC + 8;     // dS^T row stride (elements)
    static constexpr size_t bytes = sizeof(__nv_bfloat16) * (size_t)(kHaloR * kHaloC * CINP + COUT * PXP);
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_wgrad(const WgradIO io)
{
    using S = WgradShape<CIN, COUT>;
    extern __shared__ __align__(16) __nv_bfloat16 gsm[];
    __nv_bfloat16 *sA = gsm;                                   // [10 x 18][CINP]
    __nv_bfloat16 *sD = gsm + kHaloR * kHaloC * S::CINP;        // [COUT][PXP]: dS transposed
    const uint16_t *sA16 = reinterpret_cast<const uint16_t *>(sA);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int mh = io.mh, mw = io.mw;
    const int per_frame = io.tiles_r * io.tiles_c;
    const int total = io.n * per_frame;
    // this lane's B column in each of the warp's n-tiles: (tap, ci), the bias column, or nothing
    int coff[S::NPW];    // element offset of (dy, dx, ci) in the halo tile, -1 = zero column, -2 = ones
#pragma unroll
    for (int j = 0; j < S::NPW; ++j) {
        const int col = (warp * S::NPW + j) * 8 + g;
        if (col < 9 * CIN) {
            const int tap = col / CIN, ci = col % CIN;
            coff[j] = ((tap / 3) * kHaloC + tap % 3) * S::CINP + ci;
        } else {
            coff[j] = col == 9 * CIN ? -2 : -1;
        }
    }
    float acc[S::MT][S::NPW][4];
#pragma unroll
    for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
        for (int j = 0; j < S::NPW; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[mt][j][q] = 0.0f;
    const uint16_t one = 0x3f80;   // bf16 1.0
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int f = tile / per_frame, rem = tile % per_frame;
        const int y0 = (rem / io.tiles_c) * kTileR, x0 = (rem % io.tiles_c) * kTileC;
        __syncthreads();
        if constexpr (CIN == 1) {
            for (int i = tid; i < kHaloR * kHaloC; i += kConvThreads) {
                const int yy = y0 - 1 + i / kHaloC, xx = x0 - 1 + i % kHaloC;
                __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
                if (yy >= 0 && yy < mh && xx >= 0 && xx < mw)
                    v = io.A[((size_t)f * mh + yy) * mw + xx];
                sA[i * S::CINP] = v;
            }
        } else {
            for (int i = tid; i < kHaloR * kHaloC * (CIN / 8); i += kConvThreads) {
                const int cell = i / (CIN / 8), ch = i % (CIN / 8);
                const int yy = y0 - 1 + cell / kHaloC, xx = x0 - 1 + cell % kHaloC;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (yy >= 0 && yy < mh && xx >= 0 && xx < mw)
                    v = __ldg(reinterpret_cast<const uint4 *>(io.A + (((size_t)f * mh + yy) * mw + xx) * CIN) + ch);
                *reinterpret_cast<uint4 *>(sA + cell * S::CINP + ch * 8) = v;
            }
        }
        // dS of the tile's 128 cells, transposed to [co][cell]; cells outside the map are 0
        for (int i = tid; i < kTileR * kTileC * (COUT / 8); i += kConvThreads) {
            const int cell = i / (COUT / 8), ch = i % (COUT / 8);
            const int yy = y0 + cell / kTileC, xx = x0 + cell % kTileC;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (yy < mh && xx < mw)
                v = __ldg(reinterpret_cast<const uint4 *>(io.dS + (((size_t)f * mh + yy) * mw + xx) * COUT) + ch);
            const uint16_t *e = reinterpret_cast<const uint16_t *>(&v);
            uint16_t *col = reinterpret_cast<uint16_t *>(sD) + (ch * 8) * S::PXP + cell;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                col[k * S::PXP] = e[k];
        }
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < kTileR; ++r) {           // one k16 step per tile row (16 cells)
            uint32_t af[S::MT][4];
#pragma unroll
            for (int mt = 0; mt < S::MT; ++mt) {
                const __nv_bfloat16 *r0 = sD + (mt * 16 + g) * S::PXP + r * kTileC + 2 * t;
                const __nv_bfloat16 *r1 = r0 + 8 * S::PXP;
                af[mt][0] = *reinterpret_cast<const uint32_t *>(r0);
                af[mt][1] = *reinterpret_cast<const uint32_t *>(r1);
                af[mt][2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
                af[mt][3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
            }
            const int rowoff = r * kHaloC * S::CINP;
#pragma unroll
            for (int j = 0; j < S::NPW; ++j) {
                if ((warp * S::NPW + j) * 8 >= S::NCOL)
                    break;
                uint32_t b0, b1;
                if (coff[j] >= 0) {
                    const uint16_t *p = sA16 + rowoff + coff[j] + (2 * t) * S::CINP;
                    b0 = pack_raw(p[0], p[S::CINP]);
                    b1 = pack_raw(p[8 * S::CINP], p[9 * S::CINP]);
                } else {
                    b0 = coff[j] == -2 ? pack_raw(one, one) : 0u;
                    b1 = b0;
                }
#pragma unroll
                for (int mt = 0; mt < S::MT; ++mt)
                    mma16816(acc[mt][j], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
            }
        }
    }
    float *part = io.part + (size_t)blockIdx.x * COUT * S::NCOL;
#pragma unroll
    for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
        for (int j = 0; j < S::NPW; ++j) {
            const int c0 = (warp * S::NPW + j) * 8 + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int co = mt * 16 + g + (q >> 1) * 8, col = c0 + (q & 1);
                if (col < S::NCOL)
                    part[co * S::NCOL + col] = acc[mt][j][q];
            }
        }
}

// Sum the per-CTA partials in CTA order and scatter into the flat gradient (layout [co][ci][3][3], b[co]).
__global__ void k_wreduce(const float *part, int nparts, int cin, int cout, float *grad_w, float *grad_b)
{
    const int ncol = 9 * cin + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cout * ncol)
        return;
    float s = 0.0f;
    for (int k = 0; k < nparts; ++k)
        s = __fadd_rn(s, part[(size_t)k * cout * ncol + i]);
    const int co = i / ncol, col = i % ncol;
    if (col == 9 * cin)
        grad_b[co] = s;
    else
        grad_w[(co * cin + col % cin) * 9 + col / cin] = s;
}

// ---------------------------------------------------------------------------------------------------
// head + loss: z, loss term, dz, dS_4 = bf16(w_h dz [A_4 > 0]); partials (loss, dw_h[16], db_h)
// ---------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kCellThreads) k_loss(const NetArgs a, const uint8_t *labels, int n, float inv_n,
                                                       float pw, float *part)
{
    __shared__ float red[kCellThreads / 32][18];
    const int mh = a.mh, mw = a.mw;
    const long long cells = (long long)n * mh * mw;
    float whv[16];
#pragma unroll
    for (int c = 0; c < 16; ++c)
        whv[c] = __bfloat162float(a.whb[c]);
    const float bh = a.bh[0];
    float acc[18];
#pragma unroll
    for (int k = 0; k < 18; ++k)
        acc[k] = 0.0f;
    for (long long p = blockIdx.x * (long long)kCellThreads + threadIdx.x; p < cells;
         p += (long long)gridDim.x * kCellThreads) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.act[3] + p * 16);
        const uint4 q0 = src[0], q1 = src[1];
        const uint32_t w32[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        float av[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            av[2 * k] = bf_lo(w32[k]);
            av[2 * k + 1] = bf_hi(w32[k]);
        }
        float z = 0.0f;
#pragma unroll
        for (int c = 0; c < 16; ++c)
            z = __fmaf_rn(whv[c], av[c], z);
        z = __fadd_rn(z, bh);
        const float y = labels[p] ? 1.0f : 0.0f;
        const float sp = 1.0f / (1.0f + expf(-z));          // sigmoid(z)
        const float sn = 1.0f / (1.0f + expf(z));           // sigmoid(-z)
        const float spz = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));     // softplus(z)
        const float spn = fmaxf(-z, 0.0f) + log1pf(expf(-fabsf(z)));    // softplus(-z)
        acc[0] += pw * y * spn + (1.0f - y) * spz;
        const float dz = ((1.0f - y) * sp - pw * y * sn) * inv_n;
        uint32_t o[8];
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
            const float d0 = av[c] > 0.0f ? whv[c] * dz : 0.0f;
            const float d1 = av[c + 1] > 0.0f ? whv[c + 1] * dz : 0.0f;
            o[c >> 1] = pack2(d0, d1);
            acc[1 + c] = __fmaf_rn(dz, av[c], acc[1 + c]);
            acc[2 + c] = __fmaf_rn(dz, av[c + 1], acc[2 + c]);
        }
        acc[17] += dz;
        uint4 *dst = reinterpret_cast<uint4 *>(a.dS[0] + p * 16);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
        float v = acc[k];
        for (int d = 16; d > 0; d >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, d);
        if (lane == 0)
            red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 18) {
        float v = 0.0f;
        for (int w = 0; w < kCellThreads / 32; ++w)
            v += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * 18 + threadIdx.x] = v;
    }
}

// loss and the head's gradient from the k_loss partials (fixed order)
__global__ void k_loss_reduce(const float *part, int nparts, float inv_n, float *grad_head, float *loss_out)
{
    const int k = threadIdx.x;
    if (k >= 18)
        return;
    float s = 0.0f;
    for (int i = 0; i < nparts; ++i)
        s = __fadd_rn(s, part[(size_t)i * 18 + k]);
    if (k == 0) {
        if (loss_out)
            *loss_out = s * inv_n;
    } else {
        grad_head[k - 1] = s;   // wh[0..15], then bh
    }
}

// ---------------------------------------------------------------------------------------------------
// parameters: Adam step and the bf16 operand copies
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ void store_operand(const NetArgs &a, int i, float v)
{
    // flat layout: per layer W[co][ci][3][3] then b[co]; then wh[16], bh
    int base = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int ci_n = net_ch(l), co_n = net_ch(l + 1);
        const int nw = co_n * ci_n * 9;
        if (i < base + nw) {
            const int r = i - base, co = r / (ci_n * 9), ci = (r / 9) % ci_n, tap = r % 9;
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            a.wf[l][(co * 9 + tap) * ci_n + ci] = b;
            if (l > 0)
                a.wb[l][(ci * 9 + (8 - tap)) * co_n + co] = b;
            return;
        }
        base += nw + co_n;
        if (i < base)
            return;   // bias: read from the master copy
    }
    if (i < base + 16)
        a.whb[i - base] = __float2bfloat16_rn(v);
}

__global__ void k_pack(const NetArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNetParams)
        store_operand(a, i, a.theta[i]);
}

__global__ void k_adam(const NetArgs a, const float *grad, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNetParams)
        return;
    const float gi = grad[i];
    const float m = b1 * a.m[i] + (1.0f - b1) * gi;
    const float v = b2 * a.v[i] + (1.0f - b2) * gi * gi;
    a.m[i] = m;
    a.v[i] = v;
    const float th = a.theta[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);   // c1 = 1 - b1^t, c2 = 1 - b2^t
    a.theta[i] = th;
    store_operand(a, i, th);
}

// ---------------------------------------------------------------------------------------------------
// labels, scores, top-k
// ---------------------------------------------------------------------------------------------------
// one thread per (frame, lane): the Eq. 25 track of the lane's start, row by row as in the energy kernel
__global__ void k_labels(const KParams kp, const Work w, const ld_lanes *lanes, uint8_t *labels, int mh, int mw)
{
    const int f = blockIdx.x, l = threadIdx.x;
    if (l >= LD_MAX_LANES)
        return;
    const ld_lanes &L = lanes[f];
    const FrameState &fs = w.fs[f];
    if (l >= L.n_lanes || (fs.flags & (LD_F_NO_ROAD | LD_F_DEGEN_Y | LD_F_DEGEN_X)))
        return;
    const int W = kp.W, H = kp.H, vtop = fs.v_top;
    const float *Vpy = w.rows + (size_t)f * 3 * H + H;
    const float *Vpx = Vpy + H;
    uint8_t *Y = labels + (size_t)f * mh * mw;
    float u = (float)L.start_u[l];
    for (int v = H - 1; v >= vtop; --v) {
        if (v < H - 1) {
            const float vx = Vpx[v + 1], vy = Vpy[v + 1];
            const float num = __fsub_rn(__fadd_rn(vx, __fmul_rn((float)v, u)), __fmul_rn(vy, u));
            const float den = __fsub_rn((float)(v + 1), vy);
            u = __fdiv_rn(num, den);
        }
        const float c = floorf(__fadd_rn(u, 0.5f));
        if (c >= 0.0f && c < (float)W)
            Y[(v >> 2) * mw + ((int)c >> 2)] = 1;
    }
}

// one thread per (frame, coarse start c): the heatmap summed along the track in steps of four rows
__global__ void __launch_bounds__(128) k_score(const KParams kp, const Work w, const float *z, float *scores,
                                               int mh, int mw)
{
    const int f = blockIdx.y, c = blockIdx.x * 128 + threadIdx.x;
    const int nc = (kp.n_starts + 3) >> 2;
    if (c >= nc)
        return;
    const FrameState &fs = w.fs[f];
    float acc = 0.0f;
    if (!(fs.flags & LD_F_NO_LANES)) {
        const int W = kp.W, H = kp.H;
        const float *Vpy = w.rows + (size_t)f * 3 * H + H;
        const float *Vpx = Vpy + H;
        const float *zf = z + (size_t)f * mh * mw;
        float u = __fadd_rn((float)(4 * c - kp.S0), 1.5f);
        for (int v = H - 1; v >= fs.v_top; v -= 4) {
            const float col = floorf(__fadd_rn(u, 0.5f));
            if (col >= 0.0f && col < (float)W)
                acc = __fadd_rn(acc, __ldg(zf + (v >> 2) * mw + ((int)col >> 2)));
            const float step = __fdiv_rn(__fmul_rn(4.0f, __fsub_rn(Vpx[v], u)), __fsub_rn((float)v, Vpy[v]));
            u = __fadd_rn(u, step);
        }
    }
    scores[(size_t)f * nc + c] = acc;
}

// one CTA per frame: the top_k coarse scores (ties to the smaller index), flags of candidate (bit 0) and
// evaluated (bit 1) starts, and the ascending list of evaluated starts
constexpr int kTopThreads = 256;

// order-preserving integer key of a float score (-0 taken as +0, so equal scores give equal keys)
__device__ __forceinline__ uint32_t order_key(float s)
{
    const uint32_t u = __float_as_uint(s == 0.0f ? 0.0f : s);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// sum of v over the CTA (every thread gets it); red holds kTopThreads / 32 ints
__device__ __forceinline__ int cta_sum(int v, int *red)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, d);
    __syncthreads();   // earlier readers of red are done
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = 0;
#pragma unroll
    for (int k = 0; k < kTopThreads / 32; ++k)
        s += red[k];
    return s;
}

// sum of v over the threads before this one
__device__ __forceinline__ int cta_exclusive(int v, int *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d)
            x += y;
    }
    __syncthreads();
    if (lane == 31)
        red[warp] = x;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < warp; ++k)
        before += red[k];
    return before + x - v;
}

__global__ void __launch_bounds__(kTopThreads) k_topk(const KParams kp, const Work w, const float *scores, int top_k,
                                                      uint8_t *cflag, int32_t *elist, int32_t *ecnt, int ecap)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    const int f = blockIdx.x, ns = kp.n_starts, nc = (ns + 3) >> 2;
    uint32_t *key = reinterpret_cast<uint32_t *>(tsm);        // [nc]
    uint8_t *fl = tsm + sizeof(uint32_t) * ((nc + 3) & ~3);   // [ns]
    __shared__ int wsum[kTopThreads / 32];
    __shared__ int red[kTopThreads / 32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool skip = w.fs[f].flags & LD_F_NO_LANES;
    for (int i = tid; i < nc; i += kTopThreads)
        key[i] = order_key(scores[(size_t)f * nc + i]);
    for (int i = tid; i < ns; i += kTopThreads)
        fl[i] = 0;
    if (tid == 0)
        base = 0;
    __syncthreads();
    if (!skip) {
        // T = the k-th largest key, bit by bit from the top: the largest T with #(key >= T) >= k
        const int k = top_k < nc ? top_k : nc;
        const int per = (nc + kTopThreads - 1) / kTopThreads;   // contiguous chunks keep index order
        const int c0 = tid * per < nc ? tid * per : nc, c1 = c0 + per < nc ? c0 + per : nc;
        uint32_t T = 0;
        for (int bit = 31; bit >= 0; --bit) {
            const uint32_t cand = T | (1u << bit);
            int cnt = 0;
            for (int c = c0; c < c1; ++c)
                cnt += key[c] >= cand;
            if (cta_sum(cnt, red) >= k)
                T = cand;
        }
        // every key above T is chosen; of the keys equal to T, the first k - #(key > T) in index order
        int gt = 0, eq = 0;
        for (int c = c0; c < c1; ++c) {
            gt += key[c] > T;
            eq += key[c] == T;
        }
        const int need = k - cta_sum(gt, red);
        int r = cta_exclusive(eq, red);
        for (int c = c0; c < c1; ++c) {
            bool sel = key[c] > T;
            if (key[c] == T)
                sel = r++ < need;
            if (sel)
                for (int q = 0; q < 4; ++q)
                    if (4 * c + q < ns)
                        fl[4 * c + q] = 1;
        }
    }
    __syncthreads();
    // evaluated = candidate or next to one; per chunk a read phase, then the writes and an ordered compaction
    for (int i0 = 0; i0 < ns; i0 += kTopThreads) {
        const int i = i0 + tid;
        bool ev = false;
        if (i < ns)
            ev = (fl[i] & 1) || (i > 0 && (fl[i - 1] & 1)) || (i + 1 < ns && (fl[i + 1] & 1));
        __syncthreads();
        if (i < ns && ev)
            fl[i] |= 2;
        // ordered compaction of this chunk
        const unsigned bal = __ballot_sync(0xffffffffu, ev);
        if (lane == 0)
            wsum[warp] = __popc(bal);
        __syncthreads();
        int off = base;
        for (int k = 0; k < warp; ++k)
            off += wsum[k];
        off += __popc(bal & ((1u << lane) - 1u));
        if (ev && off < ecap)
            elist[(size_t)f * ecap + off] = i;
        __syncthreads();
        if (tid == 0) {
            int s = 0;
            for (int k = 0; k < kTopThreads / 32; ++k)
                s += wsum[k];
            base += s;
        }
        __syncthreads();
    }
    for (int i = tid; i < ns; i += kTopThreads)
        cflag[(size_t)f * ns + i] = fl[i];
    if (tid == 0)
        ecnt[f] = base < ecap ? base : ecap;
}

}  // namespace

// ---------------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------------
// Every kernel here stays under the default 48 KB of dynamic shared memory (k_topk: 2 bytes per start,
// at most 25 KB for the widest frame), so no opt-in is needed.

static int grid_for(int tiles, int per_sm)
{
    const int g = sm_count() * per_sm;
    return tiles < g ? tiles : g;
}

__device__ int g_tc_error;   // set when a tensor-core wait ran out (read and cleared by net_tc_status)

template <int CIN, int COUT, int EPI>
static cudaError_t conv(ConvIO io, cudaStream_t s)
{
    using S = TcSmem<CIN, COUT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)S::bytes);
        if (e != cudaSuccess)
            return e;
        attr = true;
    }
    io.tiles_r = (io.mh + kTcRows - 1) / kTcRows;
    io.tiles_c = (io.mw + kTcCols - 1) / kTcCols;
    int *err = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_tc_error);
    if (e != cudaSuccess)
        return e;
    const int tiles = io.n * io.tiles_r * io.tiles_c;
    k_conv_tc<CIN, COUT, EPI><<<grid_for(tiles, 4), kConvThreads, S::bytes, s>>>(io, err);
    return cudaGetLastError();
}

static cudaError_t net_forward_fused(const NetArgs &a, const int32_t *xsum, int n, float *z, bool heat, cudaStream_t s,
                                     const FrameState *road)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_net_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
        if (e != cudaSuccess)
            return e;
        attr = true;
    }
    FusedIO io{};
    io.xsum = xsum;
    io.w1 = a.wf[0];
    for (int l = 0; l < 3; ++l)
        io.wt[l] = a.wf[l + 1];
    for (int l = 0; l < 4; ++l)
        io.bias[l] = a.bias[l];
    io.wh = a.whb;
    io.bh = a.bh;
    io.z = z;
    io.n = n;
    io.mh = a.mh;
    io.mw = a.mw;
    io.tiles_r = (a.mh + kFR - 1) / kFR;
    io.tiles_c = (a.mw + kFC - 1) / kFC;
    io.heat = heat ? 1 : 0;
    io.fs = road;
    int *err = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_tc_error);
    if (e != cudaSuccess)
        return e;
    k_net_fused<<<grid_for(n * io.tiles_r * io.tiles_c, 1), kFusedThreads, kFusedSmem, s>>>(io, err);
    return cudaGetLastError();
}

cudaError_t net_forward(const NetArgs &a, const int32_t *xsum, int n, float *z, bool keep_a4, bool heat,
                        cudaStream_t s, const FrameState *road)
{
    if (!keep_a4 && a.fused)   // inference in one kernel, the activations never leave the SM
        return net_forward_fused(a, xsum, n, z, heat, s, road);
    const long long cells = (long long)n * a.mh * a.mw;
    const int g1 = (int)((cells + kCellThreads - 1) / kCellThreads);
    k_conv1<<<grid_for(g1, 8), kCellThreads, 0, s>>>(a, xsum, n, road);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    ConvIO io{};
    io.n = n;
    io.mh = a.mh;
    io.mw = a.mw;
    io.tiles_r = (a.mh + kTileR - 1) / kTileR;
    io.tiles_c = (a.mw + kTileC - 1) / kTileC;
    io.fs = road;
    io.in = a.act[0];
    io.wt = a.wf[1];
    io.bias = a.bias[1];
    io.out = a.act[1];
    io.depth = 2;
    if ((e = conv<16, 32, kEpiRelu>(io, s)) != cudaSuccess)
        return e;
    io.in = a.act[1];
    io.wt = a.wf[2];
    io.bias = a.bias[2];
    io.out = a.act[2];
    io.depth = 1;
    if ((e = conv<32, 32, kEpiRelu>(io, s)) != cudaSuccess)
        return e;
    io.depth = 0;
    io.in = a.act[2];
    io.wt = a.wf[3];
    io.bias = a.bias[3];
    io.out = keep_a4 ? a.act[3] : nullptr;
    io.wh = a.whb;
    io.bh = a.bh;
    io.z = z;
    io.heat = heat ? 1 : 0;
    return conv<32, 16, kEpiHead>(io, s);
}

template <int CIN, int COUT>
static cudaError_t wgrad(const NetArgs &a, const __nv_bfloat16 *dS, const __nv_bfloat16 *A, int n, float *gw,
                         float *gb, cudaStream_t s)
{
    WgradIO io{};
    io.dS = dS;
    io.A = A;
    io.part = a.part;
    io.n = n;
    io.mh = a.mh;
    io.mw = a.mw;
    io.tiles_r = (a.mh + kTileR - 1) / kTileR;
    io.tiles_c = (a.mw + kTileC - 1) / kTileC;
    const int G = grid_for(n * io.tiles_r * io.tiles_c, kWgradCtasPerSm);
    k_wgrad<CIN, COUT><<<G, kConvThreads, WgradShape<CIN, COUT>::bytes, s>>>(io);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const int outs = COUT * (9 * CIN + 1);
    k_wreduce<<<(outs + 255) / 256, 256, 0, s>>>(a.part, G, CIN, COUT, gw, gb);
    return cudaGetLastError();
}

cudaError_t net_backward(const NetArgs &a, const uint8_t *labels, int n, float pw, float *grad, float *loss,
                         cudaStream_t s)
{
    const long long cells = (long long)n * a.mh * a.mw;
    const float inv_n = 1.0f / (float)cells;
    const int gl = (int)((cells + kCellThreads - 1) / kCellThreads);
    const int GL = grid_for(gl, 4);
    k_loss<<<GL, kCellThreads, 0, s>>>(a, labels, n, inv_n, pw, a.part_head);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    k_loss_reduce<<<1, 32, 0, s>>>(a.part_head, GL, inv_n, grad + kNetParams - 17, loss);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // parameter offsets
    int off[4], cur = 0;
    for (int l = 0; l < 4; ++l) {
        off[l] = cur;
        cur += net_ch(l + 1) * net_ch(l) * 9 + net_ch(l + 1);
    }
    auto gw = [&](int l) { return grad + off[l]; };
    auto gb = [&](int l) { return grad + off[l] + net_ch(l + 1) * net_ch(l) * 9; };
    ConvIO io{};
    io.n = n;
    io.mh = a.mh;
    io.mw = a.mw;
    io.tiles_r = (a.mh + kTileR - 1) / kTileR;
    io.tiles_c = (a.mw + kTileC - 1) / kTileC;
    // layer 4: dS_4 in dS[0] (16 channels), A_3 (32)
    if ((e = wgrad<32, 16>(a, a.dS[0], a.act[2], n, gw(3), gb(3), s)) != cudaSuccess)
        return e;
    io.in = a.dS[0];
    io.wt = a.wb[3];
    io.mask = a.act[2];
    io.out = a.dS[1];
    if ((e = conv<16, 32, kEpiMask>(io, s)) != cudaSuccess)    // dS_3 (32)
        return e;
    if ((e = wgrad<32, 32>(a, a.dS[1], a.act[1], n, gw(2), gb(2), s)) != cudaSuccess)
        return e;
    io.in = a.dS[1];
    io.wt = a.wb[2];
    io.mask = a.act[1];
    io.out = a.dS[0];
    if ((e = conv<32, 32, kEpiMask>(io, s)) != cudaSuccess)    // dS_2 (32)
        return e;
    if ((e = wgrad<16, 32>(a, a.dS[0], a.act[0], n, gw(1), gb(1), s)) != cudaSuccess)
        return e;
    io.in = a.dS[0];
    io.wt = a.wb[1];
    io.mask = a.act[0];
    io.out = a.dS[1];
    if ((e = conv<32, 16, kEpiMask>(io, s)) != cudaSuccess)    // dS_1 (16)
        return e;
    return wgrad<1, 16>(a, a.dS[1], a.X, n, gw(0), gb(0), s);
}

int net_tc_status()
{
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess)
        return -1;
    if (v)
        cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    return v;
}

cudaError_t net_pack(const NetArgs &a, cudaStream_t s)
{
    k_pack<<<(kNetParams + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t net_adam(const NetArgs &a, const float *grad, float lr, float b1, float b2, float eps, float c1, float c2,
                     cudaStream_t s)
{
    k_adam<<<(kNetParams + 255) / 256, 256, 0, s>>>(a, grad, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t net_labels(const KParams &kp, const Work &w, const ld_lanes *lanes, uint8_t *labels, int mh, int mw,
                       cudaStream_t s)
{
    k_labels<<<kp.n_frames, 32, 0, s>>>(kp, w, lanes, labels, mh, mw);
    return cudaGetLastError();
}

cudaError_t net_propose(const KParams &kp, const Work &w, const float *z, int mh, int mw, int top_k, float *scores,
                        uint8_t *cflag, int32_t *elist, int32_t *ecnt, int ecap, cudaStream_t s)
{
    const int nc = (kp.n_starts + 3) >> 2;
    dim3 g1((nc + 127) / 128, kp.n_frames);
    k_score<<<g1, 128, 0, s>>>(kp, w, z, scores, mh, mw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const size_t smem = sizeof(float) * (size_t)((nc + 3) & ~3) + (size_t)kp.n_starts;
    k_topk<<<kp.n_frames, kTopThreads, smem, s>>>(kp, w, scores, top_k, cflag, elist, ecnt, ecap);
    return cudaGetLastError();
}

}  // namespace ld
