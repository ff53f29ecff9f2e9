// Dynamic programming over the two accumulators, one CTA per frame:
//
//   k_road_dp  Sec. 2.2, Eq. 11-12: from d = D-1 down to d = 1,
//              E_d(v) = -m_y(d, v) + min_{tau in [0, tau_y], v + tau <= H-1} [E_{d+1}(v + tau) + lambda_y tau],
//              backtrack buffer the size of the map (4-bit entries), path M_y = {(d, v_d)}.
//   k_vpx_dp   Sec. 2.3.2-2.3.3: the dense accumulator m_x (Alg. 5) as a sliding band of vote rows, and
//              Eq. 18 from row H-1 up to v_top,
//              E_v(u) = m_x(u, v) + min_{tau in [-tau_x, tau_x], 0 <= u + tau < W} [E_{v+1}(u + tau) + lambda_x |tau|],
//              path M_x = {(v, u_v)}.
//
// Readings: Eq. 12 as printed draws on E(v - tau)_{d+1} with -lambda tau; with rows counted from the top and
// road disparity growing downwards, the consistent form links (d, v) to (d+1, v + tau) with a +lambda tau
// penalty.  Eq. 18's "+lambda_x tau" is read as lambda_x |tau|.  Ties take the smaller |tau|, then the
// negative one; a path starts at the smallest index minimising its last row.  Alg. 5 is read from the text
// around it: m_x(u, j) = -varrho * (votes in column u of rows [j - chi, j + chi] within [v_top, H-1]).
// A path point whose cell holds no count carries no observation; the kernels hand the points with data to
// the RANSAC fit (k_fit), in increasing index order.
//
// Each DP step is one row of the map; threads own pairs of adjacent cells (one byte of 4-bit backtrack
// entries each).  Rows are padded with sentinels so the candidate loops have no bounds checks.  The
// V_px DP keeps as many backtrack rows in shared memory as fit; taller road areas are processed in
// segments, with the DP state checkpointed at segment boundaries and recomputed during the backtrack.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kRoadThreads = 512;
constexpr int kVpxThreads = 1024;
constexpr int kMaxChunks = (LD_MAX_H + 31) / 32 + 2;
constexpr int kSent = 0x3fffffff;  // larger than any DP energy (checked when the handle is created)
constexpr int kPadY = 16;          // > tau_y
constexpr int kPadX = 8;           // > tau_x

template <typename T>
__device__ __forceinline__ T *carve(unsigned char *&p, size_t count)
{
    const size_t off = ((size_t)p + 15) & ~(size_t)15;
    T *r = reinterpret_cast<T *>(off);
    p = reinterpret_cast<unsigned char *>(off + sizeof(T) * count);
    return r;
}

// Lexicographic (value, index) minimum over the block; every thread receives the index.
template <int NT>
__device__ int block_argmin(int val, int idx, int *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 16; d > 0; d >>= 1) {
        const int ov = __shfl_down_sync(0xffffffffu, val, d);
        const int oi = __shfl_down_sync(0xffffffffu, idx, d);
        if (ov < val || (ov == val && oi < idx)) {
            val = ov;
            idx = oi;
        }
    }
    if (lane == 0) {
        scratch[2 * warp] = val;
        scratch[2 * warp + 1] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int bv = scratch[0], bi = scratch[1];
        for (int w = 1; w < NT / 32; ++w)
            if (scratch[2 * w] < bv || (scratch[2 * w] == bv && scratch[2 * w + 1] < bi)) {
                bv = scratch[2 * w];
                bi = scratch[2 * w + 1];
            }
        scratch[0] = bi;
    }
    __syncthreads();
    const int r = scratch[0];
    __syncthreads();
    return r;
}

// Ascending list of j < n with flag[j]; returns the count.  chunk: >= n/32 + 2 ints.
template <int NT>
__device__ int block_compact(const uint8_t *flag, int n, int16_t *list, int *chunk)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nch = (n + 31) >> 5;
    for (int c = warp; c < nch; c += NT / 32) {
        const int j = (c << 5) + lane;
        const unsigned m = __ballot_sync(0xffffffffu, j < n && flag[j]);
        if (lane == 0)
            chunk[c] = __popc(m);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int c = 0; c < nch; ++c) {
            const int t = chunk[c];
            chunk[c] = s;
            s += t;
        }
        chunk[nch] = s;
    }
    __syncthreads();
    for (int c = warp; c < nch; c += NT / 32) {
        const int j = (c << 5) + lane;
        const bool b = j < n && flag[j];
        const unsigned m = __ballot_sync(0xffffffffu, b);
        if (b)
            list[chunk[c] + __popc(m & ((1u << lane) - 1u))] = (int16_t)j;
    }
    __syncthreads();
    const int cnt = chunk[nch];
    __syncthreads();
    return cnt;
}

// ---------------------------------------------------------------------------------------------------
// k_road_dp
// ---------------------------------------------------------------------------------------------------
constexpr int kRoadPairs = (LD_MAX_H / 2 + kRoadThreads - 1) / kRoadThreads;  // pairs per thread (2)

__global__ void __launch_bounds__(kRoadThreads) k_road_dp(const KParams kp, const Work w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int f = blockIdx.x, H = kp.H, D = kp.D, Hp = (H + 1) >> 1;
    const int tid = threadIdx.x;
    const int32_t *my = w.myT + (size_t)f * D * H;

    unsigned char *p = smem;
    int *E0 = carve<int>(p, H + kPadY);
    int *E1 = carve<int>(p, H + kPadY);
    int *sh = carve<int>(p, kMaxChunks + 2 * (kRoadThreads / 32));
    int16_t *path = carve<int16_t>(p, D);
    uint8_t *flag = carve<uint8_t>(p, D);
    int16_t *pid = carve<int16_t>(p, D);
    uint8_t *bt = carve<uint8_t>(p, (size_t)D * Hp);

    for (int v = tid; v < H + kPadY; v += kRoadThreads) {
        E0[v] = v < H ? -my[(size_t)(D - 1) * H + v] : kSent;
        E1[v] = kSent;
    }
    // data terms of the next two steps are loaded a step ahead of their use
    int cur[kRoadPairs][2], nxt[kRoadPairs][2];
#pragma unroll
    for (int q = 0; q < kRoadPairs; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int v = 2 * (tid + q * kRoadThreads) + h;
            cur[q][h] = (D - 2 >= 1 && v < H) ? my[(size_t)(D - 2) * H + v] : 0;
            nxt[q][h] = (D - 3 >= 1 && v < H) ? my[(size_t)(D - 3) * H + v] : 0;
        }
    __syncthreads();
    int *Ep = E0, *Ec = E1;
    const int tau = kp.tau_y, lam = kp.lambda_y;
    for (int d = D - 2; d >= 1; --d) {
        int nn[kRoadPairs][2];
#pragma unroll
        for (int q = 0; q < kRoadPairs; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int v = 2 * (tid + q * kRoadThreads) + h;
                nn[q][h] = (d - 2 >= 1 && v < H) ? __ldg(my + (size_t)(d - 2) * H + v) : 0;
            }
#pragma unroll
        for (int q = 0; q < kRoadPairs; ++q) {
            const int i = tid + q * kRoadThreads;
            if (i < Hp) {
                uint8_t nib = 0;
#pragma unroll
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
                        Ec[v] = -cur[q][h] + best;
                    nib |= (uint8_t)(arg << (4 * h));
                }
                bt[(size_t)d * Hp + i] = nib;
            }
        }
#pragma unroll
        for (int q = 0; q < kRoadPairs; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                cur[q][h] = nxt[q][h];
                nxt[q][h] = nn[q][h];
            }
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int v = tid; v < H; v += kRoadThreads)
        if (Ep[v] < bv) {
            bv = Ep[v];
            bi = v;
        }
    const int vstar = block_argmin<kRoadThreads>(bv, bi, sh + kMaxChunks);
    if (tid == 0) {
        path[0] = -1;
        int v = vstar;
        path[1] = (int16_t)v;
        for (int d = 1; d <= D - 2; ++d) {
            const uint8_t b = bt[(size_t)d * Hp + (v >> 1)];
            v += (v & 1) ? (b >> 4) : (b & 15);
            path[d + 1] = (int16_t)v;
        }
    }
    __syncthreads();
    for (int d = tid; d < D; d += kRoadThreads) {
        flag[d] = d >= 1 && my[(size_t)d * H + path[d]] > 0;
        w.path_y[(size_t)f * D + d] = path[d];
    }
    __syncthreads();
    const int k = block_compact<kRoadThreads>(flag, D, pid, sh);
    int16_t *gp = w.pts + (size_t)f * 2 * 3 * w.pmax;
    for (int j = tid; j < k; j += kRoadThreads) {
        gp[j] = path[pid[j]];
        gp[w.pmax + j] = pid[j];
        gp[2 * w.pmax + j] = pid[j];
    }
    if (tid == 0)
        w.npts[f * 2] = k;
}

// ---------------------------------------------------------------------------------------------------
// k_vpx_dp
// ---------------------------------------------------------------------------------------------------
struct VpxMem {
    int *E0, *E1, *band;   // E rows are padded by kPadX sentinels on both sides
    int *voff;             // [H + 1] offsets of the staged vote rows
    int16_t *vb;           // [vote_cap]
    int16_t *path;         // [H]
    uint8_t *sup;          // [H]
    int *sh;
    uint8_t *bt;           // [seg_rows][Wp]
};

__device__ __forceinline__ void band_row(const KParams &kp, const Work &w, const VpxMem &S, int f, int r, int sign,
                                         bool staged)
{
    const int cnt = w.vcount[(size_t)f * kp.H + r];
    const int16_t *src = staged ? S.vb + S.voff[r] : w.vbins + ((size_t)f * kp.H + r) * kp.W;
    for (int q = threadIdx.x; q < cnt; q += kVpxThreads)
        atomicAdd(&S.band[src[q]], sign);
}

// One Eq. 18 step for the pairs of cells owned by this thread; Ep, Ec point at column 0 of padded rows.
template <int TAU>
__device__ __forceinline__ void dp_row(const KParams &kp, const int *band, const int *Ep, int *Ec, uint8_t *btrow)
{
    const int W = kp.W, Wp = (W + 1) >> 1, lam = kp.lambda_x, rho = kp.vote_rho;
    for (int i = threadIdx.x; i < Wp; i += kVpxThreads) {
        const int u0 = 2 * i;
        int e[2 * TAU + 2];
#pragma unroll
        for (int j = 0; j < 2 * TAU + 2; ++j)
            e[j] = Ep[u0 - TAU + j];
        uint8_t nib = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int best = e[h + TAU], arg = 0;
#pragma unroll
            for (int k = 1; k <= 2 * TAU; ++k) {
                const int t = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
                const int cand = e[h + TAU + t] + lam * (t < 0 ? -t : t);
                if (cand < best) {
                    best = cand;
                    arg = t;
                }
            }
            const int u = u0 + h;
            if (u < W) {
                Ec[u] = -rho * band[u] + best;
                nib |= (uint8_t)((arg & 15) << (4 * h));
            }
        }
        btrow[i] = nib;
    }
}

__device__ __forceinline__ int bt_get(const uint8_t *bt, int Wp, int slot, int u)
{
    const uint8_t b = bt[(size_t)slot * Wp + (u >> 1)];
    const int nib = (u & 1) ? (b >> 4) : (b & 15);
    return (nib ^ 8) - 8;  // 4-bit two's complement
}

template <int TAU>
__global__ void __launch_bounds__(kVpxThreads) k_vpx_dp(const KParams kp, const Work w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int f = blockIdx.x, W = kp.W, H = kp.H, Wp = (W + 1) >> 1;
    const int tid = threadIdx.x;
    const FrameState fs0 = w.fs[f];
    if (fs0.flags & LD_F_NO_LANES)
        return;
    const int vtop = fs0.v_top, vmax = H - 1, chi = kp.chi;

    VpxMem S;
    unsigned char *p = smem;
    S.E0 = carve<int>(p, W + 2 * kPadX) + kPadX;
    S.E1 = carve<int>(p, W + 2 * kPadX) + kPadX;
    S.band = carve<int>(p, W);
    S.voff = carve<int>(p, H + 1);
    S.vb = carve<int16_t>(p, kp.vote_cap);
    S.path = carve<int16_t>(p, H);
    S.sup = carve<uint8_t>(p, H);
    S.sh = carve<int>(p, kMaxChunks + 2 * (kVpxThreads / 32));
    int16_t *pid = carve<int16_t>(p, H);
    S.bt = carve<uint8_t>(p, (size_t)kp.seg_rows * Wp);

    // ---- stage the vote rows [vtop, vmax] in shared memory when they fit ----
    for (int v = tid; v < H; v += kVpxThreads)
        S.voff[v] = v >= vtop ? w.vcount[(size_t)f * H + v] : 0;
    for (int u = tid; u < W; u += kVpxThreads)
        S.band[u] = 0;
    for (int u = tid - kPadX; u < W + kPadX; u += kVpxThreads) {
        if (u < 0 || u >= W) {
            S.E0[u] = kSent;
            S.E1[u] = kSent;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int v = 0; v < H; ++v) {
            const int c = S.voff[v];
            S.voff[v] = s;
            s += c;
        }
        S.voff[H] = s;
    }
    __syncthreads();
    const bool staged = S.voff[H] <= kp.vote_cap;
    if (staged) {
        const int lane = tid & 31, warp = tid >> 5;
        for (int v = vtop + warp; v <= vmax; v += kVpxThreads / 32) {
            const int cnt = w.vcount[(size_t)f * H + v];
            const int16_t *src = w.vbins + ((size_t)f * H + v) * W;
            for (int q = lane; q < cnt; q += 32)
                S.vb[S.voff[v] + q] = src[q];
        }
    }
    __syncthreads();

    // ---- band of row vmax: rows [max(vtop, vmax - chi), vmax] ----
    for (int r = max(vtop, vmax - chi); r <= vmax; ++r)
        band_row(kp, w, S, f, r, +1, staged);
    __syncthreads();
    for (int u = tid; u < W; u += kVpxThreads)
        S.E0[u] = -kp.vote_rho * S.band[u];
    __syncthreads();

    // ---- forward DP over rows vmax-1 .. vtop; segment k = rows [vtop + k S, vtop + (k+1) S - 1] ----
    const int SR = kp.seg_rows;
    const int nrows = vmax - vtop;
    const int nseg = (nrows + SR - 1) / SR;
    int32_t *ck = w.ckpt + (size_t)f * w.max_seg * 2 * W;
    int *Ep = S.E0, *Ec = S.E1;
    for (int v = vmax - 1; v >= vtop; --v) {
        const int seg = (v - vtop) / SR;
        if (seg > 0 && v == min(vtop + (seg + 1) * SR - 1, vmax - 1)) {
            for (int u = tid; u < W; u += kVpxThreads) {
                ck[(size_t)(2 * seg) * W + u] = Ep[u];
                ck[(size_t)(2 * seg + 1) * W + u] = S.band[u];
            }
            __syncthreads();
        }
        if (v - chi >= vtop)
            band_row(kp, w, S, f, v - chi, +1, staged);
        if (v + chi + 1 <= vmax)
            band_row(kp, w, S, f, v + chi + 1, -1, staged);
        __syncthreads();
        dp_row<TAU>(kp, S.band, Ep, Ec, S.bt + (size_t)(v - (vtop + seg * SR)) * Wp);
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    // ---- path start: smallest u minimising E_{vtop} ----
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int u = tid; u < W; u += kVpxThreads)
        if (Ep[u] < bv) {
            bv = Ep[u];
            bi = u;
        }
    const int ustar = block_argmin<kVpxThreads>(bv, bi, S.sh + kMaxChunks);
    if (tid == 0) {
        S.path[vtop] = (int16_t)ustar;
        const int hi = min(vtop + SR - 1, vmax - 1);
        for (int v = vtop; v <= hi && nseg > 0; ++v)
            S.path[v + 1] = (int16_t)(S.path[v] + bt_get(S.bt, Wp, v - vtop, S.path[v]));
    }
    __syncthreads();
    // ---- lower segments: restore the checkpoint, recompute the backtrack rows, follow them ----
    for (int seg = 1; seg < nseg; ++seg) {
        const int lo = vtop + seg * SR, hi = min(vtop + (seg + 1) * SR - 1, vmax - 1);
        for (int u = tid; u < W; u += kVpxThreads) {
            S.E0[u] = ck[(size_t)(2 * seg) * W + u];
            S.band[u] = ck[(size_t)(2 * seg + 1) * W + u];
        }
        __syncthreads();
        Ep = S.E0;
        Ec = S.E1;
        for (int v = hi; v >= lo; --v) {
            if (v - chi >= vtop)
                band_row(kp, w, S, f, v - chi, +1, staged);
            if (v + chi + 1 <= vmax)
                band_row(kp, w, S, f, v + chi + 1, -1, staged);
            __syncthreads();
            dp_row<TAU>(kp, S.band, Ep, Ec, S.bt + (size_t)(v - lo) * Wp);
            __syncthreads();
            int *tmp = Ep;
            Ep = Ec;
            Ec = tmp;
        }
        if (tid == 0)
            for (int v = lo; v <= hi; ++v)
                S.path[v + 1] = (int16_t)(S.path[v] + bt_get(S.bt, Wp, v - lo, S.path[v]));
        __syncthreads();
    }

    // ---- rows whose path cell holds votes: some vote of rows [v - chi, v + chi] in column u_v ----
    for (int v = tid; v < H; v += kVpxThreads)
        S.sup[v] = 0;
    __syncthreads();
    {
        const int lane = tid & 31, warp = tid >> 5;
        for (int r = vtop + warp; r <= vmax; r += kVpxThreads / 32) {
            const int cnt = w.vcount[(size_t)f * H + r];
            const int16_t *src = staged ? S.vb + S.voff[r] : w.vbins + ((size_t)f * H + r) * W;
            const int lo = max(vtop, r - chi), hi = min(vmax, r + chi);
            for (int q = lane; q < cnt; q += 32) {
                const int b = src[q];
                for (int v = lo; v <= hi; ++v)
                    if (S.path[v] == b)
                        S.sup[v] = 1;
            }
        }
    }
    __syncthreads();
    const int t = vmax - vtop + 1;
    const int k = block_compact<kVpxThreads>(S.sup + vtop, t, pid, S.sh);
    int16_t *gp = w.pts + ((size_t)f * 2 + 1) * 3 * w.pmax;
    for (int j = tid; j < k; j += kVpxThreads) {
        gp[j] = (int16_t)(vtop + pid[j]);
        gp[w.pmax + j] = S.path[vtop + pid[j]];
        gp[2 * w.pmax + j] = (int16_t)(vtop + pid[j]);
    }
    for (int v = tid; v < H; v += kVpxThreads)
        w.path_x[(size_t)f * H + v] = v >= vtop ? S.path[v] : (int16_t)0;
    if (tid == 0)
        w.npts[f * 2 + 1] = k;
}

size_t vpx_fixed_bytes(const KParams &kp)
{
    const size_t W = kp.W, H = kp.H;
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * (W + 2 * kPadX));
    add(4 * (W + 2 * kPadX));
    add(4 * W);
    add(4 * (H + 1));
    add(2 * (size_t)kp.vote_cap);
    add(2 * H);
    add(H);
    add(4 * (kMaxChunks + 2 * (kVpxThreads / 32)));
    add(2 * H);
    return ((s + 15) & ~(size_t)15) + 64;
}

using VpxKernel = void (*)(KParams, Work);
VpxKernel vpx_kernel(int tau)
{
    switch (tau) {
    case 0: return k_vpx_dp<0>;
    case 1: return k_vpx_dp<1>;
    case 2: return k_vpx_dp<2>;
    case 3: return k_vpx_dp<3>;
    case 4: return k_vpx_dp<4>;
    case 5: return k_vpx_dp<5>;
    case 6: return k_vpx_dp<6>;
    default: return k_vpx_dp<7>;
    }
}

}  // namespace

size_t road_smem_bytes(const KParams &kp)
{
    const size_t H = kp.H, D = kp.D, Hp = (H + 1) / 2;
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * (H + kPadY));
    add(4 * (H + kPadY));
    add(4 * (kMaxChunks + 2 * (kRoadThreads / 32)));
    add(2 * D);
    add(D);
    add(2 * D);
    add(D * Hp);
    return s + 64;
}

size_t vpx_smem_bytes(const KParams &kp)
{
    return vpx_fixed_bytes(kp) + (size_t)kp.seg_rows * ((kp.W + 1) / 2);
}

int vpx_seg_rows(const KParams &kp, size_t budget)
{
    const size_t fixed = vpx_fixed_bytes(kp);
    if (budget <= fixed)
        return 0;
    return (int)((budget - fixed) / ((kp.W + 1) / 2));
}

cudaError_t setup_dp(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_road_dp, smem_optin);
    for (int t = 0; t <= 7 && e == cudaSuccess; ++t)
        e = allow_max_smem(vpx_kernel(t), smem_optin);
    return e;
}

cudaError_t launch_road(const KParams &kp, const Work &w, cudaStream_t s)
{
    k_road_dp<<<kp.n_frames, kRoadThreads, road_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

cudaError_t launch_vpx(const KParams &kp, const Work &w, cudaStream_t s)
{
    vpx_kernel(kp.tau_x)<<<kp.n_frames, kVpxThreads, vpx_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

}  // namespace ld
