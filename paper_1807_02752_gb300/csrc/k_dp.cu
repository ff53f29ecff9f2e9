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
// Each DP step is one row of the map.  A thread owns four adjacent cells: it loads the window of the
// previous row they share once and writes their four 4-bit backtrack entries as one 16-bit word.  The CTA
// is sized to the row (one thread per four cells), so the per-row barriers involve few warps.  Rows are
// padded with sentinels so the candidate loops have no bounds checks.  The V_px DP keeps as many backtrack
// rows in shared memory as fit; taller road areas are processed in segments, with the DP state
// checkpointed at segment boundaries and recomputed during the backtrack.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kRoadThreads = 128;
constexpr int kRoadQ = (LD_MAX_H / 4 + kRoadThreads - 1) / kRoadThreads;  // quads per thread (3)
constexpr int kMaxChunks = (LD_MAX_H + 31) / 32 + 2;
constexpr int kSent = 0x3fffffff;  // larger than any DP energy (checked when the handle is created)
constexpr int kPadY = 20;          // >= 3 + tau_y
constexpr int kPadX = 16;          // >= 3 + tau_x

template <typename T>
__device__ __forceinline__ T *carve(unsigned char *&p, size_t count)
{
    const size_t off = ((size_t)p + 15) & ~(size_t)15;
    T *r = reinterpret_cast<T *>(off);
    p = reinterpret_cast<unsigned char *>(off + sizeof(T) * count);
    return r;
}

// Lexicographic (value, index) minimum over the block; every thread receives the index.
__device__ int block_argmin(int val, int idx, int *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
        for (int w = 1; w < nw; ++w)
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
__device__ int block_compact(const uint8_t *flag, int n, int16_t *list, int *chunk)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nch = (n + 31) >> 5;
    for (int c = warp; c < nch; c += nw) {
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
    for (int c = warp; c < nch; c += nw) {
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

__device__ __forceinline__ int nib16(const uint16_t *row, int i) { return (row[i >> 2] >> (4 * (i & 3))) & 15; }

// ---------------------------------------------------------------------------------------------------
// k_road_dp
// ---------------------------------------------------------------------------------------------------
template <int TMAX>
__global__ void __launch_bounds__(kRoadThreads) k_road_dp(const KParams kp, const Work w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int f = blockIdx.x, H = kp.H, D = kp.D, Hq = (H + 3) >> 2;
    const int tid = threadIdx.x;
    const int32_t *my = w.myT + (size_t)f * D * H;

    unsigned char *p = smem;
    int *E0 = carve<int>(p, H + kPadY);
    int *E1 = carve<int>(p, H + kPadY);
    int *sh = carve<int>(p, kMaxChunks + 2 * (kRoadThreads / 32));
    int16_t *path = carve<int16_t>(p, D);
    uint8_t *flag = carve<uint8_t>(p, D);
    int16_t *pid = carve<int16_t>(p, D);
    uint16_t *bt = carve<uint16_t>(p, (size_t)D * Hq);

    for (int v = tid; v < H + kPadY; v += kRoadThreads) {
        E0[v] = v < H ? -my[(size_t)(D - 1) * H + v] : kSent;
        E1[v] = kSent;
    }
    // data terms of the next two steps are loaded a step ahead of their use
    int cur[kRoadQ][4], nxt[kRoadQ][4];
#pragma unroll
    for (int q = 0; q < kRoadQ; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int v = 4 * (tid + q * kRoadThreads) + c;
            cur[q][c] = v < H ? my[(size_t)(D - 2) * H + v] : 0;
            nxt[q][c] = (D - 3 >= 1 && v < H) ? my[(size_t)(D - 3) * H + v] : 0;
        }
    __syncthreads();
    int *Ep = E0, *Ec = E1;
    const int tau = kp.tau_y, lam = kp.lambda_y;
    for (int d = D - 2; d >= 1; --d) {
        int nn[kRoadQ][4];
#pragma unroll
        for (int q = 0; q < kRoadQ; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int v = 4 * (tid + q * kRoadThreads) + c;
                nn[q][c] = (d - 2 >= 1 && v < H) ? __ldg(my + (size_t)(d - 2) * H + v) : 0;
            }
#pragma unroll
        for (int q = 0; q < kRoadQ; ++q) {
            const int i = tid + q * kRoadThreads;
            if (i < Hq) {
                const int v0 = 4 * i;
                int e[4 + TMAX];
#pragma unroll
                for (int j = 0; j < 4 + TMAX; ++j)
                    e[j] = Ep[v0 + j];
                uint32_t code = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    int best = e[c], arg = 0;
#pragma unroll
                    for (int t = 1; t <= TMAX; ++t) {
                        const int cand = e[c + t] + lam * t;
                        if (t <= tau && cand < best) {
                            best = cand;
                            arg = t;
                        }
                    }
                    if (v0 + c < H)
                        Ec[v0 + c] = -cur[q][c] + best;
                    code |= (uint32_t)arg << (4 * c);
                }
                bt[(size_t)d * Hq + i] = (uint16_t)code;
            }
        }
#pragma unroll
        for (int q = 0; q < kRoadQ; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                cur[q][c] = nxt[q][c];
                nxt[q][c] = nn[q][c];
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
    const int vstar = block_argmin(bv, bi, sh + kMaxChunks);
    if (tid == 0) {
        path[0] = -1;
        int v = vstar;
        path[1] = (int16_t)v;
        for (int d = 1; d <= D - 2; ++d) {
            v += nib16(bt + (size_t)d * Hq, v);
            path[d + 1] = (int16_t)v;
        }
    }
    __syncthreads();
    for (int d = tid; d < D; d += kRoadThreads) {
        flag[d] = d >= 1 && my[(size_t)d * H + path[d]] > 0;
        w.path_y[(size_t)f * D + d] = path[d];
    }
    __syncthreads();
    const int k = block_compact(flag, D, pid, sh);
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
    uint16_t *bt;          // [seg_rows][Wq]
};

__device__ __forceinline__ void band_row(const KParams &kp, const Work &w, const VpxMem &S, int f, int r, int sign,
                                         bool staged)
{
    // vote rows [v_top, H-1] have their counts as offset differences in shared memory
    const int cnt = S.voff[r + 1] - S.voff[r];
    const int16_t *src = staged ? S.vb + S.voff[r] : w.vbins + ((size_t)f * kp.H + r) * kp.W;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x)
        atomicAdd(&S.band[src[q]], sign);
}

// One Eq. 18 step for the quads of cells owned by this thread; Ep, Ec point at column 0 of padded rows.
template <int TAU>
__device__ __forceinline__ void dp_row(const KParams &kp, const int *band, const int *Ep, int *Ec, uint16_t *btrow)
{
    const int W = kp.W, Wq = (W + 3) >> 2, lam = kp.lambda_x, rho = kp.vote_rho;
    for (int i = threadIdx.x; i < Wq; i += blockDim.x) {
        const int u0 = 4 * i;
        int e[2 * TAU + 4];
#pragma unroll
        for (int j = 0; j < 2 * TAU + 4; ++j)
            e[j] = Ep[u0 - TAU + j];
        uint32_t code = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int best = e[c + TAU], arg = 0;
#pragma unroll
            for (int k = 1; k <= 2 * TAU; ++k) {
                const int t = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
                const int cand = e[c + TAU + t] + lam * (t < 0 ? -t : t);
                if (cand < best) {
                    best = cand;
                    arg = t;
                }
            }
            const int u = u0 + c;
            if (u < W) {
                Ec[u] = -rho * band[u] + best;
                code |= (uint32_t)(arg & 15) << (4 * c);
            }
        }
        btrow[i] = (uint16_t)code;
    }
}

__device__ __forceinline__ int bt_get(const uint16_t *bt, int Wq, int slot, int u)
{
    const int nib = nib16(bt + (size_t)slot * Wq, u);
    return (nib ^ 8) - 8;  // 4-bit two's complement
}

template <int TAU>
__global__ void __launch_bounds__(1024) k_vpx_dp(const KParams kp, const Work w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int f = blockIdx.x, W = kp.W, H = kp.H, Wq = (W + 3) >> 2;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
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
    S.sh = carve<int>(p, kMaxChunks + 64);
    int16_t *pid = carve<int16_t>(p, H);
    S.bt = carve<uint16_t>(p, (size_t)kp.seg_rows * Wq);

    // ---- stage the vote rows [vtop, vmax] in shared memory when they fit ----
    for (int v = tid; v < H; v += nt)
        S.voff[v] = v >= vtop ? w.vcount[(size_t)f * H + v] : 0;
    for (int u = tid; u < W; u += nt)
        S.band[u] = 0;
    for (int u = tid - kPadX; u < W + kPadX; u += nt) {
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
        for (int v = vtop + warp; v <= vmax; v += nw) {
            const int cnt = S.voff[v + 1] - S.voff[v];
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
    for (int u = tid; u < W; u += nt)
        S.E0[u] = -kp.vote_rho * S.band[u];
    __syncthreads();

    // ---- forward DP over rows vmax-1 .. vtop; segment k = rows [vtop + k S, vtop + (k+1) S - 1] ----
    const int SR = kp.seg_rows;
    const int nrows = vmax - vtop;
    const int nseg = (nrows + SR - 1) / SR;
    int32_t *ck = w.ckpt + (size_t)f * w.max_seg * 2 * W;
    int *Ep = S.E0, *Ec = S.E1;
    int seg = nseg - 1, seg_lo = vtop + seg * SR;
    for (int v = vmax - 1; v >= vtop; --v) {
        if (v < seg_lo) {
            --seg;
            seg_lo -= SR;
        }
        if (seg > 0 && v == min(seg_lo + SR - 1, vmax - 1)) {
            for (int u = tid; u < W; u += nt) {
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
        dp_row<TAU>(kp, S.band, Ep, Ec, S.bt + (size_t)(v - seg_lo) * Wq);
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    // ---- path start: smallest u minimising E_{vtop} ----
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int u = tid; u < W; u += nt)
        if (Ep[u] < bv) {
            bv = Ep[u];
            bi = u;
        }
    const int ustar = block_argmin(bv, bi, S.sh + kMaxChunks);
    if (tid == 0) {
        S.path[vtop] = (int16_t)ustar;
        const int hi = min(vtop + SR - 1, vmax - 1);
        for (int v = vtop; v <= hi && nseg > 0; ++v)
            S.path[v + 1] = (int16_t)(S.path[v] + bt_get(S.bt, Wq, v - vtop, S.path[v]));
    }
    __syncthreads();
    // ---- lower segments: restore the checkpoint, recompute the backtrack rows, follow them ----
    for (int sg = 1; sg < nseg; ++sg) {
        const int lo = vtop + sg * SR, hi = min(vtop + (sg + 1) * SR - 1, vmax - 1);
        for (int u = tid; u < W; u += nt) {
            S.E0[u] = ck[(size_t)(2 * sg) * W + u];
            S.band[u] = ck[(size_t)(2 * sg + 1) * W + u];
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
            dp_row<TAU>(kp, S.band, Ep, Ec, S.bt + (size_t)(v - lo) * Wq);
            __syncthreads();
            int *tmp = Ep;
            Ep = Ec;
            Ec = tmp;
        }
        if (tid == 0)
            for (int v = lo; v <= hi; ++v)
                S.path[v + 1] = (int16_t)(S.path[v] + bt_get(S.bt, Wq, v - lo, S.path[v]));
        __syncthreads();
    }

    // ---- rows whose path cell holds votes: some vote of rows [v - chi, v + chi] in column u_v ----
    for (int v = tid; v < H; v += nt)
        S.sup[v] = 0;
    __syncthreads();
    for (int r = vtop + warp; r <= vmax; r += nw) {
        const int cnt = S.voff[r + 1] - S.voff[r];
        const int16_t *src = staged ? S.vb + S.voff[r] : w.vbins + ((size_t)f * H + r) * W;
        const int lo = max(vtop, r - chi), hi = min(vmax, r + chi);
        for (int q = lane; q < cnt; q += 32) {
            const int b = src[q];
            for (int v = lo; v <= hi; ++v)
                if (S.path[v] == b)
                    S.sup[v] = 1;
        }
    }
    __syncthreads();
    const int t = vmax - vtop + 1;
    const int k = block_compact(S.sup + vtop, t, pid, S.sh);
    int16_t *gp = w.pts + ((size_t)f * 2 + 1) * 3 * w.pmax;
    for (int j = tid; j < k; j += nt) {
        gp[j] = (int16_t)(vtop + pid[j]);
        gp[w.pmax + j] = S.path[vtop + pid[j]];
        gp[2 * w.pmax + j] = (int16_t)(vtop + pid[j]);
    }
    for (int v = tid; v < H; v += nt)
        w.path_x[(size_t)f * H + v] = v >= vtop ? S.path[v] : (int16_t)0;
    if (tid == 0)
        w.npts[f * 2 + 1] = k;
}

int vpx_threads(int W)
{
    const int nq = (W + 3) / 4;
    int nt = (nq + 31) / 32 * 32;
    return nt < 64 ? 64 : nt > 1024 ? 1024 : nt;
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
    add(4 * (kMaxChunks + 64));
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

using RoadKernel = void (*)(KParams, Work);
RoadKernel road_kernel(int tau) { return tau <= 6 ? k_road_dp<6> : k_road_dp<15>; }

}  // namespace

size_t road_smem_bytes(const KParams &kp)
{
    const size_t H = kp.H, D = kp.D, Hq = (H + 3) / 4;
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * (H + kPadY));
    add(4 * (H + kPadY));
    add(4 * (kMaxChunks + 2 * (kRoadThreads / 32)));
    add(2 * D);
    add(D);
    add(2 * D);
    add(2 * D * Hq);
    return s + 64;
}

size_t vpx_smem_bytes(const KParams &kp)
{
    return vpx_fixed_bytes(kp) + (size_t)kp.seg_rows * 2 * ((kp.W + 3) / 4);
}

int vpx_seg_rows(const KParams &kp, size_t budget)
{
    const size_t fixed = vpx_fixed_bytes(kp);
    if (budget <= fixed)
        return 0;
    return (int)((budget - fixed) / (2 * ((kp.W + 3) / 4)));
}

cudaError_t setup_dp(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_road_dp<6>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_road_dp<15>, smem_optin);
    for (int t = 0; t <= 7 && e == cudaSuccess; ++t)
        e = allow_max_smem(vpx_kernel(t), smem_optin);
    return e;
}

cudaError_t launch_road(const KParams &kp, const Work &w, cudaStream_t s)
{
    road_kernel(kp.tau_y)<<<kp.n_frames, kRoadThreads, road_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

cudaError_t launch_vpx(const KParams &kp, const Work &w, cudaStream_t s)
{
    vpx_kernel(kp.tau_x)<<<kp.n_frames, vpx_threads(kp.W), vpx_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

}  // namespace ld
