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
// penalty (the printed form is kept as the dp_literal switch, k_road_dp_lit).  Eq. 18's "+lambda_x tau" is read as lambda_x |tau|.  Ties take the smaller |tau|, then the
// negative one; a path starts at the smallest index minimising its last row.  Alg. 5 is read from the text
// around it: m_x(u, j) = -varrho * (votes in column u of rows [j - chi, j + chi] within [v_top, H-1]).
// A path point whose cell holds no count carries no observation; the kernels hand the points with data to
// the RANSAC fit (k_fit), in increasing index order.
//
// Each DP step is one row of the map.  A thread owns a pair of adjacent cells (many warps per step: the
// step loops are latency-bound) and writes their two 4-bit backtrack entries as one byte.  A thread loads the window of
// the previous row its cells share once.  The CTA is sized to the row, so the per-row barriers involve few
// warps.  Rows are padded with sentinels so the candidate loops have no bounds checks.  The V_px DP keeps
// the backtrack rows of the top of the road in shared memory; the rows below go to a per-frame global
// buffer (L2-resident) and come back in blocks for the backtrack.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kMaxChunks = (LD_MAX_H + 31) / 32 + 2;
constexpr int kSent = 0x3fffffff;  // larger than any DP energy (checked when the handle is created)
constexpr int kPadY = 20;          // >= 2 + tau_y (rounded up to even)
constexpr int kPadX = 16;          // >= tau_x rounded up to even, + 1

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


// Shared-memory accesses through 32-bit shared addresses (keeps the hot DP loop on the shared-memory path
// whatever pointers the compiler can prove).
__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void atoms_add(uint32_t a, int v) { asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v)); }

// ---------------------------------------------------------------------------------------------------
// k_road_dp
// ---------------------------------------------------------------------------------------------------
template <int TMAX>
__device__ __forceinline__ void road_dp_body(const KParams &kp, const Work &w, const int f)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = kp.H, D = kp.D, Hp = (H + 1) >> 1;  // Hp: pairs of rows
    const int tid = threadIdx.x, nt = blockDim.x;
    const int32_t *my = w.myT + (size_t)f * D * H;

    unsigned char *p = smem;
    int *E0 = carve<int>(p, 2 * Hp + kPadY);
    int *E1 = carve<int>(p, 2 * Hp + kPadY);
    int *sh = carve<int>(p, kMaxChunks + 64);
    int16_t *path = carve<int16_t>(p, D);
    uint8_t *flag = carve<uint8_t>(p, D);
    int16_t *pid = carve<int16_t>(p, D);
    uint8_t *bt = carve<uint8_t>(p, (size_t)D * Hp);  // one byte per pair of rows: two 4-bit steps

    // E rows hold keys 16 E: a candidate's key 16 (E + lambda tau) + tau orders candidates by energy, then
    // by the smaller tau, so the tie-broken argmin is a plain integer minimum (|16 E| < 2^30 always holds
    // here: energies are bounded by (w + lambda_y tau_y) D).
    for (int v = tid; v < 2 * Hp + kPadY; v += nt) {
        E0[v] = v < H ? -16 * my[(size_t)(D - 1) * H + v] : kSent;
        E1[v] = kSent;
    }
    // thread i owns rows v0 = 2i, v0 + 1.  The data terms of a step are loaded kSets steps ahead into one of
    // kSets register sets (steps rotate over them), so no register copy waits for a load in flight.
    const int i = tid, v0 = 2 * i;
    const bool own = i < Hp;
    auto load_row = [&](int d, int *dst) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int v = v0 + c;
            dst[c] = (own && d >= 1 && v < H) ? __ldg(my + (size_t)d * H + v) : 0;
        }
    };
    constexpr int kSets = 16;  // steps of load latency hidden: kSets - 1
    int reg[kSets][2];
#pragma unroll
    for (int k = 0; k < kSets; ++k)
        load_row(D - 2 - k, reg[k]);
    __syncthreads();
    int *Ep = E0, *Ec = E1;
    const int tau = kp.tau_y;
    int ck[TMAX + 1];  // key offset of step t; steps beyond tau_y never win
#pragma unroll
    for (int t = 0; t <= TMAX; ++t)
        ck[t] = t <= tau ? 16 * kp.lambda_y * t + t : kSent;
    constexpr int NL = (TMAX + 3) / 2;  // 8-byte loads: rows v0 .. v0 + 1 + TMAX
    auto step = [&](int d, const int *cur) {
        if (own) {
            int e[2 * NL];
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const int2 v2 = *reinterpret_cast<const int2 *>(Ep + v0 + 2 * j);
                e[2 * j] = v2.x;
                e[2 * j + 1] = v2.y;
            }
            uint32_t code = 0;
            int out[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                int kk[TMAX + 1];
#pragma unroll
                for (int t = 0; t <= TMAX; ++t)
                    kk[t] = e[c + t] + ck[t];
#pragma unroll
                for (int st = 1; st <= TMAX; st *= 2)
#pragma unroll
                    for (int j = 0; j + st <= TMAX; j += 2 * st)
                        kk[j] = min(kk[j], kk[j + st]);
                out[c] = v0 + c < H ? -16 * cur[c] + (kk[0] & ~15) : kSent;
                code |= (uint32_t)(kk[0] & 15) << (4 * c);
            }
            *reinterpret_cast<int2 *>(Ec + v0) = make_int2(out[0], out[1]);
            bt[(size_t)d * Hp + i] = (uint8_t)code;
        }
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    };
    for (int d = D - 2; d >= 1; d -= kSets) {
#pragma unroll
        for (int k = 0; k < kSets; ++k)
            if (d - k >= 1) {
                step(d - k, reg[k]);
                load_row(d - k - kSets, reg[k]);
            }
    }
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int v = tid; v < H; v += nt)
        if (Ep[v] < bv) {
            bv = Ep[v];
            bi = v;
        }
    const int vstar = block_argmin(bv, bi, sh + kMaxChunks);
    if (tid == 0) {
        path[0] = -1;
        int v = vstar;
        path[1] = (int16_t)v;
        const uint8_t *row = bt + Hp;
        for (int d = 1; d <= D - 2; ++d, row += Hp) {
            if (LD_IN(v, H, CK_ROAD_PATH))
                v += (row[v >> 1] >> (4 * (v & 1))) & 15;
            path[d + 1] = (int16_t)v;
        }
    }
    __syncthreads();
    for (int d = tid; d < D; d += nt) {
        flag[d] = d >= 1 && LD_IN(path[d], H, CK_ROAD_PATH) && my[(size_t)d * H + path[d]] > 0;
        w.path_y[(size_t)f * D + d] = path[d];
    }
    __syncthreads();
    const int k = block_compact(flag, D, pid, sh);
    int16_t *gp = w.pts + (size_t)f * 2 * 3 * w.pmax;
    for (int j = tid; j < k; j += nt)
        if (LD_IN(j, w.pmax, CK_ROAD_PTS) && LD_IN(pid[j], D, CK_ROAD_PTS)) {
            gp[j] = path[pid[j]];
            gp[w.pmax + j] = pid[j];
            gp[2 * w.pmax + j] = pid[j];
        }
    if (tid == 0)
        w.npts[f * 2] = k;
}

// One thread per pair of rows: the tallest frame (LD_MAX_H rows) needs (LD_MAX_H + 1) / 2 threads, rounded
// up to whole warps.  The bound is kept tight so that the 16 register sets of the load pipeline fit without
// spilling.
constexpr int kRoadMaxThreads = 640;
static_assert(((LD_MAX_H + 1) / 2 + 31) / 32 * 32 <= kRoadMaxThreads, "road DP: one thread per pair of rows");

template <int TMAX>
__global__ void __launch_bounds__(kRoadMaxThreads) k_road_dp(const KParams kp, const Work w) { road_dp_body<TMAX>(kp, w, blockIdx.x); }
template <int TMAX>
__global__ void __launch_bounds__(kRoadMaxThreads) k_road_dp_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.x];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    road_dp_body<TMAX>(kp, w, 0);
}

// ---------------------------------------------------------------------------------------------------
// k_road_dp_lit: Eq. 12 as printed (dp_literal), for A/B against the reading above:
//   E_d(v) = -m_y(d, v) + min_{tau in [0, tau_y], v - tau >= 0} [E_{d+1}(v - tau) - lambda_y tau],
// ties to the smaller tau; the path starts at the smallest v minimising E_1 and steps to v - tau.  Plain
// per-row loops (a thread per pair of rows, 4-bit backtrack entries of the pair in one byte); the same
// shared-memory layout and outputs as k_road_dp.
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ void road_dp_lit_body(const KParams &kp, const Work &w, const int f)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = kp.H, D = kp.D, Hp = (H + 1) >> 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int32_t *my = w.myT + (size_t)f * D * H;
    unsigned char *p = smem;
    int *Ep = carve<int>(p, 2 * Hp + kPadY);
    int *Ec = carve<int>(p, 2 * Hp + kPadY);
    int *sh = carve<int>(p, kMaxChunks + 64);
    int16_t *path = carve<int16_t>(p, D);
    uint8_t *flag = carve<uint8_t>(p, D);
    int16_t *pid = carve<int16_t>(p, D);
    uint8_t *bt = carve<uint8_t>(p, (size_t)D * Hp);
    for (int v = tid; v < H; v += nt)
        Ep[v] = -my[(size_t)(D - 1) * H + v];
    __syncthreads();
    const int tau = kp.tau_y, lam = kp.lambda_y;
    for (int d = D - 2; d >= 1; --d) {
        for (int i = tid; i < Hp; i += nt) {
            uint32_t code = 0;
            for (int c = 0; c < 2; ++c) {
                const int v = 2 * i + c;
                if (v >= H)
                    break;
                int best = 0x7fffffff, arg = 0;
                for (int t = 0; t <= tau && v - t >= 0; ++t) {
                    const int cand = Ep[v - t] - lam * t;
                    if (cand < best) {
                        best = cand;
                        arg = t;
                    }
                }
                Ec[v] = -my[(size_t)d * H + v] + best;
                code |= (uint32_t)arg << (4 * c);
            }
            bt[(size_t)d * Hp + i] = (uint8_t)code;
        }
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int v = tid; v < H; v += nt)
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
            if (LD_IN(v, H, CK_ROAD_PATH))
                v -= (bt[(size_t)d * Hp + (v >> 1)] >> (4 * (v & 1))) & 15;
            path[d + 1] = (int16_t)v;
        }
    }
    __syncthreads();
    for (int d = tid; d < D; d += nt) {
        flag[d] = d >= 1 && LD_IN(path[d], H, CK_ROAD_PATH) && my[(size_t)d * H + path[d]] > 0;
        w.path_y[(size_t)f * D + d] = path[d];
    }
    __syncthreads();
    const int k = block_compact(flag, D, pid, sh);
    int16_t *gp = w.pts + (size_t)f * 2 * 3 * w.pmax;
    for (int j = tid; j < k; j += nt)
        if (LD_IN(j, w.pmax, CK_ROAD_PTS) && LD_IN(pid[j], D, CK_ROAD_PTS)) {
            gp[j] = path[pid[j]];
            gp[w.pmax + j] = pid[j];
            gp[2 * w.pmax + j] = pid[j];
        }
    if (tid == 0)
        w.npts[f * 2] = k;
}

__global__ void __launch_bounds__(1024) k_road_dp_lit(const KParams kp, const Work w) { road_dp_lit_body(kp, w, blockIdx.x); }
__global__ void __launch_bounds__(1024) k_road_dp_lit_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.x];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    road_dp_lit_body(kp, w, 0);
}

// ---------------------------------------------------------------------------------------------------
// k_vpx_dp
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ int2 lds2(uint32_t a)
{
    int2 v;
    asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts2(uint32_t a, int2 v)
{
    asm volatile("st.shared.v2.s32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y));
}
__device__ __forceinline__ void sts8(uint32_t a, uint32_t v) { asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v)); }
__device__ __forceinline__ uint32_t lds8(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void atoms_or(uint32_t a, uint32_t v) { asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(v)); }

// A thread owns the cell pairs j = tid + p * blockDim.x (p < NP), cells 2j and 2j + 1.  A backtrack row
// holds one byte per pair (two 4-bit entries), padded to 16 bytes (vpx_row_bytes).

// Shared-memory layout of k_vpx_dp.
struct VpxMem {
    int *E0, *E1;          // E rows, column 0 at index 0, padded by kPadX sentinels on both sides
    int *D0, *D1;          // band deltas of the next row (double-buffered), [2 pairs]
    int *voff;             // [H + 1] offsets of the staged vote rows (prefix of the per-row counts)
    int16_t *vb;           // [vote_cap]
    int16_t *path;         // [H]
    uint8_t *sup;          // [H]
    int *sh;
    int16_t *pid;          // [H]
    int4 *rinfo;           // [H] per DP row v: first staged vote and count of row v - chi (entering), of row v + chi + 1 (leaving)
    unsigned char *dyn;    // backtrack rows [seg_rows][row bytes], later the column bitmaps of the votes
};

// Vote columns of row r (staged in shared memory, else the frame's list in global memory).
struct VoteRow {
    const int16_t *p;
    int n;
};
__device__ __forceinline__ VoteRow vote_row(const KParams &kp, const Work &w, const VpxMem &S, int f, int r, bool staged)
{
    VoteRow vr;
    vr.n = S.voff[r + 1] - S.voff[r];
    vr.p = staged ? S.vb + S.voff[r] : w.vbins + ((size_t)f * kp.H + r) * kp.W;
    return vr;
}

// Scatter the band change between row v+1 and row v (votes of row v - chi enter, of row v + chi + 1 leave)
// into the delta array `delta` (shared address), by the threads t0, t0 + stride, ...
__device__ __forceinline__ void scatter_delta(const KParams &kp, const Work &w, const VpxMem &S, int f, int v, int vtop,
                                              bool staged, uint32_t delta, int t0, int stride)
{
    const int vmax = kp.H - 1, chi = kp.chi;
    if (kp.band_literal && v >= vmax - chi - 1) {
        // band_literal_bottom: rows j > vmax - chi - 1 use the band [j, vmax], so there row v enters and
        // nothing leaves; at v = vmax - chi - 1 the band [v - chi, v + chi] replaces [v + 1, vmax]
        const int r_lo = v >= vmax - chi ? v : max(vtop, v - chi);
        for (int r = max(r_lo, vtop); r <= v; ++r) {
            const VoteRow vr = vote_row(kp, w, S, f, r, staged);
            for (int q = t0; q < vr.n; q += stride)
                if (LD_IN(vr.p[q], kp.W, CK_VPX_VOTE))
                    atoms_add(delta + 4u * (uint32_t)vr.p[q], 1);
        }
        if (v == vmax - chi - 1) {
            const VoteRow vr = vote_row(kp, w, S, f, vmax, staged);
            for (int q = t0; q < vr.n; q += stride)
                if (LD_IN(vr.p[q], kp.W, CK_VPX_VOTE))
                    atoms_add(delta + 4u * (uint32_t)vr.p[q], -1);
        }
        return;
    }
    if (v - chi >= vtop) {
        const VoteRow vr = vote_row(kp, w, S, f, v - chi, staged);
        for (int q = t0; q < vr.n; q += stride)
            if (LD_IN(vr.p[q], kp.W, CK_VPX_VOTE))
                atoms_add(delta + 4u * (uint32_t)vr.p[q], 1);
    }
    if (v + chi + 1 <= vmax) {
        const VoteRow vr = vote_row(kp, w, S, f, v + chi + 1, staged);
        for (int q = t0; q < vr.n; q += stride)
            if (LD_IN(vr.p[q], kp.W, CK_VPX_VOTE))
                atoms_add(delta + 4u * (uint32_t)vr.p[q], -1);
    }
}

// The band change of DP row v from its staged descriptor: thread q takes vote q of the entering row, then
// of the leaving row (one round for up to blockDim.x votes).
__device__ __forceinline__ void scatter_staged(const VpxMem &S, int v, uint32_t delta, int W)
{
    const int4 ri = S.rinfo[v];
    for (int q = threadIdx.x; q < ri.y + ri.w; q += blockDim.x) {
        const bool enter = q < ri.y;
        const int c = S.vb[enter ? ri.x + q : ri.z + (q - ri.y)];
        if (LD_IN(c, W, CK_VPX_VOTE))
            atoms_add(delta + 4u * (uint32_t)c, enter ? 1 : -1);
    }
}

// One Eq. 18 row for the cells u0 = 2j, u0 + 1.  ep, ec: shared addresses of column 0 of E_{v+1} and E_v;
// the window [u0 - TW, u0 + 1 + TW] (TW = tau_x rounded up to even) is read as 8-byte loads.  pen[k]: the
// penalty of candidate k in tie order tau = 0, -1, +1, -2, ... (16 lambda_x |tau| + k when PACKED, so the
// tie-broken argmin is an integer minimum; lambda_x |tau| otherwise, compare-select in tie order).
// Writes E_v of the two cells (a sentinel past the last column) and returns the backtrack byte.
template <int TAU, bool PACKED>
__device__ __forceinline__ uint32_t dp_pair(const KParams &kp, int u0, int b0, int b1, const int *pen, uint32_t ep,
                                            uint32_t ec)
{
    constexpr int NK = 2 * TAU + 1;
    constexpr int TW = (TAU + 1) & ~1;
    constexpr int NL = TW + 1;  // 8-byte loads: values u0 - TW .. u0 + 1 + TW
    int e[2 * NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        const int2 v2 = lds2(ep + 4u * (uint32_t)(u0 - TW + 2 * j));
        e[2 * j] = v2.x;
        e[2 * j + 1] = v2.y;
    }
    const int band[2] = {b0, b1};
    int out[2];
    uint32_t code = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        int best, arg;
        if (PACKED) {
            int kk[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int t = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
                kk[k] = e[TW + c + t] + pen[k];
            }
#pragma unroll
            for (int st = 1; st < NK; st *= 2)
#pragma unroll
                for (int j = 0; j + st < NK; j += 2 * st)
                    kk[j] = min(kk[j], kk[j + st]);
            best = kk[0] & ~15;
            arg = kk[0] & 15;
        } else {
            best = e[TW + c];
            arg = 0;
#pragma unroll
            for (int k = 1; k < NK; ++k) {
                const int t = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
                const int cand = e[TW + c + t] + pen[k];
                if (cand < best) {
                    best = cand;
                    arg = t & 15;
                }
            }
        }
        const bool in = u0 + c < kp.W;
        out[c] = in ? (PACKED ? 16 : 1) * -kp.vote_rho * band[c] + best : kSent;
        code |= (uint32_t)(in ? arg : 0) << (4 * c);
    }
    sts2(ec + 4u * (uint32_t)u0, make_int2(out[0], out[1]));
    return code;
}

// Backtrack step at column u of a row starting at shared address rowa: tau from a 4-bit two's complement
// entry, or from the tie rank of the packed form.
__device__ __forceinline__ int bt_step(uint32_t rowa, int u, bool packed)
{
    const int nib = (int)(lds8(rowa + ((uint32_t)u >> 1)) >> (4 * (u & 1))) & 15;
    if (packed)
        return (nib & 1) ? -((nib + 1) >> 1) : (nib >> 1);
    return (nib ^ 8) - 8;
}

// Exclusive prefix sum of a[0..n) in place, a[n] = total.  chunk: >= n/32 + 2 ints.
__device__ void block_scan(int *a, int n, int *chunk)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nch = (n + 31) >> 5;
    for (int c = warp; c < nch; c += nw) {
        const int j = (c << 5) + lane;
        const int x = j < n ? a[j] : 0;
        int inc = x;
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d)
                inc += o;
        }
        if (j < n)
            a[j] = inc - x;
        if (lane == 31)
            chunk[c] = inc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // exclusive scan of the chunk totals by one warp
        int carry = 0;
        for (int c0 = 0; c0 < nch; c0 += 32) {
            const int c = c0 + threadIdx.x;
            const int x = c < nch ? chunk[c] : 0;
            int inc = x;
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, inc, d);
                if ((int)threadIdx.x >= d)
                    inc += o;
            }
            if (c < nch)
                chunk[c] = carry + inc - x;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (threadIdx.x == 0)
            a[n] = carry;
    }
    __syncthreads();
    for (int c = warp; c < nch; c += nw) {
        const int j = (c << 5) + lane;
        if (j < n)
            a[j] += chunk[c];
    }
    __syncthreads();
}

// Stage capture: m_x(u, v) = -varrho * (votes of the band of row v in column u) of cells u0, u0 + 1.
__device__ __forceinline__ void store_mx(const KParams &kp, const Work &w, int f, int v, int u0, int b0, int b1)
{
    int32_t *row = w.dbg_mx + ((size_t)f * kp.H + v) * kp.W;
    row[u0] = -kp.vote_rho * b0;
    if (u0 + 1 < kp.W)
        row[u0 + 1] = -kp.vote_rho * b1;
}

// Forward DP over rows vmax-1 .. vtop, then the backtrack.  Backtrack rows of the top seg_rows rows stay
// in shared memory; lower rows go to the frame's global buffer and come back in blocks of seg_rows rows
// for the backtrack.
template <int TAU, bool PACKED, int NP>
__device__ void vpx_dp_body(const KParams &kp, const Work &w, const VpxMem &S, int f, int vtop, bool staged)
{
    const int W = kp.W, H = kp.H, vmax = H - 1, chi = kp.chi, SR = kp.seg_rows;
    const int NPr = vpx_pairs(W), RB = vpx_row_bytes(W);
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr int NK = 2 * TAU + 1;
    int pen[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int t = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
        pen[k] = PACKED ? 16 * kp.lambda_x * (t < 0 ? -t : t) + k : kp.lambda_x * (t < 0 ? -t : t);
    }
    const uint32_t d0 = sa(S.D0), d1 = sa(S.D1), bt = sa(S.dyn);
    uint8_t *gbt = w.gbt + (size_t)f * w.max_h * vpx_row_bytes(w.max_w);
    // ---- counts of row vmax: the votes of rows [max(vtop, vmax - chi), vmax], gathered in D0 ----
    {
        const int r0 = kp.band_literal ? vmax : max(vtop, vmax - chi);   // the literal bottom band of row vmax is [vmax, vmax]
        if (staged) {
            for (int q = S.voff[r0] + tid; q < S.voff[vmax + 1]; q += nt)
                if (LD_IN(S.vb[q], W, CK_VPX_VOTE))
                    atoms_add(d0 + 4u * (uint32_t)S.vb[q], 1);
        } else {
            for (int r = r0; r <= vmax; ++r) {
                const VoteRow vr = vote_row(kp, w, S, f, r, staged);
                for (int q = tid; q < vr.n; q += nt)
                    if (LD_IN(vr.p[q], W, CK_VPX_VOTE))
                        atoms_add(d0 + 4u * (uint32_t)vr.p[q], 1);
            }
        }
    }
    __syncthreads();
    int band[NP][2];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int j = tid + p * nt;
        band[p][0] = band[p][1] = 0;
        if (j < NPr) {
            const int2 b2 = lds2(d0 + 8u * (uint32_t)j);
            band[p][0] = b2.x;
            band[p][1] = b2.y;
            sts2(d0 + 8u * (uint32_t)j, make_int2(0, 0));
            int e2[2];
#pragma unroll
            for (int c = 0; c < 2; ++c)
                e2[c] = 2 * j + c < W ? (PACKED ? 16 : 1) * -kp.vote_rho * band[p][c] : kSent;
            sts2(sa(S.E0) + 8u * (uint32_t)j, make_int2(e2[0], e2[1]));
            if (w.dbg_mx)
                store_mx(kp, w, f, vmax, 2 * j, band[p][0], band[p][1]);
        }
    }
    __syncthreads();
    int *Ep = S.E0, *Ec = S.E1;
    if (vmax - 1 >= vtop) {
        scatter_delta(kp, w, S, f, vmax - 1, vtop, staged, ((vmax - 1) & 1) ? d1 : d0, tid, nt);
        __syncthreads();
    }
    for (int v = vmax - 1; v >= vtop; --v) {
        if (v - 1 >= vtop) {
            if (staged && !kp.band_literal)
                scatter_staged(S, v - 1, ((v - 1) & 1) ? d1 : d0, W);
            else
                scatter_delta(kp, w, S, f, v - 1, vtop, staged, ((v - 1) & 1) ? d1 : d0, tid, nt);
        }
        const uint32_t dv = (v & 1) ? d1 : d0;
        const int r = v - vtop;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int j = tid + p * nt;
            if (j < NPr) {
                const int2 dl = lds2(dv + 8u * (uint32_t)j);
                sts2(dv + 8u * (uint32_t)j, make_int2(0, 0));
                band[p][0] += dl.x;
                band[p][1] += dl.y;
                if (w.dbg_mx)
                    store_mx(kp, w, f, v, 2 * j, band[p][0], band[p][1]);
                const uint32_t code = dp_pair<TAU, PACKED>(kp, 2 * j, band[p][0], band[p][1], pen, sa(Ep), sa(Ec));
                if (r < SR)
                    sts8(bt + (uint32_t)(r * RB + j), code);
                else
                    gbt[(size_t)v * RB + j] = (uint8_t)code;
            }
        }
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
    // ---- backtrack, one block of seg_rows rows at a time ----
    int u = ustar;
    for (int lo = vtop; lo <= vmax; lo += SR) {
        const int hi = min(lo + SR - 1, vmax - 1);
        if (lo > vtop) {
            // rows lo .. hi from the global buffer into shared memory (16-byte copies)
            __syncthreads();
            const int n16 = (hi - lo + 1) * (RB >> 4);
            const uint4 *src = reinterpret_cast<const uint4 *>(gbt + (size_t)lo * RB);
            uint4 *dst = reinterpret_cast<uint4 *>(S.dyn);
            for (int q = tid; q < n16; q += nt)
                dst[q] = src[q];
            __syncthreads();
        }
        if (tid == 0) {
            if (lo == vtop)
                S.path[vtop] = (int16_t)u;
            uint32_t rowa = bt;
            for (int v = lo; v <= hi; ++v, rowa += (uint32_t)RB) {
                if (LD_IN(u, W, CK_VPX_PATH))
                    u += bt_step(rowa, u, PACKED);
                S.path[v + 1] = (int16_t)u;
            }
        }
    }
    __syncthreads();
}

template <int TAU, int NP>
__device__ __forceinline__ void vpx_dp_kernel_body(const KParams &kp, const Work &w, const int f)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = kp.W, H = kp.H, NPr = vpx_pairs(W);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const FrameState fs0 = w.fs[f];
    if (fs0.flags & LD_F_NO_LANES)
        return;
    const int vtop = fs0.v_top, vmax = H - 1, chi = kp.chi;
    if (!LD_IN(vtop, H, CK_VPX_TILE))
        return;

    VpxMem S;
    unsigned char *p = smem;
    S.E0 = carve<int>(p, 2 * NPr + 2 * kPadX) + kPadX;
    S.E1 = carve<int>(p, 2 * NPr + 2 * kPadX) + kPadX;
    S.D0 = carve<int>(p, 2 * NPr);
    S.D1 = carve<int>(p, 2 * NPr);
    S.voff = carve<int>(p, H + 1);
    S.vb = carve<int16_t>(p, kp.vote_cap);
    S.path = carve<int16_t>(p, H);
    S.sup = carve<uint8_t>(p, H);
    S.sh = carve<int>(p, kMaxChunks + 64);
    S.pid = carve<int16_t>(p, H);
    S.rinfo = carve<int4>(p, H);
    S.dyn = carve<unsigned char>(p, 0);

    // ---- vote rows [vtop, vmax]: offsets by a block scan, staged in shared memory when they fit ----
    for (int v = tid; v < H; v += nt) {
        const int c = v >= vtop ? w.vcount[(size_t)f * H + v] : 0;
        S.voff[v] = LD_IN(c, W + 1, CK_VPX_VOFF) ? c : 0;   // a row holds at most W votes
    }
    for (int u = tid; u < 2 * NPr; u += nt) {
        S.D0[u] = 0;
        S.D1[u] = 0;
    }
    for (int u = tid - kPadX; u < 2 * NPr + kPadX; u += nt)
        if (u < 0 || u >= W) {
            S.E0[u] = kSent;
            S.E1[u] = kSent;
        }
    __syncthreads();
    block_scan(S.voff, H, S.sh);
    const int votes = S.voff[H];
    const bool staged = votes <= kp.vote_cap;
    if (staged) {
        // every thread takes votes q = tid + k nt; its rows come from a binary search over the offsets,
        // kStageBatch searches and loads in flight at once
        constexpr int kStageBatch = 8;
        for (int q0 = 0; q0 < votes; q0 += kStageBatch * nt) {
            int16_t val[kStageBatch];
#pragma unroll
            for (int k = 0; k < kStageBatch; ++k) {
                const int q = q0 + k * nt + tid;
                val[k] = 0;
                if (q < votes) {
                    int lo = vtop, hi = vmax + 1;  // voff[lo] <= q < voff[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (S.voff[mid] <= q)
                            lo = mid;
                        else
                            hi = mid;
                    }
                    if (LD_IN(q - S.voff[lo], W, CK_VPX_STAGE) && LD_IN(q, kp.vote_cap, CK_VPX_STAGE))
                        val[k] = __ldg(w.vbins + ((size_t)f * H + lo) * W + (q - S.voff[lo]));
                }
            }
#pragma unroll
            for (int k = 0; k < kStageBatch; ++k) {
                const int q = q0 + k * nt + tid;
                if (q < votes)
                    S.vb[q] = val[k];
            }
        }
    }
    // per DP row v the staged votes entering (row v - chi) and leaving (row v + chi + 1) the band
    if (staged && !kp.band_literal)
        for (int v = tid; v < H; v += nt) {
            int4 ri = make_int4(0, 0, 0, 0);
            if (v - chi >= vtop && v - chi <= vmax) {
                ri.x = S.voff[v - chi];
                ri.y = S.voff[v - chi + 1] - ri.x;
            }
            if (v + chi + 1 <= vmax && v + chi + 1 >= vtop) {
                ri.z = S.voff[v + chi + 1];
                ri.w = S.voff[v + chi + 2] - ri.z;
            }
            S.rinfo[v] = ri;
        }
    __syncthreads();
    // each vote enters at most 2 chi + 1 band rows, so |E| <= varrho (2 chi + 1) votes + lambda_x tau_x rows
    const bool packed = ((double)kp.vote_rho * (2.0 * chi + 1.0) * votes + (double)kp.lambda_x * kp.tau_x * H) * 16.0 <
                        536870912.0;
    if (packed)
        vpx_dp_body<TAU, true, NP>(kp, w, S, f, vtop, staged);
    else
        vpx_dp_body<TAU, false, NP>(kp, w, S, f, vtop, staged);

    // ---- rows whose path cell holds votes: a vote of rows [v - chi, v + chi] in column u_v ----
    // Column bitmaps of the vote rows (bit r - rb of column u), in the space the backtrack rows used, built
    // for blocks of B path rows at a time (a block needs the vote rows [R0 - chi, R1 + chi)).
    uint32_t *cb = reinterpret_cast<uint32_t *>(S.dyn);
    const int words = (int)(((size_t)kp.seg_rows * vpx_row_bytes(W)) / (4 * (size_t)W));
    const int B = max(32, (words * 32 - 2 * chi - 32) / 32 * 32);
    for (int R0 = vtop; R0 <= vmax; R0 += B) {
        const int R1 = min(R0 + B, vmax + 1), rb = R0 - chi;
        const int HB = (R1 + chi - rb + 31) >> 5;
        for (int j = tid; j < W * HB; j += nt)
            cb[j] = 0u;
        __syncthreads();
        const int rlo = max(vtop, R0 - chi), rhi = min(vmax, R1 - 1 + chi);
        for (int r0 = rlo + 4 * warp; r0 <= rhi; r0 += 4 * nw) {
            const int r = r0 + (lane >> 3);
            if (r <= rhi) {
                const VoteRow vr = vote_row(kp, w, S, f, r, staged);
                for (int q = lane & 7; q < vr.n; q += 8)
                    if (LD_IN(vr.p[q], W, CK_VPX_VOTE))
                        atoms_or(sa(cb + (size_t)vr.p[q] * HB + ((r - rb) >> 5)), 1u << ((r - rb) & 31));
            }
        }
        __syncthreads();
        for (int v = R0 + tid; v < R1; v += nt) {
            if (!LD_IN(S.path[v], W, CK_VPX_PATH)) {
                S.sup[v] = 0;
                continue;
            }
            const uint32_t *col = cb + (size_t)S.path[v] * HB;
            const int lo = (kp.band_literal && v > vmax - chi - 1 ? v : max(vtop, v - chi)) - rb, hi = min(vmax, v + chi) - rb;
            uint8_t sp = 0;
            for (int wd = lo >> 5; wd <= hi >> 5; ++wd) {
                uint32_t m = col[wd];
                if (wd == lo >> 5)
                    m &= 0xffffffffu << (lo & 31);
                if (wd == hi >> 5)
                    m &= 0xffffffffu >> (31 - (hi & 31));
                sp |= m != 0u;
            }
            S.sup[v] = sp;
        }
        __syncthreads();
    }
    for (int v = tid; v < vtop; v += nt)
        S.sup[v] = 0;
    __syncthreads();
    const int t = vmax - vtop + 1;
    const int k = block_compact(S.sup + vtop, t, S.pid, S.sh);
    int16_t *gp = w.pts + ((size_t)f * 2 + 1) * 3 * w.pmax;
    for (int j = tid; j < k; j += nt)
        if (LD_IN(j, w.pmax, CK_VPX_PTS) && LD_IN(S.pid[j], t, CK_VPX_PTS)) {
            gp[j] = (int16_t)(vtop + S.pid[j]);
            gp[w.pmax + j] = S.path[vtop + S.pid[j]];
            gp[2 * w.pmax + j] = (int16_t)(vtop + S.pid[j]);
        }
    for (int v = tid; v < H; v += nt)
        w.path_x[(size_t)f * H + v] = v >= vtop ? S.path[v] : (int16_t)0;
    if (tid == 0)
        w.npts[f * 2 + 1] = k;
}

template <int TAU, int NP>
__global__ void __launch_bounds__(1024) k_vpx_dp(const KParams kp, const Work w) { vpx_dp_kernel_body<TAU, NP>(kp, w, blockIdx.x); }
template <int TAU, int NP>
__global__ void __launch_bounds__(1024) k_vpx_dp_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.x];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    vpx_dp_kernel_body<TAU, NP>(kp, w, 0);
}

// Threads: one per cell pair up to 1024 (two pairs per thread past 2048 columns).
int vpx_np(int W) { return vpx_pairs(W) > 1024 ? 2 : 1; }
int vpx_threads(int W)
{
    const int np = vpx_np(W);
    int nt = ((vpx_pairs(W) + np - 1) / np + 31) / 32 * 32;
    return nt < 64 ? 64 : nt > 1024 ? 1024 : nt;
}

size_t vpx_fixed_bytes(const KParams &kp)
{
    const size_t W = kp.W, H = kp.H, NPr = vpx_pairs(kp.W);
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * (2 * NPr + 2 * kPadX));
    add(4 * (2 * NPr + 2 * kPadX));
    add(4 * 2 * NPr);
    add(4 * 2 * NPr);
    add(4 * (H + 1));
    add(2 * (size_t)kp.vote_cap);
    add(2 * H);
    add(H);
    add(4 * (kMaxChunks + 64));
    add(2 * H);
    add(16 * H);
    (void)W;
    return ((s + 15) & ~(size_t)15) + 64;
}

// Bytes of the reusable region: the backtrack rows, later the column bitmaps of blocks of vote rows.
size_t vpx_dyn_bytes(const KParams &kp) { return (size_t)kp.seg_rows * vpx_row_bytes(kp.W); }

// Words per column the bitmaps of a block of 32 path rows need: 32 + 2 chi rows, one word of alignment.
size_t vpx_min_dyn_bytes(const KParams &kp) { return (size_t)4 * kp.W * ((32 + 2 * kp.chi + 32 + 31) / 32 + 1); }

using VpxKernel = void (*)(KParams, Work);
template <int NP>
VpxKernel vpx_kernel_np(int tau)
{
    switch (tau) {
    case 0: return k_vpx_dp<0, NP>;
    case 1: return k_vpx_dp<1, NP>;
    case 2: return k_vpx_dp<2, NP>;
    case 3: return k_vpx_dp<3, NP>;
    case 4: return k_vpx_dp<4, NP>;
    case 5: return k_vpx_dp<5, NP>;
    case 6: return k_vpx_dp<6, NP>;
    default: return k_vpx_dp<7, NP>;
    }
}
VpxKernel vpx_kernel(int tau, int W) { return vpx_np(W) == 2 ? vpx_kernel_np<2>(tau) : vpx_kernel_np<1>(tau); }

using VpxKernelFd = void (*)(const FrameDesc *);
template <int NP>
VpxKernelFd vpx_kernel_fd_np(int tau)
{
    switch (tau) {
    case 0: return k_vpx_dp_fd<0, NP>;
    case 1: return k_vpx_dp_fd<1, NP>;
    case 2: return k_vpx_dp_fd<2, NP>;
    case 3: return k_vpx_dp_fd<3, NP>;
    case 4: return k_vpx_dp_fd<4, NP>;
    case 5: return k_vpx_dp_fd<5, NP>;
    case 6: return k_vpx_dp_fd<6, NP>;
    default: return k_vpx_dp_fd<7, NP>;
    }
}
VpxKernelFd vpx_kernel_fd(int tau, int W) { return vpx_np(W) == 2 ? vpx_kernel_fd_np<2>(tau) : vpx_kernel_fd_np<1>(tau); }

using RoadKernel = void (*)(KParams, Work);
RoadKernel road_kernel(int tau) { return tau <= 6 ? k_road_dp<6> : k_road_dp<15>; }

}  // namespace

size_t road_smem_bytes(const KParams &kp)
{
    const size_t H = kp.H, D = kp.D, Hp = (H + 1) / 2;
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * (2 * Hp + kPadY));
    add(4 * (2 * Hp + kPadY));
    add(4 * (kMaxChunks + 64));
    add(2 * D);
    add(D);
    add(2 * D);
    add(D * Hp);
    return s + 64;
}

// One thread per pair of rows (at least two warps).
int road_threads(int H)
{
    const int nt = ((H + 1) / 2 + 31) / 32 * 32;
    return nt < 64 ? 64 : nt;
}

size_t vpx_smem_bytes(const KParams &kp) { return vpx_fixed_bytes(kp) + vpx_dyn_bytes(kp); }

int vpx_seg_rows(const KParams &kp, size_t budget)
{
    const size_t fixed = vpx_fixed_bytes(kp);
    if (budget <= fixed + vpx_min_dyn_bytes(kp))
        return 0;
    return (int)((budget - fixed) / vpx_row_bytes(kp.W));
}

cudaError_t setup_dp(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_road_dp<6>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_road_dp_lit, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_road_dp<15>, smem_optin);
    for (int t = 0; t <= 7 && e == cudaSuccess; ++t) {
        e = allow_max_smem(vpx_kernel_np<1>(t), smem_optin);
        if (e == cudaSuccess)
            e = allow_max_smem(vpx_kernel_np<2>(t), smem_optin);
        if (e == cudaSuccess)
            e = allow_max_smem(vpx_kernel_fd_np<1>(t), smem_optin);
        if (e == cudaSuccess)
            e = allow_max_smem(vpx_kernel_fd_np<2>(t), smem_optin);
    }
    if (e == cudaSuccess)
        e = allow_max_smem(k_road_dp_fd<6>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_road_dp_fd<15>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_road_dp_lit_fd, smem_optin);
    return e;
}

cudaError_t launch_road(const KParams &kp, const Work &w, cudaStream_t s)
{
    if (kp.dp_literal)
        k_road_dp_lit<<<kp.n_frames, road_threads(kp.H), road_smem_bytes(kp), s>>>(kp, w);
    else
        road_kernel(kp.tau_y)<<<kp.n_frames, road_threads(kp.H), road_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

cudaError_t launch_road_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    if (kmax.dp_literal)
        k_road_dp_lit_fd<<<n, road_threads(kmax.H), road_smem_bytes(kmax), s>>>(fd);
    else if (kmax.tau_y <= 6)
        k_road_dp_fd<6><<<n, road_threads(kmax.H), road_smem_bytes(kmax), s>>>(fd);
    else
        k_road_dp_fd<15><<<n, road_threads(kmax.H), road_smem_bytes(kmax), s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_vpx_fd(const KParams &kmax, const FrameDesc *fd, int n, size_t smem, cudaStream_t s)
{
    vpx_kernel_fd(kmax.tau_x, kmax.W)<<<n, vpx_threads(kmax.W), smem, s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_vpx(const KParams &kp, const Work &w, cudaStream_t s)
{
    vpx_kernel(kp.tau_x, kp.W)<<<kp.n_frames, vpx_threads(kp.W), vpx_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

}  // namespace ld
