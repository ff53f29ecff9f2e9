// Sec. 2.3.1: road mask, bilateral filter (Eq. 15-16), Sobel gradients, edge test and sparse V_px votes
// (Eq. 17), for the road rows of every frame.
//
// Road pixels whose neighbourhood is provably too flat to pass the edge test are dropped first (an exact
// pruning, below): on the 1242x375 workload about three quarters of the bilateral work goes with them.
//
// One CTA covers R output rows of one frame across the full width.  It stages the image rows the
// (2 rho + 1)^2 window needs in shared memory, with a sentinel value outside the frame whose range weight
// is 0 (this is the clipped window of Eq. 15).  The bilateral output is computed only at pixels whose
// 3x3 neighbourhood holds an interior road pixel: those are the only values the Sobel stencil and the edge
// test read (Sec. 2.3.1 keeps only the road surface).  Weights are Q15 integers,
// w = (ws * wr[|I(i,j) - I(u,v)|] + 2^14) >> 15, sums are exact, and the output is
// (2 sum(w I) + sum(w)) / (2 sum(w)), so the result does not depend on the order of the taps.
//
// GB300 mapping of the bilateral (the cost of the whole path sits here):
//   - taps at equal distance share ws and the range weight depends on |I(i,j) - I(u,v)| only, so w depends
//     on (distance class, |dI|); the CTA builds one 512-entry uint16 table per class in shared memory and
//     a tap costs one absolute-difference-add (__usad), one table load and two 32-bit accumulations
//     (sum(w) and sum(w 2 I) on separate pipes).  Indexing by |dI| halves the banks the common small
//     differences occupy, which cuts the data-dependent bank conflicts of the lookups;
//   - the tile stores 2 I (a byte offset into a table), so the table address is base_c + |2 I(i,j) - 2 I(u,v)|
//     with a compile-time class offset, and sum(w 2 I) keeps the same exact arithmetic; the sentinel 2 x 511
//     outside the frame lands in the zero half of every table;
//   - a thread filters 4 horizontally adjacent pixels, sharing each window row it loads as 64-bit vectors;
//   - pixel groups that need the filter are compacted first, so warps do not diverge on the road mask.
// Staging: the image rows of a CTA (and its disparity rows) are one contiguous range of global memory,
// read with 16-byte loads that each thread issues before it uses any of them; the weight tables are
// built from registers while those loads are in flight.
//
// Each road pixel with G_x^2 + G_y^2 > thr^2 is an edge pixel.  Its vote column is
// floor(u + (v - V_py(v)) G_y / G_x + 0.5) in float32 (the line through the pixel perpendicular to the
// gradient meets row V_py there), kept when inside [0, W).  Edge pixels and votes are appended to per-row
// lists (order within a row is arbitrary; every consumer sums over them).
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kThreads = 1024;
constexpr int kTabEntries = 512;           // T_c[|dI|]: |dI| <= 255, zero from 256 on (where the sentinel lands)
constexpr int kTabBytes = kTabEntries * 2;  // one uint16 table per distance class

// Distance class of every tap (rank of dx^2 + dy^2 among the distinct values of the window), as byte
// offsets of the class tables; a compile-time table, so an unrolled tap loop folds them into the loads.
template <int RHO>
__host__ __device__ constexpr int cls_rank(int d2)
{
    int r = 0;
    for (int s = 0; s < d2; ++s) {
        bool seen = false;
        for (int dy = 0; dy <= RHO; ++dy)
            for (int dx = 0; dx <= RHO; ++dx)
                if (dx * dx + dy * dy == s)
                    seen = true;
        r += seen ? 1 : 0;
    }
    return r;
}
template <int RHO>
struct ClsOffsets {
    int v[(2 * RHO + 1) * (2 * RHO + 1)];
};
template <int RHO>
__host__ __device__ constexpr ClsOffsets<RHO> make_cls_offsets()
{
    ClsOffsets<RHO> o{};
    for (int dy = 0; dy <= 2 * RHO; ++dy)
        for (int dx = 0; dx <= 2 * RHO; ++dx)
            o.v[dy * (2 * RHO + 1) + dx] = cls_rank<RHO>((dy - RHO) * (dy - RHO) + (dx - RHO) * (dx - RHO)) * kTabBytes;
    return o;
}
constexpr int kLoadsImg = 2, kLoadsDisp = 3;  // 16-byte staging loads per thread and pass
static_assert(kThreads >= kTabEntries, "one thread per table entry builds the class tables");

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t lds_u16(uint32_t addr)
{
    uint16_t v;
    asm("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}

struct GradLayout {
    int TWP, IW, NG, TR, BR;
};

template <int RHO>
__host__ __device__ inline GradLayout grad_layout(int W, int nr)
{
    constexpr int NL = (4 + 2 * RHO + 3) / 4;  // 4-value loads per window row of a 4-pixel group
    GradLayout L;
    L.IW = (W + 3) & ~3;
    L.TWP = L.IW + 4 * NL;
    L.NG = L.IW / 4;
    L.TR = nr + 2 + 2 * RHO;
    L.BR = nr + 2;
    return L;
}

// Bilateral output of the 4 pixels (br, u0 .. u0+3); tile holds 2 I with the sentinel outside the frame.
// sum(w) <= 121 * 2^15 and sum(w 2 I) <= 121 * 2^15 * 510 < 2^31 both fit 32-bit accumulators.
template <int RHO>
__device__ __forceinline__ uint32_t bilateral4(const KParams &kp, const uint16_t *tile, int TWP, int br, int u0, int W,
                                               uint32_t tab)
{
    constexpr int N = 2 * RHO + 1;
    constexpr int NL = (4 + 2 * RHO + 3) / 4;
    const uint16_t *crow = tile + (size_t)(br + RHO) * TWP + u0 + RHO;
    uint32_t base[4], sw[4], swi[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t c2 = (u0 + p < W) ? crow[p] : 0u;  // pixels past the right edge: any valid index
        base[p] = c2;
        sw[p] = 0u;
        swi[p] = 0u;
    }
#pragma unroll
    for (int dy = 0; dy < N; ++dy) {
        const uint2 *rowp = reinterpret_cast<const uint2 *>(tile + (size_t)(br + dy) * TWP + u0);
        uint32_t q[4 * NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const uint2 v = rowp[l];
            q[4 * l] = __byte_perm(v.x, 0u, 0x4410);
            q[4 * l + 1] = __byte_perm(v.x, 0u, 0x4432);
            q[4 * l + 2] = __byte_perm(v.y, 0u, 0x4410);
            q[4 * l + 3] = __byte_perm(v.y, 0u, 0x4432);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int dx = 0; dx < N; ++dx) {
                const uint32_t qq = q[p + dx];
                constexpr ClsOffsets<RHO> kOff = make_cls_offsets<RHO>();
                const uint32_t wq = lds_u16(__usad(qq, base[p], tab) + (uint32_t)kOff.v[dy * N + dx]);
                sw[p] += wq;
                swi[p] += wq * qq;
            }
        }
    }
    uint32_t out = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t b = sw[p] ? (swi[p] + sw[p]) / (2u * sw[p]) : 0u;  // (2 sum(wI) + sum(w)) / (2 sum(w))
        out |= (b & 0xffu) << (8 * p);
    }
    return out;
}

template <int RHO>
__global__ void __launch_bounds__(kThreads, 1) k_grad(const KParams kp, const Work w, const float *__restrict__ disp,
                                                      const uint8_t *__restrict__ img, int R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = kThreads / 32;
    const int W = kp.W, H = kp.H;
    const int f = blockIdx.y;
    const int r0 = blockIdx.x * R;
    const int nr = min(R, H - r0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FrameState &fs = w.fs[f];
    const int vtop = fs.v_top;
    int32_t *ecnt = w.ecount + (size_t)f * H;
    int32_t *vcnt = w.vcount + (size_t)f * H;
    if ((fs.flags & LD_F_NO_LANES) || r0 + nr - 1 < vtop) {
        for (int r = tid; r < nr; r += kThreads) {
            ecnt[r0 + r] = 0;
            vcnt[r0 + r] = 0;
        }
        return;
    }
    const GradLayout L = grad_layout<RHO>(W, R);
    const int TR = nr + 2 + 2 * RHO, BR = nr + 2;

    unsigned char *p = smem;
    uint16_t *tabs = reinterpret_cast<uint16_t *>(p);           // [n_cls][512]
    p += (size_t)kTabBytes * kp.n_cls;
    int32_t *cnt = reinterpret_cast<int32_t *>(p);              // [2][R] edges, votes per row; [2R] groups
    p += sizeof(int32_t) * (2 * R + 4);
    float *rowF = reinterpret_cast<float *>(p);
    p += sizeof(float) * R;
    float *rowVy = reinterpret_cast<float *>(p);
    p += sizeof(float) * R;
    p = reinterpret_cast<unsigned char *>(((size_t)p + 15) & ~(size_t)15);
    uint16_t *tile = reinterpret_cast<uint16_t *>(p);           // [TR][TWP] 2 I, or 2 x sentinel
    p += sizeof(uint16_t) * (size_t)L.TR * L.TWP;
    uint8_t *ibf = p;                                           // [BR][IW] bilateral output, row br = v - r0 + 1
    p += (size_t)L.BR * L.IW;
    uint8_t *road = p;                                          // [R][IW]
    p += (size_t)R * L.IW;
    p = reinterpret_cast<unsigned char *>(((size_t)p + 15) & ~(size_t)15);
    uint16_t *glist = reinterpret_cast<uint16_t *>(p);          // [BR * NG] groups that need the filter

    // ---- staging.  The in-frame image rows [va, vb) and the disparity rows [r0, r0 + nr) are contiguous in
    // global memory; each is read as 16-byte loads of the aligned chunks inside it plus single loads of
    // its head and tail.  Every global load of this phase is issued before any is used.
    const float *rows = w.rows + (size_t)f * 3 * H;
    const int va = max(r0 - 1 - RHO, 0), vb = min(r0 + nr + RHO + 1, H);
    const uint8_t *gs = img + ((size_t)f * H + va) * W;
    const int nbytes = (vb - va) * W;
    uint16_t *tdst = tile + (size_t)(va - (r0 - 1 - RHO)) * L.TWP + RHO;  // tile cell of pixel (va, 0)
    const int headI = min((int)((16u - ((uint32_t)(uintptr_t)gs & 15u)) & 15u), nbytes);
    const int nI = (nbytes - headI) >> 4, tailI = headI + 16 * nI;
    const uint4 *bodyI = reinterpret_cast<const uint4 *>(gs + headI);
    const float *ds = disp + ((size_t)f * H + r0) * W;
    const int nel = nr * W;
    const int headD = min((int)(((16u - ((uint32_t)(uintptr_t)ds & 15u)) & 15u) >> 2), nel);
    const int nD = (nel - headD) >> 2, tailD = headD + 4 * nD;
    const float4 *bodyD = reinterpret_cast<const float4 *>(ds + headD);
    const int nsI = headI + nbytes - tailI, nsD = headD + nel - tailD;  // single loads (at most 30 and 6)
    const int ooI = tid < headI ? tid : tailI + (tid - headI);
    const int ooD = tid < headD ? tid : tailD + (tid - headD);

    const uint32_t wrk = tid < 256 ? (uint32_t)__ldg(w.wr + 256 + tid) : 0u;  // Q15 wr(|dI|)
    const float fr = tid < nr ? __ldg(rows + r0 + tid) : 0.0f;
    const float vyr = tid < nr ? __ldg(rows + H + r0 + tid) : 0.0f;
    const uint32_t bI = tid < nsI ? (uint32_t)__ldg(gs + ooI) : 0u;
    const float lD = tid < nsD ? __ldg(ds + ooD) : 0.0f;
    uint4 xi[kLoadsImg];
    float4 xd[kLoadsDisp];
#pragma unroll
    for (int k = 0; k < kLoadsImg; ++k)
        if (k * kThreads + tid < nI)
            xi[k] = __ldg(bodyI + k * kThreads + tid);
#pragma unroll
    for (int k = 0; k < kLoadsDisp; ++k)
        if (k * kThreads + tid < nD)
            xd[k] = __ldg(bodyD + k * kThreads + tid);

    // per-class weight tables T_c[a] = (ws_c * wr(a) + 2^14) >> 15 for a = |I(i,j) - I(u,v)|, one thread per a
    if (tid < kTabEntries)
        for (int c = 0; c < kp.n_cls; ++c)
            tabs[c * kTabEntries + tid] = (uint16_t)(((uint32_t)kp.cls_ws[c] * wrk + 16384u) >> 15);
    for (int i = tid; i < 2 * R + 4; i += kThreads)
        cnt[i] = 0;
    if (tid < nr) {
        // rows that hold no interior road pixel get f(v) = NaN, which fails the on-road test below
        const int v = r0 + tid;
        rowF[tid] = (v >= vtop && v >= 1 && v <= H - 2) ? fr : __int_as_float(0x7fc00000);
        rowVy[tid] = vyr;
    }
    for (int tr = warp; tr < TR; tr += NW) {
        const int v = r0 - 1 - RHO + tr;
        uint16_t *dst = tile + (size_t)tr * L.TWP;
        if (v < 0 || v >= H) {
            for (int tc = lane; tc < L.TWP; tc += 32)
                dst[tc] = (uint16_t)(2 * kSentinel);
        } else {
            for (int t = lane; t < L.TWP - W; t += 32)  // pad columns [0, rho) and [W + rho, TWP)
                dst[t < RHO ? t : W + t] = (uint16_t)(2 * kSentinel);
        }
    }
    for (int i = tid; i < nr * (L.IW - W); i += kThreads) {
        const int r = i / (L.IW - W);
        road[(size_t)r * L.IW + W + (i - r * (L.IW - W))] = 0;
    }
    __syncthreads();  // rowF

    // road mask of the interior pixels: l > 0 with |l - f(v)| <= varpi (an infinite or NaN l fails the
    // second test because f(v) is finite), v >= v_top, 1 <= u <= W-2
    auto mask = [&](int row, int col, float l) {
        const bool m = l > 0.0f && fabsf(__fsub_rn(l, rowF[row])) <= kp.varpi && col >= 1 && col <= W - 2;
        road[(size_t)row * L.IW + col] = (uint8_t)m;
    };
    if (tid < nsI) {
        const int row = ooI / W;
        tdst[row * L.TWP + ooI - row * W] = (uint16_t)(2u * bI);
    }
    if (tid < nsD) {
        const int row = ooD / W;
        mask(row, ooD - row * W, lD);
    }
    for (int pass = 0; pass * kLoadsImg * kThreads < nI || pass * kLoadsDisp * kThreads < nD; ++pass) {
        if (pass > 0) {
#pragma unroll
            for (int k = 0; k < kLoadsImg; ++k) {
                const int i = (pass * kLoadsImg + k) * kThreads + tid;
                if (i < nI)
                    xi[k] = __ldg(bodyI + i);
            }
#pragma unroll
            for (int k = 0; k < kLoadsDisp; ++k) {
                const int i = (pass * kLoadsDisp + k) * kThreads + tid;
                if (i < nD)
                    xd[k] = __ldg(bodyD + i);
            }
        }
#pragma unroll
        for (int k = 0; k < kLoadsImg; ++k) {
            const int i = (pass * kLoadsImg + k) * kThreads + tid;
            if (i < nI) {
                const uint32_t wv[4] = {xi[k].x, xi[k].y, xi[k].z, xi[k].w};
                const int off = headI + 16 * i;
                int row = off / W, col = off - row * W;
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    tdst[row * L.TWP + col] = (uint16_t)(2u * ((wv[b >> 2] >> (8 * (b & 3))) & 0xffu));
                    if (++col == W) {
                        col = 0;
                        ++row;
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kLoadsDisp; ++k) {
            const int i = (pass * kLoadsDisp + k) * kThreads + tid;
            if (i < nD) {
                const float xv[4] = {xd[k].x, xd[k].y, xd[k].z, xd[k].w};
                const int off = headD + 4 * i;
                int row = off / W, col = off - row * W;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    mask(row, col, xv[b]);
                    if (++col == W) {
                        col = 0;
                        ++row;
                    }
                }
            }
        }
    }
    __syncthreads();
    // Exact pruning: a group of 4 road pixels whose neighbourhood (the 3x3 neighbours' windows: columns
    // 4j - rho - 1 .. 4j + 4 + rho, rows v - rho - 1 .. v + rho + 1) spans an image range of at most
    // kp.flat_range cannot hold an edge pixel, whatever the values (the bound is derived and computed on
    // the host, flat_range()), so it leaves the road mask: neither its Sobel nor the bilateral outputs only
    // it would read are computed, and every edge, G and vote stays as the full computation gives them.  The
    // test reads a superset of that neighbourhood: columns 4j - rho - 4 .. 4j + rho + 5 (aligned 8-byte
    // loads of the tile).  Any tap outside the frame holds the sentinel, which makes the range too large.
    // Horizontal pass: per tile row and group, (min I, max I) packed in 16 bits, in the bilateral-output
    // buffer (written only later); vertical pass: the 2 rho + 3 rows of every output row.
    if (kp.flat_range >= 0 && TR <= 2 * BR) {
        constexpr int NLF = (2 * RHO + 10 + 3) / 4;      // 8-byte loads per tile row of a group's test region
        uint16_t *hr = reinterpret_cast<uint16_t *>(ibf);  // [TR][NG]
        for (int i = tid; i < TR * L.NG; i += kThreads) {
            const int tr = i / L.NG, j = i - tr * L.NG;
            uint32_t h = 0xff00u;                          // (min 0, max 255): never flat
            if (j >= 1) {
                const uint2 *src = reinterpret_cast<const uint2 *>(tile + (size_t)tr * L.TWP + 4 * j - 4);
                uint32_t vmn = 0xffffffffu, vmx = 0u;
#pragma unroll
                for (int l = 0; l < NLF; ++l) {
                    const uint2 v = src[l];
                    vmn = __vminu2(vmn, __vminu2(v.x, v.y));
                    vmx = __vmaxu2(vmx, __vmaxu2(v.x, v.y));
                }
                const uint32_t mn2 = min(vmn & 0xffffu, vmn >> 16), mx2 = max(vmx & 0xffffu, vmx >> 16);  // 2 I
                if (mx2 <= 510u)
                    h = (mn2 >> 1) | ((mx2 >> 1) << 8);
            }
            hr[i] = (uint16_t)h;
        }
        __syncthreads();
        for (int i = tid; i < nr * L.NG; i += kThreads) {
            const int r = i / L.NG, j = i - r * L.NG;
            uint32_t mn = 255u, mx = 0u;
#pragma unroll
            for (int t = 0; t < 2 * RHO + 3; ++t) {
                const uint32_t h = hr[(size_t)(r + t) * L.NG + j];
                mn = min(mn, h & 0xffu);
                mx = max(mx, h >> 8);
            }
            if ((int)(mx - mn) <= kp.flat_range)
                reinterpret_cast<uint32_t *>(road + (size_t)r * L.IW)[j] = 0u;
        }
        __syncthreads();
    }
    // groups of 4 pixels of the bilateral rows (r0-1 .. r0+nr) holding a pixel the Sobel stencil reads
    for (int br = warp; br < BR; br += NW) {
        for (int j0 = 0; j0 < L.NG; j0 += 32) {
            const int j = j0 + lane;
            bool need = false;
            if (j < L.NG) {
#pragma unroll
                for (int dr = -1; dr <= 1; ++dr) {
                    const int rr = br - 1 + dr;
                    if (rr < 0 || rr >= nr)
                        continue;
                    const uint32_t *rm = reinterpret_cast<const uint32_t *>(road + (size_t)rr * L.IW) + j;
                    const uint32_t left = j > 0 ? rm[-1] >> 24 : 0u;
                    const uint32_t right = j + 1 < L.NG ? rm[1] & 0xffu : 0u;
                    need |= (left | rm[0] | right) != 0u;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, need);
            int base = 0;
            if (lane == 0 && m)
                base = atomicAdd(&cnt[2 * R], __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (need)
                glist[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(br * L.NG + j);
        }
    }
    __syncthreads();
    const int ng = cnt[2 * R];
    const uint32_t tab = smem_addr(tabs);
    for (int k = tid; k < ng; k += kThreads) {
        const int g = glist[k];
        const int br = g / L.NG, u0 = 4 * (g - br * L.NG);
        uint32_t out;
        if (kp.bilateral) {
            out = bilateral4<RHO>(kp, tile, L.TWP, br, u0, W, tab);
        } else {
            const uint16_t *c = tile + (size_t)(br + RHO) * L.TWP + u0 + RHO;
            out = (uint32_t)(c[0] >> 1) | ((uint32_t)(c[1] >> 1) << 8) | ((uint32_t)(c[2] >> 1) << 16) |
                  ((uint32_t)(c[3] >> 1) << 24);
        }
        *reinterpret_cast<uint32_t *>(ibf + (size_t)br * L.IW + u0) = out;
        const int v = r0 - 1 + br;
        if (w.dbg_ibf && v >= 0 && v < H) {   // stage capture: the values this CTA computed (halo rows too)
            int16_t *drow = w.dbg_ibf + ((size_t)f * H + v) * W;
            for (int q = 0; q < 4 && u0 + q < W; ++q)
                drow[u0 + q] = (int16_t)((out >> (8 * q)) & 0xffu);
        }
    }
    __syncthreads();

    // Sobel, edge test, votes
    const int thr2 = kp.edge_thresh2;
    int16_t *edges = w.edges + (size_t)f * H * W * 4;
    int16_t *vbins = w.vbins + (size_t)f * H * W;
    // one thread per group of 4 pixels: 32-bit loads of the mask and of the three bilateral rows
    for (int k = tid; k < nr * L.NG; k += kThreads) {
        const int r = k / L.NG, j = k - r * L.NG;
        const uint32_t m4 = reinterpret_cast<const uint32_t *>(road + (size_t)r * L.IW)[j];
        if (!m4)
            continue;
        const int v = r0 + r;
        uint32_t x0[3], x1[3], x2[3];  // bytes 4j-4 .. 4j-1, 4j .. 4j+3, 4j+4 .. 4j+7 of rows v-1, v, v+1
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const uint32_t *rw = reinterpret_cast<const uint32_t *>(ibf + (size_t)(r + d) * L.IW);
            x0[d] = j > 0 ? rw[j - 1] : 0u;
            x1[d] = rw[j];
            x2[d] = j + 1 < L.NG ? rw[j + 1] : 0u;
        }
        const float vy = rowVy[r];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (!((m4 >> (8 * p)) & 0xffu))
                continue;
            const int u = 4 * j + p;
            int lf[3], cn[3], rt[3];  // I(u-1), I(u), I(u+1) of rows v-1, v, v+1
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lf[d] = p == 0 ? (int)(x0[d] >> 24) : (int)((x1[d] >> (8 * (p - 1))) & 0xffu);
                cn[d] = (int)((x1[d] >> (8 * p)) & 0xffu);
                rt[d] = p == 3 ? (int)(x2[d] & 0xffu) : (int)((x1[d] >> (8 * (p + 1))) & 0xffu);
            }
            const int gx = (rt[0] - lf[0]) + 2 * (rt[1] - lf[1]) + (rt[2] - lf[2]);
            const int gy = (lf[2] - lf[0]) + 2 * (cn[2] - cn[0]) + (rt[2] - rt[0]);
            if (gx * gx + gy * gy <= thr2)
                continue;
            int bin = -1;
            if (gx != 0) {
                const float av = __fsub_rn((float)v, vy);
                const float bv = __fmul_rn(av, (float)gy);
                const float qv = __fdiv_rn(bv, (float)gx);
                const float vs = __fadd_rn((float)u, qv);
                const float col = floorf(__fadd_rn(vs, 0.5f));
                if (col >= 0.0f && col < (float)W)
                    bin = (int)col;
            }
            const int pe = atomicAdd(&cnt[r], 1);
            const short4 e = make_short4((short)u, (short)bin, (short)gx, (short)gy);
            *reinterpret_cast<short4 *>(edges + ((size_t)v * W + pe) * 4) = e;
            if (bin >= 0) {
                const int pv = atomicAdd(&cnt[R + r], 1);
                vbins[(size_t)v * W + pv] = (int16_t)bin;
            }
        }
    }
    __syncthreads();
    for (int r = tid; r < nr; r += kThreads) {
        ecnt[r0 + r] = cnt[r];
        vcnt[r0 + r] = cnt[R + r];
    }
}

template <int RHO>
size_t grad_smem(int W, int R, int n_cls)
{
    const GradLayout L = grad_layout<RHO>(W, R);
    size_t s = (size_t)kTabBytes * n_cls + sizeof(int32_t) * (2 * R + 4) + 2 * sizeof(float) * R;
    s = (s + 15) & ~(size_t)15;
    s += sizeof(uint16_t) * (size_t)L.TR * L.TWP + (size_t)L.BR * L.IW + (size_t)R * L.IW;
    s = (s + 15) & ~(size_t)15;
    s += sizeof(uint16_t) * (size_t)L.BR * L.NG;
    return s + 16;
}

// Rows per CTA: the tuned value when set, else 28 when that fits the 220 KB shared-memory budget (fewer,
// taller tiles: less halo and fewer waves over 152 SMs), else 16; in every case reduced until it fits (one
// 1024-thread CTA per SM).
constexpr size_t kGradBudget = 220 * 1024;
template <int RHO>
int grad_rows(int W, int n_cls, int tuned)
{
    int R = tuned > 0 ? tuned : grad_smem<RHO>(W, 28, n_cls) <= kGradBudget ? 28 : 16;
    while (R > 1 && grad_smem<RHO>(W, R, n_cls) > kGradBudget)
        --R;
    return R;
}

template <int RHO>
cudaError_t launch_grad_t(const KParams &kp, const Work &w, const float *disp, const uint8_t *img, cudaStream_t s)
{
    const int R = grad_rows<RHO>(kp.W, kp.n_cls, kp.tile_grad);
    const size_t smem = grad_smem<RHO>(kp.W, R, kp.n_cls);
    dim3 grid((kp.H + R - 1) / R, kp.n_frames);
    k_grad<RHO><<<grid, kThreads, smem, s>>>(kp, w, disp, img, R);
    return cudaGetLastError();
}

}  // namespace

cudaError_t setup_grad(int smem_optin)
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad<1>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad<2>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad<3>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad<4>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad<5>, smem_optin);
    return e;
}

cudaError_t launch_grad(const KParams &kp, const Work &w, const float *disp, const uint8_t *img, cudaStream_t s)
{
    switch (kp.rho) {
    case 1: return launch_grad_t<1>(kp, w, disp, img, s);
    case 2: return launch_grad_t<2>(kp, w, disp, img, s);
    case 3: return launch_grad_t<3>(kp, w, disp, img, s);
    case 4: return launch_grad_t<4>(kp, w, disp, img, s);
    default: return launch_grad_t<5>(kp, w, disp, img, s);
    }
}

}  // namespace ld
