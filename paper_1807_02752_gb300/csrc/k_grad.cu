// Sec. 2.3.1: road mask, bilateral filter (Eq. 15-16), Sobel gradients, edge test and sparse V_px votes
// (Eq. 17), for the road rows of every frame.
//
// One CTA owns a tile of R rows x 64 four-pixel groups (256 columns) of one frame: the road test, the edge
// test and the votes of those pixels.  It stages the image region its stencils reach in shared memory as
// 2 I, with a sentinel value outside the frame whose range weight is 0 (this is the clipped window of
// Eq. 15).  Small tiles keep a CTA at about 50 KB of shared memory, so four run on an SM and one CTA's
// barriers and loads overlap the others' arithmetic.
//
// Exact pruning: a road pixel whose neighbourhood is provably too flat to pass the edge test (an image
// range of at most kp.flat_range over the windows of its 3x3 neighbours; the bound is derived and
// computed on the host, flat_range() in ld_api.cu) leaves the road mask.  On the 1242x375 workload about
// three quarters of the bilateral work goes with those pixels, and every edge, G and vote stays as the
// full computation gives them.
//
// The bilateral output is computed only at the groups holding a pixel of the 3x3 neighbourhood of a
// remaining road pixel of the tile (neighbouring tiles compute their shared border groups each).  Weights
// are Q15 integers, w = (ws * wr[|I(i,j) - I(u,v)|] + 2^14) >> 15, sums are exact, and the output is
// (2 sum(w I) + sum(w)) / (2 sum(w)), so the result does not depend on the order of the taps.
//
// GB300 mapping of the bilateral:
//   - taps at equal distance share ws and the range weight depends on |I(i,j) - I(u,v)| only, so w depends
//     on (distance class, |dI|); the CTA builds one 512-entry uint16 table per class in shared memory and
//     a tap costs one absolute-difference-add (__usad), one table load and two 32-bit accumulations
//     (sum(w) and sum(w 2 I)).  Indexing by |dI| keeps the common small differences in half of the banks;
//   - the tile stores 2 I (a byte offset into a table), so the table address is base_c + |2 I(i,j) - 2 I(u,v)|
//     with a compile-time class offset; the sentinel 2 x 511 outside the frame lands in the zero half of
//     every table;
//   - a thread filters 4 horizontally adjacent pixels, sharing each window row it loads as 64-bit vectors.
//
// Each remaining road pixel with G_x^2 + G_y^2 > thr^2 is an edge pixel.  Its vote column is
// floor(u + (v - V_py(v)) G_y / G_x + 0.5) in float32 (the line through the pixel perpendicular to the
// gradient meets row V_py there), kept when inside [0, W).  Edge pixels and votes are appended to per-row
// lists through one global atomic per group (order within a row is arbitrary; every consumer sums over
// them); the per-row counts are zeroed before the launch.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kThreads = 256;
constexpr int kGroups = 64;                // four-pixel groups per CTA (256 columns)
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

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t lds_u16(uint32_t addr)
{
    uint16_t v;
    asm("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}

// Bilateral output of 4 pixels whose windows start at tile row br and tile column u0 (the pixels sit at tile
// row br + RHO, columns u0 + RHO ..); nv of them lie inside the frame.  The tile holds 2 I with the
// sentinel outside the frame.
// sum(w) <= 121 * 2^15 and sum(w 2 I) <= 121 * 2^15 * 510 < 2^31 both fit 32-bit accumulators.
template <int RHO>
__device__ __forceinline__ uint32_t bilateral4(const KParams &kp, const uint16_t *tile, int TWP, int br, int u0, int nv,
                                               uint32_t tab)
{
    constexpr int N = 2 * RHO + 1;
    constexpr int NL = (4 + 2 * RHO + 3) / 4;
    const uint16_t *crow = tile + (size_t)(br + RHO) * TWP + u0 + RHO;
    uint32_t base[4], sw[4], swi[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t c2 = p < nv ? crow[p] : 0u;  // pixels past the right edge: any valid index
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

// Shared-memory layout of a tile (bytes; every region 16-byte aligned).
struct GradTile {
    int TWP, TR, nj, IWO, IWB, NGB;
    size_t o_tab, o_tile, o_hr, o_live, o_ibf, o_gl, o_row, bytes;
};
template <int RHO>
__host__ __device__ inline GradTile grad_tile(int nr, int nj, int n_cls)
{
    GradTile t;
    t.nj = nj;
    t.TWP = (4 * nj + 2 * RHO + 8 + 3) & ~3;  // tile columns: frame columns 4 j0 - RHO - 4 ..
    t.TR = nr + 2 * RHO + 2;                  // tile rows: frame rows r0 - RHO - 1 ..
    t.IWO = 4 * nj;                           // owned pixels per row
    t.NGB = nj + 2;                           // bilateral groups per row: j0 - 1 .. j0 + nj
    t.IWB = 4 * t.NGB;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = (o + b + 15) & ~(size_t)15;
        return r;
    };
    t.o_tab = take((size_t)kTabBytes * n_cls);
    t.o_tile = take(2 * (size_t)t.TR * t.TWP);
    t.o_hr = take(2 * (size_t)t.TR * nj);
    t.o_live = take((size_t)nr * t.IWO);
    t.o_ibf = take((size_t)(nr + 2) * t.IWB);
    t.o_gl = take(2 * (size_t)(nr + 2) * t.NGB);
    t.o_row = take(4 * (size_t)(2 * nr + 4));
    t.bytes = o;
    return t;
}

template <int RHO>
// filter: apply Eq. 15-16 (0: the image is used as it is, the median pre-filter's output or bilateral = 0)
__device__ __forceinline__ void grad_body(const KParams &kp, const Work &w, const float *__restrict__ disp,
                                          const uint8_t *__restrict__ img, int R, const int f, const int bx, const int by,
                                          const bool filter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = kThreads / 32;
    const int W = kp.W, H = kp.H, NG = (W + 3) >> 2;
    const int r0 = by * R, nr = min(R, H - r0);
    const int j0 = bx * kGroups, nj = min(kGroups, NG - j0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FrameState &fs = w.fs[f];
    const int vtop = fs.v_top;
    if ((fs.flags & LD_F_NO_LANES) || r0 + nr - 1 < vtop)
        return;   // no road pixel of the tile (the per-row counts were zeroed before the launch)
    if (!LD_IN(kp.n_cls, kClsTables + 1, CK_GRAD_TILE))   // the class tables the tile copies
        return;
    const GradTile T = grad_tile<RHO>(nr, nj, kp.n_cls);
    const int cbase = 4 * j0 - RHO - 4, rbase = r0 - RHO - 1;   // frame column / row of tile column / row 0
    uint16_t *tabs = reinterpret_cast<uint16_t *>(smem + T.o_tab);    // [n_cls][512]
    uint16_t *tile = reinterpret_cast<uint16_t *>(smem + T.o_tile);   // [TR][TWP] 2 I, or 2 x sentinel
    uint16_t *hr = reinterpret_cast<uint16_t *>(smem + T.o_hr);       // [TR][nj] (min I, max I) of a group's test columns
    uint8_t *live = smem + T.o_live;                                  // [nr][IWO] owned road pixels left after pruning
    uint8_t *ibf = smem + T.o_ibf;                                    // [nr + 2][IWB] bilateral output, row b = v - r0 + 1
    uint16_t *glist = reinterpret_cast<uint16_t *>(smem + T.o_gl);    // groups (b << 8 | g) that need the filter
    float *rowVy = reinterpret_cast<float *>(smem + T.o_row);
    int *cnt = reinterpret_cast<int *>(rowVy + 2 * nr);               // [1] groups that need the filter

    // per-class weight tables T_c[a] = (ws_c * wr(a) + 2^14) >> 15 for a = |I(i,j) - I(u,v)|, built once per
    // handle (zero from a = 256 on), copied asynchronously in 16-byte pieces (cp.async): the filter is the
    // first reader, so the copy overlaps the staging, flatness and compaction phases
    {
        const int nt16 = kp.n_cls * (kTabBytes / 16);
        const char *src = reinterpret_cast<const char *>(w.cls_tab);
        const uint32_t dst0 = smem_addr(tabs);
        for (int k = tid; k < nt16; k += kThreads)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + 16u * (uint32_t)k),
                         "l"(src + 16 * (size_t)k) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const float *rows = w.rows + (size_t)f * 3 * H;
    if (tid < nr)
        rowVy[tid] = __ldg(rows + H + r0 + tid);   // V_py(v) of the owned rows, for the votes
    if (tid == 0)
        *cnt = 0;
    // road mask of the owned pixels first: l > 0 with |l - f(v)| <= varpi (an infinite or NaN l fails the
    // second test because f(v) is finite), v >= v_top, 1 <= u <= W-2.  A warp takes two rows at a time with
    // all of their loads in flight, f(v) read directly (rows off the road get NaN, which fails the test).
    const float *dsrc = disp + ((size_t)f * H + r0) * W;
    constexpr int KX = 4 * kGroups / 32;   // 32-pixel chunks of an owned row
    for (int rr = 2 * warp; rr < nr; rr += 2 * NW) {
        float lv[2][KX], fv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = rr + q, v = r0 + r;
            fv[q] = r < nr && v >= vtop && v >= 1 && v <= H - 2 ? __ldg(rows + v) : __int_as_float(0x7fc00000);
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const int u = 4 * j0 + lane + 32 * k;
                lv[q][k] = r < nr && lane + 32 * k < T.IWO && u >= 1 && u <= W - 2 ? __ldg(dsrc + (size_t)r * W + u)
                                                                                    : 0.0f;
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const int r = rr + q, x = lane + 32 * k;
                if (r < nr && x < T.IWO)
                    live[r * T.IWO + x] = (uint8_t)(lv[q][k] > 0.0f && fabsf(__fsub_rn(lv[q][k], fv[q])) <= kp.varpi);
            }
    }
    // image region, coalesced byte loads: consecutive lanes read consecutive bytes of a row.  A warp takes
    // two tile rows at a time and issues all of their loads before its first store.
    const uint8_t *im = img + (size_t)f * H * W;
    constexpr int KC = (4 * kGroups + 2 * RHO + 11 + 31) / 32;   // 32-column chunks of a tile row (>= TWP / 32)
    for (int tr0 = 2 * warp; tr0 < T.TR; tr0 += 2 * NW) {
        uint32_t px[2][KC];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int v = rbase + tr0 + q;
            const bool vin = tr0 + q < T.TR && v >= 0 && v < H;
            const uint8_t *src = im + (size_t)(vin ? v : 0) * W;
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                const int c = cbase + lane + 32 * k;
                px[q][k] = vin && c >= 0 && c < W ? 2u * __ldg(src + c) : 2u * kSentinel;
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                const int tc = lane + 32 * k;
                if (tr0 + q < T.TR && tc < T.TWP)
                    tile[(tr0 + q) * T.TWP + tc] = (uint16_t)px[q][k];
            }
    }
    __syncthreads();
    // Exact pruning (see the comment at the top): a group is flat when the image range over columns
    // 4g - RHO - 4 .. 4g + RHO + 5 (a superset of its 3x3 neighbours' windows: tile columns 4 (g - j0) ..)
    // and rows v - RHO - 1 .. v + RHO + 1 is at most kp.flat_range; any tap outside the frame holds the
    // sentinel, which makes the range too large.
    if (kp.flat_range >= 0) {
        constexpr int NLF = (2 * RHO + 10 + 3) / 4;      // 8-byte loads per tile row of a group's test region
        for (int tr = warp; tr < T.TR; tr += NW)
            for (int g = lane; g < nj; g += 32) {
                const uint2 *src = reinterpret_cast<const uint2 *>(tile + tr * T.TWP + 4 * g);
                uint32_t vmn = 0xffffffffu, vmx = 0u;
#pragma unroll
                for (int l = 0; l < NLF; ++l) {
                    const uint2 v = src[l];
                    vmn = __vminu2(vmn, __vminu2(v.x, v.y));
                    vmx = __vmaxu2(vmx, __vmaxu2(v.x, v.y));
                }
                const uint32_t mn2 = min(vmn & 0xffffu, vmn >> 16), mx2 = max(vmx & 0xffffu, vmx >> 16);  // 2 I
                hr[tr * nj + g] = (uint16_t)(mx2 <= 510u ? (mn2 >> 1) | ((mx2 >> 1) << 8) : 0xff00u);
            }
        __syncthreads();
        for (int r = warp; r < nr; r += NW)
            for (int g = lane; g < nj; g += 32) {
                uint32_t mn = 255u, mx = 0u;
#pragma unroll
                for (int t = 0; t < 2 * RHO + 3; ++t) {
                    const uint32_t h = hr[(r + t) * nj + g];
                    mn = min(mn, h & 0xffu);
                    mx = max(mx, h >> 8);
                }
                if ((int)(mx - mn) <= kp.flat_range)
                    reinterpret_cast<uint32_t *>(live + r * T.IWO)[g] = 0u;
            }
        __syncthreads();
    }
    // groups g' = j0 - 1 + g (g < NGB) of rows v = r0 - 1 + b (b < nr + 2) holding a pixel the Sobel of a
    // remaining owned road pixel reads: owned pixels 4g - 5 .. 4g of rows b - 1 .. b + 1
    for (int b = warp; b < nr + 2; b += NW)
        for (int g0 = 0; g0 < T.NGB; g0 += 32) {
            const int g = g0 + lane;
            bool need = false;
            if (g < T.NGB) {
#pragma unroll
                for (int dr = -1; dr <= 1; ++dr) {
                    const int r = b - 1 + dr;
                    if (r < 0 || r >= nr)
                        continue;
                    const uint32_t *lw = reinterpret_cast<const uint32_t *>(live + r * T.IWO);
                    const uint32_t mid = g >= 1 && g <= nj ? lw[g - 1] : 0u;           // pixels 4g - 4 .. 4g - 1
                    const uint32_t left = g >= 2 && g <= nj + 1 ? lw[g - 2] >> 24 : 0u; // pixel 4g - 5
                    const uint32_t right = g < nj ? lw[g] & 0xffu : 0u;                 // pixel 4g
                    need |= (left | mid | right) != 0u;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, need);
            int base = 0;
            if (lane == 0 && m)
                base = atomicAdd(cnt, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            const int at = base + __popc(m & ((1u << lane) - 1u));
            if (need && LD_IN(at, (nr + 2) * T.NGB, CK_GRAD_GLIST))
                glist[at] = (uint16_t)((b << 8) | g);
        }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // this thread's table pieces have landed
    __syncthreads();
    const int ng = LD_IN(*cnt, (nr + 2) * T.NGB + 1, CK_GRAD_GLIST) ? *cnt : 0;
    const uint32_t tab = smem_addr(tabs);
    constexpr int NLW = (4 + 2 * RHO + 3) / 4;   // 8-byte loads per window row of a group
    for (int k = tid; k < ng; k += kThreads) {
        const int e = glist[k], b = e >> 8, g = e & 255;
        // the group's cell, then its windows (tile rows b .. b + 2 RHO, tile columns 4 g .. 4 g + 4 NLW - 1)
        if (!LD_IN(b, nr + 2, CK_GRAD_GROUP) || !LD_IN(g, T.NGB, CK_GRAD_GROUP) ||
            !LD_IN(b + 2 * RHO, T.TR, CK_GRAD_TAP) || !LD_IN(4 * g + 4 * NLW - 1, T.TWP, CK_GRAD_TAP))
            continue;
        const int u0 = 4 * (j0 - 1 + g), v = r0 - 1 + b;   // frame column of the group, frame row
        const int nv = min(4, W - u0);
        uint32_t out;
        // the group's windows start at tile row b (frame row v - RHO) and tile column 4 g (frame column u0 - RHO)
        if (filter) {
            out = bilateral4<RHO>(kp, tile, T.TWP, b, 4 * g, nv, tab);
        } else {
            const uint16_t *c = tile + (b + RHO) * T.TWP + 4 * g + RHO;
            out = (uint32_t)(c[0] >> 1) | ((uint32_t)(c[1] >> 1) << 8) | ((uint32_t)(c[2] >> 1) << 16) |
                  ((uint32_t)(c[3] >> 1) << 24);
        }
        *reinterpret_cast<uint32_t *>(ibf + b * T.IWB + 4 * g) = out;
        if (w.dbg_ibf && v >= 0 && v < H && u0 >= 0) {   // stage capture (groups shared with other tiles too)
            int16_t *drow = w.dbg_ibf + ((size_t)f * H + v) * W;
            for (int q = 0; q < nv; ++q)
                drow[u0 + q] = (int16_t)((out >> (8 * q)) & 0xffu);
        }
    }
    __syncthreads();

    // Sobel, edge test, votes of the remaining owned road pixels, one thread per group: 32-bit loads of the
    // mask and of the three bilateral rows (owned group g is bilateral group g + 1)
    const int thr2 = kp.edge_thresh2;
    int16_t *edges = w.edges + (size_t)f * H * W * 4;
    int16_t *vbins = w.vbins + (size_t)f * H * W;
    int32_t *ecnt = w.ecount + (size_t)f * H;
    int32_t *vcnt = w.vcount + (size_t)f * H;
    for (int r = warp; r < nr; r += NW)
        for (int g = lane; g < nj; g += 32) {
            const uint32_t m4 = reinterpret_cast<const uint32_t *>(live + r * T.IWO)[g];
            if (!m4)
                continue;
            const int v = r0 + r;
            uint32_t x0[3], x1[3], x2[3];  // bytes 4j-4 .. 4j-1, 4j .. 4j+3, 4j+4 .. 4j+7 of rows v-1, v, v+1
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const uint32_t *rw = reinterpret_cast<const uint32_t *>(ibf + (r + d) * T.IWB);
                x0[d] = rw[g];
                x1[d] = rw[g + 1];
                x2[d] = rw[g + 2];
            }
            const float vy = rowVy[r];
            short4 ent[4];
            int bins[4], ne = 0, nb = 0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (!((m4 >> (8 * p)) & 0xffu))
                    continue;
                const int u = 4 * (j0 + g) + p;
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
                ent[ne++] = make_short4((short)u, (short)bin, (short)gx, (short)gy);
                if (bin >= 0)
                    bins[nb++] = bin;
            }
            if (ne) {
                const int pe = atomicAdd(ecnt + v, ne);
                for (int k = 0; k < ne; ++k)
                    if (LD_IN(pe + k, W, CK_GRAD_EDGE))   // a row holds at most W edge entries
                        *reinterpret_cast<short4 *>(edges + ((size_t)v * W + pe + k) * 4) = ent[k];
            }
            if (nb) {
                const int pv = atomicAdd(vcnt + v, nb);
                for (int k = 0; k < nb; ++k)
                    if (LD_IN(pv + k, W, CK_GRAD_VOTE) && LD_IN(bins[k], W, CK_GRAD_VOTE))
                        vbins[(size_t)v * W + pv + k] = (int16_t)bins[k];
            }
        }
}

template <int RHO>
__global__ void __launch_bounds__(kThreads, 4) k_grad(const KParams kp, const Work w, const float *__restrict__ disp,
                                                   const uint8_t *__restrict__ img, int R)
{
    grad_body<RHO>(kp, w, disp, img, R, blockIdx.z, blockIdx.x, blockIdx.y, kp.bilateral != 0);
}

// median_input: the frame's image is its median-filtered copy in the workspace (bilateral = 2)
template <int RHO>
__global__ void __launch_bounds__(kThreads, 4) k_grad_fd(const FrameDesc *__restrict__ fd, int R, int median_input)
{
    const FrameDesc &d = fd[blockIdx.z];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    if ((int)blockIdx.y * R >= kp.H || (int)blockIdx.x * kGroups >= (kp.W + 3) / 4)
        return;
    grad_body<RHO>(kp, w, d.disp, median_input ? w.med : d.img, R, 0, blockIdx.x, blockIdx.y,
                   !median_input && kp.bilateral != 0);
}

// Rows per CTA: the tuned value when set, else 16.
template <int RHO>
int grad_rows(int tuned)
{
    return tuned > 0 ? (tuned < 64 ? tuned : 64) : 16;
}

template <int RHO>
cudaError_t launch_grad_t(const KParams &kp, const Work &w, const float *disp, const uint8_t *img, cudaStream_t s)
{
    const int R = grad_rows<RHO>(kp.tile_grad);
    const int NG = (kp.W + 3) / 4, nj = NG < kGroups ? NG : kGroups;
    const size_t smem = grad_tile<RHO>(R, nj, kp.n_cls).bytes;
    dim3 grid((NG + kGroups - 1) / kGroups, (kp.H + R - 1) / R, kp.n_frames);
    k_grad<RHO><<<grid, kThreads, smem, s>>>(kp, w, disp, img, R);
    return cudaGetLastError();
}

template <int RHO>
cudaError_t launch_grad_fd_t(const KParams &kmax, const FrameDesc *fd, int n, bool median_input, cudaStream_t s)
{
    const int R = grad_rows<RHO>(0);
    const int NG = (kmax.W + 3) / 4, nj = NG < kGroups ? NG : kGroups;
    const size_t smem = grad_tile<RHO>(R, nj, kmax.n_cls).bytes;
    dim3 grid((NG + kGroups - 1) / kGroups, (kmax.H + R - 1) / R, n);
    k_grad_fd<RHO><<<grid, kThreads, smem, s>>>(fd, R, median_input ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grad_fd(const KParams &kmax, const FrameDesc *fd, int n, bool median_input, cudaStream_t s)
{
    switch (kmax.rho) {
    case 1: return launch_grad_fd_t<1>(kmax, fd, n, median_input, s);
    case 2: return launch_grad_fd_t<2>(kmax, fd, n, median_input, s);
    case 3: return launch_grad_fd_t<3>(kmax, fd, n, median_input, s);
    case 4: return launch_grad_fd_t<4>(kmax, fd, n, median_input, s);
    default: return launch_grad_fd_t<5>(kmax, fd, n, median_input, s);
    }
}

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
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad_fd<1>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad_fd<2>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad_fd<3>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad_fd<4>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_grad_fd<5>, smem_optin);
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
