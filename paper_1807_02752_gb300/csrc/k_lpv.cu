// Sec. 2.4, lane position validation (Alg. 7):
//
//   k_m1      w_g of every road edge pixel (Eq. 23), M_0 = (2 nu + 1) x (2 varsigma + 1) box sum of
//             G_x w_g, M_1 = G * M_0 with G = [1,2,1]^T [1,0,-1] (a convolution: M_0(u+1) - M_0(u-1)),
//             evaluated through the horizontal difference D of M_0 (below).
//   k_energy  for every start s in [-floor(xi W), W + floor(xi W)) the track of Eq. 25 from the bottom
//             row up to v_top and its energy E = M_1(round(u_v), v) + lambda_g E (Eq. 24).
//   k_select  strict interior local minima of H below t = ceil(thr min H), then suppression of nearby
//             minima in increasing (energy, position) order; fills ld_lanes.
//   Both also serve the learned proposal (k_net.cu): energies of listed starts only, selection among
//   candidate starts, and the exhaustive fallback for the frames where that selected nothing.
//
// w_g reading: theta_e is the direction of the edge (the Sobel gradient turned by 90 degrees), theta_Vp
// the direction from the pixel to V_p(v); lines are undirected, so the angle is taken in [0, pi/2] through
// s = sin^2(dtheta) = (t x r)^2 / (|t|^2 |r|^2) in float32.  w_g = 0 beyond pi/6 (s > 1/4); otherwise the
// Q12 table entry at floor(sqrt(s) 2^15).  Eq. 23 is applied as printed: exp(-|dtheta| / sigma_g^2 * 36/pi).
#include <type_traits>

#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kM1Threads = 512;
constexpr int kEnThreads = 128;
constexpr int kEnBatchDefault = 8;    // track rows whose M_1 loads are in flight together
constexpr int kSelThreads = 256;

// k_m1 works on D(u, v) = M_0(u+1, v) - M_0(u-1, v).  An edge pixel at (u_e, v_e) adds g = G_x w_g to the
// (2 nu + 1)-box sums T(x, v_e) for x in [u_e - nu, u_e + nu], so on the interior columns
// D = T(x+1) - T(x-1) telescopes to +g at u_e - nu - 1 and u_e - nu, -g at u_e + nu and u_e + nu + 1
// (4 shared-memory atomics per edge instead of (2 nu + 1)(2 varsigma + 1)); M_0 is zero outside the
// frame, so column 0 holds T(1) and column W-1 holds -T(W-2).  M_1(u, v) = X(v-1) + 2 X(v) + X(v+1) with
// X(g) = sum_{|y| <= varsigma} D(u, g + y) on rows g inside the frame (0 outside), which a thread per
// column evaluates as a sliding sum.  All integer: the result does not depend on the order of the adds.
constexpr int kM1MaxEdgeRows = 64;

struct M1Layout {
    int R, Wc;  // M_1 rows per CTA, columns of D per shared-memory chunk
};

// Rows per CTA: the tuned value (1 .. 16) when set, else the most of 16 .. 8 that fit one 110 KB chunk of
// the full width (two CTAs per SM), else 16 with the columns split into chunks.
inline M1Layout m1_layout(int W, int vs, int tuned)
{
    const size_t budget = 110 * 1024;
    M1Layout L;
    if (tuned > 0) {
        L.R = tuned < 16 ? tuned : 16;
    } else {
        for (L.R = 16; L.R >= 8; --L.R)
            if ((size_t)(L.R + 2 + 2 * vs) * W * sizeof(int32_t) <= budget)
                break;
        if (L.R < 8)
            L.R = 16;
    }
    const size_t row_bytes = (size_t)(L.R + 2 + 2 * vs) * sizeof(int32_t);
    L.Wc = (size_t)W * row_bytes <= budget ? W : (int)(budget / row_bytes) & ~31;
    return L;
}

__device__ __forceinline__ void m1_body(const KParams &kp, const Work &w, int R, int Wc, const int f, int tile)
{
    extern __shared__ __align__(16) int32_t dd[];   // [nr + 2 + 2 varsigma][Wc]: rows r0-1-varsigma ..
    __shared__ int32_t eoff[kM1MaxEdgeRows + 1];
    const int W = kp.W, H = kp.H;
    const int r0 = tile * R;
    const int nr = min(R, H - r0);
    const FrameState &fs = w.fs[f];
    const int vtop = fs.v_top, vmax = H - 1;
    if ((fs.flags & LD_F_NO_LANES) || r0 + nr - 1 < vtop)
        return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nu = kp.box_nu, vs = kp.box_vs;
    const int d0 = r0 - 1 - vs;                      // frame row of D row 0
    const int ndr = nr + 2 + 2 * vs;
    // edge rows that reach the M_0 rows r0-1 .. r0+nr, and the prefix of their edge counts
    const int elo = max(vtop, d0), ehi = min(vmax, r0 + nr + vs);
    const int ner = max(0, ehi - elo + 1);           // <= kM1MaxEdgeRows (R <= 16, varsigma <= 8)
    if (!LD_IN(ner, kM1MaxEdgeRows + 1, CK_M1_CHUNK))
        return;
    if (tid < 32) {
        const int32_t *ec = w.ecount + (size_t)f * H + elo;
        int a = 2 * lane < ner ? ec[2 * lane] : 0;
        int b = 2 * lane + 1 < ner ? ec[2 * lane + 1] : 0;
        a = LD_IN(a, W + 1, CK_M1_EDGE) ? a : 0;    // a row holds at most W edge entries
        b = LD_IN(b, W + 1, CK_M1_EDGE) ? b : 0;
        int s = a + b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d)
                s += t;
        }
        eoff[2 * lane] = s - a - b;
        eoff[2 * lane + 1] = s - b;
        if (lane == 31)
            eoff[kM1MaxEdgeRows] = s;
    }
    const float *Vpy = w.rows + (size_t)f * 3 * H + H;
    const float *Vpx = Vpy + H;
    int32_t *M1 = w.M1 + (size_t)f * H * W;
    const int rs = max(r0, vtop);
    for (int c0 = 0; c0 < W; c0 += Wc) {
        const int c1 = min(W, c0 + Wc), cw = c1 - c0;
        {
            const int nz = ndr * cw;
            int4 *dd4 = reinterpret_cast<int4 *>(dd);
            for (int i = tid; i < (nz >> 2); i += kM1Threads)
                dd4[i] = make_int4(0, 0, 0, 0);
            for (int i = (nz & ~3) + tid; i < nz; i += kM1Threads)
                dd[i] = 0;
        }
        __syncthreads();
        const int total = eoff[ner];
        for (int q = tid; q < total; q += kM1Threads) {
            int lo = 0, hi = ner;  // eoff[lo] <= q < eoff[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (eoff[mid] <= q)
                    lo = mid;
                else
                    hi = mid;
            }
            const int v = elo + lo;
            const short4 e = reinterpret_cast<const short4 *>(w.edges + ((size_t)f * H + v) * W * 4)[q - eoff[lo]];
            const int u = e.x, gx = e.z, gy = e.w;
            if (!LD_IN(u, W, CK_M1_EDGE) || !LD_IN(v - d0, ndr, CK_M1_CHUNK))
                continue;
            if (u + nu + 1 < c0 || u - nu - 1 >= c1)
                if (!(c0 == 0 && abs(u - 1) <= nu) && !(c1 == W && abs(u - (W - 2)) <= nu))
                    continue;
            const float vx = Vpx[v], vy = Vpy[v];
            const float tu = (float)(-gy), tv = (float)gx;
            const float ru = __fsub_rn(vx, (float)u), rv = __fsub_rn(vy, (float)v);
            const float cr = __fsub_rn(__fmul_rn(tu, rv), __fmul_rn(tv, ru));
            const float num = __fmul_rn(cr, cr);
            const float den = __fmul_rn(__fadd_rn(__fmul_rn(tu, tu), __fmul_rn(tv, tv)),
                                        __fadd_rn(__fmul_rn(ru, ru), __fmul_rn(rv, rv)));
            int wg = 0;
            if (den > 0.0f) {
                const float s = __fdiv_rn(num, den);
                const int ti = (int)__fmul_rn(__fsqrt_rn(s), 32768.0f);
                if (s <= 0.25f && LD_IN(ti, kWgEntries, CK_M1_COL))
                    wg = __ldg(w.wg + ti);
            }
            const int g = gx * wg;
            if (g == 0)
                continue;
            // input map of the learned proposal: the CTA that owns row v and the chunk that holds column u
            // add |g| to the edge's 4x4 block (integer: the sum does not depend on the order)
            if (w.xsum && v >= r0 && v < r0 + nr && u >= c0 && u < c1)
                atomicAdd(w.xsum + ((size_t)f * ((H + 3) >> 2) + (v >> 2)) * ((W + 3) >> 2) + (u >> 2), abs(g));
            int32_t *drow = dd + (size_t)(v - d0) * cw;  // column t of the frame at drow[t - c0]
            const int tgt[4] = {u - nu - 1, u - nu, u + nu, u + nu + 1};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int t = tgt[k];
                if (t >= 1 && t <= W - 2 && t >= c0 && t < c1)
                    atomicAdd(drow + (t - c0), k < 2 ? g : -g);
            }
            if (c0 == 0 && abs(u - 1) <= nu)
                atomicAdd(drow, g);
            if (c1 == W && abs(u - (W - 2)) <= nu)
                atomicAdd(drow + (W - 1 - c0), -g);
        }
        __syncthreads();
        // column pass: pointers walk the D rows and the M_1 rows (no index products).  With an even width
        // and chunk every row starts on 8 bytes, so a thread takes two adjacent columns per 8-byte load and
        // store; otherwise one column.  Each column's sums are the same integer adds in the same order.
        const int span = 2 * vs + 1;
        if (((W | cw | c0) & 1) == 0) {
            const int cw2 = cw >> 1, W2 = W >> 1;
            for (int pc = tid; pc < cw2; pc += kM1Threads) {
                const int2 *lo = reinterpret_cast<const int2 *>(dd) + pc;   // D rows 0 .. 2 varsigma: M_0 row r0 - 1
                const int2 *hi = lo + span * cw2;
                int bx = 0, by = 0;
                for (const int2 *p = lo; p < hi; p += cw2) {
                    const int2 t = *p;
                    bx += t.x;
                    by += t.y;
                }
                int xpx = r0 - 1 >= 0 ? bx : 0, xpy = r0 - 1 >= 0 ? by : 0;   // 0 above the frame
                {
                    const int2 a = *hi, b = *lo;                               // M_0 row r0 (inside the frame)
                    bx += a.x - b.x;
                    by += a.y - b.y;
                }
                hi += cw2;
                lo += cw2;
                int xcx = bx, xcy = by;
                int2 *out = reinterpret_cast<int2 *>(M1 + (size_t)r0 * W + c0) + pc;
                for (int g = r0; g < r0 + nr; ++g, hi += cw2, lo += cw2, out += W2) {
                    const int2 a = *hi, b = *lo;                               // M_0 row g + 1
                    bx += a.x - b.x;
                    by += a.y - b.y;
                    const int xnx = g + 1 <= vmax ? bx : 0, xny = g + 1 <= vmax ? by : 0;
                    if (g >= rs)
                        *out = make_int2(xpx + 2 * xcx + xnx, xpy + 2 * xcy + xny);
                    xpx = xcx;
                    xcx = xnx;
                    xpy = xcy;
                    xcy = xny;
                }
            }
        } else {
            for (int uc = tid; uc < cw; uc += kM1Threads) {
                const int32_t *lo = dd + uc;                     // D rows 0 .. 2 varsigma: M_0 row r0 - 1
                const int32_t *hi = lo + span * cw;
                int box = 0;
                for (const int32_t *p = lo; p < hi; p += cw)
                    box += *p;
                int xp = r0 - 1 >= 0 ? box : 0;                  // 0 above the frame
                box += *hi - *lo;                                 // M_0 row r0 (inside the frame)
                hi += cw;
                lo += cw;
                int xc = box;
                int32_t *out = M1 + (size_t)r0 * W + c0 + uc;
                for (int g = r0; g < r0 + nr; ++g, hi += cw, lo += cw, out += W) {
                    box += *hi - *lo;                             // M_0 row g + 1
                    const int xn = g + 1 <= vmax ? box : 0;
                    if (g >= rs)
                        *out = xp + 2 * xc + xn;
                    xp = xc;
                    xc = xn;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kM1Threads, 2) k_m1(const KParams kp, const Work w, int R, int Wc)
{
    m1_body(kp, w, R, Wc, blockIdx.y, blockIdx.x);
}
__global__ void __launch_bounds__(kM1Threads, 2) k_m1_fd(const FrameDesc *__restrict__ fd, int R, int Wc)
{
    const FrameDesc &d = fd[blockIdx.y];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    if ((int)blockIdx.x * R >= kp.H)
        return;
    m1_body(kp, w, R, Wc, 0, blockIdx.x);
}

// MODE 0: every start of every frame; 1: the starts listed per frame (learned proposal); 2: every start of
// the frames flagged LD_F_FALLBACK (the proposal selected no lane there).
// A short list (MODE 1) is latency-bound: each start is a serial chain of divisions and gathers, so the
// list form issues the M_1 loads of 32 rows at a time instead of 8 (fewer dependent round trips).
template <int MODE, bool LAM>
__device__ __forceinline__ void energy_body(const KParams &kp, const Work &w, const int32_t *elist, const int32_t *ecnt,
                                            int ecap, const int f, const int tile)
{
    constexpr int kEnBatch = MODE == 1 ? 32 : kEnBatchDefault;
    extern __shared__ float vrow[];   // [3][H]: V_px, V_py, and the divisor of Eq. 25 for each row
    const int W = kp.W, H = kp.H;
    const FrameState &fs = w.fs[f];
    if (fs.flags & LD_F_NO_LANES)
        return;
    if (MODE == 2 && !(fs.flags & LD_F_FALLBACK))
        return;
    if (MODE == 1 && tile * kEnThreads >= ecnt[f])
        return;
    const int vtop = fs.v_top, vmax = H - 1;
    const float *rows = w.rows + (size_t)f * 3 * H;
    for (int v = threadIdx.x; v < H; v += kEnThreads) {
        vrow[v] = rows[2 * H + v];
        vrow[H + v] = rows[H + v];
        // the step into row v divides by (v + 1) - V_py(v + 1), the same for every start
        vrow[2 * H + v] = v < H - 1 ? __fsub_rn(__fadd_rn((float)v, 1.0f), rows[H + v + 1]) : 1.0f;
    }
    __syncthreads();
    int i = tile * kEnThreads + threadIdx.x;
    if (MODE == 1) {
        if (i >= ecnt[f] || !LD_IN(i, ecap, CK_EN_START))
            return;
        i = elist[(size_t)f * ecap + i];
    }
    if (i >= kp.n_starts || !LD_IN(i, kp.n_starts, CK_EN_START))
        return;
    const int32_t *M1 = w.M1 + (size_t)f * H * W;
    const float fW = (float)W;
    // The track recursion does not depend on M_1.  Each batch of kEnBatch rows first computes the track
    // columns (no load in flight while the divisions run), then issues the batch's M_1 loads back to back,
    // then adds them in row order.
    float u = (float)(i - kp.S0);
    long long E = 0;
    auto batch = [&](int v0, int nb, auto full) {
        int col[kEnBatch];
        float fv = (float)v0;  // (float)v, exact (v < 2^24)
#pragma unroll
        for (int b = 0; b < kEnBatch; ++b) {
            const int v = v0 - b;
            col[b] = -1;
            if (decltype(full)::value || b < nb) {
                if (v < vmax) {
                    const float vx = vrow[v + 1], vy = vrow[H + v + 1];
                    const float num = __fsub_rn(__fadd_rn(vx, __fmul_rn(fv, u)), __fmul_rn(vy, u));
                    u = __fdiv_rn(num, vrow[2 * H + v]);
                }
                const float c = floorf(__fadd_rn(u, 0.5f));
                if (c >= 0.0f && c < fW)
                    col[b] = (int)c;
            }
            fv = __fsub_rn(fv, 1.0f);
        }
        int32_t m[kEnBatch];
        const int rowoff = v0 * W;   // H W < 2^31
#pragma unroll
        for (int b = 0; b < kEnBatch; ++b)
            m[b] = col[b] >= 0 && LD_IN(col[b], W, CK_EN_COL) && LD_IN(v0 - b, H, CK_EN_ROW)
                       ? __ldg(M1 + (rowoff - b * W + col[b])) : 0;
#pragma unroll
        for (int b = 0; b < kEnBatch; ++b)
            if (decltype(full)::value || b < nb)
                E = LAM ? E + (long long)m[b] : (long long)m[b];
    };
    int v0 = vmax;
    for (; v0 - kEnBatch + 1 >= vtop; v0 -= kEnBatch)
        batch(v0, kEnBatch, std::true_type());
    if (v0 >= vtop)
        batch(v0, v0 - vtop + 1, std::false_type());
    w.HE[(size_t)f * kp.n_starts + i] = (int64_t)E;
}

template <int MODE>
__global__ void __launch_bounds__(kEnThreads, MODE == 1 ? 2 : 12) k_energy(const KParams kp, const Work w,
                                                                         const int32_t *elist, const int32_t *ecnt,
                                                                         int ecap)
{
    if (kp.lambda_g != 0)   // lambda_g is 0 or 1
        energy_body<MODE, true>(kp, w, elist, ecnt, ecap, blockIdx.y, blockIdx.x);
    else
        energy_body<MODE, false>(kp, w, elist, ecnt, ecap, blockIdx.y, blockIdx.x);
}
__global__ void __launch_bounds__(kEnThreads, 12) k_energy_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.y];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    if ((int)blockIdx.x * kEnThreads >= kp.n_starts)
        return;
    if (kp.lambda_g != 0)
        energy_body<0, true>(kp, w, nullptr, nullptr, 0, 0, blockIdx.x);
    else
        energy_body<0, false>(kp, w, nullptr, nullptr, 0, 0, blockIdx.x);
}

// mode 0: every start; 1: minima only at candidate starts (cflag bit 0), minimum over the evaluated ones
// (bit 1), and a frame without a lane is flagged LD_F_FALLBACK; 2: the flagged frames only, every start.
__device__ __forceinline__ void select_body(const KParams &kp, const Work &w, ld_lanes *out, const uint8_t *cflag,
                                            int mode, const int f)
{
    extern __shared__ int cand[];     // [n_starts / 2 + 2] candidate positions, then their sorted order
    __shared__ long long red[kSelThreads / 32];
    __shared__ int ncand;
    __shared__ int acc[LD_MAX_LANES];
    __shared__ int nacc;
    const int ns = kp.n_starts;
    const int tid = threadIdx.x;
    const FrameState fs = w.fs[f];
    if (mode == 2 && !(fs.flags & LD_F_FALLBACK))
        return;
    int flags = fs.flags;
    const int64_t *he = w.HE + (size_t)f * ns;
    const uint8_t *cf = mode == 1 ? cflag + (size_t)f * ns : nullptr;
    if (tid == 0) {
        ncand = 0;
        nacc = 0;
    }
    long long mn = 0;
    if (!(flags & LD_F_NO_LANES)) {
        long long m = 0x7fffffffffffffffLL;
        for (int i = tid; i < ns; i += kSelThreads)
            if (!cf || (cf[i] & 2))
                m = he[i] < m ? (long long)he[i] : m;
        for (int d = 16; d > 0; d >>= 1) {
            const long long o = __shfl_down_sync(0xffffffffu, m, d);
            m = o < m ? o : m;
        }
        if ((tid & 31) == 0)
            red[tid >> 5] = m;
        __syncthreads();
        mn = red[0];
        for (int i = 1; i < kSelThreads / 32; ++i)
            mn = red[i] < mn ? red[i] : mn;
        if (ns < 3 || mn >= 0) {
            flags |= LD_F_NO_LANES;
        } else {
            const long long t = kp.thr_abs != 0 ? kp.thr_abs : -(((-mn) * (long long)kp.thr_num) / (long long)kp.thr_den);
            int *pos = cand;
            for (int i = 1 + tid; i < ns - 1; i += kSelThreads) {
                if (cf && !(cf[i] & 1))
                    continue;
                const long long h = he[i];
                if (h < he[i - 1] && h < he[i + 1] && h < t) {
                    const int at = atomicAdd(&ncand, 1);   // strict minima: at most (ns - 1) / 2
                    if (LD_IN(at, ns / 2 + 2, CK_SEL_START))
                        pos[at] = i;
                }
            }
            __syncthreads();
            const int nc = LD_IN(ncand, ns / 2 + 3, CK_SEL_START) ? ncand : 0;
            // order by (energy, position): rank of each candidate
            int *ord = cand + nc;
            for (int a = tid; a < nc; a += kSelThreads) {
                const int ia = pos[a];
                const long long ea = he[ia];
                int rank = 0;
                for (int b = 0; b < nc; ++b) {
                    const int ib = pos[b];
                    const long long eb = he[ib];
                    rank += (eb < ea) || (eb == ea && ib < ia);
                }
                if (LD_IN(nc + rank, ns + 4, CK_SEL_START))
                    ord[rank] = ia;
            }
            __syncthreads();
            if (tid == 0) {
                int na = 0;
                for (int a = 0; a < nc && na < kp.max_lanes && LD_IN(na, LD_MAX_LANES, CK_SEL_LANES); ++a) {
                    const int c = ord[a];
                    bool ok = true;
                    for (int b = 0; b < na; ++b)
                        ok &= abs(c - acc[b]) > kp.near_px;
                    if (ok)
                        acc[na++] = c;
                }
                for (int a = 1; a < na; ++a) {
                    const int c = acc[a];
                    int b = a - 1;
                    while (b >= 0 && acc[b] > c) {
                        acc[b + 1] = acc[b];
                        --b;
                    }
                    acc[b + 1] = c;
                }
                nacc = na;
            }
            __syncthreads();
            if (nacc == 0)
                flags |= LD_F_NO_LANES;
        }
    }
    __syncthreads();
    if (mode == 1 && tid == 0 && nacc == 0 && !(fs.flags & LD_F_NO_LANES))
        w.fs[f].flags = fs.flags | LD_F_FALLBACK;
    if (tid == 0) {
        ld_lanes L;
        const int na = nacc;
        L.n_lanes = na;
        L.flags = flags;
        for (int a = 0; a < LD_MAX_LANES; ++a) {
            L.start_u[a] = a < na ? acc[a] - kp.S0 : 0;
            L.energy[a] = a < na ? he[acc[a]] : 0;
        }
        L.v_top = fs.v_top;
        L.centre = kp.centre;
        L.scale_exp = kp.e;
        L.rounds_y = fs.rounds_y;
        L.rounds_x = fs.rounds_x;
        L.reserved = 0;
        for (int i = 0; i < 3; ++i)
            L.beta[i] = fs.beta[i];
        for (int i = 0; i < 5; ++i)
            L.gamma[i] = fs.gamma[i];
        out[f] = L;
    }
}

__global__ void __launch_bounds__(kSelThreads) k_select(const KParams kp, const Work w, ld_lanes *out,
                                                        const uint8_t *cflag, int mode)
{
    select_body(kp, w, out, cflag, mode, blockIdx.x);
}
__global__ void __launch_bounds__(kSelThreads) k_select_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.x];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    select_body(kp, w, d.out, nullptr, 0, 0);
}

// Alg. 7, last step: each selected lane drawn by iterating Eq. 25 from its start (s, H-1) up to v_top, in
// the energy kernel's float32 operation order (so its rounded columns are the ones whose M_1 the lane's
// energy summed).  One thread per lane slot of a frame; rows above v_top and empty slots get NaN.
__global__ void __launch_bounds__(LD_MAX_LANES) k_tracks(const KParams kp, const Work w, const ld_lanes *lanes, float *out)
{
    const int f = blockIdx.x, k = threadIdx.x, H = kp.H;
    float *o = out + ((size_t)f * LD_MAX_LANES + k) * H;
    const ld_lanes &L = lanes[f];
    const int vtop = L.v_top;
    const bool on = k < L.n_lanes && !(L.flags & (LD_F_NO_ROAD | LD_F_DEGEN_Y | LD_F_DEGEN_X)) && vtop >= 0 && vtop < H;
    const float *vpy = w.rows + (size_t)f * 3 * H + H, *vpx = vpy + H;
    const float nanv = __int_as_float(0x7fc00000);
    float u = on ? (float)L.start_u[k] : 0.0f;
    for (int v = H - 1; v >= 0; --v) {
        if (!on || v < vtop) {
            o[v] = nanv;
            continue;
        }
        if (v < H - 1) {
            const float fv = (float)v, vx = vpx[v + 1], vy = vpy[v + 1];
            const float num = __fsub_rn(__fadd_rn(vx, __fmul_rn(fv, u)), __fmul_rn(vy, u));
            const float den = __fsub_rn(__fadd_rn(fv, 1.0f), vy);
            u = __fdiv_rn(num, den);
        }
        o[v] = u;
    }
}

}  // namespace

cudaError_t setup_lpv(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_m1, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_select, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_m1_fd, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_select_fd, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_energy_fd, smem_optin);
    return e;
}

cudaError_t launch_m1(const KParams &kp, const Work &w, cudaStream_t s)
{
    const M1Layout L = m1_layout(kp.W, kp.box_vs, kp.tile_m1);
    const size_t smem = sizeof(int32_t) * (size_t)(L.R + 2 + 2 * kp.box_vs) * L.Wc;
    dim3 grid((kp.H + L.R - 1) / L.R, kp.n_frames);
    k_m1<<<grid, kM1Threads, smem, s>>>(kp, w, L.R, L.Wc);
    return cudaGetLastError();
}

cudaError_t launch_m1_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    const M1Layout L = m1_layout(kmax.W, kmax.box_vs, 0);
    const size_t smem = sizeof(int32_t) * (size_t)(L.R + 2 + 2 * kmax.box_vs) * L.Wc;
    dim3 grid((kmax.H + L.R - 1) / L.R, n);
    k_m1_fd<<<grid, kM1Threads, smem, s>>>(fd, L.R, L.Wc);
    return cudaGetLastError();
}

cudaError_t launch_energy_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    dim3 grid((kmax.n_starts + kEnThreads - 1) / kEnThreads, n);
    k_energy_fd<<<grid, kEnThreads, sizeof(float) * 3 * kmax.H, s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_select_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    k_select_fd<<<n, kSelThreads, sizeof(int) * (size_t)(kmax.n_starts + 4), s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_energy(const KParams &kp, const Work &w, cudaStream_t s)
{
    dim3 grid((kp.n_starts + kEnThreads - 1) / kEnThreads, kp.n_frames);
    k_energy<0><<<grid, kEnThreads, sizeof(float) * 3 * kp.H, s>>>(kp, w, nullptr, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_energy_list(const KParams &kp, const Work &w, const int32_t *elist, const int32_t *ecnt, int ecap,
                               cudaStream_t s)
{
    dim3 grid((ecap + kEnThreads - 1) / kEnThreads, kp.n_frames);
    k_energy<1><<<grid, kEnThreads, sizeof(float) * 3 * kp.H, s>>>(kp, w, elist, ecnt, ecap);
    return cudaGetLastError();
}

cudaError_t launch_energy_fallback(const KParams &kp, const Work &w, cudaStream_t s)
{
    dim3 grid((kp.n_starts + kEnThreads - 1) / kEnThreads, kp.n_frames);
    k_energy<2><<<grid, kEnThreads, sizeof(float) * 3 * kp.H, s>>>(kp, w, nullptr, nullptr, 0);
    return cudaGetLastError();
}

static cudaError_t select_mode(const KParams &kp, const Work &w, ld_lanes *out, const uint8_t *cflag, int mode,
                               cudaStream_t s)
{
    const size_t smem = sizeof(int) * (size_t)(kp.n_starts + 4);
    k_select<<<kp.n_frames, kSelThreads, smem, s>>>(kp, w, out, cflag, mode);
    return cudaGetLastError();
}

cudaError_t launch_tracks(const KParams &kp, const Work &w, const ld_lanes *lanes, float *out, cudaStream_t s)
{
    k_tracks<<<kp.n_frames, LD_MAX_LANES, 0, s>>>(kp, w, lanes, out);
    return cudaGetLastError();
}

cudaError_t launch_select(const KParams &kp, const Work &w, ld_lanes *out, cudaStream_t s)
{
    return select_mode(kp, w, out, nullptr, 0, s);
}

cudaError_t launch_select_set(const KParams &kp, const Work &w, const uint8_t *cflag, ld_lanes *out, cudaStream_t s)
{
    return select_mode(kp, w, out, cflag, 1, s);
}

cudaError_t launch_select_fallback(const KParams &kp, const Work &w, ld_lanes *out, cudaStream_t s)
{
    return select_mode(kp, w, out, nullptr, 2, s);
}

}  // namespace ld
