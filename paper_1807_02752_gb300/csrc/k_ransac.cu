// RANSAC least-squares fits, one CTA per frame:
//
//   k_fit<3>  Alg. 4 on the road DP path M_y (points (v_d, d)), least squares fit of Eq. 13 -> beta; then
//             the first road row f^-1(0) on the row grid and, per road row, f(v) and V_py(v) (Eq. 14).
//   k_fit<5>  Alg. 6 on the V_px DP path M_x (points (v, u_v)), fit of Eq. 19 / Eq. 20 -> gamma; then
//             V_px(v) (Eq. 22) per road row.
//
// Reading of the loop of Alg. 4 / Alg. 6 (draw a random sample, fit it, count inliers, drop the outliers,
// repeat until the inlier fraction reaches eps, then fit the inliers):
//   - each round draws `hyps` minimal samples (M points) from the working set S, listed in increasing point
//     index; draw j takes word j & 3 of Philox4x32-10 at counter (stage << 24 | round, hypothesis, j >> 2, 0)
//     with key = seed, and picks list position floor(word * |S| / 2^32); a draw repeating a chosen point or a
//     chosen row is skipped, and after 8 M draws without M points the hypothesis is void;
//   - the sample is fitted exactly (for M points the least squares fit is the interpolant): Newton divided
//     differences in float32 over tau = (v - centre) / 2^e, in draw order;
//   - inliers are points of S with (y - g(v))^2 < tr, g evaluated in float32 in nested Newton form;
//   - the hypothesis with most inliers (lowest index on ties) wins the round and its outliers leave S;
//   - the loop ends after the first round with eps_den n_I >= eps_num |S|, when no hypothesis is valid, or
//     at the round cap; the final fit is least squares over S, by the normal equations of Eq. 20 (exact
//     integer sums over t = v - centre, rounded once to double, scaled by exact powers of two - the kappa of
//     Eq. 20 - and solved in float64 by Gaussian elimination with partial pivoting; a pivot below 2^-40 is
//     singular).
//
// GB300 mapping: every THREAD fits one hypothesis in float32 (GB300's FP64 pipe is narrow, so float64 is
// kept to the final solve); inlier counts put consecutive hypotheses on consecutive lanes against the same
// point (broadcast loads, independent iterations); the final fit reduces each exact int128 sum on its own
// warp and solves the normal equations on one warp, one column per lane.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kFitThreads = 256;
constexpr int kNW = kFitThreads / 32;

__device__ __forceinline__ double p2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Normal equations of M unknowns from exact sums S = (Sx[0 .. 2M-2], Sy[0 .. M-1]), Sx[k] = sum t^k,
// Sy[k] = sum y t^k: A[r][c] = Sx[r + c] 2^-(r+c)e, b[r] = Sy[r] 2^-re (exact power-of-two column scaling),
// Gaussian elimination with partial pivoting (first row of largest |pivot|; a pivot below 2^-40 is
// singular), then back substitution; every product, difference and quotient rounded once, no FMA.  Solved
// on one warp: lane j <= M holds column j of the augmented matrix, the pivot column is broadcast with
// shuffles and every lane applies the elimination to its own column (the same operations, in the same
// order, as the serial algorithm); lane 0 back-substitutes.  All lanes of the warp must call it.  Returns
// 0 on every lane, or -1 if singular.
template <int M>
__device__ int solve_normal_warp(const __int128 *S, int e, double *coef)
{
    const int lane = threadIdx.x & 31;
    const int c = lane <= M ? lane : M;  // lanes past M shadow column M and are never read
    double col[M];
#pragma unroll
    for (int r = 0; r < M; ++r)
        col[r] = c < M ? __dmul_rn(i128_to_f64(S[r + c]), p2d(-(r + c) * e))
                       : __dmul_rn(i128_to_f64(S[2 * M - 1 + r]), p2d(-r * e));
#pragma unroll
    for (int k = 0; k < M; ++k) {
        double pc[M];  // column k (after the previous steps), from lane k
#pragma unroll
        for (int i = 0; i < M; ++i)
            pc[i] = __shfl_sync(0xffffffffu, col[i], k);
        int piv = k;
        double pa = fabs(pc[k]);
#pragma unroll
        for (int i = k + 1; i < M; ++i)
            if (fabs(pc[i]) > pa) {
                pa = fabs(pc[i]);
                piv = i;
            }
        if (!(pa >= 0x1p-40))
            return -1;
#pragma unroll
        for (int i = k + 1; i < M; ++i)
            if (i == piv) {
                double t = col[k];
                col[k] = col[i];
                col[i] = t;
                t = pc[k];
                pc[k] = pc[i];
                pc[i] = t;
            }
        if (c > k) {
#pragma unroll
            for (int i = k + 1; i < M; ++i) {
                const double fct = __ddiv_rn(pc[i], pc[k]);
                col[i] = __dsub_rn(col[i], __dmul_rn(fct, col[k]));
            }
        }
    }
    // back substitution on lane 0, rows gathered from the column lanes
    double A[M][M + 1];
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
        for (int j = 0; j <= M; ++j)
            A[r][j] = __shfl_sync(0xffffffffu, col[r], j);
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        double s = A[k][M];
#pragma unroll
        for (int j = k + 1; j < M; ++j)
            s = __dsub_rn(s, __dmul_rn(A[k][j], coef[j]));
        coef[k] = __ddiv_rn(s, A[k][k]);
    }
    return 0;
}

__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int d)
{
    long long lo = (long long)(unsigned long long)v;
    long long hi = (long long)(v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, d);
    hi = __shfl_down_sync(0xffffffffu, hi, d);
    return ((__int128)hi << 64) | (__int128)(unsigned long long)lo;
}

// Ascending list of the indices j < n with flag[j] != 0; returns the count.  chunk: >= n/32 + 2 ints.
__device__ int block_compact(const uint8_t *flag, int n, int16_t *list, int *chunk)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nch = (n + 31) >> 5;
    for (int c = warp; c < nch; c += kNW) {
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
    for (int c = warp; c < nch; c += kNW) {
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

template <typename T>
__device__ __forceinline__ T *carve(unsigned char *&p, size_t count)
{
    const size_t off = ((size_t)p + 15) & ~(size_t)15;
    T *r = reinterpret_cast<T *>(off);
    p = reinterpret_cast<unsigned char *>(off + sizeof(T) * count);
    return r;
}

// One hypothesis: the minimal sample of Philox draws and the polynomial through it in Newton form
// (nodes = the sample's tau in draw order, c = float32 divided differences, computed in place).
template <int M>
__device__ bool hypothesis(const KParams &kp, const int16_t *xs, const int16_t *ys, const int16_t *list, int ns,
                           int stage, int round, int h, float *c, float *nodes)
{
    int pick[M];
    int got = 0;
    uint4 blk = make_uint4(0u, 0u, 0u, 0u);
    for (int j = 0; j < 8 * M && got < M; ++j) {
        if ((j & 3) == 0)
            blk = philox4x32_10(make_uint4(((uint32_t)stage << 24) | (uint32_t)round, (uint32_t)h, (uint32_t)(j >> 2), 0u),
                                kp.key0, kp.key1);
        const uint32_t wv = (j & 3) == 0 ? blk.x : (j & 3) == 1 ? blk.y : (j & 3) == 2 ? blk.z : blk.w;
        const int idx = (int)(((unsigned long long)wv * (unsigned long long)ns) >> 32);
        if (!LD_IN(idx, ns, CK_FIT_SAMPLE))
            continue;
        const int pt = list[idx];
        bool dup = false;
        for (int q = 0; q < got; ++q)
            dup |= (pick[q] == pt) | (xs[pick[q]] == xs[pt]);
        if (!dup)
            pick[got++] = pt;
    }
    if (got < M)
        return false;
    const float sc = pow2f(-kp.e);
#pragma unroll
    for (int q = 0; q < M; ++q) {
        nodes[q] = __fmul_rn((float)(xs[pick[q]] - kp.centre), sc);
        c[q] = (float)ys[pick[q]];
    }
#pragma unroll
    for (int k = 1; k < M; ++k)
#pragma unroll
        for (int i = M - 1; i >= k; --i)
            c[i] = __fdiv_rn(__fsub_rn(c[i], c[i - 1]), __fsub_rn(nodes[i], nodes[i - k]));
    return true;
}

// Inlier test of a Newton-form hypothesis: (y - p(tau))^2 < tr, nested evaluation in float32.
template <int M>
__device__ __forceinline__ bool newton_inlier(const float *c, const float *nodes, int x, int y, int centre, float sc,
                                              float tr)
{
    const float tau = __fmul_rn((float)(x - centre), sc);
    float p = c[M - 1];
#pragma unroll
    for (int k = M - 2; k >= 0; --k)
        p = __fadd_rn(__fmul_rn(p, __fsub_rn(tau, nodes[k])), c[k]);
    const float r = __fsub_rn((float)y, p);
    return __fmul_rn(r, r) < tr;
}

template <int M>
__device__ __forceinline__ void fit_body(const KParams &kp, const Work &w, const int f)
{
    constexpr int stage = M == 3 ? 0 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double coef_s[M];
    __shared__ int sh[4];
    const int H = kp.H, P = w.pmax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FrameState fs0 = w.fs[f];
    if (stage == 1 && (fs0.flags & LD_F_NO_LANES))
        return;
    const int n0 = w.npts[f * 2 + stage];
    const int n = LD_IN(n0, P + 1, CK_FIT_NPTS) ? n0 : 0;   // a point list holds at most P points
    const int16_t *gp = w.pts + ((size_t)f * 2 + stage) * 3 * P;

    unsigned char *p = smem;
    int16_t *xs = carve<int16_t>(p, P);
    int16_t *ys = carve<int16_t>(p, P);
    int16_t *pid = carve<int16_t>(p, P);
    uint8_t *member = carve<uint8_t>(p, P);
    int16_t *list = carve<int16_t>(p, P);
    int *chunk = carve<int>(p, (P + 31) / 32 + 2);
    int *hyp_ok = carve<int>(p, kMaxHyps);
    int *hyp_cnt = carve<int>(p, kMaxHyps);
    float *hyp_cf = carve<float>(p, kMaxHyps * 2 * M);  // per hypothesis: M divided differences, M nodes
    __int128 *red = carve<__int128>(p, kNW * (3 * M - 1));
    int *redc = carve<int>(p, kNW);

    for (int j = tid; j < n; j += kFitThreads) {
        xs[j] = gp[j];
        ys[j] = gp[P + j];
        pid[j] = gp[2 * P + j];
        member[j] = 1;
    }
    __syncthreads();

    const int centre = kp.centre;
    const float sc = pow2f(-kp.e);
    const float tr = stage == 0 ? kp.tr_y : kp.tr_x;
    int fl = 0, round = 0;
    for (;;) {
        const int ns = block_compact(member, n, list, chunk);
        if (ns < M) {
            fl |= 2;
            break;
        }
        if (round == kp.rounds) {
            fl |= 1;
            break;
        }
        for (int h = tid; h < kp.hyps; h += kFitThreads) {
            float c[M], nodes[M];
            const bool ok = hypothesis<M>(kp, xs, ys, list, ns, stage, round, h, c, nodes);
            hyp_ok[h] = ok;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                hyp_cf[h * 2 * M + k] = ok ? c[k] : 0.0f;
                hyp_cf[h * 2 * M + M + k] = ok ? nodes[k] : 0.0f;
            }
        }
        __syncthreads();
        // inlier counts: consecutive lanes take consecutive hypotheses against the same point (broadcast
        // point loads, independent iterations); a thread adds its count when its hypothesis changes
        for (int h = tid; h < kp.hyps; h += kFitThreads)
            hyp_cnt[h] = hyp_ok[h] ? 0 : -1;
        __syncthreads();
        {
            const int nh = kp.hyps, dh = kFitThreads % nh, dq = kFitThreads / nh;
            if (dh == 0) {
                // the thread's hypothesis is fixed: a plain strided loop the compiler can overlap
                const int h = tid % nh;
                if (hyp_ok[h]) {
                    float cf[2 * M];
#pragma unroll
                    for (int k = 0; k < 2 * M; ++k)
                        cf[k] = hyp_cf[h * 2 * M + k];
                    int c = 0;
#pragma unroll 4
                    for (int q = tid / nh; q < ns; q += dq) {
                        const int j = list[q];
                        c += newton_inlier<M>(cf, cf + M, xs[j], ys[j], centre, sc, tr);
                    }
                    if (c)
                        atomicAdd(&hyp_cnt[h], c);
                }
            } else {
                int h = tid % nh, q = tid / nh, cur = -1, c = 0;
                bool ok = false;
                float cf[2 * M];
                for (; q < ns; q += dq) {
                    if (h != cur) {
                        if (ok && c)
                            atomicAdd(&hyp_cnt[cur], c);
                        cur = h;
                        c = 0;
                        ok = hyp_ok[h] != 0;
#pragma unroll
                        for (int k = 0; k < 2 * M; ++k)
                            cf[k] = hyp_cf[h * 2 * M + k];
                    }
                    if (ok) {
                        const int j = list[q];
                        c += newton_inlier<M>(cf, cf + M, xs[j], ys[j], centre, sc, tr);
                    }
                    h += dh;
                    if (h >= nh) {
                        h -= nh;
                        ++q;
                    }
                }
                if (ok && c)
                    atomicAdd(&hyp_cnt[cur], c);
            }
        }
        __syncthreads();
        if (warp == 0) {
            int bc = -1, bh = 0x7fffffff;
            for (int h = lane; h < kp.hyps; h += 32)
                if (hyp_cnt[h] > bc) {
                    bc = hyp_cnt[h];
                    bh = h;
                }
            for (int d = 16; d > 0; d >>= 1) {
                const int oc = __shfl_down_sync(0xffffffffu, bc, d);
                const int oh = __shfl_down_sync(0xffffffffu, bh, d);
                if (oc > bc || (oc == bc && oh < bh)) {
                    bc = oc;
                    bh = oh;
                }
            }
            if (lane == 0) {
                sh[0] = bh;
                sh[1] = bc;
            }
        }
        __syncthreads();
        const int bh = sh[0], bc = sh[1];
        ++round;
        if (bc < 0) {
            fl |= 2;
            break;
        }
        float cf[2 * M];
#pragma unroll
        for (int k = 0; k < 2 * M; ++k)
            cf[k] = hyp_cf[bh * 2 * M + k];
        for (int j = tid; j < n; j += kFitThreads)
            if (member[j] && !newton_inlier<M>(cf, cf + M, xs[j], ys[j], centre, sc, tr))
                member[j] = 0;
        __syncthreads();
        if ((long long)kp.eps_den * bc >= (long long)kp.eps_num * ns)
            break;
    }
    // final least squares over the remaining set: exact sums (sum t^k for k <= 2M-2, then
    // sum y t^k for k < M), then the normal equations solved on one warp
    if (!(fl & 2)) {
        constexpr int NS = 3 * M - 1;
        if constexpr (M == 5) {
            // each thread's points: the powers of t built once per point, all NS sums at a time
            __int128 acc[NS];
#pragma unroll
            for (int k = 0; k < NS; ++k)
                acc[k] = 0;
            int cnt = 0;
            for (int j = tid; j < n; j += kFitThreads)
                if (member[j]) {
                    const __int128 t = (__int128)(xs[j] - centre), y = (__int128)ys[j];
                    __int128 pw = 1;
#pragma unroll
                    for (int k = 0; k < 2 * M - 1; ++k) {
                        acc[k] += pw;
                        if (k < M)
                            acc[2 * M - 1 + k] += y * pw;
                        pw *= t;
                    }
                    ++cnt;
                }
            // warp sums, then the warps' partial sums added by one warp (integer: the order does not matter)
#pragma unroll
            for (int k = 0; k < NS; ++k)
#pragma unroll
                for (int d = 16; d > 0; d >>= 1)
                    acc[k] += shfl_down_i128(acc[k], d);
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < NS; ++k)
                    red[warp * NS + k] = acc[k];
                redc[warp] = cnt;
            }
            __syncthreads();
            if (warp == 0) {
                __int128 s = 0;
                int c = 0;
                if (lane < NS)
                    for (int wv = 0; wv < kNW; ++wv)
                        s += red[wv * NS + lane];
                for (int wv = 0; wv < kNW; ++wv)
                    c += redc[wv];
                __syncwarp();
                if (lane < NS)
                    red[lane] = s;
                if (lane == 0)
                    redc[0] = c;
            }
            __syncthreads();
        } else {   // M = 3: one warp per sum measured faster (8 sums: one round of the 8 warps)
            for (int sidx = warp; sidx < NS; sidx += kNW) {
                const int pk = sidx < 2 * M - 1 ? sidx : sidx - (2 * M - 1);
                __int128 acc = 0;
                int cnt = 0;
                for (int j = lane; j < n; j += 32)
                    if (member[j]) {
                        const __int128 t = (__int128)(xs[j] - centre);
                        __int128 pw = sidx < 2 * M - 1 ? (__int128)1 : (__int128)ys[j];
                        for (int k = 0; k < pk; ++k)
                            pw *= t;
                        acc += pw;
                        ++cnt;
                    }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1)
                    acc += shfl_down_i128(acc, d);
                cnt = __reduce_add_sync(0xffffffffu, cnt);
                if (lane == 0) {
                    red[sidx] = acc;
                    if (sidx == 0)
                        redc[0] = cnt;
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
            double cd[M];
            int ok = redc[0] >= M ? solve_normal_warp<M>(red, kp.e, cd) == 0 : 0;
            if (lane == 0) {
                if (ok)
                    for (int k = 0; k < M; ++k)
                        coef_s[k] = cd[k];
                sh[2] = ok;
            }
        }
        __syncthreads();
        if (!sh[2])
            fl |= 2;
    }

    const double sc64 = p2d(-kp.e);
    if (stage == 0) {
        uint8_t *inl = w.inl_y + (size_t)f * kp.D;
        for (int d = tid; d < kp.D; d += kFitThreads)
            inl[d] = 0;
        __syncthreads();
        for (int j = tid; j < n; j += kFitThreads)
            if (LD_IN(pid[j], kp.D, CK_FIT_ROW))
                inl[pid[j]] = member[j];
        int flags = 0;
        if (fl & 1)
            flags |= LD_F_CAP_Y;
        if (fl & 2)
            flags |= LD_F_DEGEN_Y;
        double beta[3] = {0.0, 0.0, 0.0};
        int vtop = H;
        float *rows = w.rows + (size_t)f * 3 * H;
        if (!(fl & 2)) {
            for (int i = 0; i < 3; ++i)
                beta[i] = coef_s[i];
            // v_top: first row of the bottom run of rows with f(v) > 0 and f'(v) > 0
            int worst = -1;
            for (int v = tid; v < H; v += kFitThreads) {
                const double tau = __dmul_rn((double)(v - centre), sc64);
                const double fv = poly_f64<3>(beta, tau);
                const double dfv = __dmul_rn(__dadd_rn(beta[1], __dmul_rn(__dmul_rn(2.0, beta[2]), tau)), sc64);
                if (!(fv > 0.0 && dfv > 0.0))
                    worst = max(worst, v);
            }
            worst = __reduce_max_sync(0xffffffffu, worst);
            if (lane == 0)
                redc[warp] = worst;
            __syncthreads();
            if (tid == 0) {
                int m = -1;
                for (int i = 0; i < kNW; ++i)
                    m = max(m, redc[i]);
                sh[3] = m + 1;
            }
            __syncthreads();
            vtop = sh[3];
            for (int v = tid; v < H; v += kFitThreads) {
                float F = 0.0f, Vy = 0.0f;
                if (v >= vtop) {
                    const double tau = __dmul_rn((double)(v - centre), sc64);
                    const double fv = poly_f64<3>(beta, tau);
                    const double dfv = __dmul_rn(__dadd_rn(beta[1], __dmul_rn(__dmul_rn(2.0, beta[2]), tau)), sc64);
                    F = __double2float_rn(fv);
                    Vy = __double2float_rn(__dsub_rn((double)v, __ddiv_rn(fv, dfv)));
                }
                rows[v] = F;
                rows[H + v] = Vy;
                rows[2 * H + v] = 0.0f;
            }
            if (vtop > H - 1)
                flags |= LD_F_NO_ROAD;
        } else {
            for (int v = tid; v < 3 * H; v += kFitThreads)
                rows[v] = 0.0f;
        }
        if (flags & (LD_F_DEGEN_Y | LD_F_NO_ROAD))
            flags |= LD_F_NO_LANES;
        if (tid == 0) {
            FrameState &fs = w.fs[f];
            fs.flags = flags;
            fs.v_top = vtop;
            fs.rounds_y = round;
            fs.rounds_x = 0;
            for (int i = 0; i < 3; ++i)
                fs.beta[i] = beta[i];
            for (int i = 0; i < 5; ++i)
                fs.gamma[i] = 0.0;
        }
    } else {
        uint8_t *inl = w.inl_x + (size_t)f * H;
        for (int v = tid; v < H; v += kFitThreads)
            inl[v] = 0;
        __syncthreads();
        for (int j = tid; j < n; j += kFitThreads)
            if (LD_IN(pid[j], H, CK_FIT_ROW))
                inl[pid[j]] = member[j];
        int flags = fs0.flags;
        if (fl & 1)
            flags |= LD_F_CAP_X;
        if (fl & 2)
            flags |= LD_F_DEGEN_X | LD_F_NO_LANES;
        double gamma[5] = {0, 0, 0, 0, 0};
        if (!(fl & 2)) {
            for (int i = 0; i < 5; ++i)
                gamma[i] = coef_s[i];
            float *Vpx = w.rows + (size_t)f * 3 * H + 2 * H;
            for (int v = fs0.v_top + tid; v < H; v += kFitThreads)
                Vpx[v] = __double2float_rn(poly_f64<5>(gamma, __dmul_rn((double)(v - centre), sc64)));
        }
        if (tid == 0) {
            FrameState &fs = w.fs[f];
            fs.flags = flags;
            fs.rounds_x = round;
            for (int i = 0; i < 5; ++i)
                fs.gamma[i] = gamma[i];
        }
    }
}

template <int M>
__global__ void __launch_bounds__(kFitThreads) k_fit(const KParams kp, const Work w) { fit_body<M>(kp, w, blockIdx.x); }
template <int M>
__global__ void __launch_bounds__(kFitThreads) k_fit_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.x];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    fit_body<M>(kp, w, 0);
}

template <int M>
size_t fit_smem(int P)
{
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(2 * (size_t)P);
    add(2 * (size_t)P);
    add(2 * (size_t)P);
    add((size_t)P);
    add(2 * (size_t)P);
    add(4 * (size_t)((P + 31) / 32 + 2));
    add(4 * kMaxHyps);
    add(4 * kMaxHyps);
    add(4 * kMaxHyps * 2 * M);
    add(16 * kNW * (3 * M - 1));
    add(4 * kNW);
    return s + 16;
}

}  // namespace

cudaError_t setup_ransac(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_fit<3>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_fit_fd<3>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_fit_fd<5>, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_fit<5>, smem_optin);
    return e;
}

cudaError_t launch_fit_y(const KParams &kp, const Work &w, cudaStream_t s)
{
    k_fit<3><<<kp.n_frames, kFitThreads, fit_smem<3>(w.pmax), s>>>(kp, w);
    return cudaGetLastError();
}

cudaError_t launch_fit_y_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    k_fit_fd<3><<<n, kFitThreads, fit_smem<3>(kmax.pmax_hint), s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_fit_x_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    k_fit_fd<5><<<n, kFitThreads, fit_smem<5>(kmax.pmax_hint), s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_fit_x(const KParams &kp, const Work &w, cudaStream_t s)
{
    k_fit<5><<<kp.n_frames, kFitThreads, fit_smem<5>(w.pmax), s>>>(kp, w);
    return cudaGetLastError();
}

}  // namespace ld
