// Serial per-frame stages, one CTA per frame:
//
//   k_road  Sec. 2.2: DP over the v-disparity map (Eq. 11-12), RANSAC road profile (Alg. 4 with the
//           least squares fit of Eq. 13), first road row f^-1(0) and V_py(v) (Eq. 14).
//   k_vpx   Sec. 2.3.2-2.3.3: dense accumulator (Alg. 5) built on the fly as a sliding band of vote
//           rows, DP (Eq. 18), RANSAC quartic (Alg. 6, Eq. 19-21), V_px(v) (Eq. 22).
//
// Readings shared with the rest of the library:
//   - Eq. 12 links (d, v) to (d+1, v + tau), tau in [0, tau_y], cost +lambda_y tau; Eq. 18 links (u, v)
//     to (u + tau, v + 1), tau in [-tau_x, tau_x], cost +lambda_x |tau|.  Ties: the smaller |tau|, then the
//     negative tau; the path starts at the smallest index minimising the last row.
//   - a path point whose cell holds no count carries no observation and is left out of the fit;
//   - RANSAC: each round draws `hyps` minimal samples (3 points for beta, 5 for gamma) with Philox4x32-10
//     at counter (stage << 24 | round, hypothesis, draw >> 2, 0), keeps the sample with most inliers
//     (lowest index on ties), drops its outliers, and stops after the first round whose best count n_I
//     satisfies eps_den n_I >= eps_num n, or at the round cap; the final fit is least squares over the rest;
//   - fits solve the normal equations of Eq. 20 from exact integer sums over t = v - centre, rounded once
//     to double and scaled by exact powers of two (the kappa of Eq. 20), by Gaussian elimination with
//     partial pivoting; inlier tests evaluate the model in float32.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kRoadThreads = 512;
constexpr int kVpxThreads = 1024;
constexpr int kMaxChunks = (LD_MAX_H + 31) / 32 + 2;

__device__ __forceinline__ double p2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Normal equations of M unknowns from exact sums Sx[k] = sum t^k (k <= 2M-2), Sy[k] = sum y t^k.
// Gaussian elimination with partial pivoting (first row of largest |pivot|); a pivot below 2^-40 means
// singular.  Every operation is one IEEE rounding, in a fixed order.
template <int M>
__device__ int solve_normal(const __int128 *Sx, const __int128 *Sy, int e, double *coef)
{
    double A[M][M + 1];
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
        for (int k = 0; k < M; ++k)
            A[j][k] = __dmul_rn(i128_to_f64(Sx[j + k]), p2d(-(j + k) * e));
        A[j][M] = __dmul_rn(i128_to_f64(Sy[j]), p2d(-j * e));
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        int piv = k;
#pragma unroll
        for (int i = k + 1; i < M; ++i)
            if (fabs(A[i][k]) > fabs(A[piv][k]))
                piv = i;
        double pv = A[k][k];
#pragma unroll
        for (int i = k + 1; i < M; ++i)
            if (i == piv)
                pv = A[i][k];
        if (!(fabs(pv) >= 0x1p-40))
            return -1;
#pragma unroll
        for (int i = k + 1; i < M; ++i) {
            if (i == piv) {
#pragma unroll
                for (int j = 0; j <= M; ++j) {
                    const double t = A[k][j];
                    A[k][j] = A[i][j];
                    A[i][j] = t;
                }
            }
        }
#pragma unroll
        for (int i = k + 1; i < M; ++i) {
            const double fct = __ddiv_rn(A[i][k], A[k][k]);
#pragma unroll
            for (int j = k + 1; j <= M; ++j)
                A[i][j] = __dsub_rn(A[i][j], __dmul_rn(fct, A[k][j]));
        }
    }
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

template <int M>
__device__ __forceinline__ void add_point(__int128 *Sx, __int128 *Sy, int x, int y, int centre)
{
    const __int128 t = (__int128)(x - centre);
    __int128 pw = 1;
#pragma unroll
    for (int k = 0; k <= 2 * M - 2; ++k) {
        Sx[k] += pw;
        if (k < M)
            Sy[k] += pw * (__int128)y;
        pw *= t;
    }
}

__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int d)
{
    long long lo = (long long)(unsigned long long)v;
    long long hi = (long long)(v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, d);
    hi = __shfl_down_sync(0xffffffffu, hi, d);
    return ((__int128)hi << 64) | (__int128)(unsigned long long)lo;
}

// List (ascending) of the indices j < n with flag[j] != 0; returns the count.  chunk: >= n/32 + 2 ints.
template <int NT>
__device__ int block_compact(const uint8_t *flag, int n, int16_t *list, int *chunk)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = NT / 32;
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

// Shared-memory layout of one RANSAC run.
struct RansacMem {
    const int16_t *xs, *ys;   // points (x = row, y = d or u)
    uint8_t *member;          // [n] working set
    int16_t *list;            // [n]
    int *hyp_cnt;             // [hyps]
    float *hyp_cf;            // [hyps][M]
    int *sh;                  // >= kMaxChunks + 8 ints
    __int128 *red;            // [NT / 32][3 M - 1]
};

// Alg. 4 / Alg. 6 on n points.  Returns flags: 1 = round cap, 2 = degenerate; coef (lane 0 of thread 0
// holds it in shared memory afterwards via out) and the number of rounds.
template <int M, int NT>
__device__ int ransac_block(const KParams &kp, const RansacMem &R, int n, float tr, int stage, double *coef_out,
                            int *rounds_out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = NT / 32;
    const int centre = kp.centre;
    const float sc = pow2f(-kp.e);
    int *sh = R.sh;
    int *chunk = sh + 8;
    for (int j = threadIdx.x; j < n; j += NT)
        R.member[j] = 1;
    __syncthreads();
    int flags = 0, round = 0;
    for (;;) {
        const int ns = block_compact<NT>(R.member, n, R.list, chunk);
        if (ns < M) {
            flags |= 2;
            break;
        }
        if (round == kp.rounds) {
            flags |= 1;
            break;
        }
        for (int h = warp; h < kp.hyps; h += nw) {
            double cd[M];
#pragma unroll
            for (int k = 0; k < M; ++k)
                cd[k] = 0.0;
            int valid = 0;
            if (lane == 0) {
                int pick[M];
                int got = 0;
                uint4 blk = make_uint4(0, 0, 0, 0);
                for (int j = 0; j < 8 * M && got < M; ++j) {
                    if ((j & 3) == 0)
                        blk = philox4x32_10(make_uint4(((uint32_t)stage << 24) | (uint32_t)round, (uint32_t)h,
                                                       (uint32_t)(j >> 2), 0u),
                                            kp.key0, kp.key1);
                    const uint32_t wv = (j & 3) == 0 ? blk.x : (j & 3) == 1 ? blk.y : (j & 3) == 2 ? blk.z : blk.w;
                    const int pos = (int)(((unsigned long long)wv * (unsigned long long)ns) >> 32);
                    const int pt = R.list[pos];
                    bool dup = false;
                    for (int q = 0; q < got; ++q)
                        dup |= (pick[q] == pt) | (R.xs[pick[q]] == R.xs[pt]);
                    if (!dup)
                        pick[got++] = pt;
                }
                if (got == M) {
                    __int128 Sx[2 * M - 1], Sy[M];
#pragma unroll
                    for (int k = 0; k < 2 * M - 1; ++k)
                        Sx[k] = 0;
#pragma unroll
                    for (int k = 0; k < M; ++k)
                        Sy[k] = 0;
                    for (int q = 0; q < M; ++q)
                        add_point<M>(Sx, Sy, R.xs[pick[q]], R.ys[pick[q]], centre);
                    valid = solve_normal<M>(Sx, Sy, kp.e, cd) == 0;
                }
            }
            valid = __shfl_sync(0xffffffffu, valid, 0);
            float cf[M];
#pragma unroll
            for (int k = 0; k < M; ++k)
                cf[k] = __shfl_sync(0xffffffffu, __double2float_rn(cd[k]), 0);
            int cnt = -1;
            if (valid) {
                int c = 0;
                for (int q = lane; q < ns; q += 32) {
                    const int j = R.list[q];
                    c += inlier_test<M>(cf, R.xs[j], R.ys[j], centre, sc, tr);
                }
                cnt = __reduce_add_sync(0xffffffffu, c);
            }
            if (lane == 0) {
                R.hyp_cnt[h] = cnt;
#pragma unroll
                for (int k = 0; k < M; ++k)
                    R.hyp_cf[h * M + k] = cf[k];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int bh = -1, bc = -1;
            for (int h = 0; h < kp.hyps; ++h)
                if (R.hyp_cnt[h] > bc) {
                    bc = R.hyp_cnt[h];
                    bh = h;
                }
            sh[0] = bh;
            sh[1] = bc;
        }
        __syncthreads();
        const int bh = sh[0], bc = sh[1];
        ++round;
        if (bc < 0) {
            flags |= 2;
            break;
        }
        float cf[M];
#pragma unroll
        for (int k = 0; k < M; ++k)
            cf[k] = R.hyp_cf[bh * M + k];
        for (int j = threadIdx.x; j < n; j += NT)
            if (R.member[j] && !inlier_test<M>(cf, R.xs[j], R.ys[j], centre, sc, tr))
                R.member[j] = 0;
        __syncthreads();
        if ((long long)kp.eps_den * bc >= (long long)kp.eps_num * ns)
            break;
    }
    // final least squares over the remaining set (exact sums, reduced across the block)
    if (!(flags & 2)) {
        __int128 S[3 * M - 1];
#pragma unroll
        for (int k = 0; k < 3 * M - 1; ++k)
            S[k] = 0;
        int cnt = 0;
        for (int j = threadIdx.x; j < n; j += NT)
            if (R.member[j]) {
                add_point<M>(S, S + 2 * M - 1, R.xs[j], R.ys[j], centre);
                ++cnt;
            }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
#pragma unroll
        for (int k = 0; k < 3 * M - 1; ++k)
            for (int d = 16; d > 0; d >>= 1)
                S[k] += shfl_down_i128(S[k], d);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 3 * M - 1; ++k)
                R.red[warp * (3 * M - 1) + k] = S[k];
            chunk[warp] = cnt;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __int128 T[3 * M - 1];
            int total = 0;
#pragma unroll
            for (int k = 0; k < 3 * M - 1; ++k)
                T[k] = 0;
            for (int wi = 0; wi < nw; ++wi) {
#pragma unroll
                for (int k = 0; k < 3 * M - 1; ++k)
                    T[k] += R.red[wi * (3 * M - 1) + k];
                total += chunk[wi];
            }
            int ok = total >= M;
            if (ok)
                ok = solve_normal<M>(T, T + 2 * M - 1, kp.e, coef_out) == 0;
            sh[2] = ok;
        }
        __syncthreads();
        if (!sh[2])
            flags |= 2;
        __syncthreads();
    }
    *rounds_out = round;
    return flags;
}

template <typename T>
__device__ __forceinline__ T *carve(unsigned char *&p, size_t count)
{
    size_t off = ((size_t)p + 15) & ~(size_t)15;
    T *r = reinterpret_cast<T *>(off);
    p = reinterpret_cast<unsigned char *>(off + sizeof(T) * count);
    return r;
}

// Lexicographic (value, index) minimum over the block; every thread returns the winning index.
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

// ---------------------------------------------------------------------------------------------------
// k_road
// ---------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRoadThreads) k_road(const KParams kp, const Work w)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int f = blockIdx.x, H = kp.H, D = kp.D, Hp = (H + 1) >> 1;
    const int tid = threadIdx.x;
    const int32_t *my = w.myT + (size_t)f * D * H;

    unsigned char *p = smem;
    int *E0 = carve<int>(p, H);
    int *E1 = carve<int>(p, H);
    int *sh = carve<int>(p, kMaxChunks + 8 + 2 * (kRoadThreads / 32));
    int16_t *path = carve<int16_t>(p, D);
    unsigned char *dyn = p;                       // DP backtrack, later RANSAC scratch
    uint8_t *bt = carve<uint8_t>(p, (size_t)D * Hp);

    // ---- Eq. 12 DP, d = D-1 down to 1 ----
    for (int v = tid; v < H; v += kRoadThreads)
        E0[v] = -my[(size_t)(D - 1) * H + v];
    __syncthreads();
    int *Ep = E0, *Ec = E1;
    const int tau = kp.tau_y, lam = kp.lambda_y;
    for (int d = D - 2; d >= 1; --d) {
        const int32_t *row = my + (size_t)d * H;
        for (int i = tid; i < Hp; i += kRoadThreads) {
            uint8_t nib = 0;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int v = 2 * i + half;
                if (v < H) {
                    int best = 0x7fffffff, arg = 0;
                    for (int t = 0; t <= tau && v + t < H; ++t) {
                        const int cand = Ep[v + t] + lam * t;
                        if (cand < best) {
                            best = cand;
                            arg = t;
                        }
                    }
                    Ec[v] = -row[v] + best;
                    nib |= (uint8_t)(arg << (4 * half));
                }
            }
            bt[(size_t)d * Hp + i] = nib;
        }
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    // argmin over v of E_1, smallest v on ties
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int v = tid; v < H; v += kRoadThreads)
        if (Ep[v] < bv) {
            bv = Ep[v];
            bi = v;
        }
    const int vstar = block_argmin<kRoadThreads>(bv, bi, sh + kMaxChunks + 8);
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

    // ---- points with data: (x = v_d, y = d) for d = 1..D-1 with m_y(d, v_d) > 0 ----
    p = dyn;
    int16_t *xs = carve<int16_t>(p, D);
    int16_t *ys = carve<int16_t>(p, D);
    uint8_t *flag = carve<uint8_t>(p, D);
    int16_t *pid = carve<int16_t>(p, D);
    RansacMem R;
    R.member = carve<uint8_t>(p, D);
    R.list = carve<int16_t>(p, D);
    R.hyp_cnt = carve<int>(p, kMaxHyps);
    R.hyp_cf = carve<float>(p, kMaxHyps * 3);
    R.red = carve<__int128>(p, (kRoadThreads / 32) * 8);
    R.sh = sh;
    for (int d = tid; d < D; d += kRoadThreads)
        flag[d] = d >= 1 && my[(size_t)d * H + path[d]] > 0;
    __syncthreads();
    const int k = block_compact<kRoadThreads>(flag, D, pid, sh + 8);
    for (int j = tid; j < k; j += kRoadThreads) {
        xs[j] = path[pid[j]];
        ys[j] = pid[j];
    }
    __syncthreads();
    R.xs = xs;
    R.ys = ys;
    __shared__ double beta_s[3];
    int rounds = 0;
    const int fl = ransac_block<3, kRoadThreads>(kp, R, k, kp.tr_y, 0, beta_s, &rounds);

    int flags = 0;
    if (fl & 1)
        flags |= LD_F_CAP_Y;
    if (fl & 2)
        flags |= LD_F_DEGEN_Y;
    // outputs of the DP and the fit
    for (int d = tid; d < D; d += kRoadThreads) {
        w.path_y[(size_t)f * D + d] = path[d];
        w.inl_y[(size_t)f * D + d] = 0;
    }
    __syncthreads();
    for (int j = tid; j < k; j += kRoadThreads)
        w.inl_y[(size_t)f * D + pid[j]] = R.member[j];

    // ---- rows: v_top = first row of the bottom run with f > 0 and f' > 0; f(v), V_py(v) (Eq. 14) ----
    float *rows = w.rows + (size_t)f * 3 * H;
    double beta[3] = {0.0, 0.0, 0.0};
    int vtop = H;
    if (!(fl & 2)) {
        beta[0] = beta_s[0];
        beta[1] = beta_s[1];
        beta[2] = beta_s[2];
        const double sc = p2d(-kp.e);
        int worst = -1;
        for (int v = tid; v < H; v += kRoadThreads) {
            const double tau_v = __dmul_rn((double)(v - kp.centre), sc);
            const double fv = poly_f64<3>(beta, tau_v);
            const double dfv = __dmul_rn(__dadd_rn(beta[1], __dmul_rn(__dmul_rn(2.0, beta[2]), tau_v)), sc);
            if (!(fv > 0.0 && dfv > 0.0))
                worst = max(worst, v);
        }
        worst = __reduce_max_sync(0xffffffffu, worst);
        if ((tid & 31) == 0)
            sh[kMaxChunks + 8 + (tid >> 5)] = worst;
        __syncthreads();
        if (tid == 0) {
            int m = -1;
            for (int i = 0; i < kRoadThreads / 32; ++i)
                m = max(m, sh[kMaxChunks + 8 + i]);
            sh[2] = m + 1;
        }
        __syncthreads();
        vtop = sh[2];
        for (int v = tid; v < H; v += kRoadThreads) {
            float F = 0.0f, Vy = 0.0f;
            if (v >= vtop) {
                const double tau_v = __dmul_rn((double)(v - kp.centre), sc);
                const double fv = poly_f64<3>(beta, tau_v);
                const double dfv = __dmul_rn(__dadd_rn(beta[1], __dmul_rn(__dmul_rn(2.0, beta[2]), tau_v)), sc);
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
        for (int v = tid; v < H; v += kRoadThreads) {
            rows[v] = 0.0f;
            rows[H + v] = 0.0f;
            rows[2 * H + v] = 0.0f;
        }
    }
    if (flags & (LD_F_DEGEN_Y | LD_F_NO_ROAD))
        flags |= LD_F_NO_LANES;
    if (tid == 0) {
        FrameState &fs = w.fs[f];
        fs.flags = flags;
        fs.v_top = vtop;
        fs.rounds_y = rounds;
        fs.rounds_x = 0;
        for (int i = 0; i < 3; ++i)
            fs.beta[i] = beta[i];
        for (int i = 0; i < 5; ++i)
            fs.gamma[i] = 0.0;
    }
}

// ---------------------------------------------------------------------------------------------------
// k_vpx
// ---------------------------------------------------------------------------------------------------
struct VpxMem {
    int *E0, *E1, *band;
    int *voff;          // [H + 1] offsets of the staged vote rows
    int16_t *vb;        // [vote_cap] staged vote columns
    int16_t *path;      // [H]
    uint8_t *sup;       // [H]
    int *sh;
    uint8_t *bt;        // [seg_rows][Wp]
    unsigned char *dyn; // start of the reusable region (bt)
};

// Add (sign = +1) or remove (-1) the votes of row r to the band histogram.
__device__ __forceinline__ void band_row(const KParams &kp, const Work &w, const VpxMem &S, int f, int r, int sign,
                                         bool staged)
{
    const int cnt = w.vcount[(size_t)f * kp.H + r];
    if (staged) {
        const int16_t *src = S.vb + S.voff[r];
        for (int q = threadIdx.x; q < cnt; q += kVpxThreads)
            atomicAdd(&S.band[src[q]], sign);
    } else {
        const int16_t *src = w.vbins + ((size_t)f * kp.H + r) * kp.W;
        for (int q = threadIdx.x; q < cnt; q += kVpxThreads)
            atomicAdd(&S.band[src[q]], sign);
    }
}

// One Eq. 18 step: E_v from E_{v+1} (Ep) and the band of row v; backtrack nibbles to bt row `slot`.
__device__ __forceinline__ void dp_row(const KParams &kp, const VpxMem &S, const int *Ep, int *Ec, int slot)
{
    const int W = kp.W, Wp = (W + 1) >> 1, tau = kp.tau_x, lam = kp.lambda_x, rho = kp.vote_rho;
    for (int i = threadIdx.x; i < Wp; i += kVpxThreads) {
        uint8_t nib = 0;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int u = 2 * i + half;
            if (u < W) {
                int best = 0x7fffffff, arg = 0;
                for (int k = 0; k <= 2 * tau; ++k) {
                    const int t = (k & 1) ? -((k + 1) >> 1) : (k >> 1);
                    const int uu = u + t;
                    if (uu < 0 || uu >= W)
                        continue;
                    const int cand = Ep[uu] + lam * (t < 0 ? -t : t);
                    if (cand < best) {
                        best = cand;
                        arg = t;
                    }
                }
                Ec[u] = -rho * S.band[u] + best;
                nib |= (uint8_t)((arg & 15) << (4 * half));
            }
        }
        S.bt[(size_t)slot * Wp + i] = nib;
    }
}

__device__ __forceinline__ int bt_get(const VpxMem &S, int Wp, int slot, int u)
{
    const uint8_t b = S.bt[(size_t)slot * Wp + (u >> 1)];
    const int nib = (u & 1) ? (b >> 4) : (b & 15);
    return (nib ^ 8) - 8;  // 4-bit two's complement
}

__global__ void __launch_bounds__(kVpxThreads) k_vpx(const KParams kp, const Work w)
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
    S.E0 = carve<int>(p, W);
    S.E1 = carve<int>(p, W);
    S.band = carve<int>(p, W);
    S.voff = carve<int>(p, H + 1);
    S.vb = carve<int16_t>(p, kp.vote_cap);
    S.path = carve<int16_t>(p, H);
    S.sup = carve<uint8_t>(p, H);
    S.sh = carve<int>(p, kMaxChunks + 8 + 2 * (kVpxThreads / 32));
    S.dyn = p;
    S.bt = carve<uint8_t>(p, (size_t)kp.seg_rows * Wp);

    // ---- stage the vote rows [vtop, vmax] in shared memory when they fit ----
    for (int v = tid; v < H; v += kVpxThreads)
        S.voff[v] = v >= vtop ? w.vcount[(size_t)f * H + v] : 0;
    for (int u = tid; u < W; u += kVpxThreads)
        S.band[u] = 0;
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

    // ---- forward DP over rows vmax-1 .. vtop, segment k = rows [vtop + k S, vtop + (k+1) S - 1] ----
    const int SR = kp.seg_rows;
    const int nrows = vmax - vtop;  // rows that get a backtrack entry
    const int nseg = (nrows + SR - 1) / SR;
    int32_t *ck = w.ckpt + (size_t)f * w.max_seg * 2 * W;
    int *Ep = S.E0, *Ec = S.E1;
    for (int v = vmax - 1; v >= vtop; --v) {
        const int seg = (v - vtop) / SR;
        if (seg > 0 && v == min(vtop + (seg + 1) * SR - 1, vmax - 1)) {
            // checkpoint k = seg: E_{v+1} and the band of row v+1
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
        dp_row(kp, S, Ep, Ec, v - (vtop + seg * SR));
        __syncthreads();
        int *tmp = Ep;
        Ep = Ec;
        Ec = tmp;
    }
    // ---- start of the path: smallest u minimising E_{vtop} ----
    int bv = 0x7fffffff, bi = 0x7fffffff;
    for (int u = tid; u < W; u += kVpxThreads)
        if (Ep[u] < bv) {
            bv = Ep[u];
            bi = u;
        }
    const int ustar = block_argmin<kVpxThreads>(bv, bi, S.sh + kMaxChunks + 8);
    if (tid == 0) {
        S.path[vtop] = (int16_t)ustar;
        const int hi = min(vtop + SR - 1, vmax - 1);
        for (int v = vtop; v <= hi && nseg > 0; ++v)
            S.path[v + 1] = (int16_t)(S.path[v] + bt_get(S, Wp, v - vtop, S.path[v]));
    }
    __syncthreads();
    // ---- lower segments: restore the checkpoint, recompute the segment's backtrack, follow it ----
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
            dp_row(kp, S, Ep, Ec, v - lo);
            __syncthreads();
            int *tmp = Ep;
            Ep = Ec;
            Ec = tmp;
        }
        if (tid == 0)
            for (int v = lo; v <= hi; ++v)
                S.path[v + 1] = (int16_t)(S.path[v] + bt_get(S, Wp, v - lo, S.path[v]));
        __syncthreads();
    }

    // ---- rows whose path cell holds votes: band(u_v, v) != 0 ----
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

    // ---- RANSAC quartic on the supported rows (x = v, y = u_v) ----
    p = S.dyn;
    const int t = vmax - vtop + 1;
    int16_t *xs = carve<int16_t>(p, t);
    int16_t *ys = carve<int16_t>(p, t);
    int16_t *pid = carve<int16_t>(p, t);
    RansacMem R;
    R.member = carve<uint8_t>(p, t);
    R.list = carve<int16_t>(p, t);
    R.hyp_cnt = carve<int>(p, kMaxHyps);
    R.hyp_cf = carve<float>(p, kMaxHyps * 5);
    R.red = carve<__int128>(p, (kVpxThreads / 32) * 14);
    R.sh = S.sh;
    const int k = block_compact<kVpxThreads>(S.sup + vtop, t, pid, S.sh + 8);
    for (int j = tid; j < k; j += kVpxThreads) {
        xs[j] = (int16_t)(vtop + pid[j]);
        ys[j] = S.path[vtop + pid[j]];
    }
    __syncthreads();
    R.xs = xs;
    R.ys = ys;
    __shared__ double gamma_s[5];
    int rounds = 0;
    const int fl = ransac_block<5, kVpxThreads>(kp, R, k, kp.tr_x, 1, gamma_s, &rounds);

    for (int v = tid; v < H; v += kVpxThreads) {
        w.path_x[(size_t)f * H + v] = v >= vtop ? S.path[v] : (int16_t)0;
        w.inl_x[(size_t)f * H + v] = 0;
    }
    __syncthreads();
    for (int j = tid; j < k; j += kVpxThreads)
        w.inl_x[(size_t)f * H + vtop + pid[j]] = R.member[j];

    int flags = fs0.flags;
    if (fl & 1)
        flags |= LD_F_CAP_X;
    if (fl & 2)
        flags |= LD_F_DEGEN_X | LD_F_NO_LANES;
    double gamma[5] = {0, 0, 0, 0, 0};
    if (!(fl & 2)) {
        for (int i = 0; i < 5; ++i)
            gamma[i] = gamma_s[i];
        const double sc = p2d(-kp.e);
        float *Vpx = w.rows + (size_t)f * 3 * H + 2 * H;
        for (int v = vtop + tid; v <= vmax; v += kVpxThreads)
            Vpx[v] = __double2float_rn(poly_f64<5>(gamma, __dmul_rn((double)(v - kp.centre), sc)));
    }
    if (tid == 0) {
        FrameState &fs = w.fs[f];
        fs.flags = flags;
        fs.rounds_x = rounds;
        for (int i = 0; i < 5; ++i)
            fs.gamma[i] = gamma[i];
    }
}

}  // namespace

size_t road_smem_bytes(const KParams &kp)
{
    const size_t H = kp.H, D = kp.D, Hp = (H + 1) / 2;
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * H);
    add(4 * H);
    add(4 * (kMaxChunks + 8 + 2 * (kRoadThreads / 32)));
    add(2 * D);
    size_t dp = ((s + 15) & ~(size_t)15) + D * Hp;
    size_t rs = s;
    auto addr = [&](size_t bytes) { rs = ((rs + 15) & ~(size_t)15) + bytes; };
    addr(2 * D);
    addr(2 * D);
    addr(D);
    addr(2 * D);
    addr(D);
    addr(2 * D);
    addr(4 * kMaxHyps);
    addr(4 * kMaxHyps * 3);
    addr(16 * (kRoadThreads / 32) * 8);
    return (dp > rs ? dp : rs) + 64;
}

// Shared memory of k_vpx without the backtrack rows, and the RANSAC region that reuses them.
static size_t vpx_fixed_bytes(const KParams &kp, size_t *ransac_bytes)
{
    const size_t W = kp.W, H = kp.H;
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 15) & ~(size_t)15) + bytes; };
    add(4 * W);
    add(4 * W);
    add(4 * W);
    add(4 * (H + 1));
    add(2 * (size_t)kp.vote_cap);
    add(2 * H);
    add(H);
    add(4 * (kMaxChunks + 8 + 2 * (kVpxThreads / 32)));
    size_t r = 0;
    auto addr = [&](size_t bytes) { r = ((r + 15) & ~(size_t)15) + bytes; };
    addr(2 * H);
    addr(2 * H);
    addr(2 * H);
    addr(H);
    addr(2 * H);
    addr(4 * kMaxHyps);
    addr(4 * kMaxHyps * 5);
    addr(16 * (kVpxThreads / 32) * 14);
    *ransac_bytes = r + 16;
    return ((s + 15) & ~(size_t)15) + 64;
}

size_t vpx_smem_bytes(const KParams &kp)
{
    size_t rb;
    const size_t fixed = vpx_fixed_bytes(kp, &rb);
    const size_t btb = (size_t)kp.seg_rows * ((kp.W + 1) / 2);
    return fixed + (btb > rb ? btb : rb);
}

// Backtrack rows of k_vpx that fit in `budget` bytes of shared memory for width W, height H.
int vpx_seg_rows(const KParams &kp, size_t budget)
{
    size_t rb;
    const size_t fixed = vpx_fixed_bytes(kp, &rb);
    if (budget <= fixed + rb)
        return 0;
    return (int)((budget - fixed) / ((kp.W + 1) / 2));
}

cudaError_t setup_fit(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_road, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_vpx, smem_optin);
    return e;
}

cudaError_t launch_road(const KParams &kp, const Work &w, cudaStream_t s)
{
    k_road<<<kp.n_frames, kRoadThreads, road_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

cudaError_t launch_vpx(const KParams &kp, const Work &w, cudaStream_t s)
{
    k_vpx<<<kp.n_frames, kVpxThreads, vpx_smem_bytes(kp), s>>>(kp, w);
    return cudaGetLastError();
}

}  // namespace ld
