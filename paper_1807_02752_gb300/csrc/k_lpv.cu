// Sec. 2.4, lane position validation (Alg. 7):
//
//   k_m1      w_g of every road edge pixel (Eq. 23), M_0 = (2 nu + 1) x (2 varsigma + 1) box sum of
//             G_x w_g, M_1 = G * M_0 with G = [1,2,1]^T [1,0,-1] (a convolution: M_0(u+1) - M_0(u-1)).
//   k_energy  for every start s in [-floor(xi W), W + floor(xi W)) the track of Eq. 25 from the bottom
//             row up to v_top and its energy E = M_1(round(u_v), v) + lambda_g E (Eq. 24).
//   k_select  strict interior local minima of H below t = ceil(thr min H), then suppression of nearby
//             minima in increasing (energy, position) order; fills ld_lanes.
//
// w_g reading: theta_e is the direction of the edge (the Sobel gradient turned by 90 degrees), theta_Vp
// the direction from the pixel to V_p(v); lines are undirected, so the angle is taken in [0, pi/2] through
// s = sin^2(dtheta) = (t x r)^2 / (|t|^2 |r|^2) in float32.  w_g = 0 beyond pi/6 (s > 1/4); otherwise the
// Q12 table entry at floor(sqrt(s) 2^15).  Eq. 23 is applied as printed: exp(-|dtheta| / sigma_g^2 * 36/pi).
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kM1Threads = 512;
constexpr int kEnThreads = 256;
constexpr int kSelThreads = 256;

__global__ void __launch_bounds__(kM1Threads) k_m1(const KParams kp, const Work w, int R)
{
    extern __shared__ __align__(16) int32_t m0[];   // [R + 2][W]: M_0 rows r0-1 .. r0+R
    const int W = kp.W, H = kp.H;
    const int f = blockIdx.y;
    const int r0 = blockIdx.x * R;
    const int nr = min(R, H - r0);
    const FrameState &fs = w.fs[f];
    const int vtop = fs.v_top, vmax = H - 1;
    if ((fs.flags & LD_F_NO_LANES) || r0 + nr - 1 < vtop)
        return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nu = kp.box_nu, vs = kp.box_vs;
    for (int i = tid; i < (nr + 2) * W; i += kM1Threads)
        m0[i] = 0;
    __syncthreads();
    const float *Vpy = w.rows + (size_t)f * 3 * H + H;
    const float *Vpx = Vpy + H;
    // scatter G_x w_g of the edge pixels of rows [r0-1-vs, r0+nr+vs] into the M_0 rows they reach
    const int elo = max(vtop, r0 - 1 - vs), ehi = min(vmax, r0 + nr + vs);
    for (int v = elo + warp; v <= ehi; v += kM1Threads / 32) {
        const int cnt = w.ecount[(size_t)f * H + v];
        const short4 *src = reinterpret_cast<const short4 *>(w.edges + ((size_t)f * H + v) * W * 4);
        const float vx = Vpx[v], vy = Vpy[v];
        for (int q = lane; q < cnt; q += 32) {
            const short4 e = src[q];
            const int u = e.x, gx = e.z, gy = e.w;
            const float tu = (float)(-gy), tv = (float)gx;
            const float ru = __fsub_rn(vx, (float)u), rv = __fsub_rn(vy, (float)v);
            const float cr = __fsub_rn(__fmul_rn(tu, rv), __fmul_rn(tv, ru));
            const float num = __fmul_rn(cr, cr);
            const float den = __fmul_rn(__fadd_rn(__fmul_rn(tu, tu), __fmul_rn(tv, tv)),
                                        __fadd_rn(__fmul_rn(ru, ru), __fmul_rn(rv, rv)));
            int wg = 0;
            if (den > 0.0f) {
                const float s = __fdiv_rn(num, den);
                if (s <= 0.25f)
                    wg = __ldg(w.wg + (int)__fmul_rn(__fsqrt_rn(s), 32768.0f));
            }
            const int gw = gx * wg;
            if (gw == 0)
                continue;
            for (int y = -vs; y <= vs; ++y) {
                const int rr = v + y - (r0 - 1);
                if (rr < 0 || rr >= nr + 2 || v + y < 0 || v + y > vmax)
                    continue;
                for (int x = -nu; x <= nu; ++x) {
                    const int uu = u + x;
                    if (uu >= 0 && uu < W)
                        atomicAdd(&m0[rr * W + uu], gw);
                }
            }
        }
    }
    __syncthreads();
    // M_1 rows r0 .. r0+nr-1 (>= v_top): sum_dv (1,2,1)[dv] (M_0(u+1, v+dv) - M_0(u-1, v+dv))
    int32_t *M1 = w.M1 + (size_t)f * H * W;
    const int rstart = max(r0, vtop);
    for (int i = (rstart - r0) * W + tid; i < nr * W; i += kM1Threads) {
        const int r = i / W, u = i - r * W;
        const int32_t *a = m0 + (size_t)r * W;   // M_0 row v-1
        int s = 0;
#pragma unroll
        for (int dv = 0; dv < 3; ++dv) {
            const int32_t *row = a + dv * W;
            const int rgt = u + 1 < W ? row[u + 1] : 0;
            const int lft = u >= 1 ? row[u - 1] : 0;
            s += (dv == 1 ? 2 : 1) * (rgt - lft);
        }
        M1[(size_t)(r0 + r) * W + u] = s;
    }
}

__global__ void __launch_bounds__(kEnThreads) k_energy(const KParams kp, const Work w)
{
    extern __shared__ float vrow[];   // [2][H]: V_px, V_py
    const int W = kp.W, H = kp.H;
    const int f = blockIdx.y;
    const FrameState &fs = w.fs[f];
    if (fs.flags & LD_F_NO_LANES)
        return;
    const int vtop = fs.v_top, vmax = H - 1;
    const float *rows = w.rows + (size_t)f * 3 * H;
    for (int v = threadIdx.x; v < H; v += kEnThreads) {
        vrow[v] = rows[2 * H + v];
        vrow[H + v] = rows[H + v];
    }
    __syncthreads();
    const int i = blockIdx.x * kEnThreads + threadIdx.x;
    if (i >= kp.n_starts)
        return;
    const int32_t *M1 = w.M1 + (size_t)f * H * W;
    const float fW = (float)W;
    const long long lam = kp.lambda_g;
    float u = (float)(i - kp.S0);
    long long E = 0;
    for (int v = vmax; v >= vtop; --v) {
        if (v < vmax) {
            const float vx = vrow[v + 1], vy = vrow[H + v + 1];
            const float num = __fsub_rn(__fadd_rn(vx, __fmul_rn((float)v, u)), __fmul_rn(vy, u));
            const float den = __fsub_rn((float)(v + 1), vy);
            u = __fdiv_rn(num, den);
        }
        const float col = floorf(__fadd_rn(u, 0.5f));
        long long m = 0;
        if (col >= 0.0f && col < fW)
            m = __ldg(M1 + (size_t)v * W + (int)col);
        E = m + lam * E;
    }
    w.HE[(size_t)f * kp.n_starts + i] = (int64_t)E;
}

__global__ void __launch_bounds__(kSelThreads) k_select(const KParams kp, const Work w, ld_lanes *out)
{
    extern __shared__ int cand[];     // [n_starts / 2 + 2] candidate positions, then their sorted order
    __shared__ long long red[kSelThreads / 32];
    __shared__ int ncand;
    __shared__ int acc[LD_MAX_LANES];
    __shared__ int nacc;
    const int f = blockIdx.x, ns = kp.n_starts;
    const int tid = threadIdx.x;
    const FrameState fs = w.fs[f];
    int flags = fs.flags;
    const int64_t *he = w.HE + (size_t)f * ns;
    if (tid == 0) {
        ncand = 0;
        nacc = 0;
    }
    long long mn = 0;
    if (!(flags & LD_F_NO_LANES)) {
        long long m = 0x7fffffffffffffffLL;
        for (int i = tid; i < ns; i += kSelThreads)
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
            const long long t = -(((-mn) * (long long)kp.thr_num) / (long long)kp.thr_den);
            int *pos = cand;
            for (int i = 1 + tid; i < ns - 1; i += kSelThreads) {
                const long long h = he[i];
                if (h < he[i - 1] && h < he[i + 1] && h < t)
                    pos[atomicAdd(&ncand, 1)] = i;
            }
            __syncthreads();
            const int nc = ncand;
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
                ord[rank] = ia;
            }
            __syncthreads();
            if (tid == 0) {
                int na = 0;
                for (int a = 0; a < nc && na < kp.max_lanes; ++a) {
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

}  // namespace

cudaError_t setup_lpv(int smem_optin)
{
    cudaError_t e = allow_max_smem(k_m1, smem_optin);
    if (e == cudaSuccess)
        e = allow_max_smem(k_select, smem_optin);
    return e;
}

int m1_rows(int W)
{
    int R = 16;
    while (R > 1 && sizeof(int32_t) * (size_t)(R + 2) * W > 160 * 1024)
        --R;
    return R;
}

cudaError_t launch_m1(const KParams &kp, const Work &w, cudaStream_t s)
{
    const int R = m1_rows(kp.W);
    const size_t smem = sizeof(int32_t) * (size_t)(R + 2) * kp.W;
    dim3 grid((kp.H + R - 1) / R, kp.n_frames);
    k_m1<<<grid, kM1Threads, smem, s>>>(kp, w, R);
    return cudaGetLastError();
}

cudaError_t launch_energy(const KParams &kp, const Work &w, cudaStream_t s)
{
    dim3 grid((kp.n_starts + kEnThreads - 1) / kEnThreads, kp.n_frames);
    k_energy<<<grid, kEnThreads, sizeof(float) * 2 * kp.H, s>>>(kp, w);
    return cudaGetLastError();
}

cudaError_t launch_select(const KParams &kp, const Work &w, ld_lanes *out, cudaStream_t s)
{
    const size_t smem = sizeof(int) * (size_t)(kp.n_starts + 4);
    k_select<<<kp.n_frames, kSelThreads, smem, s>>>(kp, w, out);
    return cudaGetLastError();
}

}  // namespace ld
