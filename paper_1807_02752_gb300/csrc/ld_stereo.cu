// Stereo matching (Sec. 2.1), the stage that makes the disparity map the lane path takes as input:
// NCC block matching (Eq. 1-8) with search range propagation (Eq. 9, Alg. 2) for the left and the right
// disparity map, then the left-right consistency check (Alg. 3).  Kernels and the ld_stereo_* entry
// points of include/ld.h.
//
//   k_srp   one CTA per (frame, map): rows from H-1-rho up to rho, in order, since a row's search range
//           comes from the row below.  A ring of the 2 rho + 1 image rows of both images sits in shared
//           memory; when the window moves up one row the new top row replaces the old bottom row and
//           per-column sums of I and I^2 are updated by their difference, so the block statistics of
//           every pixel of the row are two 7-wide sums of column sums (exact integers, the quantities the
//           paper gets from integral images, Eq. 5).  A pixel keeps its own block in registers and takes
//           the candidate with the largest NCC, compared exactly: c = N / sqrt(D_a D_b) with
//           N = n P - s_a s_b and D = n Q - s^2, so c1 > c2 <=> N1 |N1| D2 > N2 |N2| D1 in 128-bit integers.
//   k_lrc   l(u, v) = l_lf(u, v) when |l_lf(u, v) - l_rt(u - l_lf(u, v), v)| <= tr, else 0; float output.
//
// Readings: blocks lie inside both images (other pixels and candidates are skipped; a pixel without a
// candidate gets 0); ties go to the smaller disparity; the first row searches [0, d_max], every later
// pixel the union of [l - tau, l + tau] over the three estimates of the row below that exist.
#include <cstring>
#include <string>

#include "ld_net.cuh"

namespace ld {

namespace {

constexpr int kSrpThreads = 512;

struct SrpArgs {
    const uint8_t *left, *right;     // [n][H][W]
    int16_t *lf, *rt;                // [n][H][W]
    int W, H, dmax, tau, Wp;         // Wp: ring row stride (W rounded up to 16)
};

// c1 > c2 for c = N / sqrt(D) (a common positive factor dropped); D = 0 means c = 0
__device__ __forceinline__ bool ncc_better(long long N1, int D1, long long N2, int D2)
{
    if (D1 == 0)
        N1 = 0;
    if (D2 == 0)
        N2 = 0;
    if (N1 == 0 || N2 == 0)
        return N2 == 0 ? N1 > 0 : N2 < 0 && N1 == 0;
    const __int128 l = (__int128)N1 * (N1 < 0 ? -N1 : N1) * D2;
    const __int128 r = (__int128)N2 * (N2 < 0 ? -N2 : N2) * D1;
    return l > r;
}

template <int RHO>
__global__ void __launch_bounds__(kSrpThreads, 1) k_srp(const SrpArgs a)
{
    constexpr int K = 2 * RHO + 1, NB = K * K;
    extern __shared__ __align__(16) unsigned char sm[];
    const int W = a.W, H = a.H, Wp = a.Wp, f = blockIdx.x, dir = blockIdx.y;
    const size_t fo = (size_t)f * H * W;
    const uint8_t *A = (dir == 0 ? a.left : a.right) + fo;   // the image whose map this is
    const uint8_t *B = (dir == 0 ? a.right : a.left) + fo;
    int16_t *out = (dir == 0 ? a.lf : a.rt) + fo;
    uint8_t *ra = sm;                                          // [K][Wp] rows of A, row y in slot y % K
    uint8_t *rb = ra + K * Wp;                                 // [K][Wp] rows of B
    int *cs = reinterpret_cast<int *>(rb + K * Wp);            // [4][W]: column sums of A, A^2, B, B^2
    int *rs = cs + 4 * W;                                      // [4][W]: block s_A, D_A, s_B, D_B of the row
    int16_t *lv = reinterpret_cast<int16_t *>(rs + 4 * W);     // [2][W]: estimates of the row below / this row
    const int tid = threadIdx.x;
    const int vb = H - 1 - RHO;
    // rows without a block are 0
    for (int i = tid; i < RHO * W; i += kSrpThreads) {
        out[i] = 0;
        out[(size_t)(H - RHO) * W + i] = 0;
    }
    if (vb < RHO)
        return;
    int cur = 0;
    for (int v = vb; v >= RHO; --v) {
        if (v == vb) {
            for (int i = tid; i < K * W; i += kSrpThreads) {
                const int r = i / W, u = i % W, y = v - RHO + r;
                ra[(y % K) * Wp + u] = A[(size_t)y * W + u];
                rb[(y % K) * Wp + u] = B[(size_t)y * W + u];
            }
            __syncthreads();
            for (int u = tid; u < W; u += kSrpThreads) {
                int s0 = 0, q0 = 0, s1 = 0, q1 = 0;
                for (int r = 0; r < K; ++r) {
                    const int x = ra[r * Wp + u], z = rb[r * Wp + u];
                    s0 += x;
                    q0 += x * x;
                    s1 += z;
                    q1 += z * z;
                }
                cs[u] = s0;
                cs[W + u] = q0;
                cs[2 * W + u] = s1;
                cs[3 * W + u] = q1;
            }
        } else {
            // row v + RHO + 1 leaves the window, row v - RHO enters (same ring slot)
            const int y = v - RHO, slot = y % K;
            for (int u = tid; u < W; u += kSrpThreads) {
                const int xo = ra[slot * Wp + u], zo = rb[slot * Wp + u];
                const int xn = A[(size_t)y * W + u], zn = B[(size_t)y * W + u];
                ra[slot * Wp + u] = (uint8_t)xn;
                rb[slot * Wp + u] = (uint8_t)zn;
                cs[u] += xn - xo;
                cs[W + u] += xn * xn - xo * xo;
                cs[2 * W + u] += zn - zo;
                cs[3 * W + u] += zn * zn - zo * zo;
            }
        }
        __syncthreads();
        for (int u = RHO + tid; u <= W - 1 - RHO; u += kSrpThreads) {
            int s0 = 0, q0 = 0, s1 = 0, q1 = 0;
#pragma unroll
            for (int x = -RHO; x <= RHO; ++x) {
                s0 += cs[u + x];
                q0 += cs[W + u + x];
                s1 += cs[2 * W + u + x];
                q1 += cs[3 * W + u + x];
            }
            rs[u] = s0;
            rs[W + u] = NB * q0 - s0 * s0;
            rs[2 * W + u] = s1;
            rs[3 * W + u] = NB * q1 - s1 * s1;
        }
        __syncthreads();
        const int16_t *below = lv + (cur ^ 1) * W;
        int16_t *here = lv + cur * W;
        for (int u = tid; u < W; u += kSrpThreads) {
            int best = 0;
            if (u >= RHO && u <= W - 1 - RHO) {
                int dhi = dir == 0 ? u - RHO : W - 1 - RHO - u;
                dhi = dhi < a.dmax ? dhi : a.dmax;
                int lo = 0, hi = dhi, l0 = -1000, l1 = -1000, l2 = -1000;
                if (v < vb) {
                    if (u - 1 >= RHO)
                        l0 = below[u - 1];
                    l1 = below[u];
                    if (u + 1 <= W - 1 - RHO)
                        l2 = below[u + 1];
                    int mn = l1, mx = l1;
                    if (l0 > -1000) {
                        mn = min(mn, l0);
                        mx = max(mx, l0);
                    }
                    if (l2 > -1000) {
                        mn = min(mn, l2);
                        mx = max(mx, l2);
                    }
                    lo = max(0, mn - a.tau);
                    hi = min(dhi, mx + a.tau);
                }
                // this pixel's block of A, kept in registers
                int blk[NB];
#pragma unroll
                for (int r = 0; r < K; ++r)
#pragma unroll
                    for (int x = 0; x < K; ++x)
                        blk[r * K + x] = ra[r * Wp + u - RHO + x];
                const int sa = rs[u], Da = rs[W + u];
                long long bN = 0;
                int bD = 0;
                bool have = false;
                for (int d = lo; d <= hi; ++d) {
                    if (v < vb && abs(d - l0) > a.tau && abs(d - l1) > a.tau && abs(d - l2) > a.tau)
                        continue;
                    const int ub = dir == 0 ? u - d : u + d;
                    int P = 0;
#pragma unroll
                    for (int r = 0; r < K; ++r)
#pragma unroll
                        for (int x = 0; x < K; ++x)
                            P += blk[r * K + x] * (int)rb[r * Wp + ub - RHO + x];
                    long long N = (long long)NB * P - (long long)sa * rs[2 * W + ub];
                    if (Da == 0)
                        N = 0;
                    const int Db = rs[3 * W + ub];
                    if (!have || ncc_better(N, Db, bN, bD)) {
                        have = true;
                        best = d;
                        bN = N;
                        bD = Db;
                    }
                }
            }
            here[u] = (int16_t)best;
            out[(size_t)v * W + u] = (int16_t)best;
        }
        __syncthreads();
        cur ^= 1;
    }
}

__global__ void k_lrc(const int16_t *lf, const int16_t *rt, int W, int H, int n, int tr, float *disp)
{
    const long long total = (long long)n * H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p % W);
        const int l = lf[p];
        const int x = u - l;
        const bool ok = x >= 0 && abs(l - (int)rt[p - l]) <= tr;
        disp[p] = ok ? (float)l : 0.0f;
    }
}

size_t srp_smem(int W, int rho)
{
    const int K = 2 * rho + 1, Wp = (W + 15) & ~15;
    return (size_t)2 * K * Wp + sizeof(int) * 8 * (size_t)W + sizeof(int16_t) * 2 * (size_t)W;
}

}  // namespace
}  // namespace ld

struct ld_stereo {
    ld_handle *h = nullptr;
    ld_stereo_params sp{};
    int max_w = 0, max_h = 0, max_n = 0;
    void *mem = nullptr;
    int16_t *lf = nullptr, *rt = nullptr;
    float *disp = nullptr;
    int last_w = 0, last_h = 0, last_n = 0;
    bool have_last = false;
    cudaEvent_t ev[3] = {};
    std::string err;
};

namespace {

std::string g_stereo_error;

int sfail(ld_stereo *st, int code, const std::string &msg)
{
    if (st)
        st->err = msg;
    else
        g_stereo_error = msg;
    return code;
}

int scuda(ld_stereo *st, cudaError_t e, const char *what)
{
    return sfail(st, LD_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_pair(ld_stereo *st, const void *left, const void *right, int w, int hh, int n, const void *out)
{
    if (!left || !right || !out)
        return sfail(st, LD_E_ARG, "null buffer");
    if (w < 16 || hh < 16 || w > st->max_w || hh > st->max_h)
        return sfail(st, LD_E_ARG, "frame size outside [16, max_w] x [16, max_h]");
    if (n < 1 || n > st->max_n)
        return sfail(st, LD_E_ARG, "n_frames outside [1, max_batch]");
    return LD_OK;
}

template <int RHO>
cudaError_t launch_srp(const ld::SrpArgs &a, int n, cudaStream_t s)
{
    const size_t smem = ld::srp_smem(a.W, RHO);
    cudaError_t e = cudaFuncSetAttribute(ld::k_srp<RHO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    ld::k_srp<RHO><<<dim3(n, 2), ld::kSrpThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// both maps and the check on the handle's stream; `timed` records an event before SRP, between, after LRC
int enqueue_stereo(ld_stereo *st, const uint8_t *left, const uint8_t *right, int w, int hh, int n, float *disp,
                   bool timed)
{
    cudaStream_t s = ld::handle_stream(st->h);
    cudaError_t e = cudaSuccess;
    if (timed && (e = cudaEventRecord(st->ev[0], s)) != cudaSuccess)
        return scuda(st, e, "event");
    ld::SrpArgs a{left, right, st->lf, st->rt, w, hh, st->sp.d_max, st->sp.tau, (w + 15) & ~15};
    switch (st->sp.rho) {
    case 1: e = launch_srp<1>(a, n, s); break;
    case 2: e = launch_srp<2>(a, n, s); break;
    default: e = launch_srp<3>(a, n, s); break;
    }
    if (e != cudaSuccess)
        return scuda(st, e, "search range propagation");
    if (timed && (e = cudaEventRecord(st->ev[1], s)) != cudaSuccess)
        return scuda(st, e, "event");
    const long long total = (long long)n * w * hh;
    const int g = (int)((total + 255) / 256);
    ld::k_lrc<<<g < 152 * 16 ? g : 152 * 16, 256, 0, s>>>(st->lf, st->rt, w, hh, n, st->sp.tr_lrc, disp);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return scuda(st, e, "consistency check");
    if (timed && (e = cudaEventRecord(st->ev[2], s)) != cudaSuccess)
        return scuda(st, e, "event");
    st->last_w = w;
    st->last_h = hh;
    st->last_n = n;
    st->have_last = true;
    return LD_OK;
}

}  // namespace

extern "C" {

void ld_stereo_params_default(ld_stereo_params *sp)
{
    if (!sp)
        return;
    std::memset(sp, 0, sizeof(*sp));
    sp->rho = 3;
    sp->tau = 1;
    sp->d_max = -1;
    sp->tr_lrc = 3;
}

int ld_stereo_create(ld_handle *h, const ld_stereo_params *sp, ld_stereo **out)
{
    if (!out)
        return sfail(nullptr, LD_E_ARG, "out is NULL");
    *out = nullptr;
    if (!h || !sp)
        return sfail(nullptr, LD_E_ARG, "null argument");
    if (sp->rho < 1 || sp->rho > 3 || sp->tau < 0 || sp->tau > 64 || sp->tr_lrc < 0 || sp->d_max < -1 ||
        sp->d_max > 1023)
        return sfail(nullptr, LD_E_ARG, "rho must be in [1, 3], tau in [0, 64], tr_lrc >= 0, d_max in [-1, 1023]");
    ld_stereo *st = new ld_stereo();
    st->h = h;
    st->sp = *sp;
    if (st->sp.d_max < 0)
        st->sp.d_max = ld::handle_params(h).n_disp - 1;
    ld::handle_dims(h, &st->max_w, &st->max_h, &st->max_n);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && ld::srp_smem(st->max_w, st->sp.rho) > (size_t)optin) {
        delete st;
        return sfail(nullptr, LD_E_ARG, "frame too wide for the shared-memory budget of the stereo kernel");
    }
    const size_t px = (size_t)st->max_n * st->max_w * st->max_h;
    if (e == cudaSuccess)
        e = cudaMalloc(&st->mem, px * (2 + 2 + 4) + 512);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete st;
        return sfail(nullptr, LD_E_NOMEM, std::string("stereo memory: ") + cudaGetErrorString(e));
    }
    char *b = (char *)st->mem;
    st->lf = (int16_t *)b;
    st->rt = (int16_t *)(b + ((px * 2 + 255) & ~(size_t)255));
    st->disp = (float *)(b + 2 * ((px * 2 + 255) & ~(size_t)255));
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = cudaEventCreate(&st->ev[k]);
    if (e != cudaSuccess) {
        scuda(nullptr, e, "event creation");
        ld_stereo_destroy(st);
        return LD_E_CUDA;
    }
    *out = st;
    return LD_OK;
}

int ld_stereo_run(ld_stereo *st, const uint8_t *left, const uint8_t *right, int32_t w, int32_t hh, int32_t n,
                  float *disp_out)
{
    if (!st)
        return LD_E_ARG;
    int rc = check_pair(st, left, right, w, hh, n, disp_out);
    return rc != LD_OK ? rc : enqueue_stereo(st, left, right, w, hh, n, disp_out, false);
}

int ld_stereo_run_timed(ld_stereo *st, const uint8_t *left, const uint8_t *right, int32_t w, int32_t hh, int32_t n,
                        float *disp_out, float *ms_out)
{
    if (!st)
        return LD_E_ARG;
    int rc = check_pair(st, left, right, w, hh, n, disp_out);
    if (rc == LD_OK && !ms_out)
        rc = sfail(st, LD_E_ARG, "ms_out is NULL");
    if (rc == LD_OK)
        rc = enqueue_stereo(st, left, right, w, hh, n, disp_out, true);
    if (rc != LD_OK)
        return rc;
    cudaError_t e = cudaEventSynchronize(st->ev[2]);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms_out[0], st->ev[0], st->ev[1]);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms_out[1], st->ev[1], st->ev[2]);
    return e == cudaSuccess ? LD_OK : scuda(st, e, "event timing");
}

int ld_detect_stereo(ld_stereo *st, const uint8_t *left, const uint8_t *right, int32_t w, int32_t hh, int32_t n,
                     ld_lanes *out_lanes)
{
    if (!st)
        return LD_E_ARG;
    int rc = check_pair(st, left, right, w, hh, n, out_lanes);
    if (rc == LD_OK)
        rc = enqueue_stereo(st, left, right, w, hh, n, st->disp, false);
    if (rc != LD_OK)
        return rc;
    rc = ld_detect(st->h, st->disp, left, w, hh, n, out_lanes);
    return rc == LD_OK ? LD_OK : sfail(st, rc, ld_last_error(st->h));
}

int ld_stereo_maps(ld_stereo *st, int32_t frame, int16_t *lf_host, int16_t *rt_host, float *disp_host)
{
    if (!st)
        return LD_E_ARG;
    if (!st->have_last)
        return sfail(st, LD_E_STATE, "no stereo call yet");
    if (frame < 0 || frame >= st->last_n)
        return sfail(st, LD_E_ARG, "frame out of range");
    cudaError_t e = cudaStreamSynchronize(ld::handle_stream(st->h));
    const size_t px = (size_t)st->last_w * st->last_h, o = (size_t)frame * px;
    if (e == cudaSuccess && lf_host)
        e = cudaMemcpy(lf_host, st->lf + o, px * 2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && rt_host)
        e = cudaMemcpy(rt_host, st->rt + o, px * 2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && disp_host)
        e = cudaMemcpy(disp_host, st->disp + o, px * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LD_OK : scuda(st, e, "map copy");
}

const char *ld_stereo_last_error(const ld_stereo *st) { return st ? st->err.c_str() : g_stereo_error.c_str(); }

void ld_stereo_destroy(ld_stereo *st)
{
    if (!st)
        return;
    cudaStreamSynchronize(ld::handle_stream(st->h));
    for (int k = 0; k < 3; ++k)
        if (st->ev[k])
            cudaEventDestroy(st->ev[k]);
    cudaFree(st->mem);
    delete st;
}

}  // extern "C"
