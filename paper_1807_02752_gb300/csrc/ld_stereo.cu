// Stereo matching (Sec. 2.1), the stage that makes the disparity map the lane path takes as input:
// NCC block matching (Eq. 1-8) with search range propagation (Eq. 9, Alg. 2) for the left and the right
// disparity map, then the left-right consistency check (Alg. 3).  Kernels and the ld_stereo_* entry
// points of include/ld.h.
//
//   k_srp   one CTA per (frame, map): rows from H-1-rho up to rho, in order, since a row's search range
//           comes from the row below.  A ring of the 2 rho + 1 image rows of both images sits in shared
//           memory, stored by column (a column's rows in 8 bytes); when the window moves up one row the new
//           top row (loaded a row ahead) replaces the old bottom row and per-column sums of I and I^2 are
//           updated by their difference, so the block statistics of every pixel of the row are two 7-wide
//           sums of column sums (exact integers, the quantities the paper gets from integral images, Eq. 5).
//           A thread takes a pixel, keeps its block's columns in registers and forms each candidate's
//           block product P from 7 column dot products (two dp4a each, in four independent chains).  The best candidate has the
//           largest NCC, compared exactly: c = N / sqrt(D_a D_b) with N = n P - s_a s_b and
//           D = n Q - s^2, so c1 > c2 <=> N1 |N1| D2 > N2 |N2| D1 (a float filter decides clear cases,
//           128-bit integers the rest).
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
    int W, H, dmax, tau;
};

// c1 > c2 for c = N / sqrt(D) (a common positive factor dropped); D = 0 means c = 0.  Decided exactly:
// c1 > c2 <=> N1 |N1| D2 > N2 |N2| D1.  Each side in float carries four roundings (the two conversions and
// two products; relative error about 2^-22), so a float gap above 2^-20 (|L| + |R|) has the sign of the
// exact one; closer pairs compare in 128-bit integers.
__device__ __forceinline__ bool ncc_better(long long N1, int D1, long long N2, int D2)
{
    if (D1 == 0)
        N1 = 0;
    if (D2 == 0)
        N2 = 0;
    if (N1 == 0 || N2 == 0)
        return N2 == 0 ? N1 > 0 : N2 < 0 && N1 == 0;
    const float f1 = (float)N1, f2 = (float)N2;
    const float L = __fmul_rn(__fmul_rn(f1, fabsf(f1)), (float)D2);
    const float R = __fmul_rn(__fmul_rn(f2, fabsf(f2)), (float)D1);
    const float gap = __fsub_rn(L, R);
    if (fabsf(gap) > 9.5367431640625e-07f * (fabsf(L) + fabsf(R)))
        return gap > 0.0f;
    const __int128 l = (__int128)N1 * (N1 < 0 ? -N1 : N1) * D2;
    const __int128 r = (__int128)N2 * (N2 < 0 ? -N2 : N2) * D1;
    return l > r;
}

constexpr int kMaxColsPerThread = 8;  // columns per thread in the row loads (the launch guarantees W <= 8 x threads)

// threads of a k_srp CTA: the pixels with a block spread evenly (every thread the same number of them),
// at most kSrpThreads, and enough threads that each loads at most kMaxColsPerThread columns of a row
inline int srp_threads(int W, int rho)
{
    const int valid = W - 2 * rho, per = (valid + kSrpThreads - 1) / kSrpThreads;
    int t = (valid + per - 1) / per;
    t = t > (W + kMaxColsPerThread - 1) / kMaxColsPerThread ? t : (W + kMaxColsPerThread - 1) / kMaxColsPerThread;
    t = t < 32 ? 32 : t;
    return t < kSrpThreads ? t : kSrpThreads;
}

template <int RHO>
__global__ void __launch_bounds__(kSrpThreads, 1) k_srp(const SrpArgs a)
{
    constexpr int K = 2 * RHO + 1, NB = K * K;
    extern __shared__ __align__(16) unsigned char sm[];
    const int W = a.W, H = a.H, f = blockIdx.x, dir = blockIdx.y;
    const size_t fo = (size_t)f * H * W;
    const uint8_t *A = (dir == 0 ? a.left : a.right) + fo;   // the image whose map this is
    const uint8_t *B = (dir == 0 ? a.right : a.left) + fo;
    int16_t *out = (dir == 0 ? a.lf : a.rt) + fo;
    // ring of the K block rows, stored by column: byte r of column c is ring slot r (row y with y % K == r),
    // byte 7 stays 0, so the dot product of two columns is two dp4a
    uint2 *ca = reinterpret_cast<uint2 *>(sm);                 // [W]
    uint2 *cb = ca + W;                                        // [W]
    int *cs = reinterpret_cast<int *>(cb + W);                 // [4][W]: column sums of A, A^2, B, B^2
    int2 *ra2 = reinterpret_cast<int2 *>(cs + 4 * W);           // [W]: block (s_A, D_A) of the row
    int2 *rb2 = ra2 + W;                                       // [W]: block (s_B, D_B)
    int16_t *lv = reinterpret_cast<int16_t *>(rb2 + W);        // [2][W]: estimates of the row below / this row
    uint8_t *ca8 = reinterpret_cast<uint8_t *>(ca), *cb8 = reinterpret_cast<uint8_t *>(cb);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int vb = H - 1 - RHO;
    for (int i = tid; i < RHO * W; i += nthr) {
        out[i] = 0;
        out[(size_t)(H - RHO) * W + i] = 0;
    }
    // initial window: rows vb - RHO .. vb + RHO
    for (int u = tid; u < W; u += nthr) {
        int s0 = 0, q0 = 0, s1 = 0, q1 = 0;
        uint8_t xa[8], xb[8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
            xa[r] = xb[r] = 0;
        for (int y = vb - RHO; y <= vb + RHO; ++y) {
            const int x = A[(size_t)y * W + u], z = B[(size_t)y * W + u];
            xa[y % K] = (uint8_t)x;
            xb[y % K] = (uint8_t)z;
            s0 += x;
            q0 += x * x;
            s1 += z;
            q1 += z * z;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            ca8[u * 8 + r] = xa[r];
            cb8[u * 8 + r] = xb[r];
        }
        cs[u] = s0;
        cs[W + u] = q0;
        cs[2 * W + u] = s1;
        cs[3 * W + u] = q1;
    }
    // the row entering next (vb - RHO - 1), loaded a row ahead
    int na[kMaxColsPerThread], nb[kMaxColsPerThread];
#pragma unroll
    for (int k = 0; k < kMaxColsPerThread; ++k) {
        const int u = tid + k * nthr, y = vb - RHO - 1;
        na[k] = (u < W && y >= 0) ? A[(size_t)y * W + u] : 0;
        nb[k] = (u < W && y >= 0) ? B[(size_t)y * W + u] : 0;
    }
    int cur = 0;
    for (int v = vb; v >= RHO; --v) {
        if (v < vb) {
            // row v + RHO + 1 leaves the window, row v - RHO enters (same ring slot)
            const int slot = (v - RHO) % K;
#pragma unroll
            for (int k = 0; k < kMaxColsPerThread; ++k) {
                const int u = tid + k * nthr;
                if (u < W) {
                    const int xo = ca8[u * 8 + slot], zo = cb8[u * 8 + slot];
                    const int xn = na[k], zn = nb[k];
                    ca8[u * 8 + slot] = (uint8_t)xn;
                    cb8[u * 8 + slot] = (uint8_t)zn;
                    cs[u] += xn - xo;
                    cs[W + u] += xn * xn - xo * xo;
                    cs[2 * W + u] += zn - zo;
                    cs[3 * W + u] += zn * zn - zo * zo;
                }
            }
            const int y = v - RHO - 1;   // prefetch the next entering row
#pragma unroll
            for (int k = 0; k < kMaxColsPerThread; ++k) {
                const int u = tid + k * nthr;
                if (u < W && y >= 0) {
                    na[k] = A[(size_t)y * W + u];
                    nb[k] = B[(size_t)y * W + u];
                }
            }
        }
        __syncthreads();
        for (int u = RHO + tid; u <= W - 1 - RHO; u += nthr) {
            int s0 = 0, q0 = 0, s1 = 0, q1 = 0;
#pragma unroll
            for (int x = -RHO; x <= RHO; ++x) {
                s0 += cs[u + x];
                q0 += cs[W + u + x];
                s1 += cs[2 * W + u + x];
                q1 += cs[3 * W + u + x];
            }
            ra2[u] = make_int2(s0, NB * q0 - s0 * s0);
            rb2[u] = make_int2(s1, NB * q1 - s1 * s1);
        }
        __syncthreads();
        const int16_t *below = lv + (cur ^ 1) * W;
        int16_t *here = lv + cur * W;
        const int umax = W - 1 - RHO;
        for (int u = RHO + tid; u <= umax; u += nthr) {
            int dhi = dir == 0 ? u - RHO : W - 1 - RHO - u;
            dhi = dhi < a.dmax ? dhi : a.dmax;
            // the search range as up to three intervals in ascending order: [0, dhi] on the first row, else
            // [l - tau, l + tau] around the sorted estimates below (duplicates skipped by starting each
            // interval after the previous one's end)
            int c0 = 0, c1 = -1000, c2 = -1000, span = dhi;   // centres (interval = [c - span, c + span])
            bool first = v == vb;
            if (!first) {
                int l0 = u - 1 >= RHO ? below[u - 1] : -1000, l1 = below[u], l2 = u + 1 <= umax ? below[u + 1] : -1000;
                // sort three values (missing ones, -1000, first)
                if (l0 > l1) { const int t = l0; l0 = l1; l1 = t; }
                if (l1 > l2) { const int t = l1; l1 = l2; l2 = t; }
                if (l0 > l1) { const int t = l0; l0 = l1; l1 = t; }
                c0 = l0;
                c1 = l1;
                c2 = l2;
                span = a.tau;
            }
            // this pixel's block of A: its K columns, each the K ring rows in 8 bytes
            uint2 acol[K];
#pragma unroll
            for (int x = 0; x < K; ++x)
                acol[x] = ca[u - RHO + x];
            const int2 sa2 = ra2[u];
            const int sa = sa2.x, Da = sa2.y;
            long long bN = 0;
            int bD = 0, best = -1, next = 0;   // next: smallest disparity not yet searched
            for (int iv = first ? 2 : 0; iv < 3; ++iv) {
                const int c = first ? span / 2 : (iv == 0 ? c0 : (iv == 1 ? c1 : c2));
                if (c <= -1000)
                    continue;
                const int from = max(next, first ? 0 : c - span), to = min(dhi, first ? dhi : c + span);
                if (from > to)
                    continue;
                for (int d = from; d <= to; ++d) {
                    const int ub = dir == 0 ? u - d : u + d;
                    uint2 bw[K];
#pragma unroll
                    for (int x = 0; x < K; ++x)
                        bw[x] = cb[ub - RHO + x];
                    unsigned p4[4] = {0u, 0u, 0u, 0u};   // four independent dp4a chains
#pragma unroll
                    for (int x = 0; x < K; ++x) {
                        p4[(2 * x) & 3] = __dp4a(acol[x].x, bw[x].x, p4[(2 * x) & 3]);
                        p4[(2 * x + 1) & 3] = __dp4a(acol[x].y, bw[x].y, p4[(2 * x + 1) & 3]);
                    }
                    const unsigned P = (p4[0] + p4[1]) + (p4[2] + p4[3]);
                    const int2 sb2 = rb2[ub];
                    long long N = (long long)NB * (long long)P - (long long)sa * sb2.x;
                    if (Da == 0)
                        N = 0;
                    if (best < 0 || ncc_better(N, sb2.y, bN, bD)) {
                        best = d;
                        bN = N;
                        bD = sb2.y;
                    }
                }
                next = max(next, to + 1);
            }
            const int16_t val = (int16_t)(best < 0 ? 0 : best);
            here[u] = val;
            out[(size_t)v * W + u] = val;
        }
        for (int u = tid; u < W; u += nthr)   // columns without a block
            if (u < RHO || u > umax) {
                here[u] = 0;
                out[(size_t)v * W + u] = 0;
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
    (void)rho;
    return sizeof(uint2) * 2 * (size_t)W + sizeof(int) * 8 * (size_t)W + sizeof(int16_t) * 2 * (size_t)W;
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
    ld::k_srp<RHO><<<dim3(n, 2), ld::srp_threads(a.W, RHO), smem, s>>>(a);
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
    ld::SrpArgs a{left, right, st->lf, st->rt, w, hh, st->sp.d_max, st->sp.tau};
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
    const int gmax = ld::sm_count() * 16;
    ld::k_lrc<<<g < gmax ? g : gmax, 256, 0, s>>>(st->lf, st->rt, w, hh, n, st->sp.tr_lrc, disp);
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
