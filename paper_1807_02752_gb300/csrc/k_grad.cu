// Sec. 2.3.1: road mask, bilateral filter (Eq. 15-16), Sobel gradients, edge test and sparse V_px votes
// (Eq. 17), for the road rows of every frame.
//
// One CTA covers R output rows of one frame across the full width.  It stages the image rows the 11x11
// window needs (R + 2 + 2 rho rows) in shared memory, with a sentinel value outside the frame whose range
// weight is 0 (this is the clipped window of Eq. 15).  The bilateral output is computed only at pixels
// whose 3x3 neighbourhood holds an interior road pixel: those are the only values the Sobel stencil and
// the edge test read (Sec. 2.3.1: "we only focus on the pixels on the road surface").  Weights are Q15
// integers, w = (ws * wr + 2^14) >> 15, sums are exact, and the output is (2 sum(w I) + sum(w)) / (2 sum(w)),
// so the result does not depend on the order of the taps.
//
// Each road pixel with G_x^2 + G_y^2 > thr^2 is an edge pixel.  Its vote column is
// floor(u + (v - V_py(v)) G_y / G_x + 0.5) in float32 (the line through the pixel perpendicular to the
// gradient meets row V_py there), kept when inside [0, W).  Edge pixels and votes are appended to per-row
// lists (order within a row is arbitrary; every consumer sums over them).
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kThreads = 512;

template <int RHO>
__global__ void __launch_bounds__(kThreads) k_grad(const KParams kp, const Work w, const float *__restrict__ disp,
                                                   const uint8_t *__restrict__ img, int R)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = kp.W, H = kp.H;
    const int f = blockIdx.y;
    const int r0 = blockIdx.x * R;
    const int nr = min(R, H - r0);
    const int tid = threadIdx.x;
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

    const int TW = W + 2 * RHO;             // tile width (columns -RHO .. W-1+RHO)
    const int TR = nr + 2 + 2 * RHO;        // tile rows (r0-1-RHO .. r0+nr+RHO)
    const int BR = nr + 2;                  // bilateral rows (r0-1 .. r0+nr)
    unsigned char *p = smem;
    int32_t *wr = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * kWrEntries;
    int32_t *cnt = reinterpret_cast<int32_t *>(p);  // [2][R]: edges, votes per row
    p += sizeof(int32_t) * 2 * R;
    float *rowF = reinterpret_cast<float *>(p);
    p += sizeof(float) * R;
    float *rowVy = reinterpret_cast<float *>(p);
    p += sizeof(float) * R;
    uint16_t *tile = reinterpret_cast<uint16_t *>(p);
    p += sizeof(uint16_t) * (size_t)TR * TW;
    p = reinterpret_cast<unsigned char *>(((size_t)p + 15) & ~(size_t)15);
    uint8_t *ibf = p;
    p += (size_t)BR * W;
    uint8_t *road = p;                      // [nr][W]

    for (int i = tid; i < kWrEntries; i += kThreads)
        wr[i] = w.wr[i];
    for (int i = tid; i < 2 * R; i += kThreads)
        cnt[i] = 0;
    const float *rows = w.rows + (size_t)f * 3 * H;
    for (int r = tid; r < nr; r += kThreads) {
        rowF[r] = rows[r0 + r];
        rowVy[r] = rows[H + r0 + r];
    }
    // image tile with the sentinel outside the frame
    const uint8_t *im = img + (size_t)f * H * W;
    for (int i = tid; i < TR * TW; i += kThreads) {
        const int tr = i / TW, tc = i - tr * TW;
        const int v = r0 - 1 - RHO + tr, u = tc - RHO;
        tile[i] = (v >= 0 && v < H && u >= 0 && u < W) ? (uint16_t)__ldg(im + (size_t)v * W + u) : (uint16_t)kSentinel;
    }
    // road mask of the interior pixels of this CTA's rows: finite l > 0 with |l - f(v)| <= varpi, v >= v_top
    const float *dsp = disp + (size_t)f * H * W;
    for (int i = tid; i < nr * W; i += kThreads) {
        const int r = i / W, u = i - r * W;
        const int v = r0 + r;
        uint8_t m = 0;
        if (v >= vtop && v >= 1 && v <= H - 2 && u >= 1 && u <= W - 2) {
            const float l = __ldg(dsp + (size_t)v * W + u);
            m = l > 0.0f && l < __int_as_float(0x7f800000) && fabsf(__fsub_rn(l, rowF[r])) <= kp.varpi;
        }
        road[i] = m;
    }
    __syncthreads();

    // bilateral output where the Sobel stencil of a road pixel reads it
    for (int i = tid; i < BR * W; i += kThreads) {
        const int br = i / W, u = i - br * W;   // bilateral row br <-> image row r0 - 1 + br
        bool need = false;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
            const int rr = br - 1 + dr;          // road-mask row
            if (rr < 0 || rr >= nr)
                continue;
#pragma unroll
            for (int du = -1; du <= 1; ++du) {
                const int uu = u + du;
                need |= uu >= 0 && uu < W && road[rr * W + uu];
            }
        }
        if (!need)
            continue;
        const uint16_t *t0 = tile + (size_t)br * TW + u;  // window rows br .. br + 2 RHO, columns u .. u + 2 RHO
        const int c = t0[RHO * TW + RHO];
        if (!kp.bilateral) {
            ibf[i] = (uint8_t)c;
            continue;
        }
        const int32_t *wrc = wr + 256 - c;
        unsigned num = 0, den = 0;
#pragma unroll
        for (int dy = 0; dy <= 2 * RHO; ++dy) {
#pragma unroll
            for (int dx = 0; dx <= 2 * RHO; ++dx) {
                const int q = t0[dy * TW + dx];
                const int wq = (kp.ws[dy * (2 * RHO + 1) + dx] * wrc[q] + 16384) >> 15;
                num += (unsigned)(wq * q);
                den += (unsigned)wq;
            }
        }
        ibf[i] = (uint8_t)((2u * num + den) / (2u * den));
    }
    __syncthreads();

    // Sobel, edge test, votes
    const int thr2 = kp.edge_thresh2;
    int16_t *edges = w.edges + (size_t)f * H * W * 4;
    int16_t *vbins = w.vbins + (size_t)f * H * W;
    for (int i = tid; i < nr * W; i += kThreads) {
        if (!road[i])
            continue;
        const int r = i / W, u = i - r * W;
        const int v = r0 + r;
        const uint8_t *a = ibf + (size_t)r * W;        // row v-1
        const uint8_t *b = a + W;                       // row v
        const uint8_t *cc = b + W;                      // row v+1
        const int gx = ((int)a[u + 1] - (int)a[u - 1]) + 2 * ((int)b[u + 1] - (int)b[u - 1]) + ((int)cc[u + 1] - (int)cc[u - 1]);
        const int gy = ((int)cc[u - 1] - (int)a[u - 1]) + 2 * ((int)cc[u] - (int)a[u]) + ((int)cc[u + 1] - (int)a[u + 1]);
        if (gx * gx + gy * gy <= thr2)
            continue;
        int bin = -1;
        if (gx != 0) {
            const float av = __fsub_rn((float)v, rowVy[r]);
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
    __syncthreads();
    for (int r = tid; r < nr; r += kThreads) {
        ecnt[r0 + r] = cnt[r];
        vcnt[r0 + r] = cnt[R + r];
    }
}

template <int RHO>
size_t grad_smem(int W, int R)
{
    const int nr = R;
    size_t s = sizeof(int32_t) * kWrEntries + sizeof(int32_t) * 2 * R + 2 * sizeof(float) * R;
    s += sizeof(uint16_t) * (size_t)(nr + 2 + 2 * RHO) * (W + 2 * RHO);
    s = (s + 15) & ~(size_t)15;
    s += (size_t)(nr + 2) * W + (size_t)nr * W;
    return s + 16;
}

template <int RHO>
cudaError_t launch_grad_t(const KParams &kp, const Work &w, const float *disp, const uint8_t *img, cudaStream_t s)
{
    int R = 8;
    while (R > 1 && grad_smem<RHO>(kp.W, R) > 100 * 1024)
        --R;
    const size_t smem = grad_smem<RHO>(kp.W, R);
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
