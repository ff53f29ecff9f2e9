// Median pre-filter (bilateral = 2): the filter of the authors' previous system that Sec. 2.3.1 compares
// the bilateral filter with, over the same (2 rho + 1)^2 window (11 x 11).  Each output pixel is the lower
// median of the window's taps inside the image: the ((n + 1) / 2)-th smallest of its n taps.
//
// One thread per pixel of an 8 x 32 tile whose halo sits in shared memory.  The median is found by value,
// bit by bit from the top: the r-th smallest value is the largest m with fewer than r taps below m, and
// each of the eight steps counts the taps below a candidate.  Integer throughout, so the result does not
// depend on the order of anything.  Only rows from v_top - 1 down are filtered (the Sobel stencil of the
// road rows reads no higher); rows above keep the raw image, and frames without a road fit are copied.
#include "ld_internal.cuh"

namespace ld {

namespace {

constexpr int kMedRows = 8, kMedCols = 32, kMedMaxRho = 5;

__device__ __forceinline__ void median_body(const KParams &kp, const Work &w, const uint8_t *img, const int f,
                                            const int bx, const int by)
{
    __shared__ uint8_t tile[(kMedRows + 2 * kMedMaxRho) * (kMedCols + 2 * kMedMaxRho)];
    const int W = kp.W, H = kp.H, rho = kp.rho;
    if (!LD_IN(rho, kMedMaxRho + 1, CK_MED_TILE))   // the halo the shared tile holds
        return;
    const int x0 = bx * kMedCols, y0 = by * kMedRows;
    const int u = x0 + (threadIdx.x & (kMedCols - 1)), v = y0 + threadIdx.x / kMedCols;
    const uint8_t *in = img + (size_t)f * H * W;
    uint8_t *out = w.med + (size_t)f * H * W;
    const FrameState &fs = w.fs[f];
    const int vfirst = (fs.flags & LD_F_NO_LANES) ? H : max(0, fs.v_top - 1);
    if (y0 + kMedRows - 1 < vfirst) {   // the whole tile lies above the filtered rows (uniform)
        if (u < W && v < H)
            out[(size_t)v * W + u] = in[(size_t)v * W + u];
        return;
    }
    const int hw = kMedCols + 2 * rho, hh = kMedRows + 2 * rho;
    for (int i = threadIdx.x; i < hw * hh; i += kMedRows * kMedCols) {
        const int yy = y0 - rho + i / hw, xx = x0 - rho + i % hw;
        tile[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? in[(size_t)yy * W + xx] : 0;
    }
    __syncthreads();
    if (u >= W || v >= H)
        return;
    if (v < vfirst) {
        out[(size_t)v * W + u] = in[(size_t)v * W + u];
        return;
    }
    // the window clipped to the image, in tile coordinates
    const int ylo = max(v - rho, 0) - (y0 - rho), yhi = min(v + rho, H - 1) - (y0 - rho);
    const int xlo = max(u - rho, 0) - (x0 - rho), xhi = min(u + rho, W - 1) - (x0 - rho);
    const int r = ((yhi - ylo + 1) * (xhi - xlo + 1) + 1) >> 1;
    int m = 0;
    for (int b = 7; b >= 0; --b) {
        const int c = m | (1 << b);
        int below = 0;
        for (int y = ylo; y <= yhi; ++y) {
            const uint8_t *row = tile + y * hw;
            for (int x = xlo; x <= xhi; ++x)
                below += row[x] < c;
        }
        if (below < r)
            m = c;
    }
    out[(size_t)v * W + u] = (uint8_t)m;
}

__global__ void __launch_bounds__(kMedRows * kMedCols) k_median(const KParams kp, const Work w, const uint8_t *img)
{
    median_body(kp, w, img, blockIdx.z, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(kMedRows * kMedCols) k_median_fd(const FrameDesc *__restrict__ fd)
{
    const FrameDesc &d = fd[blockIdx.z];
    const KParams kp = d.kp;   // the frame's parameters, loaded once into registers
    const Work w = d.w;
    if ((int)blockIdx.x * kMedCols >= kp.W || (int)blockIdx.y * kMedRows >= kp.H)
        return;
    median_body(kp, w, d.img, 0, blockIdx.x, blockIdx.y);
}

}  // namespace

cudaError_t launch_median_fd(const KParams &kmax, const FrameDesc *fd, int n, cudaStream_t s)
{
    dim3 grid((kmax.W + kMedCols - 1) / kMedCols, (kmax.H + kMedRows - 1) / kMedRows, n);
    k_median_fd<<<grid, kMedRows * kMedCols, 0, s>>>(fd);
    return cudaGetLastError();
}

cudaError_t launch_median(const KParams &kp, const Work &w, const uint8_t *img, cudaStream_t s)
{
    dim3 grid((kp.W + kMedCols - 1) / kMedCols, (kp.H + kMedRows - 1) / kMedRows, kp.n_frames);
    k_median<<<grid, kMedRows * kMedCols, 0, s>>>(kp, w, img);
    return cudaGetLastError();
}

}  // namespace ld
