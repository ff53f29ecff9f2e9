// Internal definitions of the learned lane-position proposal (kernels in k_net.cu, host runtime in
// ld_net.cu).
#pragma once

#include <cuda_bf16.h>

#include "ld_internal.cuh"

namespace ld {

// channels of the network's feature maps: input, then the outputs of the four 3x3 convolutions
__host__ __device__ constexpr int net_ch(int l) { return l == 0 ? 1 : (l == 1 ? 16 : (l == 4 ? 16 : 32)); }

// parameters, flat: per layer W[co][ci][3][3] then b[co]; then the head w[16], b
constexpr int kNetParams = (16 * 1 * 9 + 16) + (32 * 16 * 9 + 32) + (32 * 32 * 9 + 32) + (16 * 32 * 9 + 16) + 17;
static_assert(kNetParams == 18689, "parameter count");
constexpr int kWgradCtasPerSm = 4;
constexpr int kTopKMax = 256;
constexpr int kEvalPerTop = 6;      // evaluated starts per chosen coarse start, at most (4 + 2 neighbours)
constexpr float kPosWeight = 10.0f;

struct NetArgs {
    int mh, mw;                     // cell map of the call's frame size
    __nv_bfloat16 *X;               // [n][mh][mw] network input (kept for the layer-1 weight gradient)
    __nv_bfloat16 *act[4];          // A_1 .. A_4, [n][mh][mw][C_l]; A_4 only while training
    __nv_bfloat16 *dS[2];           // gradient maps, 32 channels each, used in turn
    __nv_bfloat16 *wf[4];           // forward operands W_l[co][tap][ci]
    __nv_bfloat16 *wb[4];           // backward-data operands W_l^T[ci][8 - tap][co] (layers 2-4)
    __nv_bfloat16 *whb;             // head weights, bf16
    const float *bias[4];           // b_l, inside the master copy
    const float *bh;                // head bias, inside the master copy
    float *theta, *m, *v;           // master weights and Adam moments [kNetParams]
    float *part;                    // weight-gradient partials [SMs x kWgradCtasPerSm][32][289]
    float *part_head;               // loss partials [608][18]
    int fused = 0;                  // 1: inference forward as one kernel (k_net_fused); 0: one kernel per layer
};

// logits (heat = false) or the heatmap sigmoid(z) of every cell; with road (the frames' fit states) only
// the cells on and just above each frame's road rows (v >= v_top), and nothing for frames without a road
cudaError_t net_forward(const NetArgs &a, const int32_t *xsum, int n, float *z, bool keep_a4, bool heat,
                        cudaStream_t s, const FrameState *road = nullptr);
cudaError_t net_backward(const NetArgs &a, const uint8_t *labels, int n, float pw, float *grad, float *loss,
                         cudaStream_t s);
cudaError_t net_pack(const NetArgs &a, cudaStream_t s);
// 1 when a tensor-core wait of a network kernel ran out since the last call (then cleared), 0 otherwise,
// -1 when the flag could not be read (synchronous)
int net_tc_status();
cudaError_t net_adam(const NetArgs &a, const float *grad, float lr, float b1, float b2, float eps, float c1, float c2,
                     cudaStream_t s);
cudaError_t net_labels(const KParams &kp, const Work &w, const ld_lanes *lanes, uint8_t *labels, int mh, int mw,
                       cudaStream_t s);
cudaError_t net_propose(const KParams &kp, const Work &w, const float *z, int mh, int mw, int top_k, float *scores,
                        uint8_t *cflag, int32_t *elist, int32_t *ecnt, int ecap, cudaStream_t s);

// the detector handle, as the learned proposal's runtime uses it (implemented in ld_api.cu)
int handle_fail(ld_handle *h, int code, const char *msg);
int handle_cuda_fail(ld_handle *h, cudaError_t e, const char *what);
int handle_check(ld_handle *h, const void *disp, const void *img, int w, int hh, int n, const void *out);
void handle_dims(const ld_handle *h, int *max_w, int *max_h, int *max_batch);
const ld_params &handle_params(const ld_handle *h);
cudaStream_t handle_stream(const ld_handle *h);
Work handle_work(const ld_handle *h);
KParams handle_call(ld_handle *h, int w, int hh, int n);
KParams handle_kparams(const ld_handle *h, int w, int hh, int n);
int handle_enqueue(ld_handle *h, const KParams &kp, const Work &w, const float *disp, const uint8_t *img,
                   ld_lanes *out, int first, int last, cudaStream_t s = nullptr);
Work work_view(const Work &w, const KParams &kp, int f0);

}  // namespace ld
