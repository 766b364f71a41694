// backward.cu -- gradient of a loss on (birth, death) values with respect to
// the point coordinates.
//
// Every finite birth or death of a Rips pair is the length of one edge of
// its simplex, the critical edge (u, v) attaining the diameter (eq. 5.3:
// diam = max pairwise distance).  With d = |x_u - x_v|, d d / d x_u =
// (x_u - x_v) / d and d d / d x_v = -(x_u - x_v) / d, so the chain rule
// scatters g * (x_u - x_v) / d onto u and its negative onto v.  The paper has
// no backward pass; this is the differentiable form built on its pairs.
// The difference and the length use the same single-rounding formula as the
// forward distance step.  Scatter uses float atomics (order-dependent
// rounding, within 1 ulp per addition).
#include "vr_common.cuh"

namespace vr {

// An edge with an endpoint outside 0..n-1 is skipped and reported through
// *dev_err (the host returns VR_ERR_INVALID_ARG); -1 marks "no edge".
__global__ void k_backward(const float* __restrict__ pts, int64_t n, int dim, const int32_t* __restrict__ edges,
                           int64_t num, const float* __restrict__ gb, const float* __restrict__ gd,
                           float* __restrict__ grad, int* dev_err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 2 * num;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pair = k >> 1;
        const int which = (int)(k & 1);  // 0 = birth edge, 1 = death edge
        const int u = edges[4 * pair + 2 * which], v = edges[4 * pair + 2 * which + 1];
        if (u < 0 || v < 0) continue;
        if (u >= n || v >= n) {
            atomicExch(dev_err, DEV_BAD_INPUT);
            continue;
        }
        const float g = which ? gd[pair] : gb[pair];
        if (g == 0.0f) continue;
        float acc = 0.0f;
        for (int c = 0; c < dim; ++c) {
            float diff = __fsub_rn(pts[(int64_t)u * dim + c], pts[(int64_t)v * dim + c]);
            acc = __fadd_rn(acc, __fmul_rn(diff, diff));
        }
        const float d = __fsqrt_rn(acc);
        if (!(d > 0.0f)) continue;  // coincident points: the length is not differentiable
        const float s = __fdiv_rn(g, d);
        for (int c = 0; c < dim; ++c) {
            float diff = __fsub_rn(pts[(int64_t)u * dim + c], pts[(int64_t)v * dim + c]);
            float t = __fmul_rn(s, diff);
            atomicAdd(grad + (int64_t)u * dim + c, t);
            atomicAdd(grad + (int64_t)v * dim + c, -t);
        }
    }
}

void launch_backward(const float* pts, int64_t n, int dim, const int32_t* edges, int64_t num, const float* gb,
                     const float* gd, float* grad, int* dev_err, cudaStream_t s) {
    if (num <= 0) return;
    int64_t blocks = (2 * num + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_backward<<<(unsigned)blocks, 256, 0, s>>>(pts, n, dim, edges, num, gb, gd, grad, dev_err);
    VR_CUDA(cudaGetLastError());
}

}  // namespace vr

extern "C" vr_status vr_backward(const float* pts, int64_t n, int32_t ambient_dim, const int32_t* edges, int64_t num,
                                 const float* grad_birth, const float* grad_death, float* grad_pts, void* stream) {
    if (n < 1 || ambient_dim < 1 || num < 0 || (num > 0 && (!pts || !edges || !grad_birth || !grad_death || !grad_pts)))
        return VR_ERR_INVALID_ARG;
    if (num == 0) return VR_OK;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        vr::Workspace ws(s);
        int* dev_err = ws.zeros_n<int>(1);
        vr::launch_backward(pts, n, ambient_dim, edges, num, grad_birth, grad_death, grad_pts, dev_err, s);
        int h = 0;
        VR_CUDA(cudaMemcpyAsync(&h, dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        return h == vr::DEV_OK ? VR_OK : VR_ERR_INVALID_ARG;
    } catch (const vr::Error& e) {
        return e.code;
    }
}
