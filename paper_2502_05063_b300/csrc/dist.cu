// dist.cu -- the distance step.
//
// d(i,j) = sqrt(sum_k (x_ik - x_jk)^2) with k ascending and each operation
// rounded once (explicit _rn intrinsics, which the compiler never contracts
// into fused multiply-adds; the file is also built with --fmad=false).  The
// result is the condensed lower triangle, entry (i,j), i > j, at
// i(i-1)/2 + j: the distance matrix D of Sec. 5.1 (Def 5.1.1) of the paper,
// from which every birth and death value is taken.
#include "vr_common.cuh"

namespace vr {

// One block per row i (i >= 1); threads stride over j < i.  Row i of the
// points is staged in shared memory; row j is read through the read-only
// cache.  Each row of the triangle is written contiguously (coalesced).
__global__ void k_distances(const float* __restrict__ pts, int64_t n, int dim,
                            float* __restrict__ out) {
    extern __shared__ float xi[];
    const int64_t i = (int64_t)blockIdx.x + 1;
    if (i >= n) return;
    for (int k = threadIdx.x; k < dim; k += blockDim.x) xi[k] = pts[i * dim + k];
    __syncthreads();
    const int64_t row = i * (i - 1) / 2;
    for (int64_t j = threadIdx.x; j < i; j += blockDim.x) {
        const float* xj = pts + j * dim;
        float acc = 0.0f;
        for (int k = 0; k < dim; ++k) {
            float diff = __fsub_rn(xi[k], __ldg(xj + k));
            acc = __fadd_rn(acc, __fmul_rn(diff, diff));
        }
        out[row + j] = __fsqrt_rn(acc);
    }
}

void launch_distances(const float* pts, int64_t n, int dim, float* lower_tri, cudaStream_t s) {
    if (n < 2) return;
    int threads = n - 1 >= 256 ? 256 : 128;
    k_distances<<<(unsigned)(n - 1), threads, dim * sizeof(float), s>>>(pts, n, dim, lower_tri);
    VR_CUDA(cudaGetLastError());
}

// Input check for a caller-given triangle: every entry finite and >= 0.
__global__ void k_check_lower_tri(const float* __restrict__ d, int64_t m, int* err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        float x = d[k];
        if (!(x >= 0.0f) || isinf(x)) atomicExch(err, DEV_BAD_INPUT);
    }
}

void launch_check_lower_tri(const float* lower_tri, int64_t m, int* dev_err, cudaStream_t s) {
    if (m <= 0) return;
    int64_t blocks = (m + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_check_lower_tri<<<(unsigned)blocks, 256, 0, s>>>(lower_tri, m, dev_err);
    VR_CUDA(cudaGetLastError());
}

}  // namespace vr
