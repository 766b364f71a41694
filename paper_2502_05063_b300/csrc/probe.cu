// probe.cu -- read-bandwidth probe for the roofline denominators.
//
// The fused filtration/apparent kernel gathers diameter ranks from a matrix
// that stays in the on-chip caches (1 MB for 500 points), so its roofline
// needs the bandwidth of the cache level that serves it next to the HBM
// bandwidth.  This kernel streams a buffer with 16-byte loads that bypass L1
// (ld.global.cg): a buffer well below the 126 MB L2 measures L2 read
// bandwidth, one far above it measures HBM read bandwidth.  It reads nothing
// of the method; the paper has no counterpart.
#include "vr_common.cuh"

namespace vr {
namespace {

__global__ void __launch_bounds__(512) k_read_probe(const uint4* __restrict__ p, int64_t n16, int iters,
                                                    unsigned int* __restrict__ sink) {
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it) {
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        // four independent loads in flight per thread
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride);
            const uint4 c = __ldcg(p + i + 2 * stride), d = __ldcg(p + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);  // keeps the loads live; the buffer is zeros
}

}  // namespace
}  // namespace vr

extern "C" vr_status vr_probe_read_gbs(int64_t bytes, int32_t iters, void* stream, double* out_gbs) {
    if (!out_gbs || bytes < (1 << 20) || bytes > ((int64_t)1 << 36) || iters < 1 || iters > 100000)
        return VR_ERR_INVALID_ARG;
    *out_gbs = 0.0;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        vr::Workspace ws(s);
        const int64_t n16 = bytes / 16;
        uint4* buf = ws.alloc_n<uint4>((size_t)n16);
        unsigned int* sink = ws.zeros_n<unsigned int>(1);
        VR_CUDA(cudaMemsetAsync(buf, 0, (size_t)n16 * 16, s));
        int dev = 0, sms = 148;
        VR_CUDA(cudaGetDevice(&dev));
        VR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const unsigned grid = (unsigned)sms * 4;  // 4 blocks of 512 threads per SM: every warp slot busy
        vr::k_read_probe<<<grid, 512, 0, s>>>(buf, n16, 1, sink);  // warm-up (and L2 fill)
        VR_CUDA(cudaGetLastError());
        cudaEvent_t e0, e1;
        VR_CUDA(cudaEventCreate(&e0));
        VR_CUDA(cudaEventCreate(&e1));
        VR_CUDA(cudaEventRecord(e0, s));
        vr::k_read_probe<<<grid, 512, 0, s>>>(buf, n16, iters, sink);
        VR_CUDA(cudaEventRecord(e1, s));
        VR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        VR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *out_gbs = ms > 0.f ? (double)n16 * 16.0 * iters / (ms * 1e-3) / 1e9 : 0.0;
        VR_CUDA(cudaStreamSynchronize(s));
        return VR_OK;
    } catch (const vr::Error& e) {
        return e.code;
    }
}
