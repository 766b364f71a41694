// rank.cu -- diameter ranks and the enclosing radius.
//
// The persistence pairs of a Rips filtration depend only on the order of the
// distances (Obs 5.6.8 of the paper): every comparison the method makes is
// "diam(a) < diam(b)" or "diam(a) == diam(b)".  The library therefore works
// on the dense rank of each distance among the distinct values {0} U {d(i,j)}
// and maps ranks back to the float values at the end.  Ranks are small
// integers (at most n(n-1)/2 + 1 of them), which shortens the packed sort
// keys and keeps (rank, index) row keys inside 64 bits.
//
// Enclosing radius R = min_x max_y d(x,y) (Sec. 5.2.12): truncating the
// filtration at R keeps every pair of nonzero persistence (Prop 5.2.13).
#include "vr_common.cuh"

namespace vr {

__global__ void k_float_bits(const float* __restrict__ d, int64_t m, uint32_t* __restrict__ keys) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        keys[k] = __float_as_uint(d[k]);  // d >= 0: unsigned order of the bits is the float order
}

// flag[i] = 1 if sorted[i] starts a new positive value
__global__ void k_distinct_flags(const uint32_t* __restrict__ s, int64_t m, uint32_t* __restrict__ flag) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        flag[k] = (s[k] != 0u && (k == 0 || s[k] != s[k - 1])) ? 1u : 0u;
}

__global__ void k_distinct_write(const uint32_t* __restrict__ s, const uint32_t* __restrict__ flag,
                                 const uint32_t* __restrict__ pos, int64_t m, float* __restrict__ values,
                                 int64_t* __restrict__ num_values) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        if (flag[k]) values[1 + pos[k]] = __uint_as_float(s[k]);
        if (k == m - 1) *num_values = 1 + pos[k] + flag[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        values[0] = 0.0f;
        if (m == 0) *num_values = 1;
    }
}

__device__ __forceinline__ uint32_t lower_bound_f(const float* __restrict__ v, int64_t len, float x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(v + mid) < x) lo = mid + 1; else hi = mid;
    }
    return (uint32_t)lo;
}

// One block per row i >= 1 of the triangle: rank of each d(i,j), written to
// R[i][j] and R[j][i]; the diagonal is rank 0 (distance 0).
__global__ void k_rank_matrix(const float* __restrict__ d, int64_t n, const float* __restrict__ values,
                              const int64_t* __restrict__ num_values, uint32_t* __restrict__ R, int64_t ld) {
    const int64_t i = blockIdx.x;
    const int64_t nv = *num_values;
    if (threadIdx.x == 0) R[i * ld + i] = 0;
    const int64_t row = i * (i - 1) / 2;
    for (int64_t j = threadIdx.x; j < i; j += blockDim.x) {
        uint32_t r = lower_bound_f(values, nv, d[row + j]);
        R[i * ld + j] = r;
        R[j * ld + i] = r;
    }
}

// rank of R = min over rows of the row maximum
__global__ void k_enclosing(const uint32_t* __restrict__ R, int64_t n, int64_t ld, uint32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        uint32_t m = 0;
        for (int64_t j = lane; j < n; j += 32) m = max(m, R[i * ld + j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMin(out, m);
    }
}

__global__ void k_threshold_rank(const float* __restrict__ values, const int64_t* __restrict__ num_values,
                                 float thr, uint32_t* __restrict__ out) {
    // largest rank whose value is <= thr (values[0] = 0 <= thr)
    int64_t lo = 0, hi = *num_values;  // first index with value > thr
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (values[mid] <= thr) lo = mid + 1; else hi = mid;
    }
    *out = (uint32_t)(lo - 1);
}

// Every rank above the threshold rank becomes thr + 1: no simplex with such
// an entry is in the filtration, and every comparison the method makes with
// one ("<= threshold", "<= diam(s)" for a simplex s of the filtration) has
// the same outcome, so packed keys need only bits for thr + 1.
__global__ void k_clamp_ranks(uint32_t* __restrict__ R, int64_t total, uint32_t cap) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x)
        if (R[k] > cap) R[k] = cap;
}

static unsigned grid_for(int64_t m, int threads) {
    int64_t b = (m + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 148 * 32) b = 148 * 32;
    return (unsigned)b;
}

RankInfo build_ranks(Workspace& ws, const float* lower_tri, int64_t n, HostScratch& hs) {
    RankInfo ri{};
    const int64_t m = n * (n - 1) / 2;
    ri.ld = (n + 31) / 32 * 32;
    ri.rank = ws.alloc_n<uint32_t>(n * ri.ld);
    ri.values = ws.alloc_n<float>(m + 1);
    int64_t* nv = ws.alloc_n<int64_t>(1);
    uint32_t* keys = ws.alloc_n<uint32_t>(m > 0 ? m : 1);
    uint32_t* flag = ws.alloc_n<uint32_t>(m > 0 ? m : 1);
    cudaStream_t s = ws.stream;
    if (m > 0) {
        k_float_bits<<<grid_for(m, 256), 256, 0, s>>>(lower_tri, m, keys);
        radix_sort_u32(ws, keys, nullptr, m, 32);
        k_distinct_flags<<<grid_for(m, 256), 256, 0, s>>>(keys, m, flag);
    }
    uint32_t* pos = ws.alloc_n<uint32_t>(m > 0 ? m : 1);
    if (m > 0) {
        VR_CUDA(cudaMemcpyAsync(pos, flag, m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        scan_u32_exclusive(pos, m, s);
    }
    k_distinct_write<<<grid_for(m, 256), 256, 0, s>>>(keys, flag, pos, m, ri.values, nv);
    k_rank_matrix<<<(unsigned)n, 128, 0, s>>>(lower_tri, n, ri.values, nv, ri.rank, ri.ld);
    uint32_t* enc = ws.alloc_n<uint32_t>(1);
    VR_CUDA(cudaMemsetAsync(enc, 0xFF, sizeof(uint32_t), s));
    k_enclosing<<<grid_for(n * 32, 256), 256, 0, s>>>(ri.rank, n, ri.ld, enc);
    VR_CUDA(cudaGetLastError());
    VR_CUDA(cudaMemcpyAsync(&hs.p[0], nv, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaMemcpyAsync(&hs.p[1], enc, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaStreamSynchronize(s));
    ri.num_values = hs.p[0];
    ri.enclosing_rank = (uint32_t)(hs.p[1] & 0xFFFFFFFFu);
    ri.num_values_dev = nv;
    return ri;
}

void clamp_ranks(Workspace& ws, const RankInfo& ri, int64_t n, uint32_t thr_rank) {
    const int64_t total = n * ri.ld;
    k_clamp_ranks<<<grid_for(total, 256), 256, 0, ws.stream>>>(ri.rank, total, thr_rank + 1);
    VR_CUDA(cudaGetLastError());
}

uint32_t threshold_rank(Workspace& ws, const RankInfo& ri, float threshold, HostScratch& hs) {
    if (isinf(threshold) && threshold > 0) return ri.enclosing_rank;
    uint32_t* out = ws.alloc_n<uint32_t>(1);
    k_threshold_rank<<<1, 1, 0, ws.stream>>>(ri.values, ri.num_values_dev, threshold, out);
    VR_CUDA(cudaGetLastError());
    VR_CUDA(cudaMemcpyAsync(&hs.p[2], out, sizeof(uint32_t), cudaMemcpyDeviceToHost, ws.stream));
    VR_CUDA(cudaStreamSynchronize(ws.stream));
    return (uint32_t)(hs.p[2] & 0xFFFFFFFFu);
}

}  // namespace vr
