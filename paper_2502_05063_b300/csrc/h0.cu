// h0.cu -- dimension-0 persistence (Sec. 5.2.5 of the paper).
//
// The edges that kill a connected component form the minimum spanning tree
// of the threshold graph (a forest if the threshold disconnects it).  Edges
// are compared in the simplex-wise order of Sec. 5.1.4: diameter ascending,
// then combinatorial index descending; under that strict total order the
// tree is unique.  It is grown here with Prim's algorithm in one thread
// block (dense distance matrix, no edge list), then the tree edges are
// sorted and replayed through a union-find that applies the elder rule
// (Sec. 3.2, eq. 3.88): all vertices are born at 0 and vertex n-1 is the
// oldest (largest index first), so the merging component whose oldest
// vertex has the smaller index dies and that vertex is the birth simplex.
#include "vr_common.cuh"

namespace vr {

namespace {

constexpr uint64_t NOT_REACHED = ~0ull - 1;  // a vertex no tree edge has touched yet

__device__ __forceinline__ uint64_t edge_key(uint32_t rank, int64_t u, int64_t v) {
    int64_t a = u > v ? u : v, b = u > v ? v : u;
    uint64_t e = (uint64_t)(a * (a - 1) / 2 + b);
    return ((uint64_t)rank << 32) | (0xFFFFFFFFull - e);  // ascending = filtration order
}

// Single block.  best/intree live in shared memory (n <= 16384) or in the
// global buffers passed in.
__global__ void k_prim(RankMatrix R, uint32_t thr, uint64_t* __restrict__ gbest,
                       uint8_t* __restrict__ gin, uint64_t* __restrict__ tree, int* __restrict__ tree_count,
                       int use_smem) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t n = R.n;
    uint64_t* best = use_smem ? reinterpret_cast<uint64_t*>(sm) : gbest;
    uint8_t* intree = use_smem ? sm + n * sizeof(uint64_t) : gin;
    __shared__ uint64_t red_key[32];
    __shared__ int64_t red_idx[32];
    __shared__ int64_t sel;
    __shared__ uint64_t sel_key;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) { best[v] = NOT_REACHED; intree[v] = 0; }
    int cnt = 0;
    __syncthreads();
    for (int64_t it = 0; it < n; ++it) {
        uint64_t mk = ~0ull; int64_t mi = n;
        for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
            uint64_t k = intree[v] ? ~0ull : best[v];
            if (k < mk) { mk = k; mi = v; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            uint64_t ok = __shfl_xor_sync(0xffffffffu, mk, o);
            int64_t oi = __shfl_xor_sync(0xffffffffu, mi, o);
            if (ok < mk || (ok == mk && oi < mi)) { mk = ok; mi = oi; }
        }
        if (lane == 0) { red_key[wid] = mk; red_idx[wid] = mi; }
        __syncthreads();
        if (wid == 0) {
            mk = lane < nw ? red_key[lane] : ~0ull;
            mi = lane < nw ? red_idx[lane] : n;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                uint64_t ok = __shfl_xor_sync(0xffffffffu, mk, o);
                int64_t oi = __shfl_xor_sync(0xffffffffu, mi, o);
                if (ok < mk || (ok == mk && oi < mi)) { mk = ok; mi = oi; }
            }
            if (lane == 0) { sel = mi; sel_key = mk; }
        }
        __syncthreads();
        const int64_t u = sel;
        const uint64_t uk = sel_key;
        if (threadIdx.x == 0) {
            intree[u] = 1;
            if (uk != NOT_REACHED) tree[cnt] = uk;  // the edge that reached u
        }
        if (uk != NOT_REACHED) ++cnt;
        __syncthreads();
        for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
            if (intree[v]) continue;
            uint32_t r = R(u, v);
            if (r > thr) continue;
            uint64_t k = edge_key(r, u, v);
            if (k < best[v]) best[v] = k;
        }
        __syncthreads();
    }
    // unused tail of the tree array sorts last
    for (int64_t v = cnt + threadIdx.x; v < n; v += blockDim.x) tree[v] = ~0ull;
    if (threadIdx.x == 0) *tree_count = cnt;
}

__device__ __forceinline__ void edge_vertices(uint64_t e, int64_t& a, int64_t& b) {
    int64_t x = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)e)) * 0.5);
    while (x * (x - 1) / 2 > (int64_t)e) --x;
    while ((x + 1) * x / 2 <= (int64_t)e) ++x;
    a = x;
    b = (int64_t)e - x * (x - 1) / 2;
}

// Root entries hold -1 - (oldest vertex of the component); path halving.
__device__ __forceinline__ int64_t uf_find(int64_t* parent, int64_t x) {
    while (parent[x] >= 0) {
        int64_t p = parent[x];
        if (parent[p] >= 0) parent[x] = parent[p];
        x = p;
    }
    return x;
}

// One thread: elder-rule union-find over the sorted tree edges.
__global__ void k_elder(const uint64_t* __restrict__ tree, const int* __restrict__ tree_count, int64_t n,
                        PairRec* __restrict__ out, int* __restrict__ out_count, uint32_t* __restrict__ clear1,
                        int64_t* __restrict__ gparent, int use_smem) {
    extern __shared__ __align__(16) unsigned char sm[];
    if (threadIdx.x != 0) return;
    int64_t* parent = use_smem ? reinterpret_cast<int64_t*>(sm) : gparent;  // root's entry holds -1-oldest
    for (int64_t v = 0; v < n; ++v) parent[v] = -1 - v;
    const int m = *tree_count;
    int k = 0;
    for (int i = 0; i < m; ++i) {
        const uint64_t key = tree[i];
        const uint64_t e = 0xFFFFFFFFull - (key & 0xFFFFFFFFull);
        int64_t a, b;
        edge_vertices(e, a, b);
        const int64_t ra = uf_find(parent, a), rb = uf_find(parent, b);
        const int64_t oa = -1 - parent[ra], ob = -1 - parent[rb];  // oldest = largest vertex index
        const int64_t young = oa < ob ? ra : rb, old = oa < ob ? rb : ra;
        const int64_t born = oa < ob ? oa : ob;
        parent[young] = old;
        PairRec pr;
        pr.birth_rank = 0;
        pr.death_rank = (uint32_t)(key >> 32);
        pr.birth_cidx = (uint64_t)born;
        pr.death_cidx = (int64_t)e;
        out[k++] = pr;
        if (clear1) clear1[e >> 5] |= 1u << (e & 31);
    }
    for (int64_t v = 0; v < n; ++v)
        if (parent[v] < 0) {
            PairRec pr;
            pr.birth_rank = 0;
            pr.death_rank = 0xFFFFFFFFu;
            pr.birth_cidx = (uint64_t)(-1 - parent[v]);
            pr.death_cidx = -1;
            out[k++] = pr;
        }
    *out_count = k;
}

}  // namespace

void launch_h0(const RankMatrix& R, uint32_t thr_rank, PairRec* out, int* out_count,
               uint32_t* clear_bits_dim1, int* dev_err, Workspace& ws) {
    (void)dev_err;
    const int64_t n = R.n;
    uint64_t* tree = ws.alloc_n<uint64_t>(n);
    int* tree_count = ws.alloc_n<int>(1);
    const size_t prim_smem = (size_t)n * (sizeof(uint64_t) + 1);
    const int use_smem = prim_smem <= 160 * 1024;
    uint64_t* gbest = use_smem ? nullptr : ws.alloc_n<uint64_t>(n);
    uint8_t* gin = use_smem ? nullptr : ws.alloc_n<uint8_t>(n);
    int threads = n >= 1024 ? 1024 : (int)((n + 31) / 32 * 32);
    if (threads < 64) threads = 64;
    if (use_smem)
        VR_CUDA(cudaFuncSetAttribute(k_prim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)prim_smem));
    k_prim<<<1, threads, use_smem ? prim_smem : 0, ws.stream>>>(R, thr_rank, gbest, gin, tree, tree_count, use_smem);
    VR_CUDA(cudaGetLastError());
    // tree edges in filtration order (the unused tail holds ~0 and sorts last)
    radix_sort_u64(ws, tree, nullptr, n, 64);
    const size_t uf_smem = (size_t)n * sizeof(int64_t);
    const int uf_in_smem = uf_smem <= 160 * 1024;
    int64_t* gparent = uf_in_smem ? nullptr : ws.alloc_n<int64_t>(n);
    if (uf_in_smem)
        VR_CUDA(cudaFuncSetAttribute(k_elder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)uf_smem));
    k_elder<<<1, 32, uf_in_smem ? uf_smem : 0, ws.stream>>>(tree, tree_count, n, out, out_count,
                                                            clear_bits_dim1, gparent, uf_in_smem);
    VR_CUDA(cudaGetLastError());
}

}  // namespace vr
