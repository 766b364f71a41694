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

// Keys of the vertices not yet in the tree: the filtration key of the best
// edge that reaches them (below 2^63: ranks stay below 2^31), or UNREACHED | v
// for a vertex no edge reaches yet, so that every key is distinct and the
// smallest one breaks ties to the smallest unreached vertex when a new tree
// of the forest starts.
constexpr uint64_t UNREACHED = 1ull << 63;
constexpr uint64_t IN_TREE = ~0ull;

__device__ __forceinline__ uint64_t edge_key(uint32_t rank, int64_t u, int64_t v) {
    int64_t a = u > v ? u : v, b = u > v ? v : u;
    uint64_t e = (uint64_t)(a * (a - 1) / 2 + b);
    return ((uint64_t)rank << 32) | (0xFFFFFFFFull - e);  // ascending = filtration order
}

// Single block.  best/intree live in shared memory (n <= 16384) or in the
// global buffers passed in; a thread only touches its own vertices v = t +
// k * blockDim, so one iteration needs two barriers: relax with the vertex
// added last and take the local minimum, then the block minimum.  Keys are
// distinct, so the minimum key alone identifies its vertex.
__global__ void k_prim(RankMatrix R, uint32_t thr, uint64_t* __restrict__ gbest,
                       uint8_t* __restrict__ gin, uint64_t* __restrict__ tree, int* __restrict__ tree_count,
                       int use_smem) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t n = R.n;
    uint64_t* best = use_smem ? reinterpret_cast<uint64_t*>(sm) : gbest;
    uint8_t* intree = use_smem ? sm + n * sizeof(uint64_t) : gin;
    __shared__ uint64_t red_key[32];
    __shared__ int64_t red_v[32];
    __shared__ int64_t sel;
    __shared__ uint64_t sel_key;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) { best[v] = UNREACHED | (uint64_t)v; intree[v] = 0; }
    int cnt = 0;
    int64_t u = -1;
    for (int64_t it = 0; it < n; ++it) {
        uint64_t mk = IN_TREE;
        int64_t mv = -1;
        for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
            if (intree[v]) continue;
            if (v == u) { intree[v] = 1; continue; }
            uint64_t k = best[v];
            if (u >= 0) {
                const uint32_t r = R(u, v);
                if (r <= thr) {
                    const uint64_t ek = edge_key(r, u, v);
                    if (ek < k) { k = ek; best[v] = k; }
                }
            }
            if (k < mk) { mk = k; mv = v; }
        }
        uint64_t wk = mk;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, wk, o);
            wk = y < wk ? y : wk;
        }
        if (wk == IN_TREE) {
            if (lane == 0) red_key[wid] = IN_TREE;
        } else if (mk == wk) {  // the one lane holding the warp's minimum
            red_key[wid] = wk;
            red_v[wid] = mv;
        }
        __syncthreads();
        if (wid == 0) {
            const uint64_t k = lane < nw ? red_key[lane] : IN_TREE;
            uint64_t bk = k;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t y = __shfl_xor_sync(0xffffffffu, bk, o);
                bk = y < bk ? y : bk;
            }
            if (lane < nw && k == bk) { sel = red_v[lane]; sel_key = bk; }
        }
        __syncthreads();
        u = sel;
        const uint64_t uk = sel_key;
        if (uk < UNREACHED) {  // u was reached by a tree edge (else it starts a new tree)
            if (threadIdx.x == 0) tree[cnt] = uk;
            ++cnt;
        }
    }
    // unused tail of the tree array sorts last
    for (int64_t v = cnt + threadIdx.x; v < n; v += blockDim.x) tree[v] = ~0ull;
    if (threadIdx.x == 0) *tree_count = cnt;
}

// Edge index e = a(a-1)/2 + b (a > b) back to its vertices: a float root
// estimate, corrected exactly in integers.
__device__ __forceinline__ void edge_vertices(uint64_t e, int64_t& a, int64_t& b) {
    int64_t x = (int64_t)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
    while (x > 1 && x * (x - 1) / 2 > (int64_t)e) --x;
    while ((x + 1) * x / 2 <= (int64_t)e) ++x;
    a = x;
    b = (int64_t)e - x * (x - 1) / 2;
}

// Boruvka's algorithm in one block for n <= BOR_MAXN (component labels and
// per-component minima in shared memory).  Every edge key is distinct, so
// the minimum spanning forest is unique and equals Prim's; each round every
// component takes its smallest outgoing edge (one pass over all pairs,
// rows split over warps, lanes over columns), components hook along those
// edges (a pair that picked the same edge keeps the smaller label as root)
// and labels are flattened by pointer jumping.  At most log2(n) + 1 rounds.
constexpr int BOR_MAXN = 8192;

__global__ void __launch_bounds__(1024) k_boruvka(RankMatrix R, uint32_t thr, uint64_t* __restrict__ tree,
                                                  int* __restrict__ tree_count) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = (int)R.n;
    uint64_t* mk = reinterpret_cast<uint64_t*>(sm);             // per label: smallest outgoing edge key
    int* comp = reinterpret_cast<int*>(sm + (size_t)n * 8);      // per vertex: component label (its root)
    int* par = comp + n;                                         // per label: hook target
    __shared__ int cnt, changed;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = threadIdx.x; v < n; v += blockDim.x) comp[v] = v;
    if (threadIdx.x == 0) cnt = 0;
    for (int round = 0; round < 64; ++round) {
        for (int v = threadIdx.x; v < n; v += blockDim.x) mk[v] = ~0ull;
        __syncthreads();
        // 1. smallest outgoing edge of every component: each row u (the whole
        // symmetric row, so every edge is seen from both ends) is reduced in
        // its warp and met with one shared-memory atomic
        for (int u = wid; u < n; u += nw) {
            const int cu = comp[u];
            uint64_t best = ~0ull;
            for (int v0 = 0; v0 < n; v0 += 32 * 16) {  // 16 independent row reads in flight per lane
                uint32_t r[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int v = v0 + 32 * j + lane;
                    r[j] = v < n ? R(u, v) : 0xFFFFFFFFu;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int v = v0 + 32 * j + lane;
                    if (v < n && v != u && r[j] <= thr && comp[v] != cu) {
                        const uint64_t k = edge_key(r[j], u, v);
                        best = k < best ? k : best;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t y = __shfl_xor_sync(0xffffffffu, best, o);
                best = y < best ? y : best;
            }
            if (lane == 0 && best != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(mk + cu), (unsigned long long)best);
        }
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        // 2. hook every root along its edge; record each picked edge once
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            par[c] = c;
            if (comp[c] != c || mk[c] == ~0ull) continue;
            int64_t a, b;
            edge_vertices(0xFFFFFFFFull - (mk[c] & 0xFFFFFFFFull), a, b);
            const int d = comp[a] == c ? comp[b] : comp[a];
            const bool mutual = mk[d] == mk[c];
            if (!mutual || c > d) {
                par[c] = d;
                tree[atomicAdd(&cnt, 1)] = mk[c];
                changed = 1;
            }
        }
        __syncthreads();
        if (!changed) break;
        // 3. pointer jumping over the labels, then relabel the vertices
        for (int s = 0; s < 32; ++s) {
            __shared__ int moved;
            if (threadIdx.x == 0) moved = 0;
            __syncthreads();
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const int p = par[c], pp = par[p];
                if (pp != p) { par[c] = pp; moved = 1; }
            }
            __syncthreads();
            if (!moved) break;
        }
        for (int v = threadIdx.x; v < n; v += blockDim.x) comp[v] = par[comp[v]];
        __syncthreads();
    }
    // unused tail of the tree array sorts last
    const int m = cnt;
    for (int v = m + threadIdx.x; v < n; v += blockDim.x) tree[v] = ~0ull;
    if (threadIdx.x == 0) *tree_count = m;
}

// Union-find for the elder rule: par (a root is its own parent), union by
// size (depth at most log2 n), and the oldest vertex of each component (the
// largest index) kept at its root.  The two roots of an edge are found in
// lockstep with path halving, so their load chains overlap.
__device__ __forceinline__ void uf_roots(int* par, int& x, int& y) {
    for (;;) {
        const int px = par[x], py = par[y];
        const bool dx = px == x, dy = py == y;
        if (dx && dy) return;
        if (!dx) { const int g = par[px]; par[x] = g; x = g; }
        if (!dy) { const int g = par[py]; par[y] = g; y = g; }
    }
}

// Elder-rule union-find over the tree edges in filtration order (thread 0).
// With sort_len > 0 the block first sorts the n tree keys itself (bitonic,
// padded to sort_len, in shared memory after the union-find arrays) and
// writes the pairs in parallel once thread 0 has replayed the merges.
__global__ void k_elder(const uint64_t* __restrict__ tree_in, const int* __restrict__ tree_count, int64_t n,
                        PairRec* __restrict__ out, int* __restrict__ out_count, uint32_t* __restrict__ clear1,
                        int* __restrict__ guf, int use_smem, int sort_len) {
    extern __shared__ __align__(16) unsigned char sm[];
    int* par = use_smem ? reinterpret_cast<int*>(sm) : guf;  // n parents, then n sizes, then n oldest
    int* sz = par + n;
    int* old = sz + n;
    const uint64_t* tree = tree_in;
    if (sort_len > 0) {
        uint64_t* a = reinterpret_cast<uint64_t*>(sm + (((size_t)n * 3 * sizeof(int) + 15) & ~(size_t)15));
        for (int i = threadIdx.x; i < sort_len; i += blockDim.x) a[i] = i < n ? tree_in[i] : ~0ull;
        __syncthreads();
        const int half = sort_len >> 1;
        for (int k = 2; k <= sort_len; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int p = threadIdx.x; p < half; p += blockDim.x) {
                    const int i = 2 * p - (p & (j - 1));
                    const uint64_t x = a[i], y = a[i + j];
                    if ((x > y) == ((i & k) == 0)) { a[i] = y; a[i + j] = x; }
                }
                __syncthreads();
            }
        tree = a;
    }
    for (int v = threadIdx.x; v < n; v += blockDim.x) { par[v] = v; sz[v] = 1; old[v] = v; }
    __syncthreads();
    const int m = *tree_count;
    if (sort_len > 0) {
        // thread 0 replays the merges into shared memory only (the birth of each
        // death edge); the block then writes the pairs and clearing bits
        int* bn = reinterpret_cast<int*>(const_cast<uint64_t*>(tree) + sort_len);
        if (threadIdx.x == 0) {
            for (int i = 0; i < m; ++i) {
                const uint64_t e = 0xFFFFFFFFull - (tree[i] & 0xFFFFFFFFull);
                int64_t a, b;
                edge_vertices(e, a, b);
                int ra = (int)a, rb = (int)b;
                uf_roots(par, ra, rb);
                const int oa = old[ra], ob = old[rb];
                bn[i] = oa < ob ? oa : ob;
                const int big = sz[ra] >= sz[rb] ? ra : rb, small = big == ra ? rb : ra;
                par[small] = big;
                sz[big] += sz[small];
                old[big] = oa < ob ? ob : oa;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const uint64_t key = tree[i];
            const uint64_t e = 0xFFFFFFFFull - (key & 0xFFFFFFFFull);
            PairRec pr;
            pr.birth_rank = 0;
            pr.death_rank = (uint32_t)(key >> 32);
            pr.birth_cidx = (uint64_t)bn[i];
            pr.death_cidx = (int64_t)e;
            out[i] = pr;
            if (clear1) atomicOr(clear1 + (e >> 5), 1u << (e & 31));
        }
        if (threadIdx.x == 0) {
            int k = m;
            for (int v = 0; v < n; ++v)
                if (par[v] == v) {
                    PairRec pr;
                    pr.birth_rank = 0;
                    pr.death_rank = 0xFFFFFFFFu;
                    pr.birth_cidx = (uint64_t)old[v];
                    pr.death_cidx = -1;
                    out[k++] = pr;
                }
            *out_count = k;
        }
        return;
    }
    if (threadIdx.x != 0) return;
    int k = 0;
    for (int i = 0; i < m; ++i) {
        const uint64_t key = tree[i];
        const uint64_t e = 0xFFFFFFFFull - (key & 0xFFFFFFFFull);
        int64_t a, b;
        edge_vertices(e, a, b);
        int ra = (int)a, rb = (int)b;
        uf_roots(par, ra, rb);
        const int oa = old[ra], ob = old[rb];  // oldest = largest vertex index
        const int born = oa < ob ? oa : ob;     // the younger component dies
        const int big = sz[ra] >= sz[rb] ? ra : rb, small = big == ra ? rb : ra;
        par[small] = big;
        sz[big] += sz[small];
        old[big] = oa < ob ? ob : oa;
        PairRec pr;
        pr.birth_rank = 0;
        pr.death_rank = (uint32_t)(key >> 32);
        pr.birth_cidx = (uint64_t)born;
        pr.death_cidx = (int64_t)e;
        out[k++] = pr;
        if (clear1) atomicOr(clear1 + (e >> 5), 1u << (e & 31));  // no read back: one store per edge
    }
    for (int v = 0; v < n; ++v)
        if (par[v] == v) {
            PairRec pr;
            pr.birth_rank = 0;
            pr.death_rank = 0xFFFFFFFFu;
            pr.birth_cidx = (uint64_t)old[v];
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
    if (n <= BOR_MAXN) {
        const size_t bsm = (size_t)n * (sizeof(uint64_t) + 2 * sizeof(int));
        VR_CUDA(cudaFuncSetAttribute(k_boruvka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
        k_boruvka<<<1, 1024, bsm, ws.stream>>>(R, thr_rank, tree, tree_count);
    } else {
        if (use_smem)
            VR_CUDA(cudaFuncSetAttribute(k_prim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)prim_smem));
        k_prim<<<1, threads, use_smem ? prim_smem : 0, ws.stream>>>(R, thr_rank, gbest, gin, tree, tree_count,
                                                                     use_smem);
    }
    VR_CUDA(cudaGetLastError());
    // tree edges in filtration order (the unused tail holds ~0 and sorts last):
    // sorted inside k_elder when they fit its shared memory, else radix sorted
    int sort_len = 1;
    while (sort_len < n) sort_len <<= 1;
    if (sort_len > 4096) {
        sort_len = 0;
        radix_sort_u64(ws, tree, nullptr, n, 64);
    }
    const size_t uf_smem = (((size_t)n * 3 * sizeof(int) + 15) & ~(size_t)15) + (size_t)sort_len * sizeof(uint64_t) +
                           (sort_len > 0 ? (size_t)n * sizeof(int) : 0);  // union-find, sorted keys, births
    const int uf_in_smem = uf_smem <= 160 * 1024;
    int* guf = uf_in_smem ? nullptr : ws.alloc_n<int>((size_t)n * 3);
    if (!uf_in_smem && sort_len > 0) {  // cannot happen for sort_len <= 4096 (n <= 4096)
        sort_len = 0;
        radix_sort_u64(ws, tree, nullptr, n, 64);
    }
    if (uf_in_smem)
        VR_CUDA(cudaFuncSetAttribute(k_elder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)uf_smem));
    k_elder<<<1, 512, uf_in_smem ? uf_smem : 0, ws.stream>>>(tree, tree_count, n, out, out_count, clear_bits_dim1,
                                                             guf, uf_in_smem, sort_len);
    VR_CUDA(cudaGetLastError());
}

}  // namespace vr
