// sparse.cu -- the Rips complex enumerated from neighbour lists: the sparse /
// low-threshold mode (paper, arXiv 2502.05063: Sec. 5.3.12-5.3.13 and
// Algorithm 15, cofacets of a simplex among the neighbours of its vertices;
// Sec. 5.5.3, warp-based filtering; Sec. 5.7.2, memory allocated by the size
// of the complex rather than by the number of possible simplices).
//
// With a threshold far below the enclosing radius, almost none of the
// C(n, p+1) candidate indices of the dense enumeration are simplices of the
// filtration.  Here the p-simplices of the complex are listed explicitly:
//   * the threshold graph as CSR neighbour lists (ascending), one warp per
//     vertex, ballot-compacted;
//   * the edges from the lists (already in combinatorial-index order), and
//     the (p+1)-simplices from the p-simplices by adding a larger neighbour w
//     of the largest vertex that is a neighbour of every vertex (each simplex
//     once, from the facet without its largest vertex); counted first, then
//     written into exactly the room needed, then put in index order by the
//     radix sort;
//   * the fused filter + apparent-pair kernel over the list: the apparent
//     cofacet of s (the largest w keeping the diameter) is a neighbour of every
//     vertex of s, so it is searched among the neighbours of the vertex of s
//     with the fewest, 32 per warp step from the largest down;
//   * clearing marks a (p+1)-simplex by its position in the next list
//     (binary search), so no bitmap over C(n, p+2) indices is needed.
// The pairs are exactly those of the dense path (tested): the same diameters,
// the same order, the same apparent pairs.
#include "vr_common.cuh"

namespace vr {
namespace {

constexpr int SP_WARPS = 8;
constexpr int SQCAP = 64;

// ---------------------------------------------------------------------------
// neighbour lists of the threshold graph
// ---------------------------------------------------------------------------
__global__ void k_nbr_count(RankMatrix R, uint32_t thr, uint32_t* __restrict__ deg) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int n = (int)R.n;
    for (int64_t v = warp; v < n; v += nw) {
        const uint32_t* row = R.r + (uint32_t)v * (uint32_t)R.ld;
        uint32_t cnt = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const bool ok = j < n && j != v && __ldg(row + j) <= thr;
            cnt += __popc(__ballot_sync(0xffffffffu, ok));
        }
        if (lane == 0) deg[v] = cnt;
    }
}

__global__ void k_nbr_fill(RankMatrix R, uint32_t thr, const uint32_t* __restrict__ off, uint32_t* __restrict__ nbr) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int n = (int)R.n;
    for (int64_t v = warp; v < n; v += nw) {
        const uint32_t* row = R.r + (uint32_t)v * (uint32_t)R.ld;
        uint32_t pos = off[v];
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const bool ok = j < n && j != v && __ldg(row + j) <= thr;
            const uint32_t bl = __ballot_sync(0xffffffffu, ok);
            if (ok) nbr[pos + __popc(bl & ((1u << lane) - 1u))] = (uint32_t)j;
            pos += __popc(bl);
        }
    }
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t lo, uint32_t hi,
                                                   uint32_t x) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t len, uint64_t x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// simplex lists
// ---------------------------------------------------------------------------
// edges (j < i): the neighbours of i below i, rows in order -> index order
__global__ void k_edge_count(Neighbours N, int n, uint32_t* __restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cnt[i] = lower_bound_u32(N.nbr, N.off[i], N.off[i + 1], (uint32_t)i) - N.off[i];
}

__global__ void k_edge_fill(Neighbours N, int n, const uint32_t* __restrict__ pos, uint64_t* __restrict__ cidx,
                            uint16_t* __restrict__ verts) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nw) {
        const uint32_t b = N.off[i], c = pos[i + 1] - pos[i];
        for (uint32_t k = lane; k < c; k += 32) {
            const uint32_t j = N.nbr[b + k];
            const uint64_t at = pos[i] + k;
            cidx[at] = (uint64_t)i * (uint64_t)(i - 1) / 2 + j;
            uint16_t* vv = verts + at * SIMPLEX_VSTRIDE;
            vv[0] = (uint16_t)j;
            vv[1] = (uint16_t)i;
        }
    }
}

// (p+1)-simplices from p-simplices: w > v_p among the neighbours of v_p that
// is a neighbour of every v_a (rank <= thr).  Pass 1 counts, pass 2 writes.
template <bool WRITE>
__global__ void k_extend(RankMatrix R, Binom B, Neighbours N, uint32_t thr, int p, const uint64_t* __restrict__ cidx,
                         const uint16_t* __restrict__ verts, int64_t len, uint32_t* __restrict__ cnt,
                         uint64_t* __restrict__ ocidx, uint16_t* __restrict__ overts, uint64_t* __restrict__ oidx,
                         unsigned long long* __restrict__ total) {
    unsigned long long mine = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
        int v[VR_MAX_DIM + 2];
        const uint16_t* vv = verts + k * SIMPLEX_VSTRIDE;
        for (int a = 0; a <= p; ++a) v[a] = vv[a];
        const int top = v[p];
        const uint32_t e = N.off[top + 1];
        uint32_t q = lower_bound_u32(N.nbr, N.off[top], e, (uint32_t)top + 1);
        uint32_t c = 0, at = WRITE ? cnt[k] : 0;
        const uint64_t base = WRITE ? cidx[k] : 0;
        for (; q < e; ++q) {
            const uint32_t w = __ldg(N.nbr + q);
            bool ok = true;
            for (int a = 0; a < p && ok; ++a) ok = R(w, v[a]) <= thr;
            if (!ok) continue;
            if (WRITE) {
                ocidx[at] = base + B(w, p + 2);
                oidx[at] = at;
                uint16_t* ov = overts + (uint64_t)at * SIMPLEX_VSTRIDE;
                for (int a = 0; a <= p; ++a) ov[a] = (uint16_t)v[a];
                ov[p + 1] = (uint16_t)w;
                ++at;
            } else {
                ++c;
            }
        }
        if (!WRITE) {
            cnt[k] = c;
            mine += c;
        }
    }
    if (!WRITE) {  // the exact total in 64 bits (the list offsets are 32-bit)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
    }
}

__global__ void k_gather_verts(const uint64_t* __restrict__ idx, int64_t len, const uint16_t* __restrict__ in,
                               uint16_t* __restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
        const uint4 x = *reinterpret_cast<const uint4*>(in + idx[k] * SIMPLEX_VSTRIDE);
        *reinterpret_cast<uint4*>(out + k * SIMPLEX_VSTRIDE) = x;
    }
}

// ---------------------------------------------------------------------------
// filter + apparent pairs over a simplex list
// ---------------------------------------------------------------------------
template <int P>
struct SQueue {
    uint64_t c[SQCAP];
    uint32_t r[SQCAP];
    uint32_t eq[SQCAP];
    uint16_t v[P + 1][SQCAP];
};

__host__ __device__ constexpr uint32_t pairs_without_s(int a, int nv) {
    uint32_t m = 0;
    int k = 0;
    for (int i = 1; i < nv; ++i)
        for (int j = 0; j < i; ++j) {
            if (i != a && j != a) m |= 1u << k;
            ++k;
        }
    return m;
}

struct SCount {
    uint32_t cleared = 0, kept = 0, app = 0, facet = 0;
    unsigned long long scan = 0;
};

// Apparent test of the first m queued columns: each column in turn searches,
// with the whole warp, the neighbours of its vertex of smallest degree from
// the largest down for the first w that keeps the diameter; then each lane
// finishes its own column (facet test, outputs).
template <int P>
__device__ void sparse_search(const RankMatrix& R, const Binom& B, const Neighbours& N, SQueue<P>& q, int m,
                              int cidx_bits, uint64_t rmask, const ApparentOut& o, SCount& k) {
    constexpr int NV = P + 1;
    const int lane = threadIdx.x & 31;
    const bool mine = lane < m;
    int v[NV];
    uint32_t r = 0, eq = 0;
    uint64_t c = 0;
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = mine ? (int)q.v[a][lane] : 0;
    if (mine) {
        c = q.c[lane];
        r = q.r[lane];
        eq = q.eq[lane];
    }
    __syncwarp();
    // the vertex with the fewest neighbours
    int best = 0;
    uint32_t bdeg = 0xFFFFFFFFu;
    if (mine) {
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            const uint32_t d = N.off[v[a] + 1] - N.off[v[a]];
            if (d < bdeg) { bdeg = d; best = a; }
        }
    }
    int wf = -1;
    uint32_t rw[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) rw[a] = 0;
    unsigned long long scanned = 0;
    for (int src = 0; src < m; ++src) {
        int sv[NV];
        const uint32_t* rows[NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            sv[a] = __shfl_sync(0xffffffffu, v[a], src);
            rows[a] = R.r + (uint32_t)sv[a] * (uint32_t)R.ld;
        }
        const uint32_t sr = __shfl_sync(0xffffffffu, r, src);
        const int sb = __shfl_sync(0xffffffffu, best, src);
        int u = sv[0];
#pragma unroll
        for (int a = 1; a < NV; ++a) if (a == sb) u = sv[a];
        const int64_t b0 = N.off[u], e0 = N.off[u + 1];
        int hit = -1;
        int64_t seen = 0;
        for (int64_t top = e0 - 1; top >= b0; top -= 32) {
            const int64_t q2 = top - lane;
            bool ok = q2 >= b0;
            int w = 0;
            if (ok) {
                w = (int)__ldg(N.nbr + q2);
#pragma unroll
                for (int a = 0; a < NV; ++a) ok &= (w != sv[a]) & (__ldg(rows[a] + w) <= sr);
            }
            const uint32_t bl = __ballot_sync(0xffffffffu, ok);
            if (bl) {
                const int f = __ffs(bl) - 1;
                hit = __shfl_sync(0xffffffffu, w, f);
                seen += f + 1;
                break;
            }
            seen += top - b0 + 1 < 32 ? top - b0 + 1 : 32;
        }
        if (lane == src) {
            wf = hit;
            scanned = (unsigned long long)seen;
            if (hit >= 0) {
#pragma unroll
                for (int a = 0; a < NV; ++a) rw[a] = R(v[a], hit);
            }
        }
    }
    if (mine) k.scan += scanned;
    bool apparent = false;
    if (mine && wf >= 0) {
        ++k.facet;
        uint32_t rweq = 0;
#pragma unroll
        for (int a = 0; a < NV; ++a) rweq |= (rw[a] == r ? 1u : 0u) << a;
        apparent = true;
#pragma unroll
        for (int a = 0; a < NV; ++a)
            if (v[a] > wf && ((eq & pairs_without_s(a, NV)) != 0 || (rweq & ~(1u << a)) != 0)) apparent = false;
    }
    if (apparent) {
        ++k.app;
        if (o.clear_next || o.zero_pairs) {
            uint64_t ct = 0;
            int kk = 0;
            bool placed = false;
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                if (!placed && wf < v[a]) { ct += B(wf, kk + 1); ++kk; placed = true; }
                ct += B(v[a], kk + 1);
                ++kk;
            }
            if (!placed) ct += B(wf, kk + 1);
            if (o.clear_next) {
                const int64_t pos = lower_bound_u64(o.next_list, o.next_len, ct);
                if (pos < o.next_len) atomicOr(o.clear_next + (pos >> 5), 1u << (pos & 31));
                else atomicExch(o.dev_err, DEV_INTERNAL | (6 << 8));  // a cofacet of K missing from the list
            }
            if (o.zero_pairs) {
                const unsigned long long at = atomicAdd(o.num_zero_pairs, 1ull);
                PairRec prc;
                prc.birth_rank = r; prc.death_rank = r;
                prc.birth_cidx = c; prc.death_cidx = (int64_t)ct;
                o.zero_pairs[at] = prc;
            }
        }
    }
    const bool nonapp = mine && !apparent;
    const uint32_t nb = __ballot_sync(0xffffffffu, nonapp);
    if (nb) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(o.num_nonapparent, (unsigned long long)__popc(nb));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (nonapp) {
            const unsigned long long at = base + __popc(nb & ((1u << lane) - 1u));
            if ((int64_t)at < o.capacity) o.nonapparent_keys[at] = ((~(uint64_t)r & rmask) << cidx_bits) | c;
            else atomicExch(o.dev_err, DEV_CAPACITY);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(SP_WARPS * 32)
k_sparse_filtration_apparent(RankMatrix R, Binom B, Neighbours N, const uint64_t* __restrict__ lc,
                             const uint16_t* __restrict__ lv, int64_t len, const uint32_t* __restrict__ clear_bits,
                             int clear_by_pos, int cidx_bits, uint64_t rmask, ApparentOut o) {
    constexpr int NV = P + 1;
    constexpr int NPS = NV * (NV - 1) / 2;
    __shared__ SQueue<P> queues[SP_WARPS];
    SQueue<P>& q = queues[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    SCount k;
    int qn = 0;
    for (int64_t base = warp * 32; base < len; base += nw * 32) {
        const int64_t i = base + lane;
        bool kept = false;
        uint32_t r = 0, eq = 0;
        uint64_t c = 0;
        int v[NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = 0;
        if (i < len) {
            c = lc[i];
            const uint16_t* vv = lv + i * SIMPLEX_VSTRIDE;
#pragma unroll
            for (int a = 0; a < NV; ++a) v[a] = vv[a];
            uint32_t pr[NPS];
            int kk = 0;
#pragma unroll
            for (int a = 1; a < NV; ++a) {
                const uint32_t* row = R.r + (uint32_t)v[a] * (uint32_t)R.ld;
#pragma unroll
                for (int b = 0; b < a; ++b) {
                    pr[kk] = __ldg(row + v[b]);
                    r = max(r, pr[kk]);
                    ++kk;
                }
            }
#pragma unroll
            for (int j = 0; j < NPS; ++j) eq |= (pr[j] == r ? 1u : 0u) << j;
            const uint64_t bit = clear_by_pos ? (uint64_t)i : c;
            if (clear_bits && ((__ldg(clear_bits + (bit >> 5)) >> (bit & 31)) & 1u)) ++k.cleared;
            else { kept = true; ++k.kept; }
        }
        const uint32_t kb = __ballot_sync(0xffffffffu, kept);
        if (kept) {
            const int at = qn + __popc(kb & ((1u << lane) - 1u));
            q.c[at] = c;
            q.r[at] = r;
            q.eq[at] = eq;
#pragma unroll
            for (int a = 0; a < NV; ++a) q.v[a][at] = (uint16_t)v[a];
        }
        qn += __popc(kb);
        __syncwarp();
        if (qn >= 32) {
            sparse_search<P>(R, B, N, q, 32, cidx_bits, rmask, o, k);
            const int rest = qn - 32;
            if (lane < rest) {
                q.c[lane] = q.c[32 + lane];
                q.r[lane] = q.r[32 + lane];
                q.eq[lane] = q.eq[32 + lane];
#pragma unroll
                for (int a = 0; a < NV; ++a) q.v[a][lane] = q.v[a][32 + lane];
            }
            qn = rest;
            __syncwarp();
        }
    }
    if (qn > 0) sparse_search<P>(R, B, N, q, qn, cidx_bits, rmask, o, k);
    unsigned long long t[5] = {k.cleared, k.kept, k.app, k.scan, k.facet};
#pragma unroll
    for (int x = 0; x < 5; ++x)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t[x] += __shfl_xor_sync(0xffffffffu, t[x], off);
    if (lane == 0) {
        if (t[0]) atomicAdd(o.counters + 1, t[0]);
        if (t[1]) atomicAdd(o.counters + 2, t[1]);
        if (t[2]) atomicAdd(o.counters + 3, t[2]);
        if (t[3]) atomicAdd(o.counters + 6, t[3]);
        if (t[4]) atomicAdd(o.counters + 7, t[4]);
    }
}

unsigned grid_of(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 148 * 16 ? 148 * 16 : b));
}

template <int P>
void launch_sparse_p(const RankMatrix& R, const Binom& B, const Neighbours& N, const SimplexList& L,
                     const uint32_t* clear_bits, bool clear_by_pos, int cidx_bits, uint64_t rmask,
                     const ApparentOut& o, cudaStream_t s) {
    int64_t blocks = (L.len + 32 * SP_WARPS - 1) / (32 * SP_WARPS);
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (blocks < 1) blocks = 1;
    k_sparse_filtration_apparent<P><<<(unsigned)blocks, SP_WARPS * 32, 0, s>>>(
        R, B, N, L.cidx, L.verts, L.len, clear_bits, clear_by_pos ? 1 : 0, cidx_bits, rmask, o);
    VR_CUDA(cudaGetLastError());
}

}  // namespace

Neighbours build_neighbours(Workspace& ws, const RankMatrix& R, uint32_t thr, HostScratch& hs) {
    const int64_t n = R.n;
    Neighbours N;
    N.off = ws.alloc_n<uint32_t>(n + 1);
    k_nbr_count<<<grid_of(n * 32, 256), 256, 0, ws.stream>>>(R, thr, N.off);
    VR_CUDA(cudaGetLastError());
    VR_CUDA(cudaMemsetAsync(N.off + n, 0, sizeof(uint32_t), ws.stream));
    scan_u32_exclusive(N.off, n + 1, ws.stream);
    VR_CUDA(cudaMemcpyAsync(&hs.p[42], N.off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, ws.stream));
    VR_CUDA(cudaStreamSynchronize(ws.stream));
    N.num = (int64_t)(hs.p[42] & 0xFFFFFFFFu);
    N.nbr = ws.alloc_n<uint32_t>(N.num > 0 ? N.num : 1);
    k_nbr_fill<<<grid_of(n * 32, 256), 256, 0, ws.stream>>>(R, thr, N.off, N.nbr);
    VR_CUDA(cudaGetLastError());
    return N;
}

SimplexList edge_list(Workspace& ws, const RankMatrix& R, const Neighbours& N, HostScratch& hs) {
    const int n = (int)R.n;
    uint32_t* pos = ws.alloc_n<uint32_t>(n + 1);
    k_edge_count<<<grid_of(n, 256), 256, 0, ws.stream>>>(N, n, pos);
    VR_CUDA(cudaGetLastError());
    VR_CUDA(cudaMemsetAsync(pos + n, 0, sizeof(uint32_t), ws.stream));
    scan_u32_exclusive(pos, n + 1, ws.stream);
    VR_CUDA(cudaMemcpyAsync(&hs.p[43], pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, ws.stream));
    VR_CUDA(cudaStreamSynchronize(ws.stream));
    SimplexList L;
    L.len = (int64_t)(hs.p[43] & 0xFFFFFFFFu);
    L.cidx = ws.alloc_n<uint64_t>(L.len > 0 ? L.len : 1);
    L.verts = ws.alloc_n<uint16_t>((L.len > 0 ? L.len : 1) * SIMPLEX_VSTRIDE);
    k_edge_fill<<<grid_of((int64_t)n * 32, 256), 256, 0, ws.stream>>>(N, n, pos, L.cidx, L.verts);
    VR_CUDA(cudaGetLastError());
    return L;
}

SimplexList next_list(Workspace& ws, const RankMatrix& R, const Binom& B, const Neighbours& N, uint32_t thr,
                      const SimplexList& L, int p, int out_cidx_bits, HostScratch& hs) {
    SimplexList out;
    out.len = 0;
    uint32_t* cnt = ws.alloc_n<uint32_t>(L.len + 1);
    unsigned long long* total = ws.zeros_n<unsigned long long>(1);
    VR_CUDA(cudaMemsetAsync(cnt + L.len, 0, sizeof(uint32_t), ws.stream));
    if (L.len > 0) {
        k_extend<false><<<grid_of(L.len, 128), 128, 0, ws.stream>>>(R, B, N, thr, p, L.cidx, L.verts, L.len, cnt,
                                                                     nullptr, nullptr, nullptr, total);
        VR_CUDA(cudaGetLastError());
    }
    VR_CUDA(cudaMemcpyAsync(&hs.p[45], total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ws.stream));
    VR_CUDA(cudaStreamSynchronize(ws.stream));
    VR_CHECK((uint64_t)hs.p[45] < (1ull << 32), VR_ERR_OOM);  // the list offsets are 32-bit
    scan_u32_exclusive(cnt, L.len + 1, ws.stream);
    out.len = hs.p[45];
    const int64_t m = out.len > 0 ? out.len : 1;
    out.cidx = ws.alloc_n<uint64_t>(m);
    out.verts = ws.alloc_n<uint16_t>(m * SIMPLEX_VSTRIDE);
    if (out.len > 0) {
        uint64_t* idx = ws.alloc_n<uint64_t>(m);
        uint16_t* tmp = ws.alloc_n<uint16_t>(m * SIMPLEX_VSTRIDE);
        k_extend<true><<<grid_of(L.len, 128), 128, 0, ws.stream>>>(R, B, N, thr, p, L.cidx, L.verts, L.len, cnt,
                                                                    out.cidx, tmp, idx, nullptr);
        VR_CUDA(cudaGetLastError());
        radix_sort_u64(ws, out.cidx, idx, out.len, out_cidx_bits);
        k_gather_verts<<<grid_of(out.len, 256), 256, 0, ws.stream>>>(idx, out.len, tmp, out.verts);
        VR_CUDA(cudaGetLastError());
    }
    return out;
}

void launch_sparse_filtration_apparent(int p, const RankMatrix& R, const Binom& B, const Neighbours& N,
                                       const SimplexList& L, const uint32_t* clear_bits, bool clear_by_pos,
                                       int cidx_bits, int rank_bits, const ApparentOut& o, cudaStream_t s) {
    const uint64_t rmask = rank_bits >= 64 ? ~0ull : ((1ull << rank_bits) - 1);
    switch (p) {
        case 1: launch_sparse_p<1>(R, B, N, L, clear_bits, clear_by_pos, cidx_bits, rmask, o, s); break;
        case 2: launch_sparse_p<2>(R, B, N, L, clear_bits, clear_by_pos, cidx_bits, rmask, o, s); break;
        case 3: launch_sparse_p<3>(R, B, N, L, clear_bits, clear_by_pos, cidx_bits, rmask, o, s); break;
        case 4: launch_sparse_p<4>(R, B, N, L, clear_bits, clear_by_pos, cidx_bits, rmask, o, s); break;
        case 5: launch_sparse_p<5>(R, B, N, L, clear_bits, clear_by_pos, cidx_bits, rmask, o, s); break;
        case 6: launch_sparse_p<6>(R, B, N, L, clear_bits, clear_by_pos, cidx_bits, rmask, o, s); break;
        default: throw Error{VR_ERR_INVALID_ARG};
    }
}

}  // namespace vr
