// apparent.cu -- filtration construction with clearing fused with the
// apparent-pair search, for the p-simplices of one dimension.
//
// Paper (arXiv 2502.05063): Algorithm 17 keeps a p-simplex s iff it is not
// the death simplex of a (p-1)-pair (clearing lemma, Sec. 5.2.3) and
// diam(s) <= threshold; Algorithm 18 launches one thread per candidate
// index and sorts the kept columns; Algorithm 13 then tests each column with
// the Apparent Pairs Lemma (Lemma 5.3.6): t is the first cofacet of s, in
// decreasing combinatorial index, with diam(t) = diam(s), and no facet s' of
// t with diam(s') = diam(s) has a smaller index than s.  By Cor 5.3.7 the
// test is independent per column and by Prop 5.3.9 it may run after
// clearing.
//
// B300 design (differs from the paper's thread-per-column kernel):
//  * no sort of the kept columns: the apparent test does not need the
//    coboundary order, so filtering and the search run in one kernel and
//    only the non-apparent columns (about 0.1-1% of them) are written out, as
//    packed (rank, index) keys for the later radix sort;
//  * enumeration: a warp takes tasks of up to 256 consecutive candidate indices.
//    It decodes the first index once (eq. 5.6, binomial table in shared
//    memory when it fits) and every lane reaches its own simplex by stepping
//    through the combinatorial number system (add to the smallest vertex,
//    carry into the next when it reaches it): no per-lane search;
//  * filtering: each lane computes the diameter rank of its candidate (the
//    C(p+1,2) pairwise ranks), tests the threshold and the clearing bit, and
//    a ballot appends the kept columns to a per-warp queue in shared memory,
//    so that above-threshold and cleared candidates leave no idle lanes in
//    the search;
//  * search, 32 queued columns at a time: first every lane tests the same
//    added vertices w = n-1, n-2, ... for its own column (the lanes read one
//    row w of the symmetric rank matrix, whose columns are their vertices:
//    few cache lines per load), for a bounded number of steps; a column
//    still open then searches warp-cooperatively, 32 vertices w per step
//    (row v_i of the matrix at columns w..w-31, one coalesced load per vertex
//    of s), and a ballot picks the largest qualifying w;
//  * the facet test needs only the ranks among the p+2 vertices of t: a bit
//    mask of the pairs of s that attain diam(s) (kept with the column) and
//    the ranks of the new pairs (w, v_i).
// Apparent pairs have zero persistence (diam(s) = diam(t)); they are only
// counted, marked in the clearing bitmap of dimension p+1, and written out
// when zero-length pairs are requested.
#include <map>
#include <mutex>

#include "vr_common.cuh"

namespace vr {

namespace {

constexpr int AP_WARPS = 8;        // warps per block
constexpr int QCAP = 64;           // queued columns per warp (a chunk adds at most 32 to fewer than 32)
constexpr int TASK_CHUNKS = 8;     // chunks of 32 consecutive candidates per task (at most)
constexpr int LOCKSTEP = 10;       // added vertices every lane tests for its own column first
constexpr int64_t SMEM_BINOM_BYTES = 48 * 1024;  // largest binomial table copied to shared memory

// Binomial table access (same [k][v] layout as Binom), from shared or global memory.
template <bool SB>
struct BinomAt {
    const uint64_t* t;
    int64_t n;
    __device__ __forceinline__ uint64_t operator()(int64_t v, int k) const {
        if (SB) return t[(size_t)k * (size_t)(n + 1) + (size_t)v];
        return __ldg(t + (size_t)k * (size_t)(n + 1) + (size_t)v);
    }
};

template <int P>
struct ColQueue {
    uint64_t c[QCAP];         // combinatorial index of s
    uint32_t r[QCAP];         // diameter rank of s
    uint32_t eq[QCAP];        // bit k: pair k of s (pair order below) has rank r
    uint16_t v[P + 1][QCAP];  // vertices of s, ascending (n <= 65536)
};

// Bit mask of the pairs (i, j), i > j, of an nv-vertex set (enumerated i = 1..,
// j = 0..i-1) that do not contain vertex position a.
__host__ __device__ constexpr uint32_t pairs_without(int a, int nv) {
    uint32_t m = 0;
    int k = 0;
    for (int i = 1; i < nv; ++i)
        for (int j = 0; j < i; ++j) {
            if (i != a && j != a) m |= 1u << k;
            ++k;
        }
    return m;
}

// The simplex `add` places later in the combinatorial number system (eq. 5.6):
// the smallest vertex grows; when it reaches the next vertex it wraps to 0
// and the prefix (v_1..v_p) moves to its successor (v_1 + 1, or a carry
// into higher vertices, each reset to its smallest value).  The row of a
// prefix holds v_1 simplices, so `add` <= 32 costs one pass of the loop for
// v_1 >= 32.
template <int P>
__device__ __forceinline__ void step_simplex(int* v, int add) {
    int r = v[0] + add;
    while (r >= v[1]) {
        r -= v[1];
        ++v[1];
#pragma unroll
        for (int i = 1; i < P; ++i) {
            if (v[i] < v[i + 1]) break;
            v[i] = i;
            ++v[i + 1];
        }
    }
    v[0] = r;
}

struct Counters {  // per lane; only `scan` can pass 2^32 (n cofacets per column)
    uint32_t above = 0, cleared = 0, kept = 0, app = 0, facet = 0;
    unsigned long long scan = 0;
};

// Apparent-pair test of the first m (<= 32) queued columns, one per lane,
// and their outputs.  Warp-uniform m.
template <int P, bool SB>
__device__ __forceinline__ void search_batch(const RankMatrix& R, const BinomAt<SB>& B, ColQueue<P>& q, int m,
                                             int cidx_bits, uint64_t rmask, const ApparentOut& o, Counters& k) {
    constexpr int NV = P + 1;
    const int lane = threadIdx.x & 31;
    const int64_t n = R.n;
    const bool mine = lane < m;
    int v[NV];
    uint32_t r = 0, eq = 0;
    uint64_t c = 0;
    if (mine) {
        c = q.c[lane];
        r = q.r[lane];
        eq = q.eq[lane];
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = q.v[a][lane];
    } else {
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = 0;
    }
    __syncwarp();  // every entry is in registers before the queue is rewritten

    // 1. lock-step: all lanes test the same w for their own columns
    // (vertex indices are below 2^16, so row offsets fit 32 bits)
    bool open = mine;
    int wf = -1;
    uint32_t rw[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) rw[a] = 0;
    const int nn = (int)n;
    for (int step = 0; step < LOCKSTEP; ++step) {
        const int w = nn - 1 - step;
        if (w < 0 || !__any_sync(0xffffffffu, open)) break;
        const uint32_t* row = R.r + (uint32_t)w * (uint32_t)R.ld;  // row w, one per warp
        uint32_t rr[NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) rr[a] = __ldg(row + v[a]);  // the diagonal when w is a vertex of s
        bool ok = open;
#pragma unroll
        for (int a = 0; a < NV; ++a) ok &= (w != v[a]) & (rr[a] <= r);
        if (ok) {
            wf = w;
            open = false;
#pragma unroll
            for (int a = 0; a < NV; ++a) rw[a] = rr[a];
        }
    }
    // 2. columns still open: warp-cooperative, 32 vertices w per step
    const int base0 = nn - 1 - LOCKSTEP;
    uint32_t rem = __ballot_sync(0xffffffffu, open && base0 >= 0);
    while (rem) {
        const int src = __ffs(rem) - 1;
        rem &= rem - 1;
        int sv[NV];
        const uint32_t* rows[NV];  // rows v_a of the matrix
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            sv[a] = __shfl_sync(0xffffffffu, v[a], src);
            rows[a] = R.r + (uint32_t)sv[a] * (uint32_t)R.ld;
        }
        const uint32_t sr = __shfl_sync(0xffffffffu, r, src);
        int hit = -1;
        for (int base = base0; base >= 0; base -= 32) {
            const int w = base - lane;
            bool ok = w >= 0;
            if (ok) {
#pragma unroll
                for (int a = 0; a < NV; ++a) ok &= (w != sv[a]) & (__ldg(rows[a] + w) <= sr);
            }
            const uint32_t bl = __ballot_sync(0xffffffffu, ok);
            if (bl) {
                hit = base - (__ffs(bl) - 1);
                break;
            }
        }
        if (lane == src && hit >= 0) {
            wf = hit;
#pragma unroll
            for (int a = 0; a < NV; ++a) rw[a] = R(v[a], wf);
        }
    }
    if (mine) k.scan += wf >= 0 ? (unsigned long long)(n - wf) : (unsigned long long)n;

    // 3. facet test: a facet t - {v_a} with v_a > wf has a smaller index than s
    //    and must not keep the diameter; its pairs are the pairs of s without
    //    v_a and the pairs (wf, v_b), b != a
    bool apparent = false;
    if (mine && wf >= 0) {
        ++k.facet;
        uint32_t rweq = 0;
#pragma unroll
        for (int a = 0; a < NV; ++a) rweq |= (rw[a] == r ? 1u : 0u) << a;
        apparent = true;
#pragma unroll
        for (int a = 0; a < NV; ++a)
            if (v[a] > wf && ((eq & pairs_without(a, NV)) != 0 || (rweq & ~(1u << a)) != 0)) apparent = false;
    }

    // 4. outputs
    if (apparent) {
        ++k.app;
        if (o.clear_next || o.zero_pairs) {
            uint64_t ct = 0;  // index of t: wf inserted into the ascending vertices of s
            int kk = 0;
            bool placed = false;
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                if (!placed && wf < v[a]) {
                    ct += B(wf, kk + 1);
                    ++kk;
                    placed = true;
                }
                ct += B(v[a], kk + 1);
                ++kk;
            }
            if (!placed) ct += B(wf, kk + 1);
            if (o.clear_next) atomicOr(o.clear_next + (ct >> 5), 1u << (ct & 31));
            if (o.zero_pairs) {
                const unsigned long long at = atomicAdd(o.num_zero_pairs, 1ull);
                PairRec prc;
                prc.birth_rank = r;
                prc.death_rank = r;
                prc.birth_cidx = c;
                prc.death_cidx = (int64_t)ct;
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
            if ((int64_t)at < o.capacity)
                o.nonapparent_keys[at] = ((~(uint64_t)r & rmask) << cidx_bits) | c;
            else
                atomicExch(o.dev_err, DEV_CAPACITY);
        }
    }
}

template <int P, bool SB>
__global__ void __launch_bounds__(AP_WARPS * 32, P <= 2 ? 4 : 2)
k_filtration_apparent(RankMatrix R, Binom Bg, uint32_t thr, const uint32_t* __restrict__ clear_bits,
                      int cidx_bits, uint64_t rmask, uint64_t num_cand, int task_chunks, ApparentOut o) {
    constexpr int NV = P + 1;
    constexpr int NPS = NV * (NV - 1) / 2;  // vertex pairs of s
    extern __shared__ __align__(16) unsigned char ap_smem[];
    ColQueue<P>& q = reinterpret_cast<ColQueue<P>*>(ap_smem)[threadIdx.x >> 5];
    const int64_t n = R.n;
    BinomAt<SB> B{Bg.t, n};
    if (SB) {  // rows k = 0..p+2 of the table: decoding (k <= p+1) and cofacet indices (k <= p+2)
        uint64_t* tab = reinterpret_cast<uint64_t*>(ap_smem + AP_WARPS * sizeof(ColQueue<P>));
        const int64_t cnt = (int64_t)(P + 3) * (n + 1);
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) tab[i] = __ldg(Bg.t + i);
        B.t = tab;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t TASK = 32ull * (uint64_t)task_chunks;
    const uint64_t ntasks = (num_cand + TASK - 1) / TASK;
    Counters k;
    int qn = 0;  // queued columns (warp-uniform)

    for (uint64_t task = warp; task < ntasks; task += nwarps) {
        const uint64_t c0 = task * TASK;
        int v[NV];
        warp_decode_simplex<P>(B, c0, n - 1, v);
        step_simplex<P>(v, lane);
        for (int ch = 0; ch < task_chunks; ++ch) {
            const uint64_t c = c0 + 32ull * ch + lane;
            if (c0 + 32ull * ch >= num_cand) break;  // warp-uniform
            uint32_t r = 0, eq = 0;
            bool kept = false;
            if (c < num_cand) {
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
                if (r > thr) ++k.above;
                else if (clear_bits && ((__ldg(clear_bits + (c >> 5)) >> (c & 31)) & 1u)) ++k.cleared;
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
                search_batch<P, SB>(R, B, q, 32, cidx_bits, rmask, o, k);
                const int rest = qn - 32;  // move entries 32.. to the front
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
            // next chunk: one past lane 31's simplex, plus the lane
            int nx[NV];
#pragma unroll
            for (int a = 0; a < NV; ++a) nx[a] = __shfl_sync(0xffffffffu, v[a], 31);
            step_simplex<P>(nx, lane + 1);
#pragma unroll
            for (int a = 0; a < NV; ++a) v[a] = nx[a];
        }
    }
    if (qn > 0) search_batch<P, SB>(R, B, q, qn, cidx_bits, rmask, o, k);

    // counters (sums over the warp in 64 bits)
    unsigned long long t[6] = {k.above, k.cleared, k.kept, k.app, k.scan, k.facet};
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t[i] += __shfl_xor_sync(0xffffffffu, t[i], off);
    if (lane == 0) {
        if (t[0]) atomicAdd(o.counters + 0, t[0]);
        if (t[1]) atomicAdd(o.counters + 1, t[1]);
        if (t[2]) atomicAdd(o.counters + 2, t[2]);
        if (t[3]) atomicAdd(o.counters + 3, t[3]);
        if (t[4]) atomicAdd(o.counters + 6, t[4]);
        if (t[5]) atomicAdd(o.counters + 7, t[5]);
    }
}

template <int P, bool SB>
void launch_ps(const RankMatrix& R, const Binom& B, uint32_t thr, const uint32_t* clear_bits, int cidx_bits,
               uint64_t rmask, uint64_t num_cand, const ApparentOut& o, cudaStream_t s) {
    const size_t smem = AP_WARPS * sizeof(ColQueue<P>) + (SB ? (size_t)(P + 3) * (size_t)(R.n + 1) * 8 : 0);
    auto kern = k_filtration_apparent<P, SB>;
    // launch shape per device and shared-memory size, queried once (the queries
    // would otherwise sit between the stage's timing events)
    struct Shape { size_t smem; int sms, per_sm; };
    static std::mutex mu;
    static std::map<int, Shape> shapes;
    int dev = 0;
    VR_CUDA(cudaGetDevice(&dev));
    Shape sh{0, 0, 0};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = shapes.find(dev);
        if (it != shapes.end() && it->second.smem >= smem) sh = it->second;
    }
    if (sh.sms == 0) {
        VR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sh.smem = smem;
        VR_CUDA(cudaDeviceGetAttribute(&sh.sms, cudaDevAttrMultiProcessorCount, dev));
        VR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.per_sm, kern, AP_WARPS * 32, smem));
        std::lock_guard<std::mutex> lock(mu);
        shapes[dev] = sh;
    }
    const int sms = sh.sms, per_sm = sh.per_sm < 1 ? 1 : sh.per_sm;
    // tasks of up to TASK_CHUNKS chunks; shorter ones when the launch is too small
    // to give every resident warp a few full tasks
    const uint64_t cap = (uint64_t)sms * (uint64_t)per_sm;  // one wave of resident blocks
    const uint64_t chunks = (num_cand + 31) / 32;
    uint64_t tc = chunks / (cap * AP_WARPS * 4);
    const int task_chunks = (int)(tc < 1 ? 1 : (tc > TASK_CHUNKS ? TASK_CHUNKS : tc));
    const uint64_t tasks = (chunks + task_chunks - 1) / task_chunks;
    uint64_t blocks = (tasks + AP_WARPS - 1) / AP_WARPS;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, AP_WARPS * 32, smem, s>>>(R, B, thr, clear_bits, cidx_bits, rmask, num_cand,
                                                        task_chunks, o);
    VR_CUDA(cudaGetLastError());
}

template <int P>
void launch_p(const RankMatrix& R, const Binom& B, uint32_t thr, const uint32_t* clear_bits, int cidx_bits,
              uint64_t rmask, uint64_t num_cand, const ApparentOut& o, cudaStream_t s) {
    // the table needs rows 0..p+2, and the launch needs K >= p+2
    VR_CHECK(B.K >= P + 2, VR_ERR_INTERNAL);
    if ((int64_t)(P + 3) * (R.n + 1) * 8 <= SMEM_BINOM_BYTES)
        launch_ps<P, true>(R, B, thr, clear_bits, cidx_bits, rmask, num_cand, o, s);
    else
        launch_ps<P, false>(R, B, thr, clear_bits, cidx_bits, rmask, num_cand, o, s);
}

}  // namespace

void launch_filtration_apparent(int p, const RankMatrix& R, const Binom& B, uint32_t thr_rank,
                                const uint32_t* clear_bits, int cidx_bits, int rank_bits, uint64_t num_cand,
                                const ApparentOut& o, cudaStream_t s) {
    const uint64_t rmask = rank_bits >= 64 ? ~0ull : ((1ull << rank_bits) - 1);
    switch (p) {
        case 1: launch_p<1>(R, B, thr_rank, clear_bits, cidx_bits, rmask, num_cand, o, s); break;
        case 2: launch_p<2>(R, B, thr_rank, clear_bits, cidx_bits, rmask, num_cand, o, s); break;
        case 3: launch_p<3>(R, B, thr_rank, clear_bits, cidx_bits, rmask, num_cand, o, s); break;
        case 4: launch_p<4>(R, B, thr_rank, clear_bits, cidx_bits, rmask, num_cand, o, s); break;
        case 5: launch_p<5>(R, B, thr_rank, clear_bits, cidx_bits, rmask, num_cand, o, s); break;
        case 6: launch_p<6>(R, B, thr_rank, clear_bits, cidx_bits, rmask, num_cand, o, s); break;
        default: throw Error{VR_ERR_INVALID_ARG};
    }
}

}  // namespace vr
