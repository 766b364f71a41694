// batched.cu -- barcodes of many small clouds in one persistent launch.
//
// The paper computes one point cloud at a time (Ch. 5).  For workloads of
// thousands of small clouds (n <= 256, H0-H1) a launch per cloud would be
// dominated by launch and synchronisation costs, so this kernel keeps every
// SM busy with whole clouds taken from a work queue ordered by decreasing
// size.  One 512-thread block owns a cloud from its points to its sorted
// pairs:
//   1. distances by the single-precision formula, kept as the bit patterns of
//      the non-negative floats (ordered like the values, so the integer
//      comparisons of the rank-based kernels apply unchanged);
//   2. enclosing radius (Sec. 5.2.12) unless a threshold is given;
//   3. warp 0: minimum spanning tree (Prim, strict order of Sec. 5.1.4) and
//      elder-rule pairing (Sec. 5.2.5) -> H0 and the clearing set;
//      warps 1-15 meanwhile: apparent-pair search over every edge within the
//      threshold (Lemma 5.3.6; clearing may come after it, Prop 5.3.9);
//   4. drop cleared edges, sort the non-apparent ones into coboundary order;
//   5. reduction (Algorithm 12): all columns once in parallel without
//      additions, finalized in order by the prefix-minimum rule of reduce.cu,
//      the rest in order by the bitmap engine (a bit per triangle, pivots
//      through diameter buckets; see its section below);
//   6. pairs sorted per cloud and appended to the output.
// A cloud that outgrows a per-block buffer is flagged and recomputed by the
// host through the single-cloud path.
#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "reduce_device.cuh"

namespace vr {
namespace {

constexpr int BMAXN = VR_BATCH_MAX_N;  // 256
constexpr int BMAXDIM = 16;
constexpr int BLD = BMAXN;             // row stride of a cloud's square matrix
constexpr int CCAP = 8192;             // non-apparent columns per cloud
constexpr int HCAP = 16384;            // hash slots per cloud (power of two, >= 2 CCAP)
constexpr int64_t BACKCAP = 1 << 20;   // per-cloud global scratch of the bitmap engine, in 8-byte units (8 MB)
constexpr int EDGE_BITS = 15;          // C(256,2) - 1 < 2^15
constexpr int TRI_BITS = 22;           // C(256,3) - 1 < 2^22
constexpr int64_t POOLCAP = 1 << 15;   // stored reduced columns per cloud

struct BatchArgs {
    const float* pts;
    const int64_t* offs;   // num + 1
    const int32_t* order;  // clouds by decreasing size
    int num;
    int dim;
    int dmax;
    uint32_t thr_bits;     // used when !thr_inf
    int thr_inf;
    int want_edges;
    int64_t pool_cap;      // stored generators per cloud (POOLCAP; smaller under VR_BATCH_POOL_CAP, for tests)
    // per-slot scratch
    uint32_t* mat;
    uint64_t* hkeys;
    uint32_t* hvals;
    uint64_t* cols;
    uint64_t* cur_key;
    uint8_t* status;
    uint32_t* ulist;
    PairRec* h1tmp;
    uint64_t* back;
    uint64_t* wstage;      // slots x HW x STAGE
    uint64_t* pool;        // slots x POOLCAP
    unsigned long long* pool_used;  // per slot
    uint64_t* rc_off;      // slots x CCAP
    uint32_t* rc_len;      // slots x CCAP
    uint32_t* adds;        // slots x CCAP
    const uint64_t* binom;  // C(v,k), v <= 256, k <= 3
    // outputs (per dimension p = 0, 1)
    PairRec* recs[2];
    int32_t* edges[2];
    unsigned long long* used;  // [2]
    int64_t cap[2];
    int64_t* start[2];     // per cloud
    int32_t* count[2];
    float* thr_used;
    int32_t* cloud_err;
    unsigned long long* work;
    unsigned long long* stats;  // [0] candidates [1] apparent [2] columns [3] additions
    unsigned long long* prof;   // VR_LOG only: cycles per phase, summed over clouds (thread 0 of each block)
};

struct BatchSmem {
    HeavySmem S;  // first: the bitmap engine addresses its arena from the start of shared memory
    float pts[BMAXN * BMAXDIM];
    uint32_t clear[(BMAXN * (BMAXN - 1) / 2 + 31) / 32];
    uint64_t tree[BMAXN];
    int32_t parent[BMAXN];
    PairRec h0[BMAXN];
    int h0n;
    int ncols;
    int nh1;
    int nu;
    int overflow;
    uint32_t thr;
    uint64_t carry_min;
    int carry_cnt;
    uint64_t wmin[HW];
    int wcnt[HW];
};
static_assert(offsetof(BatchSmem, S) == 0, "the engine arena starts the shared memory");


__device__ __forceinline__ void edge_of(int e, int& a, int& b) {
    int x = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
    while (x * (x - 1) / 2 > e) --x;
    while ((x + 1) * x / 2 <= e) ++x;
    a = x;
    b = e - x * (x - 1) / 2;
}

__device__ __forceinline__ bool rec_less(const PairRec& x, const PairRec& y) {
    if (x.birth_rank != y.birth_rank) return x.birth_rank < y.birth_rank;
    if (x.death_rank != y.death_rank) return x.death_rank < y.death_rank;
    return x.birth_cidx < y.birth_cidx;
}

// block bitonic sort of records (len a power of two, padded by the caller),
// one compare pair per thread and step as in block_bitonic
__device__ void block_sort_recs(PairRec* a, int len) {
    const int half = len >> 1;
    for (int k = 2; k <= len; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < half; p += HT) {
                const int i = 2 * p - (p & (j - 1));
                const PairRec x = a[i], y = a[i + j];
                const bool up = (i & k) == 0;
                if (rec_less(y, x) == up) { a[i] = y; a[i + j] = x; }
            }
            __syncthreads();
        }
}

// edge (u > v) of the q-simplex attaining its diameter, ties -> largest C(u,2)+v
__device__ void crit_edge(const RankMatrix& R, const Binom& B, uint64_t cidx, int q, int& cu, int& cv) {
    int v[3];
    if (q == 1) decode_simplex<1>(B, cidx, R.n - 1, v);
    else decode_simplex<2>(B, cidx, R.n - 1, v);
    uint32_t best = 0;
    cu = -1; cv = -1;
    for (int i = 1; i <= q; ++i)
        for (int j = 0; j < i; ++j) {
            const uint32_t r = R(v[i], v[j]);
            const int e = v[i] * (v[i] - 1) / 2 + v[j];
            const int be = cu < 0 ? -1 : cu * (cu - 1) / 2 + cv;
            if (cu < 0 || r > best || (r == best && e > be)) { best = r; cu = v[i]; cv = v[j]; }
        }
}

// Append `cnt` sorted records of dimension p for cloud `cloud` to the output.
__device__ void emit_block(const BatchArgs& A, BatchSmem& M, int p, int cloud, const PairRec* src, int cnt,
                           const RankMatrix& R, const Binom& B) {
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) {
        base = atomicAdd(A.used + p, (unsigned long long)cnt);
        A.start[p][cloud] = (int64_t)base;
        A.count[p][cloud] = cnt;
        if ((int64_t)(base + cnt) > A.cap[p]) M.overflow = 1;  // the host grows the buffer and reruns
    }
    __syncthreads();
    if ((int64_t)(base + cnt) > A.cap[p]) return;
    for (int i = threadIdx.x; i < cnt; i += HT) {
        const PairRec r = src[i];
        A.recs[p][base + i] = r;
        if (A.want_edges) {
            int bu = -1, bv = -1, du = -1, dv = -1;
            if (p > 0) crit_edge(R, B, r.birth_cidx, p, bu, bv);
            if (r.death_cidx >= 0) crit_edge(R, B, (uint64_t)r.death_cidx, p + 1, du, dv);
            int32_t* e = A.edges[p] + 4 * (base + i);
            e[0] = bu; e[1] = bv; e[2] = du; e[3] = dv;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// 5c. The bitmap engine (dimension 1, n <= 256).  A cloud's working column
// W is one bit per triangle, at the triangle's index (eq. 5.6, below 2^22),
// so W <- W + D_s flips the bits of the cofacets of s and nothing is sorted
// or merged.  The pivot of W is its smallest row in coboundary order: the
// smallest diameter, then the largest index.  Rows are bucketed by the
// dense rank of their diameter among the distinct distances within the
// threshold; a triangle of diameter rank r holds an edge of rank r, so the
// rows of bucket r are found among the triangles {a, b, w} over the edges
// (a, b) of rank r (one edge unless distances tie) and the third vertices
// w.  One bit per bucket marks those that may hold a row: a bucket's bit is
// set whenever one of its rows flips, and cleared when its search finds
// nothing or when the rows of the last pivot's bucket, counted, run out.
// No bucket below the last pivot's holds a row, so each search starts
// there; the warps covering the vertices find the lowest set bit themselves
// and search the bucket, with one barrier per search.
// Owners follow the block engine's rule: the pivot of a finished column
// (hash), else the apparent owner of Def 5.3.4 recomputed; a finished
// column is added as its reduced form, the sum of the coboundaries of the
// generators it records (its column of V).
// The column loop runs on the warps covering the cloud's vertices plus one
// that probes the hash, on a named barrier (bit_sync); the block's other
// warps wait for the whole reduction at a block barrier.
// Three variants by the cloud's size (bit_variant): the bitmap, the bucket
// starts and the ranks in shared memory (n <= 128); the ranks only (n <=
// 172); neither.  The head, the bucket bits and the edges by distance are
// always in shared memory, the rest in the slot's global scratch.
// Shared data are addressed from the dynamic shared array itself, so the
// accesses compile to shared-space instructions.
// ---------------------------------------------------------------------------
extern __shared__ __align__(16) unsigned char g_bsm[];

constexpr int BIT_VCAP = 1 << 16;  // generators of the column being reduced
// per-slot global scratch carved from `back` (in 8-byte units)
constexpr int64_t BIT_KEYS = 0;                                                // sort keys, 32768
constexpr int64_t BIT_RK = BIT_KEYS + 32768;                                   // u16 dense ranks
constexpr int64_t BIT_G = BIT_RK + 8192;                                       // u16 bucket starts
constexpr int64_t BIT_ES = BIT_G + 8200;                                       // u16 edges by distance
constexpr int64_t BIT_BITS = BIT_ES + 8192;                                    // u32 bitmap, C(256,3) bits
constexpr int64_t BIT_V = BIT_BITS + ((int64_t)BMAXN * (BMAXN - 1) * (BMAXN - 2) / 6 + 63) / 64;
constexpr int64_t BIT_KEYS2 = BIT_V + BIT_VCAP;  // partitioned sort keys, 32768, then room to sort a crowded range
static_assert(BIT_KEYS2 + 65536 <= BACKCAP, "the bitmap engine's scratch fits the back buffer");
constexpr int BIT_CHUNK = 8192;  // keys sorted at once in shared memory
constexpr int BAT_DSM_N = 197;   // largest n whose distances (upper triangle) fit the arena in steps 1-3
constexpr int BAT_LOCK = 8;      // lock-step candidate vertices of the apparent search
static_assert(BMAXN * (BMAXN - 1) / 2 < 0xFFFF, "dense ranks fit 16 bits below the above-threshold mark");

struct BitHead {
    uint32_t best[3];         // pivot search results (packed, see bit_pivot), the largest wins; used in rotation
    int cnt[3];               // rows found by the same searches (a tie may count a row twice)
    int rr[3];                // the buckets they searched (-1: W is zero)
    uint32_t lo, hi;          // setup: the smallest and largest distance bits within the threshold
    int dcnt;                 // rows of the last pivot's bucket the last addition set (+1) or cleared (-1)
    int opos;                 // position of the finished column owning the pivot, or -1
    int fail;                 // a buffer was too small: the cloud goes to the single-cloud path
    unsigned long long poff;  // where the finished column's generators go in the pool
    int ws[HW + 1];
};

struct BitEng {
    uint32_t o_h0, o_G, o_Es, o_bits, o_rk;  // byte offsets in the dynamic shared memory
    const uint16_t* gG;   // [nR + 1]: bucket r holds the edges Es[G[r] .. G[r+1])
    const uint16_t* gEs;  // edges within the threshold by distance, as (a << 8) | b, a > b
    uint32_t* gbits;      // the working column, [nbw] words
    const uint16_t* grk;  // dense rank per edge index, 0xFFFF above the threshold
    uint64_t* vbuf;       // generators of the current column (edge indices)
    int n, nbw, nR;
    int nt;               // threads of the column loop: the warps covering the n vertices, then one for the hash
    bool ident;           // every bucket holds one edge (no two distances tie): bucket r is Es[r]
};

// The column loop runs on the first E.nt threads (the warps covering the
// cloud's vertices and one more, which probes the hash), synchronized by
// named barrier 1; the block's other warps wait for the whole reduction at
// a block barrier instead of taking part in every step.
__device__ __forceinline__ void bit_sync(const BitEng& E) {
    asm volatile("bar.sync 1, %0;" ::"r"(E.nt) : "memory");
}
__device__ __forceinline__ int bit_sync_or(const BitEng& E, int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred), "r"(E.nt)
        : "memory");
    return r;
}

__device__ __forceinline__ BitHead& bit_hd() { return *reinterpret_cast<BitHead*>(g_bsm); }
__device__ __forceinline__ uint32_t* bit_h0(const BitEng& E) { return reinterpret_cast<uint32_t*>(g_bsm + E.o_h0); }
// SB: the bitmap and the bucket starts in shared memory (n <= 128); SR: the
// ranks too (n <= 172).  The edges by distance always are.
template <bool SB>
__device__ __forceinline__ const uint16_t* bit_G(const BitEng& E) {
    if constexpr (SB) return reinterpret_cast<const uint16_t*>(g_bsm + E.o_G); else return E.gG;
}
__device__ __forceinline__ const uint16_t* bit_Es(const BitEng& E) {
    return reinterpret_cast<const uint16_t*>(g_bsm + E.o_Es);
}
template <bool SR>
__device__ __forceinline__ const uint16_t* bit_rk(const BitEng& E) {
    if constexpr (SR) return reinterpret_cast<const uint16_t*>(g_bsm + E.o_rk); else return E.grk;
}
template <bool SB>
__device__ __forceinline__ uint32_t* bit_bits(const BitEng& E) {
    if constexpr (SB) return reinterpret_cast<uint32_t*>(g_bsm + E.o_bits); else return E.gbits;
}
// a word of W after a barrier: shared memory as is, global past the L1 (flipped by atomics)
template <bool SB>
__device__ __forceinline__ uint32_t bit_word(const BitEng& E, uint32_t i) {
    if constexpr (SB) return bit_bits<true>(E)[i]; else return __ldcg(E.gbits + i);
}

__device__ __forceinline__ uint32_t bit_eidx(uint32_t u, uint32_t v) {  // u != v
    const uint32_t x = u > v ? u : v, y = u > v ? v : u;
    return x * (x - 1) / 2 + y;
}

// index of the triangle {u, v, w} (distinct vertices), eq. 5.6
__device__ __forceinline__ uint32_t bit_tidx(uint32_t u, uint32_t v, uint32_t w) {
    const uint32_t x0 = min(u, min(v, w)), x2 = max(u, max(v, w)), x1 = u + v + w - x0 - x2;
    return x2 * (x2 - 1) * (x2 - 2) / 6 + x1 * (x1 - 1) / 2 + x0;
}

// Clear bucket r's bit; every thread may do it at once (the same value is written).
__device__ __forceinline__ void bit_clear_bucket(const BitEng& E, int r) {
    uint32_t* h0 = bit_h0(E);
    h0[r >> 5] = h0[r >> 5] & ~(1u << (r & 31));
}

// Flip row `t` (bucket d) of W if `on`; every lane of the warp calls this.
// Rows of the last pivot's bucket rp (many rows of the added coboundary
// lie at its diameter) leave its bit alone (set, and cleared only by the
// count) and count whether they were set or cleared, summed per warp.
// (Combining the other buckets' bits per warp first, lanes grouped by
// target word, measured slower: 765 -> 3.8 K cycles per addition.  So did
// flipping without counting, leaving an emptied bucket to its next search:
// 2.89 -> 3.30 ms on 256 circles, 62.0 -> 65.9 ms on 4096 clouds.)
template <bool SB, bool SR>
__device__ __forceinline__ void bit_flip(const BitEng& E, bool on, uint32_t t, uint32_t d, int rp) {
    int delta = 0;
    if (on) {
        const uint32_t m = 1u << (t & 31);
        uint32_t* w = bit_bits<SB>(E) + (t >> 5);
        if ((int)d == rp) {
            delta = (atomicXor(w, m) & m) ? -1 : 1;
        } else {
            atomicXor(w, m);
            atomicOr(bit_h0(E) + (d >> 5), 1u << (d & 31));
        }
    }
    if (rp >= 0) {
        const int sum = __reduce_add_sync(0xffffffffu, delta);
        if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&bit_hd().dcnt, sum);
    }
}

// The row of D_s for the edge s = (u, v) of rank rs and this thread's
// vertex w (none if w < 0): flipped if its diameter is within the threshold.
template <bool SB, bool SR>
__device__ __forceinline__ void bit_cob(const BitEng& E, int u, int v, uint32_t rs, int w, int rp) {
    bool on = false;
    uint32_t t = 0, d = 0;
    if (w >= 0 && w != u && w != v) {
        const uint16_t* rk = bit_rk<SR>(E);
        const uint32_t mx = max(rs, max((uint32_t)rk[bit_eidx(u, w)], (uint32_t)rk[bit_eidx(v, w)]));
        on = mx != 0xFFFFu;
        d = mx;
        t = bit_tidx(u, v, w);
    }
    bit_flip<SB, SR>(E, on, t, d, rp);
}

// W <- W + sum of D_g over the generators g (edge indices) in list[0..len),
// one generator per pass of the loop's threads (more than n of them).
template <bool SB, bool SR>
__device__ void bit_add_list(const BitEng& E, const uint64_t* list, int len, int rp) {
    const int w = (int)threadIdx.x < E.n ? (int)threadIdx.x : -1;
    for (int gi = 0; gi < len; ++gi) {
        const int e = (int)list[gi];
        int u, v;
        edge_of(e, u, v);
        bit_cob<SB, SR>(E, u, v, bit_rk<SR>(E)[e], w, rp);
    }
}

// The pivot of W: false if W is zero, else the triangle {a, b, w} (a > b an
// edge of bucket r) with the largest index among the rows of the lowest
// non-empty bucket r, and whether the edges (a, w) and (b, w) also have rank
// r (eq_aw, eq_bw): a search result packs (index << 10) | (w << 2) |
// (eq_aw << 1) | eq_bw.  rp, cp: the previous pivot's bucket (-1: none) and
// the rows its search found; with the rows the last addition set or
// cleared there (H.dcnt) they tell whether it emptied, in which case its
// bit is cleared first.  Each warp covering the third vertices finds the
// lowest set bucket bit itself (a warp minimum over the words, no barrier)
// and searches its share; the bucket and the result reach every thread
// through the result slots after one barrier.  A bucket whose search finds
// nothing is cleared and the next one searched.  `it` is the result slot
// of the column's next search, counting searches mod 3: the slot of search i
// + 2 (i - 1's) is zeroed after search i's barrier, when it has been read.
template <bool SB, bool SR>
__device__ bool bit_pivot(const BitEng& E, int rp, int cp, int& it, int& r_out, uint32_t& a_out, uint32_t& b_out,
                          uint32_t& w_out, uint32_t& t_out, int& c_out, bool& eq_aw, bool& eq_bw) {
    BitHead& H = bit_hd();
    const uint16_t* G = bit_G<SB>(E);
    const uint16_t* Es = bit_Es(E);
    const uint16_t* rk = bit_rk<SR>(E);
    const uint32_t* h0 = bit_h0(E);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (E.nR + 31) >> 5;
    // the warps covering the n third vertices search; the others wait at the
    // barrier and take the bucket from the result slot
    const int sw = (E.n + 31) >> 5;
    const bool searcher = wid < sw;
    if (searcher && rp >= 0 && cp + H.dcnt <= 0) bit_clear_bucket(E, rp);
    // no bucket below the last pivot's holds a row (the pivot was the
    // column's smallest row, and an addition's sum has no row below it, though
    // the coboundaries of a finished column's generators may leave cancelled
    // rows' bits there), so the search starts at that floor: its word, masked
    // below it, is usually the answer, read by every lane at once
    int fb = rp >= 0 ? rp : 0;
    for (;;) {
        const int sl = it;  // the slot of this search (it runs 0, 1, 2, 0, ...)
        int rs = -1;        // the searchers' bucket and its first edge, kept in registers
        uint32_t abs0 = 0;
        if (searcher) {
            const int fw = fb >> 5;
            uint32_t lw = 0xFFFFFFFFu, x0 = 0;
            if (fw < nw) x0 = h0[fw] & (0xFFFFFFFFu << (fb & 31));
            if (x0) {
                lw = (uint32_t)fw;
            } else {
                // the lowest non-empty word above: eight words per lane loaded at
                // once, lane i taking words i, i + 32, ... of a batch; a batch with
                // a set bit ends it
                for (int base = fw + 1; base < nw; base += 256) {
                    uint32_t v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = base + u * 32 + lane;
                        v[u] = i < nw ? h0[i] : 0u;
                    }
#pragma unroll
                    for (int u = 7; u >= 0; --u)
                        if (v[u]) lw = (uint32_t)(base + u * 32 + lane);
                    if (__any_sync(0xffffffffu, lw != 0xFFFFFFFFu)) break;
                }
                lw = __reduce_min_sync(0xffffffffu, lw);
            }
            const int r = lw == 0xFFFFFFFFu ? -1 : (int)(lw * 32 + __ffs((int)lw == fw ? x0 : h0[lw]) - 1);
            if (threadIdx.x == 0) H.rr[sl] = r;
            rs = r;
            if (r >= 0) {
                const int g0 = E.ident ? r : (int)G[r], k = E.ident ? 1 : (int)G[r + 1] - g0;
                const uint32_t ab0 = Es[g0];  // the bucket's first (usually only) edge
                abs0 = ab0;
                int found = 0;
                for (int idx = threadIdx.x; idx < k * E.n; idx += sw * 32) {
                    const int ei = k == 1 ? 0 : idx / E.n, w = idx - ei * E.n;
                    const uint32_t ab = ei == 0 ? ab0 : Es[g0 + ei], a = ab >> 8, b = ab & 0xFFu;
                    if (w == (int)a || w == (int)b) continue;
                    const uint32_t t = bit_tidx(a, b, w);
                    const uint32_t word = bit_word<SB>(E, t >> 5), ra = rk[bit_eidx(a, w)], rb = rk[bit_eidx(b, w)];
                    if (!((word >> (t & 31)) & 1u) || ra > (uint32_t)r || rb > (uint32_t)r) continue;  // absent, or another bucket's
                    ++found;
                    atomicMax(&H.best[sl], (t << 10) | ((uint32_t)w << 2) | ((ra == (uint32_t)r) << 1) | (rb == (uint32_t)r));
                }
                if (found) atomicAdd(&H.cnt[sl], found);
            }
        }
        bit_sync(E);
        const int r = searcher ? rs : H.rr[sl];
        const uint32_t best = H.best[sl];
        const int cnt = H.cnt[sl];
        const int zs = sl == 0 ? 2 : sl - 1;  // the slot two searches on (the previous search's)
        if (threadIdx.x == 0) { H.best[zs] = 0; H.cnt[zs] = 0; }
        it = sl == 2 ? 0 : sl + 1;
        if (r < 0) return false;
        if (cnt) {
            const int g0 = E.ident ? r : (int)G[r], k = E.ident ? 1 : (int)G[r + 1] - g0;
            const uint32_t t = best >> 10, w = (best >> 2) & 0xFFu;
            const uint32_t ab = searcher ? abs0 : Es[g0];
            uint32_t a = ab >> 8, b = ab & 0xFFu;
            for (int ei = 1; ei < k && !(a != w && b != w && bit_tidx(a, b, w) == t); ++ei) {  // ties only
                a = Es[g0 + ei] >> 8;
                b = Es[g0 + ei] & 0xFFu;
            }
            r_out = r; t_out = t; w_out = w; a_out = a; b_out = b; c_out = cnt;
            eq_aw = (best >> 1) & 1u;
            eq_bw = best & 1u;
            if (threadIdx.x == 0) H.dcnt = 0;  // counted from the caller's next barrier on
            return true;
        }
        if (searcher) bit_clear_bucket(E, r);  // bucket r is empty, and every one below it
        fb = r + 1;
    }
}

// Sort keys[0..m) ((distance bits << 16) | edge, distance bits in [lo, hi])
// in global memory, using the arena from byte hb: BIT_CHUNK keys, then the
// partition's tables.  The keys are partitioned into 256 ranges of distance
// bits (a histogram, a scan and a scatter into tmp), consecutive ranges are
// grouped into chunks of at most BIT_CHUNK keys, and each chunk is sorted by
// a bitonic network in shared memory and written back; the ranges being
// ordered, the chunks follow one another.  A range above BIT_CHUNK keys
// (distances crowded into a narrow band) is sorted in global memory, in
// tmp[32768..).
__device__ void bit_sort_keys(uint64_t* keys, uint64_t* tmp, int m, uint32_t lo, uint32_t hi, uint32_t hb) {
    uint64_t* sk = reinterpret_cast<uint64_t*>(g_bsm + hb);
    int* rstart = reinterpret_cast<int*>(g_bsm + hb + BIT_CHUNK * 8);  // [257]
    int* rcur = rstart + 257;                                          // [256]
    int* cbeg = rcur + 256;                                            // [257], then the chunk count
    const uint64_t span = (uint64_t)hi - lo + 1;
    auto range_of = [&](uint64_t k) { return (int)((((k >> 16) - lo) * 256) / span); };
    for (int i = threadIdx.x; i < 256; i += HT) rcur[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += HT) atomicAdd(&rcur[range_of(keys[i])], 1);
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 counts by one warp, 8 per lane
        int v[8], sum = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) { v[u] = rcur[threadIdx.x * 8 + u]; sum += v[u]; }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)threadIdx.x >= o) incl += y;
        }
        int run = incl - sum;
#pragma unroll
        for (int u = 0; u < 8; ++u) { rstart[threadIdx.x * 8 + u] = run; rcur[threadIdx.x * 8 + u] = run; run += v[u]; }
        if (threadIdx.x == 31) rstart[256] = run;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += HT) {
        const uint64_t k = keys[i];
        tmp[atomicAdd(&rcur[range_of(k)], 1)] = k;
    }
    if (threadIdx.x == 0) {  // chunks: maximal runs of ranges within BIT_CHUNK keys
        int c = 0, b = 0;
        cbeg[0] = 0;
        while (b < 256) {
            int e = b + 1;
            while (e < 256 && rstart[e + 1] - rstart[b] <= BIT_CHUNK) ++e;
            cbeg[++c] = rstart[e];
            b = e;
        }
        cbeg[257] = c;
    }
    __syncthreads();
    const int nch = cbeg[257];
    for (int ch = 0; ch < nch; ++ch) {
        const int c0 = cbeg[ch], len = cbeg[ch + 1] - c0;
        int l2 = 1;
        while (l2 < len) l2 <<= 1;
        uint64_t* buf = len > BIT_CHUNK ? tmp + 32768 : sk;  // a crowded range: global room of 32768
        for (int i = threadIdx.x; i < l2; i += HT) buf[i] = i < len ? tmp[c0 + i] : EMPTY;
        __syncthreads();
        block_bitonic(buf, l2);
        for (int i = threadIdx.x; i < len; i += HT) keys[c0 + i] = buf[i];
        __syncthreads();
    }
}

// Which variant a cloud of n points takes, for the worst case (every edge
// within the threshold, all distances distinct): 0 = SB and SR (head,
// bucket bits, bucket starts, edges by distance and bitmap in the arena, the
// sort keys there first, the ranks in the second arena), 1 = SR only, 2 =
// neither (the edges by distance still in the arena).
__device__ __forceinline__ int bit_variant(int n, size_t arena_bytes, size_t arena2_bytes) {
    const size_t ne = (size_t)n * (n - 1) / 2, ntri = (size_t)n * (n - 1) * (n - 2) / 6;
    const size_t hb = (sizeof(BitHead) + 15) & ~(size_t)15;
    size_t lmax = 1;
    while (lmax < ne) lmax <<= 1;
    const size_t h0b = ((ne + 31) / 32 * 4 + 15) & ~(size_t)15;
    const size_t gb = ((ne + 1) * 2 + 15) & ~(size_t)15, eb = (ne * 2 + 15) & ~(size_t)15;
    const size_t bb = ((ntri + 31) / 32 * 4 + 15) & ~(size_t)15;
    const bool sr = ne * 2 <= arena2_bytes;
    if (sr && hb + lmax * 8 <= arena_bytes && hb + h0b + gb + eb + bb <= arena_bytes) return 0;
    return sr ? 1 : 2;
}

// Per cloud: dense ranks of the edges within the threshold (a sort by
// distance), the buckets, and the engine's storage (see bit_variant).
template <bool SB, bool SR>
__device__ BitEng bit_setup(uint64_t* back, const uint32_t* mat, int n, uint32_t thr, uint32_t arena2_off) {
    BitEng E;
    BitHead& H = bit_hd();
    E.n = n;
    E.vbuf = back + BIT_V;
    uint16_t* Gg = reinterpret_cast<uint16_t*>(back + BIT_G);
    uint16_t* Esg = reinterpret_cast<uint16_t*>(back + BIT_ES);
    const int ne = n * (n - 1) / 2;
    const uint32_t hb = (sizeof(BitHead) + 15) & ~15u;
    uint64_t* keys = SB ? reinterpret_cast<uint64_t*>(g_bsm + hb) : back + BIT_KEYS;
    uint16_t* rk;
    if constexpr (SR) {
        rk = reinterpret_cast<uint16_t*>(g_bsm + arena2_off);
        E.o_rk = arena2_off;
    } else {
        rk = reinterpret_cast<uint16_t*>(back + BIT_RK);
    }
    E.grk = reinterpret_cast<const uint16_t*>(back + BIT_RK);
    // 1. the edges within the threshold, as (distance bits << 16) | edge, in
    // any order (they are sorted next); four distances in flight per thread
    if (threadIdx.x == 0) { H.cnt[0] = 0; H.lo = 0xFFFFFFFFu; H.hi = 0; }  // append counter (search slots are zeroed per column)
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    for (int base = 0; base < ne; base += 4 * HT) {
        uint32_t d[4];
        int e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            e[u] = base + u * HT + (int)threadIdx.x;
            d[u] = 0xFFFFFFFFu;
            if (e[u] < ne) {
                int a, b;
                edge_of(e[u], a, b);
                d[u] = mat[a * BLD + b];
                rk[e[u]] = 0xFFFFu;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool keep = e[u] < ne && d[u] <= thr;
            const uint32_t bl = __ballot_sync(0xffffffffu, keep);
            int at = 0;
            if (lane == 0 && bl) at = atomicAdd(&H.cnt[0], __popc(bl));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (keep) {
                keys[at + __popc(bl & ((1u << lane) - 1u))] = ((uint64_t)d[u] << 16) | (uint64_t)e[u];
                lo = min(lo, d[u]);
                hi = max(hi, d[u]);
            }
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) { atomicMin(&H.lo, lo); atomicMax(&H.hi, hi); }
    __syncthreads();
    const int m = H.cnt[0];
    int len = 1;
    while (len < m) len <<= 1;
    if constexpr (SB) {  // all keys fit the arena
        for (int i = m + (int)threadIdx.x; i < len; i += HT) keys[i] = EMPTY;
        __syncthreads();
        block_bitonic(keys, len);
    } else {
        bit_sort_keys(keys, back + BIT_KEYS2, m, H.lo, H.hi, hb);
    }
    // 2. buckets: runs of equal distance
    int nR = 0;
    for (int base = 0; base < m; base += HT) {
        const int p = base + (int)threadIdx.x;
        bool first = false;
        int e = 0;
        if (p < m) {
            const uint64_t k = keys[p];
            e = (int)(k & 0xFFFFu);
            first = p == 0 || (keys[p - 1] >> 16) != (k >> 16);
        }
        int tot;
        const int pos = block_excl_scan(first, H.ws, &tot);
        if (p < m) {
            const int g = nR + pos + (first ? 0 : -1);
            int a, b;
            edge_of(e, a, b);
            rk[e] = (uint16_t)g;
            Esg[p] = (uint16_t)((a << 8) | b);
            if (first) Gg[g] = (uint16_t)p;
        }
        nR += tot;
    }
    if (threadIdx.x == 0) Gg[nR] = (uint16_t)m;
    E.nR = nR;
    E.ident = nR == m;
    E.nt = 32 * ((n + 31) / 32 + 1);
    const int64_t ntri = (int64_t)n * (n - 1) * (n - 2) / 6;
    E.nbw = (int)((ntri + 31) / 32);
    __syncthreads();
    // 3. storage: bucket bits after the head (the keys are done with), then
    // the edges by distance, then (SB) the bucket starts and the bitmap
    uint32_t off = hb;
    E.o_h0 = off;
    off += (((uint32_t)(nR + 31) / 32) * 4 + 15) & ~15u;
    E.gG = Gg;
    E.gbits = reinterpret_cast<uint32_t*>(back + BIT_BITS);
    const int ev = (m + 7) / 8;  // 16-byte vectors of 8 entries
    E.o_Es = off;
    off += (uint32_t)ev * 16;
    uint4* es = reinterpret_cast<uint4*>(g_bsm + E.o_Es);
    for (int i = threadIdx.x; i < ev; i += HT) es[i] = reinterpret_cast<const uint4*>(Esg)[i];
    const int nbv = (E.nbw + 3) / 4;  // bitmap words in 16-byte vectors
    if constexpr (SB) {
        const int gv = (nR + 1 + 7) / 8;
        E.o_G = off;
        off += (uint32_t)gv * 16;
        E.o_bits = off;
        uint4* gs = reinterpret_cast<uint4*>(g_bsm + E.o_G);
        for (int i = threadIdx.x; i < gv; i += HT) gs[i] = reinterpret_cast<const uint4*>(Gg)[i];
        uint4* bw = reinterpret_cast<uint4*>(g_bsm + E.o_bits);
        for (int i = threadIdx.x; i < nbv; i += HT) bw[i] = make_uint4(0, 0, 0, 0);
    } else {
        uint4* bw = reinterpret_cast<uint4*>(E.gbits);
        for (int i = threadIdx.x; i < nbv; i += HT) bw[i] = make_uint4(0, 0, 0, 0);
    }
    uint32_t* h0 = bit_h0(E);
    for (int i = threadIdx.x; i < (nR + 31) / 32; i += HT) h0[i] = 0;
    if (threadIdx.x == 0) H.fail = 0;
    __syncthreads();
    return E;
}

// Reduce column j (position in cols) to completion on an empty W; returns
// its pivot as a row key ((distance bits << TRI_BITS) | (mask - index)), or
// EMPTY for a zero column.  `adds` receives the additions made and `vl` the
// generators recorded in E.vbuf (R_j = D_j + sum of their D_g).  Sets
// H.fail when a buffer is too small (the cloud is then recomputed by the
// single-cloud path).  All threads take the same branches (vl, adds and
// the owner are the same in every thread).
template <bool SB, bool SR>
__device__ uint64_t bit_column(const BitEng& E, const Ctx& c, const uint32_t* mat, int j, unsigned long long& adds,
                               int& vl) {
    BitHead& H = bit_hd();
    const uint16_t* rk = bit_rk<SR>(E);
    const uint64_t self_key = c.cols[j];
    const int ej = (int)(self_key & c.cmask);
    const uint32_t rj = rk[ej];
    int ja, jb;
    edge_of(ej, ja, jb);
    const int x = (int)threadIdx.x;  // this thread's third vertex
    bit_cob<SB, SR>(E, ja, jb, rj, x < E.n ? x : -1, -1);
    if (threadIdx.x < 3) { H.best[threadIdx.x] = 0; H.cnt[threadIdx.x] = 0; }
    bit_sync(E);
    uint64_t key = EMPTY;
    adds = 0;
    vl = 0;
    int it = 0, rp = -1, cp = 0;
    for (;;) {
        int r, cf;
        uint32_t a, b, w, t;
        bool eq_aw, eq_bw;
        if (!bit_pivot<SB, SR>(E, rp, cp, it, r, a, b, w, t, cf, eq_aw, eq_bw)) break;
        rp = r;
        cp = cf;
        // the loop's last warp (no vertex of its own) probes the hash of finished columns;
        // meanwhile every thread finds the candidate apparent owner s' (the
        // facet left by dropping the largest vertex whose opposite edge keeps
        // the diameter; w's is (a, b)) and tests its own cofacet of s'
        if ((int)threadIdx.x >= E.nt - 32) {  // the last warp of the loop, with no vertex of its own
            const int64_t hp = warp_hash_find(c, t);
            if ((int)threadIdx.x == E.nt - 32) H.opos = (int)hp;
        }
        uint32_t wd = w;
        if (eq_bw && a > wd) wd = a;  // the edge opposite a is (b, w)
        if (eq_aw && b > wd) wd = b;
        const uint32_t su = wd == a ? b : a, sv = wd == w ? b : w;  // s' = {a, b, w} - {wd}
        bool row = false, older = false;
        uint32_t rt = 0, d = 0;
        if (x < E.n && x != (int)su && x != (int)sv) {
            const uint32_t mx = max((uint32_t)rk[bit_eidx(su, x)], (uint32_t)rk[bit_eidx(sv, x)]);
            older = (uint32_t)x > wd && mx <= (uint32_t)r;  // s' + {x} is an older cofacet of s'
            d = max((uint32_t)r, mx);
            row = d != 0xFFFFu;
            rt = bit_tidx(su, sv, x);
        }
        const int any_older = bit_sync_or(E, older);
        const int opos = H.opos;
        if (opos < 0 && any_older) {  // the pivot has no owner: the column is complete
            key = ((uint64_t)mat[a * BLD + b] << TRI_BITS) | (c.rcmask - t);
            break;
        }
        if (adds >= (1ull << 22)) {  // far beyond any column of n <= 256
            if (threadIdx.x == 0) H.fail = 1;
            break;
        }
        ++adds;
        if (opos >= 0) {
            // the pivot of the finished column opos: add its reduced form
            const uint32_t len = c.rc_len[opos];
            const uint64_t* lst = reinterpret_cast<const uint64_t*>(c.rc_ptr[opos]);
            const uint64_t eo = c.cols[opos] & c.cmask;
            const int add = len ? (int)len : 1;
            if (vl + add > BIT_VCAP) {
                if (threadIdx.x == 0) H.fail = 1;
                break;
            }
            if (len) {
                bit_add_list<SB, SR>(E, lst, (int)len, r);
                for (int i = threadIdx.x; i < (int)len; i += E.nt) E.vbuf[vl + i] = lst[i];
            } else {
                int oa, ob;
                edge_of((int)eo, oa, ob);
                bit_cob<SB, SR>(E, oa, ob, rk[eo], x < E.n ? x : -1, r);
                if (threadIdx.x == 0) E.vbuf[vl] = eo;
            }
            vl += add;
        } else {
            // the apparent owner s', which precedes column j in coboundary order
            // (larger distance, or equal distance and smaller index)
            const uint32_t es = bit_eidx(su, sv);
            if (threadIdx.x == 0 && !((uint32_t)r > rj || ((uint32_t)r == rj && (int)es < ej)))
                atomicExch(c.err, DEV_INTERNAL | (5 << 8));
            if (vl + 1 > BIT_VCAP) {
                if (threadIdx.x == 0) H.fail = 1;
                break;
            }
            bit_flip<SB, SR>(E, row, rt, d, r);
            if (threadIdx.x == 0) E.vbuf[vl] = es;
            vl += 1;
        }
        bit_sync(E);
    }
    bit_sync(E);  // H.fail is read by every thread of the loop after the return
    return key;
}

// Empty W after column j (generators vbuf[0..vl)): a few coboundaries are
// flipped back, a longer record is cheaper to wipe; the bucket bits are reset.
template <bool SB, bool SR>
__device__ void bit_clear(const BitEng& E, int ej, int vl) {
    bit_sync(E);
    if (!SB && vl < 8) {
        int ja, jb;
        edge_of(ej, ja, jb);
        const int x = (int)threadIdx.x;
        bit_cob<SB, SR>(E, ja, jb, bit_rk<SR>(E)[ej], x < E.n ? x : -1, -1);
        bit_add_list<SB, SR>(E, E.vbuf, vl, -1);
    } else {
        uint4* bw = reinterpret_cast<uint4*>(bit_bits<SB>(E));
        for (int i = threadIdx.x; i < (E.nbw + 3) / 4; i += E.nt) bw[i] = make_uint4(0, 0, 0, 0);
    }
    bit_sync(E);
    uint32_t* h0 = bit_h0(E);
    for (int i = threadIdx.x; i < (E.nR + 31) / 32; i += E.nt) h0[i] = 0;
    bit_sync(E);
}

// 5c for one cloud: the columns ucur[0..nu) in order, each reduced to
// completion; pairs appended to h1tmp (count *nh1), the pivots to the hash.
// The hash moves to the second arena's free part when it fits.  Returns
// false when a buffer was too small (the cloud is then recomputed singly).
template <bool SB, bool SR>
__device__ bool bit_reduce(Ctx c, const uint32_t* mat, uint64_t* back, int n, uint32_t thr, const uint32_t* ucur,
                           int nu, uint32_t arena2_off, size_t arena2_bytes, PairRec* h1tmp, int* nh1,
                           unsigned long long& adds) {
    const BitEng E = bit_setup<SB, SR>(back, mat, n, thr, arena2_off);
    BitHead& H = bit_hd();
    const size_t used2 = SR ? (((size_t)n * (n - 1) + 15) & ~(size_t)15) : 0;  // the ranks (2 bytes per edge)
    const size_t hsz = (size_t)c.hmask + 1;
    if (used2 + hsz * 12 <= arena2_bytes) {
        uint64_t* hk = reinterpret_cast<uint64_t*>(g_bsm + arena2_off + used2);
        uint32_t* hv = reinterpret_cast<uint32_t*>(g_bsm + arena2_off + used2 + hsz * 8);
        for (size_t i = threadIdx.x; i < hsz; i += HT) { hk[i] = c.hkeys[i]; hv[i] = c.hvals[i]; }
        c.hkeys = hk;
        c.hvals = hv;
        __syncthreads();
    }
    adds = 0;
    if ((int)threadIdx.x < E.nt) {  // the column loop (the other warps wait at the barrier below)
        for (int q = 0; q < nu; ++q) {
            const int j = (int)ucur[q];
            const uint64_t self_key = c.cols[j];
            unsigned long long col_adds;
            int vl;
            const uint64_t key = bit_column<SB, SR>(E, c, mat, j, col_adds, vl);
            adds += col_adds;
            if (H.fail) break;
            if (col_adds) {  // keep R_j as its generators: j, then those recorded
                if (threadIdx.x == 0) H.poff = atomicAdd(c.pool_used, (unsigned long long)(vl + 1));
                bit_sync(E);
                const unsigned long long off = H.poff;
                if ((int64_t)(off + vl + 1) > c.pool_cap) {
                    if (threadIdx.x == 0) H.fail = 1;
                    break;
                }
                for (int i = threadIdx.x; i <= vl; i += E.nt)
                    c.pool[off + i] = i == 0 ? (self_key & c.cmask) : E.vbuf[i - 1];
                if (threadIdx.x == 0) {
                    c.rc_ptr[j] = (uint64_t)(c.pool + off);
                    c.rc_len[j] = (uint32_t)(vl + 1);
                }
            }
            if (threadIdx.x == 0) {
                Simplex<1> s;
                load_col<1>(c, self_key, s);
                PairRec pr;
                pr.birth_rank = s.r;
                pr.birth_cidx = s.cidx;
                bool out = true;
                if (key == EMPTY) {
                    pr.death_rank = 0xFFFFFFFFu; pr.death_cidx = -1;
                } else {
                    pr.death_rank = (uint32_t)(key >> TRI_BITS);
                    pr.death_cidx = (int64_t)(c.rcmask - (key & c.rcmask));
                    hash_insert(c, (uint64_t)pr.death_cidx, (uint32_t)j);
                    out = pr.death_rank > pr.birth_rank;
                }
                if (out) h1tmp[(*nh1)++] = pr;
            }
            if (q + 1 < nu) bit_clear<SB, SR>(E, (int)(self_key & c.cmask), vl);
            bit_sync(E);
        }
    }
    __syncthreads();
    return !H.fail;
}

__global__ void __launch_bounds__(HT, 2) k_batched(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char bsm[];
    BatchSmem& M = *reinterpret_cast<BatchSmem*>(bsm);
    HeavySmem& S = M.S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t slot = blockIdx.x;
    uint32_t* mat = A.mat + slot * (int64_t)BMAXN * BLD;
    uint64_t* cols = A.cols + slot * (int64_t)CCAP;
    uint64_t* cur_key = A.cur_key + slot * (int64_t)CCAP;
    uint8_t* status = A.status + slot * (int64_t)CCAP;
    uint32_t* ulist = A.ulist + slot * (int64_t)(2 * CCAP);
    PairRec* h1tmp = A.h1tmp + slot * (int64_t)CCAP;
    uint64_t* back = A.back + slot * BACKCAP;
    const Binom B{A.binom, BMAXN, 3};
    __shared__ int next_cloud;

    for (;;) {
        if (threadIdx.x == 0) next_cloud = (int)atomicAdd(A.work, 1ull);
        __syncthreads();
        const int k = next_cloud;
        __syncthreads();
        if (k >= A.num) break;
        const int cloud = A.order[k];
        const int64_t o0 = A.offs[cloud];
        const int n = (int)(A.offs[cloud + 1] - o0);
        const int ne = n * (n - 1) / 2;
        if (threadIdx.x == 0) { M.h0n = 0; M.ncols = 0; M.nh1 = 0; M.nu = 0; M.overflow = 0; }
        long long tp = clock64();
        const long long t_cloud = tp;
#define VR_PHASE(i)                                                          \
    do {                                                                     \
        if (A.prof && threadIdx.x == 0) {                                    \
            const long long t_ = clock64();                                  \
            atomicAdd(A.prof + (i), (unsigned long long)(t_ - tp));          \
            tp = t_;                                                         \
        }                                                                    \
    } while (0)
        // ---- 1. points and distances (bits of the single-precision formula);
        // up to BAT_DSM_N points the upper triangle is also kept in the arena
        // (the engine's space, unused until 5c) for the spanning tree and the
        // apparent search
        const bool dsh = n <= BAT_DSM_N;
        uint32_t* dsm = reinterpret_cast<uint32_t*>(g_bsm);
        for (int i = threadIdx.x; i < n * A.dim; i += HT) M.pts[i] = A.pts[o0 * A.dim + i];
        for (int i = threadIdx.x; i < (ne + 31) / 32; i += HT) M.clear[i] = 0;
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * n; idx += HT) {
            const int i = idx / n, j = idx % n;
            uint32_t bits = 0;
            if (i != j) {
                const int a = i > j ? i : j, b = i > j ? j : i;
                float acc = 0.0f;
                for (int q = 0; q < A.dim; ++q) {
                    const float diff = __fsub_rn(M.pts[a * A.dim + q], M.pts[b * A.dim + q]);
                    acc = __fadd_rn(acc, __fmul_rn(diff, diff));
                }
                bits = __float_as_uint(__fsqrt_rn(acc));
            }
            mat[i * BLD + j] = bits;
            if (dsh && i > j) dsm[i * (i - 1) / 2 + j] = bits;
        }
        __syncthreads();
        const RankMatrix R{mat, n, BLD};
        // distances for steps 2-3: the arena's copy when it holds one (shared
        // memory), else the matrix in global memory
        auto D = [&](int i, int j) -> uint32_t {
            if (dsh) return i == j ? 0u : dsm[i > j ? i * (i - 1) / 2 + j : j * (j - 1) / 2 + i];
            return R(i, j);
        };
        // ---- 2. threshold: enclosing radius unless given
        if (threadIdx.x == 0) M.thr = A.thr_inf ? 0xFFFFFFFFu : A.thr_bits;
        __syncthreads();
        if (A.thr_inf) {
            for (int i = wid; i < n; i += HW) {
                uint32_t m = 0;
                for (int j = lane; j < n; j += 32) m = max(m, D(i, j));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) atomicMin(&M.thr, m);
            }
            __syncthreads();
        }
        const uint32_t thr = M.thr;
        if (threadIdx.x == 0) A.thr_used[cloud] = __uint_as_float(thr);
        VR_PHASE(0);
        // ---- 3a. warp 0: spanning tree and elder rule
        if (wid == 0) {
            uint64_t best[BMAXN / 32];
            uint32_t intree = 0;
#pragma unroll
            for (int q = 0; q < BMAXN / 32; ++q) best[q] = ~0ull - 1;
            int cnt = 0;
            for (int it = 0; it < n; ++it) {
                uint64_t mk = ~0ull;
                int mi = BMAXN;
#pragma unroll
                for (int q = 0; q < BMAXN / 32; ++q) {
                    const int v = lane + 32 * q;
                    if (v < n && !((intree >> q) & 1u) && best[q] < mk) { mk = best[q]; mi = v; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t ok = __shfl_xor_sync(0xffffffffu, mk, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
                    if (ok < mk || (ok == mk && oi < mi)) { mk = ok; mi = oi; }
                }
                const int u = mi;
                if ((u & 31) == lane) intree |= 1u << (u >> 5);
                if (mk != ~0ull - 1) {
                    if (lane == 0) M.tree[cnt] = mk;
                    ++cnt;
                }
#pragma unroll
                for (int q = 0; q < BMAXN / 32; ++q) {
                    const int v = lane + 32 * q;
                    if (v < n && !((intree >> q) & 1u)) {
                        const uint32_t r = D(u, v);
                        if (r <= thr) {
                            const int a = u > v ? u : v, b = u > v ? v : u;
                            const uint64_t key = ((uint64_t)r << 32) | (0xFFFFFFFFull - (uint64_t)(a * (a - 1) / 2 + b));
                            if (key < best[q]) best[q] = key;
                        }
                    }
                }
            }
            for (int i = cnt + lane; i < BMAXN; i += 32) M.tree[i] = ~0ull;
            __syncwarp();
            warp_bitonic(M.tree, BMAXN);
            if (lane == 0) {
                for (int v = 0; v < n; ++v) M.parent[v] = -1 - v;
                int h = 0;
                for (int i = 0; i < cnt; ++i) {
                    const uint64_t key = M.tree[i];
                    const int e = (int)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
                    int a, b;
                    edge_of(e, a, b);
                    int ra = a; while (M.parent[ra] >= 0) ra = M.parent[ra];
                    int rb = b; while (M.parent[rb] >= 0) rb = M.parent[rb];
                    const int oa = -1 - M.parent[ra], ob = -1 - M.parent[rb];
                    const int young = oa < ob ? ra : rb, old = oa < ob ? rb : ra;
                    const uint32_t dr = (uint32_t)(key >> 32);
                    if (dr != 0) {  // zero-length classes (coincident points) are not reported
                        PairRec pr;
                        pr.birth_rank = 0; pr.death_rank = dr;
                        pr.birth_cidx = (uint64_t)(oa < ob ? oa : ob); pr.death_cidx = e;
                        M.h0[h++] = pr;
                    }
                    M.parent[young] = old;
                    M.clear[e >> 5] |= 1u << (e & 31);
                }
                for (int v = 0; v < n; ++v)
                    if (M.parent[v] < 0) {
                        PairRec pr;
                        pr.birth_rank = 0; pr.death_rank = 0xFFFFFFFFu;
                        pr.birth_cidx = (uint64_t)(-1 - M.parent[v]); pr.death_cidx = -1;
                        M.h0[h++] = pr;
                    }
                M.h0n = h;
            }
        } else if (A.dmax >= 1) {
            // ---- 3b. warps 1..15: apparent pairs of the edges within the threshold.
            // Each lane takes an edge s = (a, b) of the chunk and tests, in lock
            // step with the other lanes, the candidate vertices w = n-1, n-2, ...
            // (the oldest cofacet of s is s + {w} for the largest w keeping the
            // diameter) for BAT_LOCK steps; the edges still open then search the
            // rest one at a time, 32 candidates per warp step.
            unsigned long long c_app = 0, c_cand = 0;
            for (int ch = wid - 1; ch * 32 < ne; ch += HW - 1) {
                const int e = ch * 32 + lane;
                int va = 0, vb = 0;
                uint32_t r = 0;
                bool kept = false;
                if (e < ne) {
                    edge_of(e, va, vb);
                    r = D(va, vb);
                    kept = r <= thr;
                    c_cand += kept;
                }
                int wf = -1;
                bool open = kept;
#pragma unroll
                for (int k = 0; k < BAT_LOCK; ++k) {
                    const int w = n - 1 - k;
                    if (open && w >= 0 && w != va && w != vb && D(va, w) <= r && D(vb, w) <= r) {
                        wf = w;
                        open = false;
                    }
                }
                if (n - 1 - BAT_LOCK < 0) open = false;  // every candidate tested
                uint32_t om = __ballot_sync(0xffffffffu, open);
                while (om) {
                    const int src = __ffs(om) - 1;
                    om &= om - 1;
                    const int a = __shfl_sync(0xffffffffu, va, src), b = __shfl_sync(0xffffffffu, vb, src);
                    const uint32_t sr = __shfl_sync(0xffffffffu, r, src);
                    int f = -1;
                    for (int base = n - 1 - BAT_LOCK; base >= 0; base -= 32) {
                        const int w = base - lane;
                        const bool ok = w >= 0 && w != a && w != b && D(a, w) <= sr && D(b, w) <= sr;
                        const uint32_t bl = __ballot_sync(0xffffffffu, ok);
                        if (bl) { f = base - (__ffs(bl) - 1); break; }
                    }
                    if (lane == src) wf = f;
                }
                // facet t - {x} for a vertex x > wf of s must not keep the diameter
                bool apparent = kept && wf >= 0;
                if (apparent && va > wf && D(vb, wf) == r) apparent = false;
                if (apparent && vb > wf && D(va, wf) == r) apparent = false;
                c_app += apparent;
                const bool col = kept && !apparent;
                const uint32_t cm = __ballot_sync(0xffffffffu, col);
                int at = 0;
                if (lane == 0 && cm) at = atomicAdd(&M.ncols, __popc(cm));
                at = __shfl_sync(0xffffffffu, at, 0) + __popc(cm & ((1u << lane) - 1u));
                if (col) {
                    if (at < CCAP) cols[at] = ((~(uint64_t)r & 0xFFFFFFFFull) << EDGE_BITS) | (uint64_t)e;
                    else M.overflow = 1;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c_cand += __shfl_xor_sync(0xffffffffu, c_cand, o);
                c_app += __shfl_xor_sync(0xffffffffu, c_app, o);
            }
            if (lane == 0 && c_app) atomicAdd(A.stats + 1, c_app);
            if (lane == 0 && c_cand) atomicAdd(A.stats + 0, c_cand);
        }
        __syncthreads();
        VR_PHASE(1);
        if (M.overflow) {
            if (threadIdx.x == 0) A.cloud_err[cloud] = 1;
            __syncthreads();
            continue;
        }
        // ---- H0 output
        {
            const int h = M.h0n;
            int len = 1;
            while (len < h) len <<= 1;
            for (int i = h + threadIdx.x; i < len; i += HT) {
                M.h0[i].birth_rank = 0xFFFFFFFFu; M.h0[i].death_rank = 0xFFFFFFFFu; M.h0[i].birth_cidx = ~0ull;
            }
            __syncthreads();
            if (len <= BMAXN) block_sort_recs(M.h0, len);
            emit_block(A, M, 0, cloud, M.h0, h, R, B);
        }
        VR_PHASE(2);
        if (A.dmax < 1) continue;
        // ---- 4. drop cleared columns, sort the rest into coboundary order
        int m = M.ncols;
        {
            int kept_total = 0;
            for (int base = 0; base < m; base += HT) {
                const int i = base + threadIdx.x;
                const uint64_t key = i < m ? cols[i] : EMPTY;
                const int e = (int)(key & ((1ull << EDGE_BITS) - 1));
                const bool keep = i < m && !((M.clear[e >> 5] >> (e & 31)) & 1u);
                int tot;
                const int pos = block_excl_scan(keep, S.ws, &tot);
                if (keep) cols[kept_total + pos] = key;
                kept_total += tot;
            }
            m = kept_total;
            int len = 1;
            while (len < m) len <<= 1;
            for (int i = m + threadIdx.x; i < len; i += HT) cols[i] = EMPTY;
            __syncthreads();
            block_bitonic(cols, len);
            if (threadIdx.x == 0) atomicAdd(A.stats + 2, (unsigned long long)m);
        }
        VR_PHASE(3);
        // ---- 5. reduction
        Ctx c;
        c.R = R;
        c.B = B;
        c.thr = thr;
        c.cb = EDGE_BITS;
        c.rcb = TRI_BITS;
        c.cmask = (1ull << EDGE_BITS) - 1;
        c.rcmask = (1ull << TRI_BITS) - 1;
        c.rmask = 0xFFFFFFFFull;
        c.cols = cols;
        c.num_cols = m;
        c.hkeys = A.hkeys + slot * (int64_t)HCAP;
        c.hvals = A.hvals + slot * (int64_t)HCAP;
        uint64_t hsz = 64;
        while (hsz < 2 * (uint64_t)m) hsz <<= 1;
        c.hmask = hsz - 1;
        c.err = A.cloud_err + cloud;
        c.pool = A.pool + slot * POOLCAP;
        c.pool_used = A.pool_used + slot;
        c.pool_cap = A.pool_cap;
        c.rc_ptr = A.rc_off + slot * (int64_t)CCAP;
        c.mode = MODE_EXPLICIT;
        c.rc_len = A.rc_len + slot * (int64_t)CCAP;
        uint32_t* adds_j = A.adds + slot * (int64_t)CCAP;
        for (uint64_t i = threadIdx.x; i < hsz; i += HT) c.hkeys[i] = EMPTY;
        if (threadIdx.x == 0) *c.pool_used = 0;
        __syncthreads();
        // 5a/5b. one round over the columns, one warp each, without additions:
        // it finds every pivot and settles, in order by the prefix-minimum rule,
        // the columns whose pivot has no owner.  The rest go to the bitmap engine
        // (measured faster on these clouds than warp rounds with additions: with
        // up to 8 additions per column here, 4096 clouds 29.6 -> 31.1 ms).
        uint32_t* ucur = ulist;
        uint32_t* unext = ulist + CCAP;
        for (int i = threadIdx.x; i < m; i += HT) ucur[i] = (uint32_t)i;
        int nu = m;
        constexpr int budget = 0;
        __syncthreads();
        if (nu > 0) {
            {
                uint64_t* wst = A.wstage + (slot * HW + wid) * (int64_t)STAGE;
                for (int q = wid; q < nu; q += HW) {
                    const int j = ucur[q];
                    uint64_t key;
                    uint8_t st;
                    uint32_t ad;
                    reduce_one<1>(c, j, budget, wst, key, st, ad);
                    if (lane == 0) { cur_key[j] = key; status[j] = st; adds_j[j] = ad; }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) { M.carry_min = EMPTY; M.carry_cnt = 0; }
            __syncthreads();
            for (int base = 0; base < nu; base += HT) {
                const bool valid = base + (int)threadIdx.x < nu;
                const int j = valid ? (int)ucur[base + threadIdx.x] : 0;
                const uint64_t key = valid ? cur_key[j] : EMPTY;
                const uint8_t st = valid ? status[j] : ST_COMPLETE;
                uint64_t incl = key;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o && y < incl) incl = y;
                }
                if (lane == 31) M.wmin[wid] = incl;
                __syncthreads();
                uint64_t pm = M.carry_min;
                for (int w = 0; w < wid; ++w) pm = min(pm, M.wmin[w]);
                const uint64_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
                if (lane > 0) pm = min(pm, excl);
                const bool fin = valid && st == ST_COMPLETE && (key == EMPTY || key < pm);
                const bool keep = valid && !fin;
                if (fin) {
                    if (adds_j[j]) atomicAdd(A.stats + 3, (unsigned long long)adds_j[j]);
                    const uint64_t ck = cols[j];
                    PairRec pr;
                    pr.birth_rank = (uint32_t)(~(ck >> EDGE_BITS));
                    pr.birth_cidx = ck & c.cmask;
                    bool out = true;
                    if (key == EMPTY) {
                        pr.death_rank = 0xFFFFFFFFu; pr.death_cidx = -1;
                    } else {
                        pr.death_rank = (uint32_t)(key >> TRI_BITS);
                        pr.death_cidx = (int64_t)(c.rcmask - (key & c.rcmask));
                        hash_insert(c, (uint64_t)pr.death_cidx, (uint32_t)j);
                        out = pr.death_rank > pr.birth_rank;
                    }
                    if (out) h1tmp[atomicAdd(&M.nh1, 1)] = pr;
                }
                const uint32_t kb = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) M.wcnt[wid] = __popc(kb);
                __syncthreads();
                int before = 0, total = 0;
                for (int w = 0; w < HW; ++w) {
                    if (w < wid) before += M.wcnt[w];
                    total += M.wcnt[w];
                }
                if (keep) unext[M.carry_cnt + before + __popc(kb & ((1u << lane) - 1u))] = (uint32_t)j;
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint64_t cm = M.carry_min;
                    for (int w = 0; w < HW; ++w) cm = min(cm, M.wmin[w]);
                    M.carry_min = cm;
                    M.carry_cnt += total;
                }
                __syncthreads();
            }
            const int nn = M.carry_cnt;
            uint32_t* t = ucur; ucur = unext; unext = t;
            nu = nn;
        }
        VR_PHASE(5);
        // 5c. the remaining columns in order, each to completion (bitmap engine)
        if (A.prof && threadIdx.x == 0) atomicAdd(A.prof + 8, (unsigned long long)nu);
        unsigned long long adds = 0;
        if (nu > 0) {
            // the block engine's shared space is the arena; the per-point buffers (points,
            // clearing bits, tree, H0 records), no longer needed, the second arena
            constexpr uint32_t a2 = (uint32_t)offsetof(BatchSmem, pts);
            constexpr size_t a2b = offsetof(BatchSmem, h0) + sizeof(PairRec) * BMAXN - offsetof(BatchSmem, pts);
            const int var = bit_variant(n, sizeof(HeavySmem), a2b);
            const bool ok = var == 0   ? bit_reduce<true, true>(c, mat, back, n, thr, ucur, nu, a2, a2b, h1tmp, &M.nh1, adds)
                            : var == 1 ? bit_reduce<false, true>(c, mat, back, n, thr, ucur, nu, a2, a2b, h1tmp, &M.nh1, adds)
                                       : bit_reduce<false, false>(c, mat, back, n, thr, ucur, nu, a2, a2b, h1tmp, &M.nh1,
                                                                  adds);
            if (!ok) {
                if (threadIdx.x == 0) M.overflow = 1;
                __syncthreads();
            }
        }
        if (threadIdx.x == 0 && adds) atomicAdd(A.stats + 3, adds);
        VR_PHASE(6);
        if (M.overflow) {
            if (threadIdx.x == 0) A.cloud_err[cloud] = 1;
            __syncthreads();
            continue;
        }
        // ---- 6. H1 output, sorted
        {
            const int h = M.nh1;
            int len = 1;
            while (len < h) len <<= 1;
            for (int i = h + threadIdx.x; i < len; i += HT) {
                h1tmp[i].birth_rank = 0xFFFFFFFFu; h1tmp[i].death_rank = 0xFFFFFFFFu; h1tmp[i].birth_cidx = ~0ull;
            }
            __syncthreads();
            block_sort_recs(h1tmp, len);
            emit_block(A, M, 1, cloud, h1tmp, h, R, B);
        }
        VR_PHASE(7);
        if (A.prof && threadIdx.x == 0 && cloud >= 0 && cloud < A.num)
            A.prof[16 + cloud] = (unsigned long long)(clock64() - t_cloud);
    }
#undef VR_PHASE
}

// Ordered copy of the appended records: cloud i's pairs of dimension p go to
// out[off[i] .. off[i+1]), converted to float values.
__global__ void k_batch_gather(const PairRec* __restrict__ recs, const int32_t* __restrict__ edges,
                               const int64_t* __restrict__ start, const int32_t* __restrict__ count,
                               const int64_t* __restrict__ off, const int64_t* __restrict__ poffs, int num,
                               int64_t cap, vr_pair* __restrict__ out, int32_t* __restrict__ out_edges) {
    for (int cl = blockIdx.x; cl < num; cl += gridDim.x) {
        const int64_t s = start[cl], o = off[cl];
        const int cnt = count[cl];
        // past the planned room (the host then grows the buffers and reruns):
        // neither the records nor the output hold these pairs
        if (cnt <= 0 || s < 0 || s + cnt > cap || o + cnt > cap) continue;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const PairRec r = recs[s + i];
            vr_pair v;
            v.birth = __uint_as_float(r.birth_rank);
            v.death = r.death_rank == 0xFFFFFFFFu ? __int_as_float(0x7f800000) : __uint_as_float(r.death_rank);
            v.birth_simplex = r.birth_cidx;
            v.death_simplex = r.death_cidx;
            out[o + i] = v;
            if (out_edges)  // rows of the packed point array
                for (int q = 0; q < 4; ++q) {
                    const int32_t e = edges[4 * (s + i) + q];
                    out_edges[4 * (o + i) + q] = e >= 0 ? (int32_t)(e + poffs[cl]) : -1;
                }
        }
    }
}

__global__ void k_exclusive_scan_i64(const int32_t* __restrict__ count, int num, int64_t* __restrict__ off) {
    // one block: sequential chunks with a running carry (num is at most a few thousand)
    __shared__ int64_t carry;
    __shared__ int64_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < num; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int64_t x = i < num ? count[i] : 0;
        int64_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        int64_t before = carry;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        if (i < num) off[i] = before + incl - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[num] = carry;
}

// ---------------------------------------------------------------------------
// host side: buffers, CUDA graph and the launch-shape autotuner
// ---------------------------------------------------------------------------
struct BatchPlan {
    int device = -1;
    int num = 0, dim = 0, dmax = 0, want_edges = 0, thr_inf = 1;
    uint32_t thr_bits = 0;
    int64_t total = 0;
    int slots = 0;
    int64_t cap[2] = {0, 0};
    // device buffers
    float* pts = nullptr;
    int64_t* offs = nullptr;
    int32_t* order = nullptr;
    char* scratch = nullptr;
    char* outbuf = nullptr;
    BatchArgs args{};
    int64_t* off[2] = {nullptr, nullptr};
    vr_pair* pairs[2] = {nullptr, nullptr};
    int32_t* edges[2] = {nullptr, nullptr};
    cudaGraphExec_t exec = nullptr;
    cudaStream_t captured_on = nullptr;
    // pinned staging of host results (device-to-host copies into pageable
    // memory run at a fraction of the link's rate), grown on demand
    char* pin = nullptr;
    size_t pin_bytes = 0;
};

// Copy `bytes` from device memory into pageable host memory through the
// plan's pinned staging buffer (chunks of at most 8 MB, the copy of one
// chunk overlapping the host copy of the previous one).
void copy_to_host(BatchPlan& P, void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    constexpr size_t CH = (size_t)8 << 20;
    if (!P.pin) {
        VR_CUDA(cudaMallocHost((void**)&P.pin, 2 * CH));
        P.pin_bytes = 2 * CH;
    }
    cudaEvent_t done[2];
    VR_CUDA(cudaEventCreateWithFlags(&done[0], cudaEventDisableTiming));
    VR_CUDA(cudaEventCreateWithFlags(&done[1], cudaEventDisableTiming));
    const size_t nch = (bytes + CH - 1) / CH;
    for (size_t k = 0; k <= nch; ++k) {
        if (k < nch) {  // queue chunk k into half k % 2
            const size_t len = std::min(CH, bytes - k * CH);
            VR_CUDA(cudaMemcpyAsync(P.pin + (k & 1) * CH, static_cast<const char*>(src) + k * CH, len,
                                    cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaEventRecord(done[k & 1], s));
        }
        if (k > 0) {  // chunk k - 1 is on the host once its event completes
            const size_t j = k - 1, len = std::min(CH, bytes - j * CH);
            VR_CUDA(cudaEventSynchronize(done[j & 1]));
            memcpy(static_cast<char*>(dst) + j * CH, P.pin + (j & 1) * CH, len);
        }
    }
    cudaEventDestroy(done[0]);
    cudaEventDestroy(done[1]);
}

std::mutex g_batch_mutex;
BatchPlan* g_plan = nullptr;
std::map<std::pair<int, int64_t>, int> g_tuned;  // (device, size bucket) -> slots per SM

size_t slot_bytes() {
    return (size_t)BMAXN * BLD * 4 + (size_t)HCAP * 12 +
           (size_t)CCAP * (8 + 8 + 1 + 8 + sizeof(PairRec) + 8 + 4 + 4) + (size_t)BACKCAP * 8 +
           (size_t)HW * STAGE * 8 + (size_t)POOLCAP * 8 + 16 * 256;
}

void free_plan(BatchPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->pin) cudaFreeHost(p->pin);
    cudaFree(p->pts); cudaFree(p->offs); cudaFree(p->order); cudaFree(p->scratch); cudaFree(p->outbuf);
    delete p;
}

template <class T>
T* carve(char*& cur, size_t n) {
    T* p = reinterpret_cast<T*>(cur);
    cur += (n * sizeof(T) + 255) / 256 * 256;
    return p;
}

void record_launches(BatchPlan& P, cudaStream_t s) {
    BatchArgs& A = P.args;
    VR_CUDA(cudaMemsetAsync(A.work, 0, 8 * sizeof(unsigned long long), s));  // work, used[2], stats[4]
    VR_CUDA(cudaMemsetAsync(A.cloud_err, 0, P.num * sizeof(int32_t), s));
    // a cloud recomputed by the host (cloud_err) emits no pairs of some dimension:
    // its count must read 0, not what a previous launch or the allocation left
    for (int p = 0; p <= P.dmax; ++p) VR_CUDA(cudaMemsetAsync(A.count[p], 0, P.num * sizeof(int32_t), s));
    k_batched<<<P.slots, HT, sizeof(BatchSmem), s>>>(A);
    for (int p = 0; p <= P.dmax; ++p) {
        k_exclusive_scan_i64<<<1, 1024, 0, s>>>(A.count[p], P.num, P.off[p]);
        k_batch_gather<<<std::min(P.num, 4096), 128, 0, s>>>(A.recs[p], A.edges[p], A.start[p], A.count[p], P.off[p],
                                                             P.offs, P.num, A.cap[p], P.pairs[p],
                                                             P.want_edges ? P.edges[p] : nullptr);
    }
    VR_CUDA(cudaGetLastError());
}

BatchPlan* make_plan(int dev, int num, int dim, int dmax, int want_edges, int thr_inf, uint32_t thr_bits,
                     int64_t total, int slots, const int64_t cap[2]) {
    BatchPlan* P = new BatchPlan();
    P->device = dev; P->num = num; P->dim = dim; P->dmax = dmax; P->want_edges = want_edges;
    P->thr_inf = thr_inf; P->thr_bits = thr_bits; P->total = total; P->slots = slots;
    P->cap[0] = cap[0]; P->cap[1] = cap[1];
    try {
        VR_CUDA(cudaMalloc(&P->pts, std::max<int64_t>(total * dim, 1) * sizeof(float)));
        VR_CUDA(cudaMalloc(&P->offs, (num + 1) * sizeof(int64_t)));
        VR_CUDA(cudaMalloc(&P->order, std::max(num, 1) * sizeof(int32_t)));
        const size_t sb = slot_bytes() * (size_t)slots + (size_t)4 * 1024 * 1024;
        VR_CUDA(cudaMalloc(&P->scratch, sb));
        size_t ob = 0;
        for (int p = 0; p < 2; ++p)
            ob += (cap[p] + 1) * (sizeof(PairRec) + sizeof(vr_pair) + 32) + (size_t)(num + 1) * 32 + 4096;
        ob += (size_t)num * 16 + 4096;
        VR_CUDA(cudaMalloc(&P->outbuf, ob));
        BatchArgs& A = P->args;
        char* cur = P->scratch;
        A.mat = carve<uint32_t>(cur, (size_t)slots * BMAXN * BLD);
        A.hkeys = carve<uint64_t>(cur, (size_t)slots * HCAP);
        A.hvals = carve<uint32_t>(cur, (size_t)slots * HCAP);
        A.cols = carve<uint64_t>(cur, (size_t)slots * CCAP);
        A.cur_key = carve<uint64_t>(cur, (size_t)slots * CCAP);
        A.status = carve<uint8_t>(cur, (size_t)slots * CCAP);
        A.ulist = carve<uint32_t>(cur, (size_t)slots * 2 * CCAP);
        A.h1tmp = carve<PairRec>(cur, (size_t)slots * CCAP);
        A.back = carve<uint64_t>(cur, (size_t)slots * BACKCAP);
        A.wstage = carve<uint64_t>(cur, (size_t)slots * HW * STAGE);
        A.pool = carve<uint64_t>(cur, (size_t)slots * POOLCAP);
        A.pool_cap = POOLCAP;
        if (const char* pc = getenv("VR_BATCH_POOL_CAP")) {  // test-only: force the single-cloud recompute
            const long long v = atoll(pc);
            A.pool_cap = v < 1 ? 1 : (v > POOLCAP ? POOLCAP : v);
        }
        A.pool_used = carve<unsigned long long>(cur, (size_t)slots);
        A.rc_off = carve<uint64_t>(cur, (size_t)slots * CCAP);
        A.rc_len = carve<uint32_t>(cur, (size_t)slots * CCAP);
        A.adds = carve<uint32_t>(cur, (size_t)slots * CCAP);
        uint64_t* binom = carve<uint64_t>(cur, (size_t)4 * (BMAXN + 1));
        A.work = carve<unsigned long long>(cur, 8);
        A.prof = log_enabled() ? carve<unsigned long long>(cur, 16 + (size_t)num) : nullptr;
        if (A.prof) VR_CUDA(cudaMemset(A.prof, 0, (16 + (size_t)num) * sizeof(unsigned long long)));
        A.used = A.work + 1;
        A.stats = A.work + 3;
        std::vector<uint64_t> hb = host_binomials(BMAXN, 3);
        VR_CUDA(cudaMemcpy(binom, hb.data(), hb.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
        A.binom = binom;
        char* oc = P->outbuf;
        for (int p = 0; p < 2; ++p) {
            A.recs[p] = carve<PairRec>(oc, cap[p] + 1);
            A.edges[p] = carve<int32_t>(oc, 4 * (cap[p] + 1));
            A.start[p] = carve<int64_t>(oc, num + 1);
            A.count[p] = carve<int32_t>(oc, num + 1);
            P->off[p] = carve<int64_t>(oc, num + 1);
            P->pairs[p] = carve<vr_pair>(oc, cap[p] + 1);
            P->edges[p] = carve<int32_t>(oc, 4 * (cap[p] + 1));
            A.cap[p] = cap[p];
        }
        A.thr_used = carve<float>(oc, num + 1);
        A.cloud_err = carve<int32_t>(oc, num + 1);
        A.pts = P->pts; A.offs = P->offs; A.order = P->order;
        A.num = num; A.dim = dim; A.dmax = dmax;
        A.thr_bits = thr_bits; A.thr_inf = thr_inf; A.want_edges = want_edges;
        VR_CUDA(cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem)));
    } catch (...) {
        free_plan(P);
        throw;
    }
    return P;
}

// Launch shape: persistent blocks per SM (1 or 2), picked by timing both on
// the first batch of more clouds than SMs of a given size bucket (mean cloud
// size and number of clouds) and remembered per device.
int tuned_slots(BatchPlan& P, cudaStream_t s, int sms, int64_t bucket) {
    // no more clouds than SMs: one block per SM runs every cloud at once, each
    // alone on its SM; nothing is timed or remembered (a batch this small would
    // time both shapes alike and fix the choice for larger batches)
    if (P.num <= sms) return 1;
    const auto key = std::make_pair(P.device, bucket);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
    const char* env = getenv("VR_BATCH_BLOCKS_PER_SM");
    if (env && (env[0] == '1' || env[0] == '2')) return g_tuned[key] = env[0] - '0';
    // one untimed launch (module load, caches), then each choice twice in
    // alternation; the smaller of each pair counts (a single timing each
    // picked the slower choice often enough to swing the batched rate by 1.5x)
    float best[3] = {0.f, 1e30f, 1e30f};
    cudaEvent_t e0, e1;
    VR_CUDA(cudaEventCreate(&e0));
    VR_CUDA(cudaEventCreate(&e1));
    P.slots = sms * 2;  // the scratch is sized for 2 blocks per SM
    record_launches(P, s);
    for (int rep = 0; rep < 2; ++rep)
        for (int per = 1; per <= 2; ++per) {
            P.slots = sms * per;
            VR_CUDA(cudaEventRecord(e0, s));
            record_launches(P, s);
            VR_CUDA(cudaEventRecord(e1, s));
            VR_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            VR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best[per] = std::min(best[per], ms);
        }
    const int pick = best[1] <= best[2] ? 1 : 2;
    if (log_enabled()) fprintf(stderr, "[vr] batch launch shape: %.3f ms at 1 block per SM, %.3f ms at 2: %d\n",
                               best[1], best[2], pick);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return g_tuned[key] = pick;
}

}  // namespace
}  // namespace vr

namespace vr {
namespace {

// The batched computation; with `dres` the pairs and critical edges end in
// device memory (dev->pairs / dev->critical_edges, cudaMalloc) instead of
// the host arrays of *out (whose pairs / critical_edges are then NULL).
vr_status batched_impl(const float* pts, const int64_t* offsets, int32_t num_clouds, int32_t ambient_dim,
                       int32_t dmax, float threshold, uint32_t flags, void* stream, vr_batch_result** out,
                       vr_batch_device_result* dres) {
    if (!out) return VR_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_clouds < 0 || !offsets || (num_clouds > 0 && !pts) || ambient_dim < 1 || ambient_dim > BMAXDIM ||
        dmax < 0 || dmax > 1 || std::isnan(threshold) || (flags & ~(uint32_t)(VR_CRITICAL_EDGES | VR_DEBUG_CHECKS)))
        return VR_ERR_INVALID_ARG;
    if (offsets[0] != 0) return VR_ERR_INVALID_ARG;
    int64_t total = 0, sumsq = 0;
    for (int i = 0; i < num_clouds; ++i) {
        const int64_t n = offsets[i + 1] - offsets[i];
        if (n < 1 || n > BMAXN) return VR_ERR_INVALID_ARG;
        total += n;
        sumsq += n * (n - 1) / 2;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    vr_batch_result* res = nullptr;
    try {
        res = (vr_batch_result*)calloc(1, sizeof(vr_batch_result));
        if (!res) throw Error{VR_ERR_OOM};
        res->num_clouds = num_clouds;
        res->dmax = dmax;
        res->thresholds = (float*)calloc(num_clouds + 1, sizeof(float));
        for (int p = 0; p < 2; ++p) res->pair_offsets[p] = (int64_t*)calloc(num_clouds + 1, sizeof(int64_t));
        if (!res->thresholds || !res->pair_offsets[0] || !res->pair_offsets[1]) throw Error{VR_ERR_OOM};
        if (num_clouds == 0 || threshold < 0) {
            for (int p = 0; p <= dmax; ++p) {
                if (dres) {
                    VR_CUDA(cudaMallocAsync((void**)&dres->pairs[p], sizeof(vr_pair), s));
                    if (flags & VR_CRITICAL_EDGES)
                        VR_CUDA(cudaMallocAsync((void**)&dres->critical_edges[p], 4 * sizeof(int32_t), s));
                } else {
                    res->pairs[p] = (vr_pair*)malloc(sizeof(vr_pair));
                }
            }
            for (int i = 0; i < num_clouds; ++i) res->thresholds[i] = threshold;
            *out = res;
            return VR_OK;
        }
        int dev = 0;
        VR_CUDA(cudaGetDevice(&dev));
        int sms = 148;
        VR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int want_edges = (flags & VR_CRITICAL_EDGES) ? 1 : 0;
        const int thr_inf = (std::isinf(threshold) && threshold > 0) ? 1 : 0;
        uint32_t thr_bits = 0;
        if (!thr_inf) memcpy(&thr_bits, &threshold, 4);
        int64_t cap[2] = {total, (int64_t)num_clouds * 64 + 1024};
        // plan (device buffers and graph) reused while the shape is unchanged
        BatchPlan* P = g_plan;
        const bool same = P && P->device == dev && P->num == num_clouds && P->dim == ambient_dim && P->dmax == dmax &&
                          P->want_edges == want_edges && P->thr_inf == thr_inf && P->thr_bits == thr_bits &&
                          P->total == total;
        if (!same) {
            free_plan(g_plan);
            g_plan = nullptr;
            P = g_plan = make_plan(dev, num_clouds, ambient_dim, dmax, want_edges, thr_inf, thr_bits, total, 2 * sms,
                                   cap);
        }
        // inputs
        std::vector<int32_t> order(num_clouds);
        for (int i = 0; i < num_clouds; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
        });
        cudaPointerAttributes pa;
        bool dev_in = cudaPointerGetAttributes(&pa, pts) == cudaSuccess &&
                      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        VR_CUDA(cudaMemcpyAsync(P->pts, pts, total * ambient_dim * sizeof(float),
                                dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        VR_CUDA(cudaMemcpyAsync(P->offs, offsets, (num_clouds + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        VR_CUDA(cudaMemcpyAsync(P->order, order.data(), num_clouds * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        // tuned per (mean cloud size / 32, number of clouds rounded up to a power of
        // two): the better shape depends on both
        int lg = 0;
        while ((1 << lg) < num_clouds) ++lg;
        const int64_t bucket = (total / num_clouds / 32) * 64 + lg;
        const int per = tuned_slots(*P, s, sms, bucket);
        if (P->slots != per * sms || !P->exec || P->captured_on != s) {
            P->slots = per * sms;
            if (P->exec) { cudaGraphExecDestroy(P->exec); P->exec = nullptr; }
            cudaGraph_t g;
            cudaStream_t cs;
            VR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            VR_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            record_launches(*P, cs);
            VR_CUDA(cudaStreamEndCapture(cs, &g));
            VR_CUDA(cudaGraphInstantiate(&P->exec, g, 0));
            cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            P->captured_on = s;
        }
        VR_CUDA(cudaGraphLaunch(P->exec, s));
        // host reads, one wait: usage, per-cloud errors, thresholds, pair offsets
        unsigned long long used[2] = {0, 0};
        std::vector<int32_t> cerr(num_clouds);
        auto read_back = [&]() {
            VR_CUDA(cudaMemcpyAsync(used, P->args.used, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaMemcpyAsync(cerr.data(), P->args.cloud_err, num_clouds * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaMemcpyAsync(res->thresholds, P->args.thr_used, num_clouds * sizeof(float),
                                    cudaMemcpyDeviceToHost, s));
            for (int p = 0; p <= dmax; ++p)
                VR_CUDA(cudaMemcpyAsync(res->pair_offsets[p], P->off[p], (num_clouds + 1) * sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
        };
        read_back();
        if ((int64_t)used[0] > P->cap[0] || (int64_t)used[1] > P->cap[1]) {
            // output larger than planned: rebuild with room and rerun once
            int64_t ncap[2] = {std::max<int64_t>(P->cap[0], used[0]), std::max<int64_t>(P->cap[1], used[1] + 1024)};
            free_plan(g_plan);
            P = g_plan = make_plan(dev, num_clouds, ambient_dim, dmax, want_edges, thr_inf, thr_bits, total, per * sms,
                                   ncap);
            VR_CUDA(cudaMemcpyAsync(P->pts, pts, total * ambient_dim * sizeof(float),
                                    dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
            VR_CUDA(cudaMemcpyAsync(P->offs, offsets, (num_clouds + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            VR_CUDA(cudaMemcpyAsync(P->order, order.data(), num_clouds * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            record_launches(*P, s);
            read_back();
        }
        if (P->args.prof) {
            unsigned long long pr[16], st[4];
            VR_CUDA(cudaMemcpy(pr, P->args.prof, sizeof pr, cudaMemcpyDeviceToHost));
            VR_CUDA(cudaMemcpy(st, P->args.stats, sizeof st, cudaMemcpyDeviceToHost));
            const char* names[8] = {"distances+threshold", "H0 tree + apparent", "H0 output", "clear+sort",
                                    "first pass", "finalize", "bitmap engine", "H1 output"};
            for (int i = 0; i < 8; ++i) fprintf(stderr, "[vr] batch %-20s %14llu cycles (all clouds, cumulative)\n", names[i], pr[i]);
            fprintf(stderr, "[vr] batch: candidates %llu apparent %llu columns %llu additions %llu, block-engine columns %llu\n",
                    st[0], st[1], st[2], st[3], pr[8]);
            std::vector<unsigned long long> pc(num_clouds);
            VR_CUDA(cudaMemcpy(pc.data(), P->args.prof + 16, num_clouds * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost));
            std::vector<int> ix(num_clouds);
            for (int i = 0; i < num_clouds; ++i) ix[i] = i;
            std::sort(ix.begin(), ix.end(), [&](int a, int b) { return pc[a] > pc[b]; });
            for (int t = 0; t < std::min(num_clouds, 8); ++t)
                fprintf(stderr, "[vr] batch slowest cloud %d: n=%lld, %llu cycles\n", ix[t],
                        (long long)(offsets[ix[t] + 1] - offsets[ix[t]]), pc[ix[t]]);
            VR_CUDA(cudaMemset(P->args.prof, 0, 16 * sizeof(unsigned long long)));
        }
        // results in cloud order
        std::vector<int> bad;
        int codes[8] = {0};
        for (int i = 0; i < num_clouds; ++i)
            if (cerr[i]) { bad.push_back(i); codes[cerr[i] & 7]++; }
        res->recomputed = (int32_t)bad.size();
        if (log_enabled() && !bad.empty())
            fprintf(stderr, "[vr] batch: %zu clouds recomputed singly (codes 1:%d 2:%d 3:%d 4:%d)\n", bad.size(),
                    codes[1], codes[2], codes[3], codes[4]);
        // clouds that outgrew a per-block buffer: recompute with the single-cloud path
        std::vector<vr_result*> redo(bad.size(), nullptr);
        for (size_t b = 0; b < bad.size(); ++b) {
            const int i = bad[b];
            const int64_t n = offsets[i + 1] - offsets[i];
            vr_status st = vr_barcodes_points(P->pts + offsets[i] * ambient_dim, n, ambient_dim, dmax, threshold,
                                              flags, stream, &redo[b]);
            if (st != VR_OK) {
                for (auto r : redo) vr_result_free(r);
                throw Error{st};
            }
        }
        for (int p = 0; p <= dmax; ++p) {
            std::vector<int64_t> cnt(num_clouds);
            for (int i = 0; i < num_clouds; ++i) cnt[i] = res->pair_offsets[p][i + 1] - res->pair_offsets[p][i];
            for (size_t b = 0; b < bad.size(); ++b) cnt[bad[b]] = redo[b]->count[p];
            std::vector<int64_t> off(num_clouds + 1, 0);
            for (int i = 0; i < num_clouds; ++i) off[i + 1] = off[i] + cnt[i];
            if (dres) {
                const int64_t tot = std::max<int64_t>(off[num_clouds], 1);
                VR_CUDA(cudaMallocAsync((void**)&dres->pairs[p], tot * sizeof(vr_pair), s));
                if (want_edges) VR_CUDA(cudaMallocAsync((void**)&dres->critical_edges[p], tot * 4 * sizeof(int32_t), s));
                if (bad.empty()) {  // already in cloud order on the device
                    VR_CUDA(cudaMemcpyAsync(dres->pairs[p], P->pairs[p], off[num_clouds] * sizeof(vr_pair),
                                            cudaMemcpyDeviceToDevice, s));
                    if (want_edges)
                        VR_CUDA(cudaMemcpyAsync(dres->critical_edges[p], P->edges[p],
                                                off[num_clouds] * 4 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                    // stream-ordered: the caller reads the arrays on `stream` (no wait here)
                    memcpy(res->pair_offsets[p], off.data(), (num_clouds + 1) * sizeof(int64_t));
                    continue;
                }
            }
            res->pairs[p] = (vr_pair*)malloc(std::max<int64_t>(off[num_clouds], 1) * sizeof(vr_pair));
            if (want_edges)
                res->critical_edges[p] = (int32_t*)malloc(std::max<int64_t>(off[num_clouds], 1) * 4 * sizeof(int32_t));
            if (!res->pairs[p] || (want_edges && !res->critical_edges[p])) throw Error{VR_ERR_OOM};
            if (bad.empty()) {
                copy_to_host(*P, res->pairs[p], P->pairs[p], off[num_clouds] * sizeof(vr_pair), s);
                if (want_edges)
                    copy_to_host(*P, res->critical_edges[p], P->edges[p], off[num_clouds] * 4 * sizeof(int32_t), s);
            } else {
                std::vector<vr_pair> dv(std::max<int64_t>(res->pair_offsets[p][num_clouds], 1));
                std::vector<int32_t> de(want_edges ? 4 * dv.size() : 0);
                VR_CUDA(cudaMemcpyAsync(dv.data(), P->pairs[p], res->pair_offsets[p][num_clouds] * sizeof(vr_pair),
                                        cudaMemcpyDeviceToHost, s));
                if (want_edges)
                    VR_CUDA(cudaMemcpyAsync(de.data(), P->edges[p],
                                            res->pair_offsets[p][num_clouds] * 4 * sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, s));
                VR_CUDA(cudaStreamSynchronize(s));
                size_t b = 0;
                for (int i = 0; i < num_clouds; ++i) {
                    if (b < bad.size() && bad[b] == i) {
                        memcpy(res->pairs[p] + off[i], redo[b]->pairs[p], cnt[i] * sizeof(vr_pair));
                        if (want_edges)
                            for (int64_t q = 0; q < 4 * cnt[i]; ++q) {
                                const int32_t e = redo[b]->critical_edges[p][q];
                                res->critical_edges[p][4 * off[i] + q] = e >= 0 ? (int32_t)(e + offsets[i]) : -1;
                            }
                        if (p == 0) res->thresholds[i] = redo[b]->threshold;
                        ++b;
                    } else {
                        memcpy(res->pairs[p] + off[i], dv.data() + res->pair_offsets[p][i], cnt[i] * sizeof(vr_pair));
                        if (want_edges) memcpy(res->critical_edges[p] + 4 * off[i], de.data() + 4 * res->pair_offsets[p][i],
                                               cnt[i] * 4 * sizeof(int32_t));
                    }
                }
            }
            memcpy(res->pair_offsets[p], off.data(), (num_clouds + 1) * sizeof(int64_t));
            if (dres) {  // clouds recomputed on the host path: upload the assembled arrays
                VR_CUDA(cudaMemcpyAsync(dres->pairs[p], res->pairs[p], off[num_clouds] * sizeof(vr_pair),
                                        cudaMemcpyHostToDevice, s));
                if (want_edges)
                    VR_CUDA(cudaMemcpyAsync(dres->critical_edges[p], res->critical_edges[p],
                                            off[num_clouds] * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
                VR_CUDA(cudaStreamSynchronize(s));
                free(res->pairs[p]);
                free(res->critical_edges[p]);
                res->pairs[p] = nullptr;
                res->critical_edges[p] = nullptr;
            }
        }
        for (auto r : redo) vr_result_free(r);
        (void)sumsq;
        if ((flags & VR_DEBUG_CHECKS) && !dres) {
            // per cloud: n_i - 1 finite H0 pairs at most, one essential H0 class at least,
            // birth <= death, and the documented order within the cloud
            for (int p = 0; p <= dmax; ++p)
                for (int i = 0; i < num_clouds; ++i) {
                    const int64_t a0 = res->pair_offsets[p][i], a1 = res->pair_offsets[p][i + 1];
                    int64_t ess = 0;
                    for (int64_t k = a0; k < a1; ++k) {
                        const vr_pair& x = res->pairs[p][k];
                        VR_CHECK(x.birth <= x.death && x.birth >= 0.0f, VR_ERR_INTERNAL);
                        ess += x.death_simplex < 0;
                        if (k > a0) {
                            const vr_pair& y = res->pairs[p][k - 1];
                            VR_CHECK(y.birth < x.birth || (y.birth == x.birth && (y.death < x.death ||
                                     (y.death == x.death && y.birth_simplex <= x.birth_simplex))), VR_ERR_INTERNAL);
                        }
                    }
                    if (p == 0) VR_CHECK(ess >= 1 && a1 - a0 <= offsets[i + 1] - offsets[i], VR_ERR_INTERNAL);
                }
        }
        *out = res;
        return VR_OK;
    } catch (const Error& e) {
        vr_batch_result_free(res);
        return e.code;
    } catch (const std::bad_alloc&) {
        vr_batch_result_free(res);
        return VR_ERR_OOM;
    }
}

}  // namespace
}  // namespace vr

extern "C" vr_status vr_barcodes_batched(const float* pts, const int64_t* offsets, int32_t num_clouds,
                                         int32_t ambient_dim, int32_t dmax, float threshold, uint32_t flags,
                                         void* stream, vr_batch_result** out) {
    return vr::batched_impl(pts, offsets, num_clouds, ambient_dim, dmax, threshold, flags, stream, out, nullptr);
}

extern "C" vr_status vr_barcodes_batched_device(const float* pts, const int64_t* offsets, int32_t num_clouds,
                                                int32_t ambient_dim, int32_t dmax, float threshold, uint32_t flags,
                                                void* stream, vr_batch_device_result** out) {
    if (!out) return VR_ERR_INVALID_ARG;
    *out = nullptr;
    vr_batch_device_result* d = (vr_batch_device_result*)calloc(1, sizeof(vr_batch_device_result));
    if (!d) return VR_ERR_OOM;
    d->stream = stream;
    vr_batch_result* r = nullptr;
    const vr_status st =
        vr::batched_impl(pts, offsets, num_clouds, ambient_dim, dmax, threshold, flags, stream, &r, d);
    if (st != VR_OK) {
        vr_batch_device_result_free(d);
        return st;
    }
    d->num_clouds = r->num_clouds;
    d->dmax = r->dmax;
    for (int p = 0; p < 2; ++p) {  // the host offsets and thresholds move over
        d->pair_offsets[p] = r->pair_offsets[p];
        r->pair_offsets[p] = nullptr;
    }
    d->thresholds = r->thresholds;
    r->thresholds = nullptr;
    d->recomputed = r->recomputed;
    vr_batch_result_free(r);
    *out = d;
    return VR_OK;
}

extern "C" void vr_batch_device_result_free(vr_batch_device_result* r) {
    if (!r) return;
    for (int p = 0; p < 2; ++p) {
        free(r->pair_offsets[p]);
        if (r->pairs[p]) cudaFreeAsync(r->pairs[p], (cudaStream_t)r->stream);
        if (r->critical_edges[p]) cudaFreeAsync(r->critical_edges[p], (cudaStream_t)r->stream);
    }
    free(r->thresholds);
    free(r);
}

extern "C" void vr_batch_result_free(vr_batch_result* r) {
    if (!r) return;
    for (int p = 0; p < 2; ++p) {
        free(r->pair_offsets[p]);
        free(r->pairs[p]);
        free(r->critical_edges[p]);
    }
    free(r->thresholds);
    free(r);
}
