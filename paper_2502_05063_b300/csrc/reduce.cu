// reduce.cu -- Z/2 reduction of the non-apparent columns of the coboundary
// matrix (paper: Algorithm 12, oblivious column reduction, Lemma 5.2.10;
// cohomology, Sec. 5.2.4; implicit matrix, Sec. 5.2.8; two-layer pair store,
// Sec. 5.5.1).
//
// Rows are (p+1)-simplices identified by a 64-bit row key
//     (diameter rank << row_cidx_bits) | (row_mask - cidx),
// so the pivot ("low") of a column -- the cofacet first in the simplex-wise
// filtration order -- is its smallest row key.  A column is the sum over Z/2
// of the coboundaries D_x of a set of p-simplices; D_x is never stored but
// generated from the vertices of x (one lane per added vertex w).
//
// Parallel schedule (B300 design; the paper reduces these columns
// sequentially on the CPU).  Columns c_0 < c_1 < ... are in coboundary
// order.  Each round, every unfinished column is reduced independently
// against the pivots known so far (apparent pairs + finalized columns) until
// its pivot is unknown, or a per-round budget of additions runs out.  Then,
// in order, column j is finalized iff its reduction completed and its pivot
// key is smaller than the current pivot key of every earlier unfinished
// column.  This is exact: the finished low of column i is the smallest low
// over D_i + span(D_<i), so every partial state of i bounds its final pivot
// key from below; a pivot key of j below all those bounds cannot be the
// final pivot of any earlier column, and a vector of D_j + span(D_<j) whose
// low is no earlier column's pivot has the low of the fully reduced column
// (the argument behind Lemma 5.2.10).  Columns finalized in one round have
// strictly decreasing keys, hence distinct pivots.  When a round makes no
// progress or few columns remain, one warp finishes them in order, which is
// Algorithm 12 verbatim.
//
// Pivot lookup (the paper's two-layer store, Fig 5.10): first a device hash
// of pivots found by this reduction, then the apparent pairs, which are not
// stored at all: t is owned by an apparent column iff its youngest facet s'
// (drop the largest vertex whose removal keeps diam) has t as its oldest
// cofacet (no larger added vertex keeps diam) -- Def 5.3.4 evaluated on the
// fly in one warp.  No wait in this file spins on another thread.
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "vr_common.cuh"

namespace vr {

namespace {

constexpr uint64_t EMPTY = ~0ull;
constexpr int RED_WARPS = 4;      // warps per block, round mode
constexpr int STAGE = 1024;       // per-warp shared staging of generated rows
constexpr uint8_t ST_COMPLETE = 0, ST_BUDGET = 1, ST_OVERFLOW = 2;

struct Ctx {
    RankMatrix R;
    Binom B;
    uint32_t thr;
    int cb, rcb;
    uint64_t cmask, rcmask, rmask;
    const uint64_t* cols;
    int64_t num_cols;
    uint64_t* hkeys;   // pivot cidx (EMPTY = free)
    uint32_t* hvals;   // column position
    uint64_t hmask;
    int* err;
    // finished columns that needed additions keep their reduced form R_j here,
    // so a later column adds R_j (standard reduction) instead of D_j
    uint64_t* pool;
    unsigned long long* pool_used;
    int64_t pool_cap;
    uint64_t* rc_off;  // per column position
    uint32_t* rc_len;  // 0: the column is its own coboundary D_j
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
    return x;
}

template <int P>
struct Simplex {
    int v[P + 1];   // ascending
    uint32_t r;     // diameter rank
    uint64_t cidx;
};

template <int P>
__device__ __forceinline__ void load_col(const Ctx& c, uint64_t key, Simplex<P>& s) {
    s.cidx = key & c.cmask;
    s.r = (uint32_t)((~(key >> c.cb)) & c.rmask);
    decode_simplex<P>(c.B, s.cidx, c.R.n - 1, s.v);
}

template <int P>
__device__ __forceinline__ uint64_t col_key(const Ctx& c, const Simplex<P>& s) {
    return ((~(uint64_t)s.r & c.rmask) << c.cb) | s.cidx;
}

// index of s + {w}, w not a vertex of s (eq. 5.6 with w inserted in place)
template <int P>
__device__ __forceinline__ uint64_t cofacet_cidx(const Binom& B, const int* v, int64_t w) {
    uint64_t ct = 0;
    int k = 0;
    bool placed = false;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
        if (!placed && w < v[a]) { ct += B(w, k + 1); ++k; placed = true; }
        ct += B(v[a], k + 1);
        ++k;
    }
    if (!placed) ct += B(w, k + 1);
    return ct;
}

template <int P>
__device__ __forceinline__ uint64_t row_key(const Ctx& c, const Simplex<P>& s, int64_t w, uint32_t rt) {
    return ((uint64_t)rt << c.rcb) | (c.rcmask - cofacet_cidx<P>(c.B, s.v, w));
}

// Pivot of the unreduced column D_s: smallest (rank asc, w desc) cofacet.
template <int P>
__device__ uint64_t warp_column_pivot(const Ctx& c, const Simplex<P>& s) {
    const int lane = threadIdx.x & 31;
    const int64_t n = c.R.n;
    uint32_t brt = 0xFFFFFFFFu;
    int64_t bw = -1;
    for (int64_t base = n - 1; base >= 0; base -= 32) {
        const int64_t w = base - lane;
        bool ok = w >= 0;
#pragma unroll
        for (int a = 0; a <= P; ++a) ok = ok && (w != s.v[a]);
        if (ok) {
            uint32_t rt = s.r;
#pragma unroll
            for (int a = 0; a <= P; ++a) rt = max(rt, c.R(s.v[a], w));
            if (rt <= c.thr && rt < brt) { brt = rt; bw = w; }  // w only decreases per lane
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint32_t ort = __shfl_xor_sync(0xffffffffu, brt, o);
        int64_t ow = __shfl_xor_sync(0xffffffffu, bw, o);
        if (ort < brt || (ort == brt && ow > bw)) { brt = ort; bw = ow; }
    }
    if (bw < 0) return EMPTY;
    return row_key<P>(c, s, bw, brt);
}

// Bitonic sort of stage[0..len) (len a power of two >= 32) by one warp.
__device__ void warp_bitonic(uint64_t* stage, int len) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= len; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < len; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = stage[i], b = stage[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { stage[i] = b; stage[ixj] = a; }
                }
            }
            __syncwarp();
        }
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t len, uint64_t x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// out = in XOR S (symmetric difference of two sorted sets), returns the new
// size or -1 if it would exceed cap.
__device__ int64_t warp_xor_merge(const uint64_t* in, int64_t a, const uint64_t* S, int64_t b, uint64_t* out,
                                  int64_t cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int64_t matched = 0;
    bool over = false;
    for (int64_t base = 0; base < a; base += 32) {
        const int64_t i = base + lane;
        const uint64_t x = i < a ? in[i] : EMPTY;
        int64_t bs = 0;
        bool m = false;
        if (i < a) {
            bs = lower_bound_u64(S, b, x);
            m = bs < b && S[bs] == x;
        }
        const uint32_t mb = __ballot_sync(0xffffffffu, m);
        const int64_t mw = matched + __popc(mb & lt);
        if (i < a && !m) {
            const int64_t pos = i + bs - 2 * mw;
            if (pos < cap) out[pos] = x; else over = true;
        }
        matched += __popc(mb);
    }
    int64_t matched2 = 0;
    for (int64_t base = 0; base < b; base += 32) {
        const int64_t k = base + lane;
        const uint64_t y = k < b ? S[k] : EMPTY;
        int64_t bw = 0;
        bool m = false;
        if (k < b) {
            bw = lower_bound_u64(in, a, y);
            m = bw < a && in[bw] == y;
        }
        const uint32_t mb = __ballot_sync(0xffffffffu, m);
        const int64_t ms = matched2 + __popc(mb & lt);
        if (k < b && !m) {
            const int64_t pos = k + bw - 2 * ms;
            if (pos < cap) out[pos] = y; else over = true;
        }
        matched2 += __popc(mb);
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, over)) return -1;
    return a + b - 2 * matched;
}

// W <- W + D_x.  W lives in *W (size a) and the spare buffer *spare; the
// pointers are swapped as pieces are merged.  Returns the new size or -1.
template <int P>
__device__ int64_t warp_add_coboundary(const Ctx& c, const Simplex<P>& x, uint64_t* stage, uint64_t*& W,
                                       uint64_t*& spare, int64_t a, int64_t cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t n = c.R.n;
    int64_t base = n - 1;
    while (base >= 0) {
        int fill = 0;
        while (base >= 0 && fill <= STAGE - 32) {
            const int64_t w = base - lane;
            bool ok = w >= 0;
#pragma unroll
            for (int q = 0; q <= P; ++q) ok = ok && (w != x.v[q]);
            uint32_t rt = x.r;
            if (ok) {
#pragma unroll
                for (int q = 0; q <= P; ++q) rt = max(rt, c.R(x.v[q], w));
                ok = rt <= c.thr;
            }
            const uint32_t b = __ballot_sync(0xffffffffu, ok);
            if (ok) stage[fill + __popc(b & lt)] = row_key<P>(c, x, w, rt);
            fill += __popc(b);
            base -= 32;
        }
        int len = 32;
        while (len < fill) len <<= 1;
        for (int i = fill + lane; i < len; i += 32) stage[i] = EMPTY;
        __syncwarp();
        warp_bitonic(stage, len);
        const int64_t na = warp_xor_merge(W, a, stage, fill, spare, cap);
        __syncwarp();
        if (na < 0) return -1;
        uint64_t* t = W; W = spare; spare = t;
        a = na;
    }
    return a;
}

// Position of the finished column whose pivot is the (p+1)-simplex ct, or -1;
// one warp probes 32 slots of the open-addressing table at a time.
__device__ int64_t warp_hash_find(const Ctx& c, uint64_t ct) {
    const int lane = threadIdx.x & 31;
    const uint64_t slot0 = mix64(ct) & c.hmask;
    for (uint64_t probe = 0; probe <= c.hmask; probe += 32) {
        const uint64_t sl = (slot0 + probe + lane) & c.hmask;
        const uint64_t k = c.hkeys[sl];
        const uint32_t hit = __ballot_sync(0xffffffffu, k == ct);
        const uint32_t emp = __ballot_sync(0xffffffffu, k == EMPTY);
        if (hit && (!emp || __ffs(hit) < __ffs(emp)))
            return (int64_t)__shfl_sync(0xffffffffu, c.hvals[sl], __ffs(hit) - 1);
        if (emp) break;
    }
    return -1;
}

// Owner of pivot row key rk among the columns before `self_key` in order:
// returns true and fills `o`, or false if rk is no known pivot.
template <int P>
__device__ bool warp_owner(const Ctx& c, uint64_t rk, uint64_t self_key, Simplex<P>& o, int64_t& opos) {
    constexpr int NT = P + 2;
    constexpr int NPAIR = NT * (NT - 1) / 2;
    const int lane = threadIdx.x & 31;
    const int64_t n = c.R.n;
    const uint32_t rt = (uint32_t)(rk >> c.rcb);
    const uint64_t ct = c.rcmask - (rk & c.rcmask);
    // 1. pivots of reduced columns
    {
        const int64_t pos = warp_hash_find(c, ct);
        if (pos >= 0) {
            const uint64_t okey = c.cols[pos];
            if (!(okey < self_key)) atomicExch(c.err, DEV_INTERNAL);
            load_col<P>(c, okey, o);
            opos = pos;
            return true;
        }
    }
    // 2. apparent pairs (Def 5.3.4), recomputed
    int tv[NT];
    decode_simplex<P + 1>(c.B, ct, n - 1, tv);
    bool eq = false;
    int pi = 0, pj = 0;
    if (lane < NPAIR) {
        int k = lane;
        pi = 1;
        while (k >= pi) { k -= pi; ++pi; }
        pj = k;
        eq = c.R(tv[pi], tv[pj]) == rt;
    }
    int drop = -1;
#pragma unroll
    for (int m = NT - 1; m >= 0; --m) {  // largest vertex first = smallest facet index
        if (drop < 0 && __ballot_sync(0xffffffffu, eq && pi != m && pj != m)) drop = m;
    }
    if (drop < 0) return false;
    int k = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q)
        if (q != drop) o.v[k++] = tv[q];
    const int64_t wd = tv[drop];
    for (int64_t base = n - 1; base > wd; base -= 32) {
        const int64_t w = base - lane;
        bool ok = w > wd;
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (w != o.v[q]);
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (c.R(o.v[q], w) <= rt);
        if (__ballot_sync(0xffffffffu, ok)) return false;  // an older cofacet of s' exists
    }
    o.r = rt;
    uint64_t cs = 0;
#pragma unroll
    for (int q = 0; q <= P; ++q) cs += c.B(o.v[q], q + 1);
    o.cidx = cs;
    if (!(col_key<P>(c, o) < self_key)) atomicExch(c.err, DEV_INTERNAL);
    opos = -1;
    return true;
}

// W <- W + R_o: the stored reduced column of a finished column, or its
// coboundary when none is stored (apparent columns, zero-addition columns).
template <int P>
__device__ int64_t warp_add_owner(const Ctx& c, const Simplex<P>& o, int64_t opos, uint64_t* stage, uint64_t*& W,
                                  uint64_t*& spare, int64_t a, int64_t cap) {
    if (opos >= 0) {
        const uint32_t len = c.rc_len[opos];
        if (len) {
            const int64_t na = warp_xor_merge(W, a, c.pool + c.rc_off[opos], len, spare, cap);
            __syncwarp();
            if (na < 0) return -1;
            uint64_t* t = W; W = spare; spare = t;
            return na;
        }
    }
    return warp_add_coboundary<P>(c, o, stage, W, spare, a, cap);
}

// Keep the reduced column of position j (W[0..a)) for later additions.
__device__ void store_reduced(const Ctx& c, int64_t j, const uint64_t* W, int64_t a) {
    const int lane = threadIdx.x & 31;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(c.pool_used, (unsigned long long)a);
    off = __shfl_sync(0xffffffffu, off, 0);
    const bool fits = (int64_t)(off + a) <= c.pool_cap && a <= 0xFFFFFFFFll;
    if (fits)
        for (int64_t i = lane; i < a; i += 32) c.pool[off + i] = W[i];
    __syncwarp();
    if (lane == 0) {
        c.rc_off[j] = off;
        c.rc_len[j] = fits ? (uint32_t)a : 0u;  // no room: later additions regenerate D_j
    }
}

// Reduce column j (position in cols) against the known pivots.  At most
// `budget` additions; on completion with additions the result is stored.
template <int P>
__device__ void reduce_one(const Ctx& c, int64_t j, int budget, uint64_t* stage, uint64_t* bufA, uint64_t* bufB,
                           int64_t cap, uint64_t& out_key, uint8_t& out_status, uint32_t& out_adds) {
    const int lane = threadIdx.x & 31;
    const uint64_t self_key = c.cols[j];
    Simplex<P> s, o;
    int64_t opos = -1;
    load_col<P>(c, self_key, s);
    uint64_t piv = warp_column_pivot<P>(c, s);
    out_adds = 0;
    if (lane == 0) c.rc_len[j] = 0;
    if (piv == EMPTY) { out_key = EMPTY; out_status = ST_COMPLETE; return; }
    if (!warp_owner<P>(c, piv, self_key, o, opos)) { out_key = piv; out_status = ST_COMPLETE; return; }
    uint64_t* W = bufA;
    uint64_t* spare = bufB;
    int64_t a = warp_add_coboundary<P>(c, s, stage, W, spare, 0, cap);
    if (a < 0) { out_key = piv; out_status = ST_OVERFLOW; return; }
    uint32_t adds = 0;
    for (;;) {
        if ((int)adds >= budget) { out_key = piv; out_status = ST_BUDGET; out_adds = adds; return; }
        const int64_t na = warp_add_owner<P>(c, o, opos, stage, W, spare, a, cap);
        if (na < 0) { out_key = piv; out_status = ST_OVERFLOW; out_adds = adds; return; }
        ++adds;
        a = na;
        if (a == 0) { out_key = EMPTY; out_status = ST_COMPLETE; out_adds = adds; return; }
        piv = W[0];
        if (!warp_owner<P>(c, piv, self_key, o, opos)) {
            out_key = piv;
            out_status = ST_COMPLETE;
            out_adds = adds;
            store_reduced(c, j, W, a);
            return;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(RED_WARPS * 32)
k_reduce_round(Ctx c, const uint32_t* __restrict__ U, int64_t u, int budget, uint64_t* __restrict__ cur_key,
               uint8_t* __restrict__ status, uint32_t* __restrict__ adds, uint64_t* __restrict__ scratch,
               int64_t cap, unsigned long long* __restrict__ work) {
    __shared__ uint64_t stage_all[RED_WARPS][STAGE];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t slot = (int64_t)blockIdx.x * RED_WARPS + wid;
    uint64_t* bufA = scratch + slot * 2 * cap;
    uint64_t* bufB = bufA + cap;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(work, 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        if ((int64_t)k >= u) break;
        const int64_t j = U[k];
        uint64_t key;
        uint8_t st;
        uint32_t ad;
        reduce_one<P>(c, j, budget, stage_all[wid], bufA, bufB, cap, key, st, ad);
        if (lane == 0) { cur_key[j] = key; status[j] = st; adds[j] = ad; }
    }
}

__device__ void hash_insert(const Ctx& c, uint64_t key, uint32_t val) {
    uint64_t sl = mix64(key) & c.hmask;
    for (uint64_t probe = 0; probe <= c.hmask; ++probe) {
        const unsigned long long prev =
            atomicCAS(reinterpret_cast<unsigned long long*>(c.hkeys + sl), (unsigned long long)EMPTY,
                      (unsigned long long)key);
        if (prev == EMPTY || prev == key) { c.hvals[sl] = val; return; }
        sl = (sl + 1) & c.hmask;
    }
    atomicExch(c.err, DEV_CAPACITY);
}

struct Emit {
    PairRec* pairs;
    unsigned long long* num_pairs;
    uint32_t* clear_next;
    unsigned long long* counters;  // [0] additions [1] pairs [2] essential
    int keep_zero;
};

// Record the finished column j with pivot key `key` (EMPTY = zero column).
__device__ void finish_column(const Ctx& c, const Emit& e, int64_t j, uint64_t key, uint32_t adds) {
    const uint64_t ckey = c.cols[j];
    const uint64_t cs = ckey & c.cmask;
    const uint32_t rs = (uint32_t)((~(ckey >> c.cb)) & c.rmask);
    PairRec pr;
    pr.birth_rank = rs;
    pr.birth_cidx = cs;
    if (adds) atomicAdd(e.counters + 0, (unsigned long long)adds);
    if (key == EMPTY) {  // zero column of an uncleared simplex: essential class
        pr.death_rank = 0xFFFFFFFFu;
        pr.death_cidx = -1;
        atomicAdd(e.counters + 2, 1ull);
        e.pairs[atomicAdd(e.num_pairs, 1ull)] = pr;
        return;
    }
    const uint32_t rt = (uint32_t)(key >> c.rcb);
    const uint64_t ct = c.rcmask - (key & c.rcmask);
    hash_insert(c, ct, (uint32_t)j);
    if (e.clear_next) atomicOr(e.clear_next + (ct >> 5), 1u << (ct & 31));
    atomicAdd(e.counters + 1, 1ull);
    if (rt > rs || e.keep_zero) {
        pr.death_rank = rt;
        pr.death_cidx = (int64_t)ct;
        e.pairs[atomicAdd(e.num_pairs, 1ull)] = pr;
    }
}

// One block: exclusive prefix-min of the pivot keys over U in order decides
// which columns are final; the rest are compacted, in order, into Unext.
__global__ void __launch_bounds__(1024)
k_finalize(Ctx c, Emit e, const uint32_t* __restrict__ U, int64_t u, const uint64_t* __restrict__ cur_key,
           const uint8_t* __restrict__ status, const uint32_t* __restrict__ adds, uint32_t* __restrict__ Unext,
           unsigned long long* __restrict__ u_next, unsigned long long* __restrict__ first_status) {
    __shared__ uint64_t wmin[32];
    __shared__ uint32_t wcnt[32];
    __shared__ uint64_t carry_min;
    __shared__ uint32_t carry_cnt;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) { carry_min = EMPTY; carry_cnt = 0; }
    __syncthreads();
    for (int64_t base = 0; base < u; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        const bool valid = k < u;
        const uint32_t j = valid ? U[k] : 0;
        const uint64_t key = valid ? cur_key[j] : EMPTY;
        const uint8_t st = valid ? status[j] : ST_COMPLETE;
        // inclusive min-scan within the warp
        uint64_t incl = key;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o && y < incl) incl = y;
        }
        if (lane == 31) wmin[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint64_t t = wmin[lane];
            uint64_t ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o && y < ti) ti = y;
            }
            uint64_t ex = __shfl_up_sync(0xffffffffu, ti, 1);
            wmin[lane] = lane == 0 ? EMPTY : ex;  // exclusive over warps
        }
        __syncthreads();
        uint64_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = EMPTY;
        uint64_t pm = carry_min;
        if (wmin[wid] < pm) pm = wmin[wid];
        if (excl < pm) pm = excl;
        const bool fin = valid && st == ST_COMPLETE && (key == EMPTY || key < pm);
        if (k == 0) *first_status = st;
        if (fin) finish_column(c, e, j, key, adds[j]);
        const bool keep = valid && !fin;
        const uint32_t kb = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcnt[wid] = __popc(kb);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < wid) before += wcnt[w];
            total += wcnt[w];
        }
        if (keep) Unext[carry_cnt + before + __popc(kb & lt)] = j;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            uint64_t cm = carry_min;
            if (wmin[wid] < cm) cm = wmin[wid];
            if (incl < cm) cm = incl;
            carry_min = cm;
            carry_cnt += total;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *u_next = carry_cnt;
}

// ---------------------------------------------------------------------------
// Heavy columns: one 512-thread block per column, state kept across rounds.
//
// A column that needs many additions (the cocycle of a long bar can reach
// hundreds of thousands of rows) is never merged as a whole.  Its rows are
// split at a key Ks: the front F (rows < Ks, sorted, unique, at most FC of
// them) lives in shared memory and is the only part the pivot search reads;
// the back B (rows >= Ks) is an unsorted multiset in global memory to which
// new rows are appended without sorting.  When F runs empty, a most-
// significant-digit radix select over B finds a split T with at most FC/2
// rows below it; those rows are sorted, rows of even multiplicity cancel
// (Z/2), and the rest become the new front with Ks = T.  An addition thus
// costs O(rows added + |F|), independent of the column's size.
// ---------------------------------------------------------------------------
constexpr int HT = 512;          // threads per block
constexpr int HW = HT / 32;
constexpr int FC = 4096;         // front capacity
constexpr int FKEEP = FC - 1024; // front size kept after a spill
constexpr int HSTAGE = 1024;     // rows generated or copied per pass (power of two >= HT)
constexpr int REFILL = FC / 2;   // rows promoted from the back per refill (at most)

struct HeavyState {
    uint64_t* F;       // slots x FC, the front saved between rounds
    uint64_t* B;       // slots x bcap
    int64_t bcap;
    uint64_t* Ks;      // per slot
    int32_t* fsize;
    int64_t* bsize;
    uint8_t* init;     // 0: the column has not been started (or must restart)
    uint32_t* adds;
    unsigned long long* prof;  // VR_LOG only: cycles {refill, lookup, add, resume}, counts {adds, lookups}
};

struct HeavySmem {
    uint64_t buf[2][FC];   // the front and its merge target, swapped after each merge
    uint64_t stage[HSTAGE];
    int ws[HW + 1];
    uint32_t hist[256];
    uint64_t Ks;
    int64_t bsize;
    int64_t opos;
    int fsize;
    int cur;               // which buf holds the front
    int flag;
    int ov[VR_MAX_DIM + 2];
    uint32_t orank;
    uint64_t sel;          // radix-select result
};

// exclusive block scan of one int per thread; *total receives the sum
__device__ __forceinline__ int block_excl_scan(int x, int* ws, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < HW ? ws[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < HW) ws[lane] = ti - t;
        if (lane == HW - 1) ws[HW] = ti;
    }
    __syncthreads();
    const int r = ws[wid] + incl - x;
    *total = ws[HW];
    __syncthreads();
    return r;
}

__device__ void block_bitonic(uint64_t* a, int len) {
    for (int k = 2; k <= len; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < len; i += HT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t x = a[i], y = a[ixj];
                    if ((x > y) == ((i & k) == 0)) { a[i] = y; a[ixj] = x; }
                }
            }
            __syncthreads();
        }
}

// Sort stage[0..cnt) ascending (pads to a power of two with EMPTY).
__device__ void stage_sort(HeavySmem& S, int cnt) {
    if (cnt <= 1) return;
    int len = 2;
    while (len < cnt) len <<= 1;
    for (int i = cnt + threadIdx.x; i < len; i += HT) S.stage[i] = EMPTY;
    __syncthreads();
    block_bitonic(S.stage, len);
}

__device__ __forceinline__ int lower_bound_sm(const uint64_t* a, int len, uint64_t x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Append rows to B; false (and nothing written) if B is full.
__device__ bool heavy_append(HeavySmem& S, uint64_t* B, int64_t bcap, const uint64_t* src, int cnt) {
    const int64_t bs = S.bsize;
    if (bs + cnt > bcap) return false;
    for (int i = threadIdx.x; i < cnt; i += HT) B[bs + i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) S.bsize = bs + cnt;
    __syncthreads();
    return true;
}

// front <- front XOR stage[0..b), stage sorted, unique and entirely below Ks.
__device__ bool heavy_merge_front(HeavySmem& S, uint64_t* B, int64_t bcap, int b) {
    if (b == 0) return true;
    const uint64_t* run = S.stage;
    const uint64_t* F = S.buf[S.cur];
    uint64_t* F2 = S.buf[S.cur ^ 1];
    const int a = S.fsize;
    // rows of F below run[0] keep their place
    const int p0 = lower_bound_sm(F, a, run[0]);
    for (int i = threadIdx.x; i < p0; i += HT) F2[i] = F[i];
    const int rest = a - p0;
    const int chunkF = (rest + HT - 1) / HT;
    const int f0 = p0 + min(rest, (int)threadIdx.x * chunkF), f1 = min(a, f0 + chunkF);
    int mloc = 0;
    for (int i = f0; i < f1; ++i) {
        int q = lower_bound_sm(run, b, F[i]);
        mloc += (q < b && run[q] == F[i]);
    }
    int mtot;
    int m = block_excl_scan(mloc, S.ws, &mtot);
    for (int i = f0; i < f1; ++i) {
        const uint64_t x = F[i];
        const int q = lower_bound_sm(run, b, x);
        if (q < b && run[q] == x) { ++m; continue; }
        F2[i + q - 2 * m] = x;
    }
    const int chunkR = (b + HT - 1) / HT;
    const int r0 = min(b, (int)threadIdx.x * chunkR), r1 = min(b, r0 + chunkR);
    int mloc2 = 0;
    for (int k = r0; k < r1; ++k) {
        const int q = lower_bound_sm(F, a, run[k]);
        mloc2 += (q < a && F[q] == run[k]);
    }
    int mt2;
    int m2 = block_excl_scan(mloc2, S.ws, &mt2);
    for (int k = r0; k < r1; ++k) {
        const uint64_t y = run[k];
        const int q = lower_bound_sm(F, a, y);
        if (q < a && F[q] == y) { ++m2; continue; }
        F2[k + q - 2 * m2] = y;
    }
    __syncthreads();
    int na = a + b - 2 * mtot;
    if (threadIdx.x == 0) S.cur ^= 1;
    __syncthreads();
    if (na > FKEEP) {  // spill the top of the front to B and lower the split
        if (!heavy_append(S, B, bcap, S.buf[S.cur] + FKEEP, na - FKEEP)) return false;
        if (threadIdx.x == 0) S.Ks = S.buf[S.cur][FKEEP];
        na = FKEEP;
    }
    if (threadIdx.x == 0) S.fsize = na;
    __syncthreads();
    return true;
}

// W <- W + run for a sorted, unique run in stage[0..b) (any keys).
__device__ bool heavy_add_run(HeavySmem& S, uint64_t* B, int64_t bcap, int b) {
    const int lo = lower_bound_sm(S.stage, b, S.Ks);
    if (!heavy_append(S, B, bcap, S.stage + lo, b - lo)) return false;
    return heavy_merge_front(S, B, bcap, lo);
}

// Refill an empty front from B.  Returns false if the column is zero.
__device__ bool heavy_refill(HeavySmem& S, uint64_t* B, int keybits) {
    for (;;) {
        __syncthreads();
        const int64_t bsz = S.bsize;
        if (bsz == 0) return false;
        // 1. split T with at most REFILL rows below it (MSD radix select)
        uint64_t T = EMPTY;
        if (bsz > REFILL) {
            uint64_t prefix = 0;
            int shift = ((keybits + 7) / 8) * 8 - 8;
            if (shift < 0) shift = 0;
            int64_t below = 0;
            for (;;) {
                for (int i = threadIdx.x; i < 256; i += HT) S.hist[i] = 0;
                __syncthreads();
                for (int64_t i = threadIdx.x; i < bsz; i += HT) {
                    const uint64_t k = B[i];
                    const bool in = shift + 8 >= 64 || (k >> (shift + 8)) == (prefix >> (shift + 8));
                    if (in) atomicAdd(&S.hist[(k >> shift) & 0xFF], 1u);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    int d = 0;
                    int64_t bl = below;
                    while (d < 256 && bl + S.hist[d] <= REFILL) bl += S.hist[d++];
                    const uint64_t hi_mask = (shift + 8 >= 64) ? 0ull : ~((1ull << (shift + 8)) - 1);
                    S.sel = (prefix & hi_mask) | ((uint64_t)d << shift);
                    S.flag = bl > 0 ? 1 : (shift == 0 ? 2 : 0);  // 1 done, 2 one key, 0 descend
                    S.ws[HW] = (int)bl;
                }
                __syncthreads();
                const int fl = S.flag;
                if (fl == 1) { T = S.sel; break; }
                if (fl == 2) { T = S.sel + 1; break; }
                prefix = S.sel;
                below = S.ws[HW];
                shift -= 8;
                __syncthreads();
            }
        }
        // 2. move rows < T to the spare buffer (tile by tile: B is compacted in place)
        uint64_t* G = S.buf[S.cur ^ 1];
        int nlt = 0;
        int64_t nge = 0;
        for (int64_t base = 0; base < bsz; base += HT) {
            const int64_t i = base + threadIdx.x;
            const uint64_t k = i < bsz ? B[i] : EMPTY;
            const bool lt = i < bsz && k < T;
            const bool ge = i < bsz && !lt;
            int tot;
            const int packed = block_excl_scan((int)lt | ((int)ge << 16), S.ws, &tot);
            if (lt && nlt + (packed & 0xFFFF) < FC) G[nlt + (packed & 0xFFFF)] = k;
            if (ge) B[nge + (packed >> 16)] = k;
            nlt += tot & 0xFFFF;
            nge += tot >> 16;
        }
        __syncthreads();
        if (nlt > FC) {  // a single key with more copies than fit: keep its parity only
            if (threadIdx.x == 0) {
                S.buf[S.cur][0] = T - 1;
                S.fsize = (nlt & 1) ? 1 : 0;
                S.bsize = nge;
                S.Ks = T;
            }
            __syncthreads();
            if (S.fsize) return true;
            continue;
        }
        int len = 1;
        while (len < nlt) len <<= 1;
        for (int i = nlt + threadIdx.x; i < len; i += HT) G[i] = EMPTY;
        __syncthreads();
        block_bitonic(G, len);
        // 3. keep the rows of odd multiplicity
        uint64_t* F = S.buf[S.cur];
        const int chunk = (nlt + HT - 1) / HT;
        const int c0 = min(nlt, (int)threadIdx.x * chunk), c1 = min(nlt, c0 + chunk);
        int keep = 0;
        for (int i = c0; i < c1; ++i) {
            if (i > 0 && G[i - 1] == G[i]) continue;
            int e = i;
            while (e + 1 < nlt && G[e + 1] == G[i]) ++e;
            keep += ((e - i + 1) & 1);
        }
        int tk;
        int pos = block_excl_scan(keep, S.ws, &tk);
        for (int i = c0; i < c1; ++i) {
            if (i > 0 && G[i - 1] == G[i]) continue;
            int e = i;
            while (e + 1 < nlt && G[e + 1] == G[i]) ++e;
            if ((e - i + 1) & 1) F[pos++] = G[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            S.fsize = tk;
            S.bsize = nge;
            S.Ks = T;
        }
        __syncthreads();
        if (tk > 0) return true;
    }
}

// W <- W + D_x for the p-simplex x (vertices ascending, diameter rank xr):
// rows at or above the split go straight to B, only the few below it are
// sorted and merged into the front.
template <int P>
__device__ bool heavy_add_coboundary(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, const Simplex<P>& x) {
    const int64_t n = c.R.n;
    for (int64_t base = n - 1; base >= 0; base -= HT) {
        const int64_t w = base - (int64_t)threadIdx.x;
        bool ok = w >= 0;
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (w != x.v[q]);
        uint32_t rt = x.r;
        uint64_t key = EMPTY;
        if (ok) {
#pragma unroll
            for (int q = 0; q <= P; ++q) rt = max(rt, c.R(x.v[q], w));
            ok = rt <= c.thr;
            if (ok) key = row_key<P>(c, x, w, rt);
        }
        const bool lt = ok && key < S.Ks;
        const bool ge = ok && !lt;
        int tot;
        const int packed = block_excl_scan((int)lt | ((int)ge << 16), S.ws, &tot);
        const int nlt = tot & 0xFFFF, nge = tot >> 16;
        const int64_t bs = S.bsize;
        if (bs + nge > bcap) return false;
        if (ge) B[bs + (packed >> 16)] = key;
        if (lt) S.stage[packed & 0xFFFF] = key;
        __syncthreads();
        if (threadIdx.x == 0) S.bsize = bs + nge;
        __syncthreads();
        stage_sort(S, nlt);
        if (!heavy_merge_front(S, B, bcap, nlt)) return false;
    }
    return true;
}

// W <- W + R_o where R_o is a stored reduced column (sorted, unique).
__device__ bool heavy_add_stored(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, int64_t opos) {
    const uint64_t* run = c.pool + c.rc_off[opos];
    const int64_t len = c.rc_len[opos];
    for (int64_t base = 0; base < len; base += HSTAGE) {
        const int cnt = (int)min((int64_t)HSTAGE, len - base);
        for (int i = threadIdx.x; i < cnt; i += HT) S.stage[i] = run[base + i];
        __syncthreads();
        if (!heavy_add_run(S, B, bcap, cnt)) return false;
    }
    return true;
}

// Owner of pivot rk (see warp_owner); result in S.opos / S.ov / S.orank.
template <int P>
__device__ bool heavy_owner(const Ctx& c, HeavySmem& S, uint64_t rk, uint64_t self_key) {
    constexpr int NT = P + 2;
    constexpr int NPAIR = NT * (NT - 1) / 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = c.R.n;
    const uint32_t rt = (uint32_t)(rk >> c.rcb);
    const uint64_t ct = c.rcmask - (rk & c.rcmask);
    if (wid == 0) {
        int64_t pos = warp_hash_find(c, ct);
        int flag = 0;  // 1 = stored column owner, 2 = candidate apparent owner, 0 = none
        int drop = -1;
        int tv[NT];
        if (pos >= 0) {
            flag = 1;
        } else {
            decode_simplex<P + 1>(c.B, ct, n - 1, tv);
            bool eq = false;
            int pi = 0, pj = 0;
            if (lane < NPAIR) {
                int k = lane;
                pi = 1;
                while (k >= pi) { k -= pi; ++pi; }
                pj = k;
                eq = c.R(tv[pi], tv[pj]) == rt;
            }
#pragma unroll
            for (int m = NT - 1; m >= 0; --m)
                if (drop < 0 && __ballot_sync(0xffffffffu, eq && pi != m && pj != m)) drop = m;
            if (drop >= 0) flag = 2;
        }
        if (lane == 0) {
            S.flag = flag;
            S.opos = pos;
            if (flag == 2) {
                int k = 0;
                for (int q = 0; q < NT; ++q)
                    if (q != drop) S.ov[k++] = tv[q];
                S.ov[P + 1] = tv[drop];  // the dropped vertex
                S.orank = rt;
            }
        }
    }
    __syncthreads();
    const int flag = S.flag;
    if (flag == 0) return false;
    if (flag == 1) {
        if (threadIdx.x == 0) {
            const uint64_t okey = c.cols[S.opos];
            if (!(okey < self_key)) atomicExch(c.err, DEV_INTERNAL);
        }
        return true;
    }
    // apparent iff no vertex w above the dropped one keeps the diameter of s'
    int ov[P + 1];
#pragma unroll
    for (int q = 0; q <= P; ++q) ov[q] = S.ov[q];
    const int64_t wd = S.ov[P + 1];
    bool older = false;
    for (int64_t base = n - 1; base > wd; base -= HT) {
        const int64_t w = base - (int64_t)threadIdx.x;
        bool ok = w > wd;
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (w != ov[q]);
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (c.R(ov[q], w) <= rt);
        older = older || ok;
    }
    return !__syncthreads_or(older);
}

template <int P>
__global__ void __launch_bounds__(HT)
k_reduce_heavy(Ctx c, const uint32_t* __restrict__ U, int64_t u, const uint32_t* __restrict__ slot_of,
               HeavyState hs, int budget, int keybits, uint64_t* __restrict__ cur_key, uint8_t* __restrict__ status,
               uint32_t* __restrict__ adds_out) {
    extern __shared__ __align__(16) unsigned char hsm[];
    HeavySmem& S = *reinterpret_cast<HeavySmem*>(hsm);
    const int64_t k = blockIdx.x;
    if (k >= u) return;
    const int64_t j = U[k];
    const int64_t slot = slot_of[j];
    uint64_t* B = hs.B + slot * hs.bcap;
    const uint64_t self_key = c.cols[j];
    Simplex<P> s;
    load_col<P>(c, self_key, s);
    uint32_t adds;
    bool ok = true;
    if (!hs.init[slot]) {
        if (threadIdx.x == 0) { S.fsize = 0; S.bsize = 0; S.Ks = EMPTY; S.cur = 0; }
        __syncthreads();
        adds = 0;
        ok = heavy_add_coboundary<P>(c, S, B, hs.bcap, s);
    } else {
        if (threadIdx.x == 0) { S.fsize = hs.fsize[slot]; S.bsize = hs.bsize[slot]; S.Ks = hs.Ks[slot]; S.cur = 0; }
        adds = hs.adds[slot];
        __syncthreads();
        for (int i = threadIdx.x; i < S.fsize; i += HT) S.buf[0][i] = hs.F[slot * FC + i];
        __syncthreads();
    }
    uint64_t key = ok ? EMPTY : 0;  // 0: no consistent state yet, the smallest (always valid) bound
    uint8_t st = ST_COMPLETE;
    int done = 0;
    long long t0 = clock64(), t_ref = 0, t_look = 0, t_add = 0, n_look = 0;
    const long long t_resume = t0;
    while (ok) {
        long long ta = clock64();
        if (S.fsize == 0 && !heavy_refill(S, B, keybits)) { key = EMPTY; break; }  // zero column
        long long tb = clock64();
        t_ref += tb - ta;
        key = S.buf[S.cur][0];
        const bool owned = heavy_owner<P>(c, S, key, self_key);
        long long tc = clock64();
        t_look += tc - tb;
        ++n_look;
        if (!owned) break;  // pivot unknown: complete
        if (done >= budget) { st = ST_BUDGET; break; }
        if (S.flag == 1) {
            const int64_t opos = S.opos;
            if (c.rc_len[opos]) {
                ok = heavy_add_stored(c, S, B, hs.bcap, opos);
            } else {
                Simplex<P> o;
                load_col<P>(c, c.cols[opos], o);
                ok = heavy_add_coboundary<P>(c, S, B, hs.bcap, o);
            }
        } else {
            Simplex<P> o;
#pragma unroll
            for (int q = 0; q <= P; ++q) o.v[q] = S.ov[q];
            o.r = S.orank;
            ok = heavy_add_coboundary<P>(c, S, B, hs.bcap, o);
        }
        ++adds;
        ++done;
        __syncthreads();
        t_add += clock64() - tc;
    }
    if (hs.prof && threadIdx.x == 0) {
        atomicAdd(hs.prof + 0, (unsigned long long)t_ref);
        atomicAdd(hs.prof + 1, (unsigned long long)t_look);
        atomicAdd(hs.prof + 2, (unsigned long long)t_add);
        atomicAdd(hs.prof + 3, (unsigned long long)(clock64() - t_resume - t_ref - t_look - t_add));
        atomicAdd(hs.prof + 4, (unsigned long long)done);
        atomicAdd(hs.prof + 5, (unsigned long long)n_look);
    }
    if (!ok) st = ST_OVERFLOW;  // key holds the last consistent pivot, a valid bound
    for (int i = threadIdx.x; i < S.fsize && ok; i += HT) hs.F[slot * FC + i] = S.buf[S.cur][i];
    if (threadIdx.x == 0) {
        hs.fsize[slot] = S.fsize;
        hs.bsize[slot] = S.bsize;
        hs.Ks[slot] = S.Ks;
        hs.adds[slot] = adds;
        hs.init[slot] = ok ? 1 : 0;  // an overflowed column restarts from scratch
        cur_key[j] = key;
        status[j] = st;
        adds_out[j] = adds;
    }
}

__global__ void k_assign_slots(const uint32_t* __restrict__ U, int64_t u, uint32_t* __restrict__ slot_of,
                               uint8_t* __restrict__ init) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x) {
        slot_of[U[k]] = (uint32_t)k;
        init[k] = 0;
    }
}

// One warp finishes the remaining columns in order (Algorithm 12 verbatim).
template <int P>
__global__ void __launch_bounds__(32)
k_reduce_seq(Ctx c, Emit e, const uint32_t* __restrict__ U, int64_t u, uint64_t* bufA, uint64_t* bufB, int64_t cap) {
    __shared__ uint64_t stage[STAGE];
    const int lane = threadIdx.x & 31;
    for (int64_t k = 0; k < u; ++k) {
        const int64_t j = U[k];
        uint64_t key;
        uint8_t st;
        uint32_t ad;
        reduce_one<P>(c, j, 0x7FFFFFFF, stage, bufA, bufB, cap, key, st, ad);
        if (st != ST_COMPLETE) {
            if (lane == 0) atomicExch(c.err, DEV_CAPACITY);
            return;
        }
        if (lane == 0) finish_column(c, e, j, key, ad);
        __threadfence_block();
        __syncwarp();
    }
}

__global__ void k_iota(uint32_t* U, int64_t m) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        U[k] = (uint32_t)k;
}

template <int P>
void run_p(const Ctx& c, const Emit& e, Workspace& ws, HostScratch& hs) {
    const int64_t m = c.num_cols;
    cudaStream_t s = ws.stream;
    uint32_t* U = ws.alloc_n<uint32_t>(m);
    uint32_t* Un = ws.alloc_n<uint32_t>(m);
    uint64_t* cur_key = ws.alloc_n<uint64_t>(m);
    uint8_t* status = ws.alloc_n<uint8_t>(m);
    uint32_t* adds = ws.alloc_n<uint32_t>(m);
    unsigned long long* ctr = ws.zeros_n<unsigned long long>(3);  // [0] work [1] u_next [2] first status
    k_iota<<<(unsigned)((m + 255) / 256 < 4096 ? (m + 255) / 256 : 4096), 256, 0, s>>>(U, m);
    VR_CUDA(cudaGetLastError());
    int64_t u = m;
    const int keybits = bits_for(c.rmask) + c.rcb;
    // Phase 1: one warp per column, at most 8 additions, every column at once.
    {
        const int64_t max_slots = 148 * 4 * RED_WARPS;
        int64_t slots = u < max_slots ? u : max_slots;
        slots = (slots + RED_WARPS - 1) / RED_WARPS * RED_WARPS;
        const int64_t cap = 8192;
        uint64_t* scratch = ws.alloc_n<uint64_t>((size_t)slots * 2 * cap);
        VR_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s));
        k_reduce_round<P><<<(unsigned)(slots / RED_WARPS), RED_WARPS * 32, 0, s>>>(c, U, u, 8, cur_key, status, adds,
                                                                                   scratch, cap, ctr);
        k_finalize<<<1, 1024, 0, s>>>(c, e, U, u, cur_key, status, adds, Un, ctr + 1, ctr + 2);
        VR_CUDA(cudaGetLastError());
        VR_CUDA(cudaMemcpyAsync(&hs.p[8], ctr + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        if (log_enabled())
            fprintf(stderr, "[vr] dim%d warp round: %lld -> %lld unfinished\n", P, (long long)u, (long long)hs.p[8]);
        uint32_t* t = U; U = Un; Un = t;
        u = hs.p[8];
    }
    // Phase 2: one block per remaining column, state kept between rounds; the
    // first unfinished column always finishes once its budget suffices (no
    // earlier column can block it), so budgets double every round.
    int rounds = 0;
    if (u > 0) {
        const size_t smem = sizeof(HeavySmem);
        VR_CUDA(cudaFuncSetAttribute(k_reduce_heavy<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t nslot = u;
        HeavyState h;
        h.bcap = std::max<int64_t>((int64_t)1 << 16, std::min<int64_t>((int64_t)1 << 22, ((int64_t)1 << 27) / nslot));
        h.F = ws.alloc_n<uint64_t>((size_t)nslot * FC);
        h.B = ws.alloc_n<uint64_t>((size_t)nslot * h.bcap);
        h.Ks = ws.alloc_n<uint64_t>(nslot);
        h.fsize = ws.alloc_n<int32_t>(nslot);
        h.bsize = ws.alloc_n<int64_t>(nslot);
        h.init = ws.alloc_n<uint8_t>(nslot);
        h.adds = ws.alloc_n<uint32_t>(nslot);
        h.prof = log_enabled() ? ws.zeros_n<unsigned long long>(8) : nullptr;
        uint32_t* slot_of = ws.alloc_n<uint32_t>(m);
        k_assign_slots<<<(unsigned)((u + 255) / 256), 256, 0, s>>>(U, u, slot_of, h.init);
        int budget = 64;
        while (u > 0) {
            k_reduce_heavy<P><<<(unsigned)u, HT, smem, s>>>(c, U, u, slot_of, h, budget, keybits, cur_key, status, adds);
            k_finalize<<<1, 1024, 0, s>>>(c, e, U, u, cur_key, status, adds, Un, ctr + 1, ctr + 2);
            VR_CUDA(cudaGetLastError());
            VR_CUDA(cudaMemcpyAsync(&hs.p[8], ctr + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
            const int64_t un = hs.p[8];
            const int64_t first = hs.p[9];
            ++rounds;
            if (log_enabled())
                fprintf(stderr, "[vr] dim%d block round %d: budget %d bcap %lld: %lld -> %lld unfinished\n", P,
                        rounds, budget, (long long)h.bcap, (long long)u, (long long)un);
            uint32_t* t = U; U = Un; Un = t;
            const bool stalled = un == u;
            u = un;
            if (stalled && first == ST_OVERFLOW) {
                // the first column outgrew its back buffer: give the remaining
                // columns the whole arena (they restart from scratch)
                const int64_t nb = ((int64_t)1 << 27) / (u > 0 ? u : 1);
                if (nb <= h.bcap) throw Error{VR_ERR_OOM};
                h.bcap = std::min<int64_t>(nb, (int64_t)1 << 27);
                h.B = ws.alloc_n<uint64_t>((size_t)u * h.bcap);
                k_assign_slots<<<(unsigned)((u + 255) / 256), 256, 0, s>>>(U, u, slot_of, h.init);
                VR_CUDA(cudaGetLastError());
            }
            if (budget < (1 << 24)) budget *= 2;
        }
        if (h.prof) {
            VR_CUDA(cudaMemcpyAsync(&hs.p[16], h.prof, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
            const double ad = hs.p[20] ? (double)hs.p[20] : 1.0, lk = hs.p[21] ? (double)hs.p[21] : 1.0;
            fprintf(stderr,
                    "[vr] dim%d block engine: %lld additions, %lld lookups; cycles/add %.0f, cycles/lookup %.0f, "
                    "refill total %lld, other total %lld\n",
                    P, (long long)hs.p[20], (long long)hs.p[21], hs.p[18] / ad, hs.p[17] / lk, (long long)hs.p[16],
                    (long long)hs.p[19]);
        }
    }
    if (log_enabled()) {
        VR_CUDA(cudaMemcpyAsync(&hs.p[10], c.pool_used, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        fprintf(stderr, "[vr] dim%d reduction: %d block rounds, stored rows %lld of %lld\n", P, rounds,
                (long long)hs.p[10], (long long)c.pool_cap);
    }
}

}  // namespace

void run_reduction(const ReduceIn& in, const ReduceOut& out, bool keep_zero, Workspace& ws, HostScratch& hs) {
    if (in.num_cols <= 0) return;
    Ctx c;
    c.R = in.R;
    c.B = in.B;
    c.thr = in.thr_rank;
    c.cb = in.cidx_bits;
    c.rcb = in.row_cidx_bits;
    c.cmask = in.cidx_bits >= 64 ? ~0ull : ((1ull << in.cidx_bits) - 1);
    c.rcmask = in.row_cidx_bits >= 64 ? ~0ull : ((1ull << in.row_cidx_bits) - 1);
    c.rmask = in.rank_bits >= 64 ? ~0ull : ((1ull << in.rank_bits) - 1);
    c.cols = in.cols;
    c.num_cols = in.num_cols;
    uint64_t hcap = 1024;
    while (hcap < 2 * (uint64_t)in.num_cols) hcap <<= 1;
    c.hkeys = ws.alloc_n<uint64_t>(hcap);
    c.hvals = ws.alloc_n<uint32_t>(hcap);
    VR_CUDA(cudaMemsetAsync(c.hkeys, 0xFF, hcap * sizeof(uint64_t), ws.stream));
    c.hmask = hcap - 1;
    c.err = out.dev_err;
    c.pool_cap = std::min<int64_t>((int64_t)1 << 24, std::max<int64_t>((int64_t)1 << 16, in.num_cols * 2048));
    c.pool = ws.alloc_n<uint64_t>((size_t)c.pool_cap);
    c.pool_used = ws.zeros_n<unsigned long long>(1);
    c.rc_off = ws.alloc_n<uint64_t>((size_t)in.num_cols);
    c.rc_len = ws.zeros_n<uint32_t>((size_t)in.num_cols);
    Emit e;
    e.pairs = out.pairs;
    e.num_pairs = out.num_pairs;
    e.clear_next = out.clear_next;
    e.counters = out.counters;
    e.keep_zero = keep_zero ? 1 : 0;
    switch (in.p) {
        case 1: run_p<1>(c, e, ws, hs); break;
        case 2: run_p<2>(c, e, ws, hs); break;
        case 3: run_p<3>(c, e, ws, hs); break;
        case 4: run_p<4>(c, e, ws, hs); break;
        case 5: run_p<5>(c, e, ws, hs); break;
        case 6: run_p<6>(c, e, ws, hs); break;
        default: throw Error{VR_ERR_INVALID_ARG};
    }
}

}  // namespace vr
