// reduce_device.cuh -- device-side pieces of the Z/2 reduction shared by the
// single-cloud schedule (reduce.cu) and the batched kernel (batched.cu): row
// keys, coboundary generation, pivot lookup (hash of finished columns, then
// apparent pairs recomputed from Def 5.3.4), the warp engine for light columns
// and the block engine (front/back split) for heavy columns.  See reduce.cu for
// the method and its justification.
#pragma once

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
    // finished columns that needed additions keep their reduced form R_j as
    // its generators (column j of V, R_j = sum of D_g), so a later column adds
    // R_j (standard reduction) instead of D_j
    uint64_t* pool;
    unsigned long long* pool_used;
    int64_t pool_cap;
    uint64_t* rc_ptr;  // per column position: device address of its generator list
    uint32_t* rc_len;  // 0: the column is its own coboundary D_j
    // reduction mode (Sec. 5.2.9): 0 = phase-2 columns keep R_j explicitly
    // (front and back), 1 = every column keeps V_j (generators) only,
    // 2 = oblivious (Algorithm 12 as printed: nothing is kept, owners add D_o)
    int mode;
    // sparse mode (Sec. 5.3.12): CSR lists of the threshold graph, ascending;
    // null: cofacets are enumerated over every vertex
    const uint32_t* nb_off = nullptr;
    const uint32_t* nb = nullptr;
};
constexpr int MODE_EXPLICIT = 0, MODE_V = 1, MODE_OBLIVIOUS = 2;

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

// Candidate vertices w of the cofacets x + {w} of a simplex, largest first:
// every vertex, or in sparse mode the neighbour list of x's vertex with the
// fewest neighbours (Alg 15: a cofacet within the threshold is adjacent to
// every vertex of x; the rank test made on each candidate excludes the rest).
struct Cands {
    const uint32_t* list;  // null: all vertices
    int64_t cnt;
    __device__ __forceinline__ int64_t operator[](int64_t i) const {  // the i-th largest, i < cnt
        return list ? (int64_t)list[cnt - 1 - i] : cnt - 1 - i;
    }
};
template <int P>
__device__ __forceinline__ Cands cofacet_cands(const Ctx& c, const int* v) {
    if (!c.nb_off) return Cands{nullptr, c.R.n};
    uint32_t b = c.nb_off[v[0]], e = c.nb_off[v[0] + 1];
#pragma unroll
    for (int q = 1; q <= P; ++q) {
        const uint32_t bq = c.nb_off[v[q]], eq = c.nb_off[v[q] + 1];
        if (eq - bq < e - b) {
            b = bq;
            e = eq;
        }
    }
    return Cands{c.nb + b, (int64_t)(e - b)};
}

template <int P>
__device__ __forceinline__ void load_col(const Ctx& c, uint64_t key, Simplex<P>& s) {
    s.cidx = key & c.cmask;
    s.r = (uint32_t)((~(key >> c.cb)) & c.rmask);
    warp_decode_simplex<P>(c.B, s.cidx, c.R.n - 1, s.v);  // callers are whole warps
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

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
    const uint32_t hi = __reduce_min_sync(0xffffffffu, (uint32_t)(x >> 32));
    const uint32_t lo = __reduce_min_sync(0xffffffffu, (uint32_t)(x >> 32) == hi ? (uint32_t)x : 0xffffffffu);
    return ((uint64_t)hi << 32) | lo;
}

// The K smallest row keys of D_x above `cut` (all rows if !has_cut), in
// ascending order, EMPTY-padded, by one warp: the cofacets x + {w} one lane
// each, every lane keeping its K smallest in registers (a key and its
// binomial reads only when its diameter rank can still enter), then K
// rounds of a warp minimum, the lane holding it moving on.  Every lane
// returns the same out[].
constexpr int RC = 4;
template <int P, int K = RC>
__device__ void warp_rows_above(const Ctx& c, const Simplex<P>& x, bool has_cut, uint64_t cut, uint64_t* out) {
    const int lane = threadIdx.x & 31;
    const Cands cw = cofacet_cands<P>(c, x.v);
    const uint32_t rcut = has_cut ? (uint32_t)(cut >> c.rcb) : 0u;
    uint64_t t[K];
#pragma unroll
    for (int r = 0; r < K; ++r) t[r] = EMPTY;
    for (int64_t i0 = 0; i0 < cw.cnt; i0 += 32) {
        const int64_t i = i0 + lane;
        const int64_t w = i < cw.cnt ? cw[i] : -1;
        bool ok = w >= 0;
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (w != x.v[q]);
        if (ok) {
            uint32_t rt = x.r;
#pragma unroll
            for (int q = 0; q <= P; ++q) rt = max(rt, c.R(x.v[q], w));
            if (rt <= c.thr && rt >= rcut && ((uint64_t)rt << c.rcb) <= t[K - 1]) {
                uint64_t key = row_key<P>(c, x, w, rt);
                if ((!has_cut || key > cut) && key < t[K - 1]) {
                    t[K - 1] = key;
#pragma unroll
                    for (int r = K - 1; r > 0; --r) {
                        const uint64_t lo = t[r - 1] < t[r] ? t[r - 1] : t[r], hi = t[r - 1] < t[r] ? t[r] : t[r - 1];
                        t[r - 1] = lo;
                        t[r] = hi;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint64_t m = warp_min_u64(t[0]);
        out[r] = m;
        const uint32_t own = __ballot_sync(0xffffffffu, m != EMPTY && t[0] == m);
        if (own && lane == __ffs(own) - 1) {  // keys of one coboundary are distinct: one owner
#pragma unroll
            for (int q = 0; q < K - 1; ++q) t[q] = t[q + 1];
            t[K - 1] = EMPTY;
        }
    }
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
            if (!(okey < self_key)) atomicExch(c.err, DEV_INTERNAL | (2 << 8));
            load_col<P>(c, okey, o);
            opos = pos;
            return true;
        }
    }
    // 2. apparent pairs (Def 5.3.4), recomputed
    int tv[NT];
    warp_decode_simplex<P + 1>(c.B, ct, n - 1, tv);
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
    const Cands cw = cofacet_cands<P>(c, o.v);
    for (int64_t i0 = 0; i0 < cw.cnt && cw[i0] > wd; i0 += 32) {  // largest first: stop below wd
        const int64_t i = i0 + lane;
        const int64_t w = i < cw.cnt ? cw[i] : -1;
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
    if (!(col_key<P>(c, o) < self_key)) atomicExch(c.err, DEV_INTERNAL | (3 << 8));
    opos = -1;
    return true;
}

// Keep the reduced column of position j as the list of simplices whose
// coboundaries add up to it (its column of V: R_j = D_j + sum of D_g), as
// column keys, for later additions.
template <int P>
__device__ void store_generators(const Ctx& c, int64_t j, const Simplex<P>* gs, int m) {
    const int lane = threadIdx.x & 31;
    unsigned long long off = 0;
    if (c.mode == MODE_OBLIVIOUS) return;  // Algorithm 12 keeps no reduced form
    if (lane == 0) off = atomicAdd(c.pool_used, (unsigned long long)m);
    off = __shfl_sync(0xffffffffu, off, 0);
    const bool fits = (int64_t)(off + m) <= c.pool_cap;
    if (fits && lane < m) c.pool[off + lane] = col_key<P>(c, gs[lane]);
    __syncwarp();
    if (lane == 0) {
        c.rc_ptr[j] = (uint64_t)(c.pool + off);
        c.rc_len[j] = fits ? (uint32_t)m : 0u;
        // without its reduced form a later column could only add D_j, which need
        // not cancel the shared pivot: report the shortage instead
        if (!fits) atomicExch(c.err, DEV_CAPACITY);
    }
}

// Reduce column j (position in cols) against the known pivots, with at most
// `budget` additions (and at most RGEN - 1).  The column is kept implicitly
// as its generators g (j itself and the owners added so far): a row r has
// multiplicity #{g : g is a facet of r}, and each generator caches the RC
// smallest rows of D_g above the rows already known to cancel.  The pivot
// is the smallest current row if it occurs an odd number of times;
// otherwise it cancels, the generators holding it move to their next
// cached row (looking up RC more when the cache runs out), and the search
// goes on.  Nothing is sorted or merged.  Only apparent owners are added
// here (this runs before any column of the dimension is finalized); a
// pivot owned by a finished column ends the call with ST_BUDGET.  On
// completion with additions the generators are stored (store_generators).
constexpr int RGEN = 16;
template <int P>
__device__ void reduce_one(const Ctx& c, int64_t j, int budget, uint64_t* stage, uint64_t& out_key,
                           uint8_t& out_status, uint32_t& out_adds) {
    static_assert(RGEN * (RC + 1 + sizeof(Simplex<P>) / 8 + 1) <= STAGE, "generators fit the stage");
    const int lane = threadIdx.x & 31;
    const uint64_t self_key = c.cols[j];
    Simplex<P> s, o;
    int64_t opos = -1;
    load_col<P>(c, self_key, s);
    uint64_t* gc = stage;                                                      // [RGEN][RC] cached rows
    int* gh = reinterpret_cast<int*>(stage + RGEN * RC);                       // [RGEN] position in the cache
    Simplex<P>* gs = reinterpret_cast<Simplex<P>*>(stage + RGEN * (RC + 1));  // [RGEN] generators
    uint64_t rows[RC];
    warp_rows_above<P, 1>(c, s, false, 0, rows);  // the pivot of D_j; more rows only if it is added to
    uint64_t piv = rows[0];
    out_adds = 0;
    if (lane == 0) c.rc_len[j] = 0;
    if (piv == EMPTY) { out_key = EMPTY; out_status = ST_COMPLETE; return; }
    if (!warp_owner<P>(c, piv, self_key, o, opos)) { out_key = piv; out_status = ST_COMPLETE; return; }
    if (budget <= 0) { out_key = piv; out_status = ST_BUDGET; return; }  // the pivot has an owner: not settled here
    // a generator enters with its smallest row as the last cached one: when
    // that row cancels, the next RC are looked up
    if (lane == 0) {
        gs[0] = s;
        gh[0] = RC - 1;
        gc[RC - 1] = piv;
    }
    __syncwarp();
    int m = 1;
    uint32_t adds = 0;
    auto current = [&](int i) -> uint64_t { const int h = gh[i]; return h < RC ? gc[i * RC + h] : EMPTY; };
    for (;;) {
        if ((int)adds >= budget || m >= RGEN || opos >= 0) {
            out_key = piv; out_status = ST_BUDGET; out_adds = adds;
            return;
        }
        // W <- W + D_o: its smallest row is piv (o owns it)
        if (lane == 0) {
            gs[m] = o;
            gh[m] = RC - 1;
            gc[m * RC + RC - 1] = piv;
        }
        __syncwarp();
        ++m;
        ++adds;
        for (;;) {
            uint64_t cm = EMPTY;
            int cnt = 0;
            for (int i = 0; i < m; ++i) {
                const uint64_t x = current(i);
                if (x < cm) { cm = x; cnt = 1; } else if (x == cm) ++cnt;
            }
            if (cm == EMPTY || (cnt & 1)) { piv = cm; break; }
            for (int i = 0; i < m; ++i) {  // cm cancels: the generators holding it move on
                if (current(i) != cm) continue;
                const int h = gh[i] + 1;
                const uint64_t last = gc[i * RC + RC - 1];
                __syncwarp();
                if (h < RC || last == EMPTY) {  // the next cached row, or none left
                    if (lane == 0) gh[i] = h < RC ? h : RC;
                } else {
                    const Simplex<P> g = gs[i];
                    warp_rows_above<P>(c, g, true, last, rows);
                    if (lane == 0) {
                        gh[i] = 0;
#pragma unroll
                        for (int r = 0; r < RC; ++r) gc[i * RC + r] = rows[r];
                    }
                }
                __syncwarp();
            }
        }
        if (piv == EMPTY) { out_key = EMPTY; out_status = ST_COMPLETE; out_adds = adds; return; }
        if (!warp_owner<P>(c, piv, self_key, o, opos)) {
            out_key = piv;
            out_status = ST_COMPLETE;
            out_adds = adds;
            store_generators<P>(c, j, gs, m);
            return;
        }
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
    const uint64_t* next_list;     // sparse mode: clear_next by position in this sorted list (else NULL)
    int64_t next_len;
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
    if (e.clear_next) {
        uint64_t bit = ct;
        if (e.next_list) {  // position of ct among the listed (p+1)-simplices
            int64_t lo = 0, hi = e.next_len;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (e.next_list[mid] < ct) lo = mid + 1; else hi = mid;
            }
            bit = (uint64_t)lo;
            if (lo >= e.next_len) atomicExch(c.err, DEV_INTERNAL | (7 << 8));
        }
        if (!e.next_list || (int64_t)bit < e.next_len) atomicOr(e.clear_next + (bit >> 5), 1u << (bit & 31));
    }
    atomicAdd(e.counters + 1, 1ull);
    if (rt > rs || e.keep_zero) {
        pr.death_rank = rt;
        pr.death_cidx = (int64_t)ct;
        e.pairs[atomicAdd(e.num_pairs, 1ull)] = pr;
    }
}

// One block: exclusive prefix-min of the pivot keys over U in order decides
// which columns are final; the rest are compacted, in order, into Unext.
// ---------------------------------------------------------------------------
// Heavy columns: one 512-thread block per column, state kept across rounds.
//
// A column that needs many additions (the cocycle of a long bar can reach
// hundreds of thousands of rows) is never merged as a whole.  Its rows are
// split at a key Ks: the front F (rows < Ks, sorted, unique, at most FC of
// them) lives in shared memory and is the only part the pivot search reads;
// the back B (rows >= Ks) is an unsorted multiset in global memory to which
// new rows are appended without sorting.  When F runs empty, a sampled
// split T with at most FC rows below it is found; those rows are taken out
// of B (leaving holes), sorted, rows of even multiplicity cancel (Z/2), and
// the rest become the new front with Ks = T.  An addition thus
// costs O(rows added + |F|), independent of the column's size.
// ---------------------------------------------------------------------------
constexpr int HT = 512;          // threads per block
constexpr int HW = HT / 32;
constexpr int FC = 4096;         // front capacity
// Front size kept after a spill.  Every addition rewrites the front in its
// merge, so a smaller front makes additions cheaper, until refills from the
// back come too often (torus500 step, alternating runs on one GPU: 19.9 ms at
// 3072 rows, 19.4 ms at 2048 and at 2560, 19.8 ms at 1536, 20.4 ms at 1024).
constexpr int FKEEP = FC / 2;
constexpr int HSTAGE = 1024;     // rows generated or copied per pass (power of two >= HT)
static_assert(HSTAGE == 2 * HT, "a flushed stage holds two rows per thread");
static_assert(FKEEP + HSTAGE <= FC, "a merge writes a front of FKEEP rows and a run of HSTAGE into FC");
constexpr int REFILL_MAX = FC - HT;  // rows a refill may leave in the front
static_assert(REFILL_MAX + HT <= FC, "a pass of generated rows (at most HT) fits after a refill");
constexpr int pow2_ceil(int x) { return x <= 1 ? 1 : 2 * pow2_ceil((x + 1) / 2); }
static_assert(pow2_ceil(REFILL_MAX) <= FC, "a refill sorts its rows in a front buffer, padded to a power of two");
static_assert(HW <= 32, "block scans keep one total per warp in one warp");
static_assert(FC < (1 << 16) && HSTAGE < (1 << 16), "merge splits pack two 16-bit indices");

struct HeavyState {
    uint64_t* F;       // slots x FC, the front saved between rounds
    uint64_t** B;      // per slot: its back buffer (a regrowth moves the unfinished columns'
    int64_t* bcap;     // buffers; a finished column keeps its reduced form) and its rows
    uint64_t* Ks;      // per slot
    int32_t* fsize;
    int64_t* bsize;
    uint8_t* init;     // 0: the column has not been started (or must restart)
    uint32_t* adds;
    int64_t* holes;    // per slot: holes (EMPTY rows) in B
    unsigned long long* prof;  // VR_LOG only: cycles {refill, lookup, add, resume}, counts {adds, lookups}
    // V mode: per slot, the column's generators so far (an unsorted multiset of
    // column keys: j itself, then every simplex whose coboundary was added;
    // duplicates cancel when the coboundaries are generated)
    uint64_t** V;
    int64_t* vcap;
    int64_t* vlen;
    // windowed engine (V and oblivious modes): only the first `nslot`
    // unfinished columns hold a slot; a finalized column returns its slot
    // here (its reduced form is not needed: its generators, if any, move to
    // the pool) and the next column in order takes it.  NULL: every column
    // has a fixed slot (default mode, whose finished columns keep R_j in it).
    int32_t* free_slots;
    int32_t* free_top;
};

// VR_LOG instrumentation of the block engine (-DVR_HPROF builds): {refills, rows to front, rows
// to back, merges}
__device__ unsigned long long g_heavy_counts[4];

struct HeavySmem {
    uint64_t buf[2][FC];   // the front and its merge target, swapped after each merge
    uint64_t stage[HSTAGE];
    uint32_t msplit[HT];               // merge: (front index << 16) | run index at each thread's diagonal
    uint32_t eqbits[HSTAGE / 32];      // merge: run rows that cancel a front row
    int ws[HW + 1];
    uint32_t hist[256];
    uint64_t Ks;
    int64_t bsize;
    int64_t holes;         // EMPTY rows in B (left by refills)
    int64_t opos;
    int64_t vlen;          // V mode: generators recorded so far
    int fsize;
    int cur;               // which buf holds the front
    int flag;
    int na;                // merge result size (written by the merge group)
    int pkind;             // owner kind of the next pivot, probed during the merge (0: not probed)
    int ov[VR_MAX_DIM + 2];
    uint32_t orank;
    uint64_t sel;          // the next pivot, when found during a merge
    long long tp[20];      // VR_LOG only (thread 0): sub-phase cycles
};
// Sub-phase cycle counters of the block engine (thread 0, into S.tp), printed
// with VR_LOG=1; compiled in only with -DVR_HPROF, since their clock reads sit
// on the per-addition critical path.
#ifdef VR_HPROF
#define HCLK() clock64()
#define HPROF_T0() long long _hp_t = clock64()
#define HPROF_LAP(i) do { if (threadIdx.x == 0) { long long _n = clock64(); S.tp[i] += _n - _hp_t; _hp_t = _n; } } while (0)
#else
#define HCLK() 0ll
#define HPROF_T0() do { } while (0)
#define HPROF_LAP(i) do { } while (0)
#endif

// exclusive block scan of one int per thread; *total receives the sum.
// Warp scans, one barrier to publish the warp totals, then every warp sums
// the totals before it itself (no second scan stage); the trailing barrier
// lets the next call reuse ws.
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
    const int v = lane < HW ? ws[lane] : 0;
    int before = lane < wid ? v : 0, all = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    *total = all;
    __syncthreads();
    return before + incl - x;
}

// Bitonic sort of a[0..len), len a power of two.  Each thread takes compare
// pairs, not elements: pair p of a stage with distance j joins i = 2p - (p mod
// j) and i + j, so no lane idles on the upper half of a pair.
__device__ void block_bitonic(uint64_t* a, int len) {
    const int half = len >> 1;
    for (int k = 2; k <= len; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < half; p += HT) {
                const int i = 2 * p - (p & (j - 1));
                const uint64_t x = a[i], y = a[i + j];
                if ((x > y) == ((i & k) == 0)) { a[i] = y; a[i + j] = x; }
            }
            __syncthreads();
        }
}

// Sort stage[0..cnt) ascending; returns where the sorted rows are.  Up to
// HT rows: each thread ranks its row by comparing it with every row
// (broadcast shared reads, stable for equal rows) and places it in the
// upper half of the stage, which costs one barrier instead of the log^2
// barrier stages of a bitonic network; more rows are sorted in place by the
// bitonic network.
// DISTINCT: the rows are known to differ (one pass of one coboundary), so a
// row's rank needs no tie-break.
template <bool DISTINCT = false>
__device__ const uint64_t* stage_sort(HeavySmem& S, int cnt) {
    if (cnt <= 1) return S.stage;
    if (cnt <= HT && cnt <= HSTAGE / 2) {
        const int i = threadIdx.x;
        if (i < cnt) {
            const uint64_t x = S.stage[i];
            int rank = 0;
            if (DISTINCT) {
#pragma unroll 8
                for (int j = 0; j < cnt; ++j) rank += S.stage[j] < x;
            } else {
                for (int j = 0; j < cnt; ++j) {
                    const uint64_t y = S.stage[j];
                    rank += (y < x) || (y == x && j < i);
                }
            }
            S.stage[HSTAGE / 2 + rank] = x;
        }
        __syncthreads();
        return S.stage + HSTAGE / 2;
    }
    int len = 2;
    while (len < cnt) len <<= 1;
    for (int i = cnt + threadIdx.x; i < len; i += HT) S.stage[i] = EMPTY;
    __syncthreads();
    block_bitonic(S.stage, len);
    return S.stage;
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

// Named barrier `id` over `n` threads (whole warps); id 0 with n = HT is
// the block barrier.
__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// F2 <- F XOR run (F = buf[cur] with a rows, run[0..b) in the stage, both sorted
// and unique), computed by threads [t0, t0 + nt) of the block (t0 and nt
// multiples of 32), which meet at barrier `bar`; returns the merged size.
// No barrier follows the writes of F2 (the caller's does).
//
// Merge path: the merged sequence (a + b rows before cancellation) is cut
// into equal diagonals, one per thread, so rows that cluster in one gap of
// the front still spread over the threads.  Each thread finds the split of
// its diagonal by a binary search no longer than log2(b) (equal rows ordered
// front first; a boundary between a front row and an equal run row moves
// before the front row, so every cancelling pair stays in one thread's
// range) and reads the end of its range from the next thread.  Meanwhile
// each run row looks itself up in the front: the cancelled ones form a bit
// mask (one ballot per 32 rows), so after one barrier a thread's output
// offset is its diagonal minus twice the cancelled run rows before its
// range, and a single walk writes its part.
__device__ int merge_group(HeavySmem& S, const uint64_t* run, int cur, int a, int b, int t0, int nt, int bar) {
    const uint64_t* F = S.buf[cur];
    uint64_t* F2 = S.buf[cur ^ 1];
    const int g = (int)threadIdx.x - t0;
    const int lane = threadIdx.x & 31;
    const int tot = a + b;
    const int per = (tot + nt - 1) / nt;
    const int d = min(tot, g * per);
    // k0: run rows among the first d of the merged sequence, the largest k in
    // [max(0, d - a), min(d, b)] with run[k-1] < F[d-k] (fixed power-of-two
    // steps: no data-dependent branches in the search)
    const int klo = max(0, d - a), khi = min(d, b);
    int k0 = klo;
    for (int st = khi > klo ? 1 << (31 - __clz(khi - klo)) : 0; st > 0; st >>= 1) {
        const int t = k0 + st;
        if (t <= khi && run[t - 1] < F[d - t]) k0 = t;
    }
    int i0 = d - k0;
    if (i0 > 0 && k0 < b && F[i0 - 1] == run[k0]) --i0;
    S.msplit[g] = ((uint32_t)i0 << 16) | (uint32_t)k0;
    // run rows kb + lane (kb: this warp's block of 32, stepping by nt) that cancel
    for (int kb = g - lane; kb < b; kb += nt) {
        const int k = kb + lane;
        bool eq = false;
        if (k < b) {
            const uint64_t y = run[k];
            int q = 0;  // front rows below y, by fixed steps
            for (int st = a > 0 ? 1 << (31 - __clz(a)) : 0; st > 0; st >>= 1) {
                const int t = q + st;
                if (t <= a && F[t - 1] < y) q = t;
            }
            eq = q < a && F[q] == y;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) S.eqbits[kb >> 5] = m;
    }
    bar_sync(bar, nt);
    const uint32_t nx = g + 1 < nt ? S.msplit[g + 1] : (((uint32_t)a << 16) | (uint32_t)b);
    const int i1 = (int)(nx >> 16), k1 = (int)(nx & 0xFFFFu);
    int eb = 0, et = 0;
    for (int w = 0; w < ((b + 31) >> 5); ++w) {
        const uint32_t m = S.eqbits[w];
        const int base = w << 5;
        et += __popc(m);
        eb += base + 32 <= k0 ? __popc(m) : (base < k0 ? __popc(m & ((1u << (k0 - base)) - 1u)) : 0);
    }
    int pos = i0 + k0 - 2 * eb;
    int i = i0, k = k0;
    while (i < i1 || k < k1) {
        const uint64_t x = i < i1 ? F[i] : EMPTY;
        const uint64_t y = k < k1 ? run[k] : EMPTY;
        const bool tx = x <= y, ty = y <= x;  // both: a cancelling pair
        if (tx != ty) F2[pos++] = tx ? x : y;
        i += tx;
        k += ty;
    }
    return tot - 2 * et;
}

// After a merge into buf[cur ^ 1] of na rows (cur and fsize already
// published): spill the top of the front to B and lower the split.
__device__ bool heavy_spill(HeavySmem& S, uint64_t* B, int64_t bcap, int na) {
    if (na <= FKEEP) return true;
    uint64_t* F2 = S.buf[S.cur];
    if (!heavy_append(S, B, bcap, F2 + FKEEP, na - FKEEP)) return false;
    if (threadIdx.x == 0) S.Ks = F2[FKEEP];
    __syncthreads();
    return true;
}

// front <- front XOR run[0..b) (rows in the stage, sorted, unique and
// entirely below Ks; the whole block merges, see merge_group).
__device__ bool heavy_merge_front(HeavySmem& S, uint64_t* B, int64_t bcap, const uint64_t* run, int b) {
    if (b == 0) return true;
    if (S.fsize + b > FC) {
        // a run of more than HT rows into a refilled front (up to REFILL_MAX
        // rows): the front's top rows go to B first and the split drops to the
        // first of them; the run rows at or above it follow them
        const int keep = FC - b;
        const uint64_t* F0 = S.buf[S.cur];
        const uint64_t nks = F0[keep];
        if (!heavy_append(S, B, bcap, F0 + keep, S.fsize - keep)) return false;
        const int lo = lower_bound_sm(run, b, nks);
        if (!heavy_append(S, B, bcap, run + lo, b - lo)) return false;
        if (threadIdx.x == 0) {
            S.Ks = nks;
            S.fsize = keep;
        }
        __syncthreads();
        b = lo;
        if (b == 0) return true;
    }
    const int cur = S.cur, a = S.fsize;
    HPROF_T0();
    const int na = merge_group(S, run, cur, a, b, 0, HT, 0);
    HPROF_LAP(10);
    if (threadIdx.x == 0) {  // every read of cur and fsize happened before the merge's first barrier
        S.cur = cur ^ 1;
        S.fsize = min(na, FKEEP);
    }
    __syncthreads();
    HPROF_LAP(11);
    const bool ok = heavy_spill(S, B, bcap, na);
    HPROF_LAP(12);
    return ok;
}

// W <- W + run for a sorted, unique run in stage[0..b) (any keys).
__device__ bool heavy_add_run(HeavySmem& S, uint64_t* B, int64_t bcap, int b) {
    const int lo = lower_bound_sm(S.stage, b, S.Ks);
    if (!heavy_append(S, B, bcap, S.stage + lo, b - lo)) return false;
    return heavy_merge_front(S, B, bcap, S.stage, lo);
}

// Remove the holes (EMPTY) from B in place, keeping the order of the rest.
__device__ void heavy_compact_back(HeavySmem& S, uint64_t* B) {
    const int64_t bsz = S.bsize;
    constexpr int PER = 8;
    // the next tile is loaded before this one is written back: writes land
    // below the current tile's end, so they never touch the rows read
    uint64_t nk[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int64_t i = (int64_t)q * HT + threadIdx.x;
        nk[q] = i < bsz ? B[i] : EMPTY;
    }
    int64_t nkeep = 0;
    for (int64_t base = 0; base < bsz; base += (int64_t)HT * PER) {
        uint64_t k[PER];
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            k[q] = nk[q];
            cnt += k[q] != EMPTY;
        }
        if (base + (int64_t)HT * PER < bsz) {
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int64_t i = base + (int64_t)HT * (PER + q) + threadIdx.x;
                nk[q] = i < bsz ? B[i] : EMPTY;
            }
        }
        int tot;
        int64_t pos = nkeep + block_excl_scan(cnt, S.ws, &tot);  // all of the tile is read
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (k[q] != EMPTY) B[pos++] = k[q];
        nkeep += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) S.bsize = nkeep;
    __syncthreads();
}

// Refill an empty front from B.  Returns false if the column is zero.
// A refilled front holds at most REFILL_MAX = FC - HT rows: a pass of
// generated rows (at most HT) still fits beside it, and heavy_merge_front
// spills before a longer run.  Two splits Ta < Tb come from a sorted sample
// of B (its quantiles for about 0.5 and 0.9 REFILL_MAX rows).  One pass
// over B collects the positions of the rows below Tb (room for 2 FC); if
// they fit the front they are taken, else, if the rows below Ta among them
// do, those are -- so a
// refill takes close to a full front without a second pass over B (a pass
// costs the same for either, and fewer, larger refills are cheaper).  If
// neither fits, the splits move and the pass repeats.  The rows are
// gathered, replaced by holes (EMPTY, above every row key), sorted, and the
// rows of odd multiplicity become the front (Z/2).  B is only read in
// full; it is compacted once holes make up half of it.
// UN: rows each thread loads per step of the pass (independent loads in flight).
template <int UN = 16>
__device__ bool heavy_refill(HeavySmem& S, uint64_t* B) {
    constexpr int NS = 2048;  // samples (fit the empty front buffer)
    static_assert(NS <= FC, "the sample lives in the front buffer");
    __shared__ int cnt_sh;
    __shared__ unsigned long long min_sh;
    const int lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();
        const int64_t bsz = S.bsize;
        if (bsz == 0) return false;
        HPROF_T0();
#ifdef VR_HPROF
        if (threadIdx.x == 0) { atomicAdd(&g_heavy_counts[0], 1ull); S.tp[9] += 1; }
#endif
        uint64_t* Sm = S.buf[S.cur];  // the sample (the front is empty), then the gathered rows
        uint32_t* P = reinterpret_cast<uint32_t*>(S.buf[S.cur ^ 1]);  // positions of the rows below Tb (2 FC)
        uint64_t Ta = EMPTY, Tb = EMPTY;
        int qa = 0, qb = 0;
        if (bsz > (FKEEP * 7) / 10) {
            const int64_t stride = bsz / NS;
            for (int i = threadIdx.x; i < NS; i += HT) Sm[i] = B[(int64_t)i * stride];
            __syncthreads();
            block_bitonic(Sm, NS);
            qa = (int)((double)REFILL_MAX * 0.5 * NS / (double)bsz);
            qb = (int)((double)REFILL_MAX * 0.9 * NS / (double)bsz);
            qa = qa < 1 ? 1 : (qa > NS - 2 ? NS - 2 : qa);
            qb = qb <= qa ? qa + 1 : (qb > NS - 1 ? NS - 1 : qb);
            Ta = Sm[qa];
            Tb = Sm[qb];
        }
        HPROF_LAP(4);
        // 2. positions of the rows below Tb (one pass; the smallest row is
        //    only looked for when the splits must drop to it)
        int cnt, nsel = 0;
        bool filtered = false;
        uint64_t T = Tb;
        uint64_t bmin = EMPTY;
        bool have_min = false;
        for (;;) {
            if (threadIdx.x == 0) cnt_sh = 0;
            __syncthreads();
            // UN rows per thread per step; a mask of the rows below Tb, and the
            // rare hits placed by one shared-memory atomic per lane
            for (int64_t w0 = threadIdx.x; w0 < bsz; w0 += (int64_t)HT * UN) {
                uint64_t kk[UN];
#pragma unroll
                for (int u = 0; u < UN; ++u) {
                    const int64_t i = w0 + (int64_t)u * HT;
                    kk[u] = i < bsz ? B[i] : EMPTY;
                }
                uint32_t mask = 0;
#pragma unroll
                for (int u = 0; u < UN; ++u) mask |= (uint32_t)(kk[u] < Tb) << u;
                if (mask) {
                    int slot = atomicAdd(&cnt_sh, __popc(mask));
#pragma unroll
                    for (int u = 0; u < UN; ++u)
                        if ((mask >> u) & 1u) {
                            if (slot < 2 * FC) P[slot] = (uint32_t)(w0 + (int64_t)u * HT);
                            ++slot;
                        }
                }
            }
            __syncthreads();
            cnt = cnt_sh;
            __syncthreads();
            if (cnt >= 1 && cnt <= REFILL_MAX) { T = Tb; nsel = cnt; break; }
            int ca = -1;  // rows below Ta, when known
            if (cnt > REFILL_MAX && cnt <= 2 * FC && Ta < Tb) {
                int c = 0;
                for (int i = threadIdx.x; i < cnt; i += HT) c += B[P[i]] < Ta;
                int tot;
                block_excl_scan(c, S.ws, &tot);
                ca = tot;
                if (ca >= 1 && ca <= REFILL_MAX) { T = Ta; nsel = ca; filtered = true; break; }
            }
            if (cnt > REFILL_MAX && have_min && Tb == bmin + 1) { T = Tb; nsel = cnt; break; }  // one key, more copies than fit
            if (!have_min) {
                if (threadIdx.x == 0) min_sh = EMPTY;
                __syncthreads();
                uint64_t mn = EMPTY;
                for (int64_t i = threadIdx.x; i < bsz; i += HT) {
                    const uint64_t k = B[i];
                    mn = k < mn ? k : mn;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, mn, o);
                    mn = y < mn ? y : mn;
                }
                if (lane == 0) atomicMin(&min_sh, (unsigned long long)mn);
                __syncthreads();
                bmin = min_sh;
                have_min = true;
                __syncthreads();
                if (bmin == EMPTY) {  // only holes left: the column is zero
                    if (threadIdx.x == 0) S.bsize = 0;
                    __syncthreads();
                    return false;
                }
            }
            if (ca == 0 && qb - qa > 1) {  // Ta too low, Tb too high: split the difference
                qb = (qa + qb) >> 1;
                Tb = Sm[qb];
            } else if (cnt == 0 || qa <= 1) {
                Ta = bmin + 1;  // the smallest key alone
                Tb = Ta;
                qa = qb = 0;
            } else {
                qb = qa;
                Tb = Ta;
                qa >>= 1;
                Ta = Sm[qa];
            }
        }
        HPROF_LAP(5);
        if (nsel > REFILL_MAX) {  // every copy of bmin becomes a hole; its parity decides
            for (int64_t i = threadIdx.x; i < bsz; i += HT)
                if (B[i] == bmin) B[i] = EMPTY;
            __syncthreads();
            if (threadIdx.x == 0) {
                S.buf[S.cur][0] = bmin;
                S.fsize = nsel & 1;
                S.Ks = T;
            }
            __syncthreads();
        } else {
            // gather the rows into the sample's buffer and leave holes
            if (!filtered) {
                for (int i = threadIdx.x; i < nsel; i += HT) {
                    const int64_t pos = (int64_t)P[i];
                    Sm[i] = B[pos];
                    B[pos] = EMPTY;
                }
            } else {  // the rows below Ta among those below Tb
                int c = 0;
                for (int i = threadIdx.x; i < cnt; i += HT) c += B[P[i]] < Ta;
                int tot;
                int o = block_excl_scan(c, S.ws, &tot);
                for (int i = threadIdx.x; i < cnt; i += HT) {
                    const int64_t pos = (int64_t)P[i];
                    const uint64_t k = B[pos];
                    if (k < Ta) {
                        Sm[o++] = k;
                        B[pos] = EMPTY;
                    }
                }
            }
            int len = 1;
            while (len < nsel) len <<= 1;
            for (int i = nsel + threadIdx.x; i < len; i += HT) Sm[i] = EMPTY;
            __syncthreads();
            HPROF_LAP(6);
            block_bitonic(Sm, len);
            // keep the rows of odd multiplicity, in the other buffer
            uint64_t* F = S.buf[S.cur ^ 1];
            const int chunk = (nsel + HT - 1) / HT;
            const int c0 = min(nsel, (int)threadIdx.x * chunk), c1 = min(nsel, c0 + chunk);
            int keep = 0;
            for (int i = c0; i < c1; ++i) {
                if (i > 0 && Sm[i - 1] == Sm[i]) continue;
                int e = i;
                while (e + 1 < nsel && Sm[e + 1] == Sm[i]) ++e;
                keep += ((e - i + 1) & 1);
            }
            int tk;
            int pos = block_excl_scan(keep, S.ws, &tk);  // its barriers: every position was read
            for (int i = c0; i < c1; ++i) {
                if (i > 0 && Sm[i - 1] == Sm[i]) continue;
                int e = i;
                while (e + 1 < nsel && Sm[e + 1] == Sm[i]) ++e;
                if ((e - i + 1) & 1) F[pos++] = Sm[i];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                S.cur ^= 1;
                S.fsize = tk;
                S.Ks = T;
            }
            __syncthreads();
        }
        const int64_t holes = S.holes + nsel;
        if (holes == bsz) {
            if (threadIdx.x == 0) { S.bsize = 0; S.holes = 0; }
            __syncthreads();
        } else if (2 * holes > bsz) {
            heavy_compact_back(S, B);
            if (threadIdx.x == 0) S.holes = 0;
            __syncthreads();
        } else {
            if (threadIdx.x == 0) S.holes = holes;
            __syncthreads();
        }
        HPROF_LAP(7);
        if (S.fsize > 0) return true;
    }
}

// Place one pass of generated rows (thread t holds `key` if `ok`): rows at
// or above the split go straight to B, the few below it are sorted and
// merged into the front.
__device__ bool heavy_cob_place(HeavySmem& S, uint64_t* B, int64_t bcap, bool ok, uint64_t key) {
    HPROF_T0();
    const int64_t bs = S.bsize;  // read before the scan's barriers, rewritten after them
    const bool lt = ok && key < S.Ks;
    const bool ge = ok && !lt;
    int tot;
    const int packed = block_excl_scan((int)lt | ((int)ge << 16), S.ws, &tot);
    const int nlt = tot & 0xFFFF, nge = tot >> 16;
    if (bs + nge > bcap) return false;
    if (ge) B[bs + (packed >> 16)] = key;
    if (lt) S.stage[packed & 0xFFFF] = key;
    if (threadIdx.x == 0) {
        S.bsize = bs + nge;
#ifdef VR_HPROF
        atomicAdd(&g_heavy_counts[1], (unsigned long long)nlt);
        atomicAdd(&g_heavy_counts[2], (unsigned long long)nge);
        atomicAdd(&g_heavy_counts[3], 1ull);
#endif
    }
    __syncthreads();
    HPROF_LAP(0);
    const uint64_t* srt = stage_sort<true>(S, nlt);
    HPROF_LAP(1);
    if (!heavy_merge_front(S, B, bcap, srt, nlt)) return false;
    HPROF_LAP(2);
    return true;
}

template <int P, bool GROUP = false>
__device__ int heavy_owner_probe(const Ctx& c, HeavySmem& S, uint64_t rk, uint64_t self_key);

// heavy_cob_place for the last (here: only) pass of an addition, with the
// owner probe of the next pivot overlapped with the merge.  The next pivot
// is the smallest row of F XOR run; warp 0 finds it from the first 32 rows
// of each (merged by a bitonic network in registers, where a row survives
// unless an equal row sits next to it; the result is certain when it
// precedes row 32 of both), then warps 0 and 1 probe its owner while warps
// 2..15 merge.  S.pkind receives the probe's kind, or 0
// when the pivot was not certain from the heads (or the column emptied);
// every thread returns it in *next_kind (3 = probed, no owner).
template <int P>
__device__ bool heavy_cob_place_next(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, bool ok, uint64_t key,
                                     uint64_t self_key, int* next_kind) {
    HPROF_T0();
    const int64_t bs = S.bsize;
    const bool lt = ok && key < S.Ks;
    const bool ge = ok && !lt;
    int tot;
    const int packed = block_excl_scan((int)lt | ((int)ge << 16), S.ws, &tot);
    const int nlt = tot & 0xFFFF, nge = tot >> 16;
    if (bs + nge > bcap) return false;
    if (ge) B[bs + (packed >> 16)] = key;
    if (lt) S.stage[packed & 0xFFFF] = key;
    if (threadIdx.x == 0) {
        S.bsize = bs + nge;
        S.pkind = 0;
#ifdef VR_HPROF
        atomicAdd(&g_heavy_counts[1], (unsigned long long)nlt);
        atomicAdd(&g_heavy_counts[2], (unsigned long long)nge);
        atomicAdd(&g_heavy_counts[3], 1ull);
#endif
    }
    __syncthreads();
    HPROF_LAP(0);
    const uint64_t* srt = stage_sort<true>(S, nlt);
    HPROF_LAP(1);
    *next_kind = 0;
    if (nlt == 0) return true;
    const int cur = S.cur, a = S.fsize;  // read by every thread before the groups part
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= 2) {
#ifdef VR_HPROF
        const long long tm = clock64();
#endif
        const int na = merge_group(S, srt, cur, a, nlt, 64, HT - 64, 1);
        if (threadIdx.x == 64) {
#ifdef VR_HPROF
            S.tp[16] += clock64() - tm;  // merge group alone
            S.tp[17] += a;
            S.tp[18] += nlt;
            S.tp[19] += 1;
#endif
            S.na = na;
            S.cur = cur ^ 1;
            S.fsize = min(na, FKEEP);
        }
    } else {
        const uint64_t* F = S.buf[cur];
        const uint64_t* run = srt;
        uint64_t pn = EMPTY;
        bool certain = false;
        if (wid == 0) {
            // the smallest row of F XOR run among the two 32-row heads: a row
            // survives unless the other head holds it (both arrays are unique),
            // exact for rows below row 32 of both
            const int fa = min(a, 32), fr = min(nlt, 32);
            const uint64_t f = lane < a ? F[lane] : EMPTY, r = lane < nlt ? run[lane] : EMPTY;
            int qf = 0, qr = 0;  // rows of the other head below f / r, by fixed steps
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                if (qf + st <= fr && run[qf + st - 1] < f) qf += st;
                if (qr + st <= fa && F[qr + st - 1] < r) qr += st;
            }
            const bool fs = f != EMPTY && !(qf < fr && run[qf] == f);
            const bool rs = r != EMPTY && !(qr < fa && F[qr] == r);
            // both heads ascend with the lane: each one's smallest survivor is
            // its first surviving lane
            const unsigned bf = __ballot_sync(0xffffffffu, fs), br = __ballot_sync(0xffffffffu, rs);
            const uint64_t f0 = __shfl_sync(0xffffffffu, f, bf ? __ffs(bf) - 1 : 0);
            const uint64_t r0 = __shfl_sync(0xffffffffu, r, br ? __ffs(br) - 1 : 0);
            pn = bf ? (br && r0 < f0 ? r0 : f0) : (br ? r0 : EMPTY);
            const uint64_t f32 = a > 32 ? F[32] : EMPTY, r32 = nlt > 32 ? run[32] : EMPTY;
            certain = pn < (f32 < r32 ? f32 : r32);
            if (lane == 0) { S.sel = certain ? pn : EMPTY; }
        }
        bar_sync(2, 64);
        HPROF_LAP(10);  // head check
        pn = S.sel;
        if (pn != EMPTY) {
            const int kind = heavy_owner_probe<P, true>(c, S, pn, self_key);
            if (threadIdx.x == 0) S.pkind = kind == 0 ? 3 : kind;  // 3: the pivot has no owner
        }
    }
    __syncthreads();
    HPROF_LAP(11);  // wait for the merge group
    const int na = S.na;
    *next_kind = S.pkind;
    const bool r = heavy_spill(S, B, bcap, na);
    HPROF_LAP(12);
    return r;
}

// Row key of x + {w} for the thread's w, if w is no vertex of x and the
// cofacet is within the threshold.
template <int P>
__device__ __forceinline__ bool cob_row(const Ctx& c, const Simplex<P>& x, int64_t w, uint64_t& key) {
    bool ok = w >= 0;
#pragma unroll
    for (int q = 0; q <= P; ++q) ok = ok && (w != x.v[q]);
    if (!ok) return false;
    uint32_t rt = x.r;
#pragma unroll
    for (int q = 0; q <= P; ++q) rt = max(rt, c.R(x.v[q], w));
    if (rt > c.thr) return false;
    key = row_key<P>(c, x, w, rt);
    return true;
}

// W <- W + D_x for the p-simplex x (vertices ascending, diameter rank x.r),
// HT candidate vertices w per pass, largest first, from the first-th.
template <int P>
__device__ bool heavy_add_coboundary(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, const Simplex<P>& x,
                                     int64_t first) {
    const Cands cw = cofacet_cands<P>(c, x.v);
    for (int64_t i0 = first; i0 < cw.cnt; i0 += HT) {
        const int64_t i = i0 + threadIdx.x;
        uint64_t key = EMPTY;
        const bool ok = cob_row<P>(c, x, i < cw.cnt ? cw[i] : -1, key);
        if (!heavy_cob_place(S, B, bcap, ok, key)) return false;
    }
    return true;
}
template <int P>
__device__ bool heavy_add_coboundary(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, const Simplex<P>& x) {
    return heavy_add_coboundary<P>(c, S, B, bcap, x, 0);
}

// Sort stage[0..cnt) (cnt <= HSTAGE), keep one row of every run of odd
// length (Z/2) and add the result to W.
__device__ bool heavy_flush_stage(HeavySmem& S, uint64_t* B, int64_t bcap, int cnt) {
    const uint64_t* srt = stage_sort(S, cnt);
    bool keep0 = false, keep1 = false;
    const int i0 = threadIdx.x, i1 = threadIdx.x + HT;
    uint64_t v0 = 0, v1 = 0;
    if (i0 < cnt && (i0 == 0 || srt[i0 - 1] != srt[i0])) {
        int e = i0;
        while (e + 1 < cnt && srt[e + 1] == srt[i0]) ++e;
        keep0 = ((e - i0 + 1) & 1) != 0;
        v0 = srt[i0];
    }
    if (i1 < cnt && (srt[i1 - 1] != srt[i1])) {
        int e = i1;
        while (e + 1 < cnt && srt[e + 1] == srt[i1]) ++e;
        keep1 = ((e - i1 + 1) & 1) != 0;
        v1 = srt[i1];
    }
    // rows 0..HT-1 first, then HT..2HT-1, so the kept rows stay in order
    int tot0, tot1;
    const int pos0 = block_excl_scan((int)keep0, S.ws, &tot0);  // syncs: all reads are done
    const int pos1 = block_excl_scan((int)keep1, S.ws, &tot1);
    if (keep0) S.stage[pos0] = v0;
    if (keep1) S.stage[tot0 + pos1] = v1;
    __syncthreads();
    return heavy_add_run(S, B, bcap, tot0 + tot1);
}

// W <- W + R_o where R_o is stored as its generators (store_generators):
// their coboundaries' rows are generated in turn, the rows at or above the
// split go straight to the back and the rest collect in the stage, which is
// flushed (sorted, cancelled, merged) only when the next pass might not fit
// -- one merge for several coboundaries instead of one addition each.
template <int P>
__device__ bool heavy_add_stored(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, int64_t opos) {
    const uint64_t* gk = reinterpret_cast<const uint64_t*>(c.rc_ptr[opos]);
    const int64_t len = c.rc_len[opos];
    int sc = 0;  // rows in the stage
    for (int64_t i = 0; i < len; ++i) {
        Simplex<P> g;
        load_col<P>(c, gk[i], g);
        const Cands cw = cofacet_cands<P>(c, g.v);
        for (int64_t i0 = 0; i0 < cw.cnt; i0 += HT) {
            const int64_t iw = i0 + threadIdx.x;
            uint64_t key = EMPTY;
            const bool ok = cob_row<P>(c, g, iw < cw.cnt ? cw[iw] : -1, key);
            const bool lt = ok && key < S.Ks, ge = ok && !lt;
            int tot;
            const int packed = block_excl_scan((int)lt | ((int)ge << 16), S.ws, &tot);
            const int nlt = tot & 0xFFFF, nge = tot >> 16;
            if (sc + nlt > HSTAGE) {  // flushing may lower Ks: rows kept below the old split stay valid
                if (!heavy_flush_stage(S, B, bcap, sc)) return false;
                sc = 0;
            }
            const int64_t bs = S.bsize;
            if (bs + nge > bcap) return false;
            if (ge) B[bs + (packed >> 16)] = key;
            if (lt) S.stage[sc + (packed & 0xFFFF)] = key;
            sc += nlt;
            __syncthreads();
            if (threadIdx.x == 0) S.bsize = bs + nge;
            __syncthreads();
        }
    }
    return sc == 0 || heavy_flush_stage(S, B, bcap, sc);
}

// W <- W + R_o where R_o = rows[0..len) is any multiset of rows (for example
// the front and the unsorted back of a column finished by the block engine;
// holes, EMPTY, are skipped).
// Rows at or above the split go straight to the back; rows below it collect
// in the stage, which is flushed (sorted, cancelled, merged) whenever the
// next tile might not fit.  The next tile is loaded before the current one
// is placed, so one memory latency per tile overlaps the block scan.
__device__ bool heavy_add_multiset(HeavySmem& S, uint64_t* B, int64_t bcap, const uint64_t* rows, int64_t len) {
    HPROF_T0();
    if (threadIdx.x == 0) S.tp[8] += 1;
    constexpr int PER = HSTAGE / HT;
    uint64_t nk[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int64_t i = (int64_t)q * HT + threadIdx.x;
        nk[q] = i < len ? rows[i] : EMPTY;
    }
    int sc = 0;  // rows in the stage
    for (int64_t base = 0; base < len; base += HSTAGE) {
        uint64_t k[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) k[q] = nk[q];
        if (base + HSTAGE < len) {
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int64_t i = base + HSTAGE + (int64_t)q * HT + threadIdx.x;
                nk[q] = i < len ? rows[i] : EMPTY;
            }
        }
        const uint64_t Ks = S.Ks;
        int cl = 0, cg = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (k[q] != EMPTY) {  // out of range, or a hole of a block-engine back
                if (k[q] < Ks) ++cl; else ++cg;
            }
        }
        int tot;
        const int packed = block_excl_scan(cl | (cg << 16), S.ws, &tot);
        const int nlt = tot & 0xFFFF, nge = tot >> 16;
        if (sc + nlt > HSTAGE) {  // flushing may lower Ks: rows kept below the old split stay valid
            if (!heavy_flush_stage(S, B, bcap, sc)) return false;
            sc = 0;
        }
        const int64_t bs = S.bsize;
        if (bs + nge > bcap) return false;
        int pl = sc + (packed & 0xFFFF);
        int64_t pg = bs + (packed >> 16);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (k[q] != EMPTY) {
                if (k[q] < Ks) S.stage[pl++] = k[q]; else B[pg++] = k[q];
            }
        }
        sc += nlt;
        __syncthreads();
        if (threadIdx.x == 0) S.bsize = bs + nge;
        __syncthreads();
    }
    const bool ok = sc == 0 || heavy_flush_stage(S, B, bcap, sc);
    HPROF_LAP(3);
    return ok;
}

// V mode: append `len` generator keys to the column's list; false if it has
// no room (the column then restarts with larger buffers).
__device__ bool heavy_v_append(HeavySmem& S, uint64_t* V, int64_t vcap, const uint64_t* src, int64_t len) {
    const int64_t at = S.vlen;
    if (at + len > vcap) return false;
    for (int64_t i = threadIdx.x; i < len; i += HT) V[at + i] = src[i];
    __syncthreads();  // every thread has read S.vlen
    if (threadIdx.x == 0) S.vlen = at + len;
    __syncthreads();
    return true;
}
__device__ bool heavy_v_append1(HeavySmem& S, uint64_t* V, int64_t vcap, uint64_t key) {
    const int64_t at = S.vlen;
    if (at + 1 > vcap) return false;
    __syncthreads();  // every thread has read S.vlen
    if (threadIdx.x == 0) {
        V[at] = key;
        S.vlen = at + 1;
    }
    __syncthreads();
    return true;
}
// Column key of the candidate apparent owner s' found by the last probe
// (S.ov[0..P], diameter rank S.orank).
template <int P>
__device__ uint64_t probed_owner_key(const Ctx& c, const HeavySmem& S) {
    uint64_t cidx = 0;
#pragma unroll
    for (int q = 0; q <= P; ++q) cidx += c.B(S.ov[q], q + 1);
    return ((~(uint64_t)S.orank & c.rmask) << c.cb) | cidx;
}

// Owner probe for pivot row rk: 1 = the pivot of a finished column (in
// S.opos), 2 = a candidate apparent owner s' (Def 5.3.4: the facet left by
// dropping the largest vertex whose removal keeps the diameter; S.ov[0..P],
// the dropped vertex in S.ov[P+1], the diameter rank in S.orank), 0 = none.
// A row has at most one owner: warp 1 probes the hash of finished columns
// while warp 0 decodes the pivot and finds the dropped vertex.
// With GROUP the probe is made by warps 0 and 1 alone (named barrier 2),
// while the rest of the block merges; the result is then read by those two
// warps only, until the block meets again.
template <int P, bool GROUP>
__device__ int heavy_owner_probe(const Ctx& c, HeavySmem& S, uint64_t rk, uint64_t self_key) {
    constexpr int NT = P + 2;
    constexpr int NPAIR = NT * (NT - 1) / 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = c.R.n;
    const uint32_t rt = (uint32_t)(rk >> c.rcb);
    const uint64_t ct = c.rcmask - (rk & c.rcmask);
    HPROF_T0();
    if (wid == 1) {
        const int64_t hp = warp_hash_find(c, ct);
        if (lane == 0) {
            S.opos = hp;
            if (hp >= 0 && !(c.cols[hp] < self_key)) atomicExch(c.err, DEV_INTERNAL | (4 << 8));  // owners come earlier
        }
    }
    if (wid == 0) {
        int drop = -1;
        int tv[NT];
        warp_decode_simplex<P + 1>(c.B, ct, n - 1, tv);
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
        if (lane == 0) {
            S.flag = drop >= 0 ? 2 : 0;
            if (drop >= 0) {
                int k = 0;
                for (int q = 0; q < NT; ++q)
                    if (q != drop) S.ov[k++] = tv[q];
                S.ov[P + 1] = tv[drop];
                S.orank = rt;
            }
        }
    }
    if (GROUP) bar_sync(2, 64); else __syncthreads();
    HPROF_LAP(13);
    return S.opos >= 0 ? 1 : S.flag;
}

// For a probe that returned 2: whether s' owns the pivot, i.e. no vertex w
// above the dropped one keeps the diameter of s' (s' has no older cofacet).
template <int P>
__device__ bool heavy_apparent_check(const Ctx& c, HeavySmem& S) {
    int ov[P + 1];
#pragma unroll
    for (int q = 0; q <= P; ++q) ov[q] = S.ov[q];
    const int64_t wd = S.ov[P + 1];
    const uint32_t rt = S.orank;
    const Cands cw = cofacet_cands<P>(c, ov);
    bool older = false;
    for (int64_t i0 = 0; i0 < cw.cnt && cw[i0] > wd; i0 += HT) {  // largest first: stop below wd
        const int64_t i = i0 + (int64_t)threadIdx.x;
        const int64_t w = i < cw.cnt ? cw[i] : -1;
        bool ok = w > wd;
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (w != ov[q]);
#pragma unroll
        for (int q = 0; q <= P; ++q) ok = ok && (c.R(ov[q], w) <= rt);
        older = older || ok;
    }
    return !__syncthreads_or(older);
}

// For a probe that returned 2: if s' owns the pivot, W <- W + D_{s'} and 1;
// -1 if it does not (the pivot has no owner); 0 if B overflowed.
// *next_kind: the owner kind of the next pivot when it was probed during
// the merge (see heavy_cob_place_next), else 0.  When one
// pass of HT vertices covers every w above the dropped vertex, the ownership
// test and the first pass of D_{s'} share their rank reads: each thread's
// w is an older cofacet of s' exactly when its diameter stays at s''s.
template <int P, bool OVERLAP = true>
__device__ int heavy_apparent_add(const Ctx& c, HeavySmem& S, uint64_t* B, int64_t bcap, uint64_t self_key,
                                  int* next_kind) {
    *next_kind = 0;
    Simplex<P> o;
#pragma unroll
    for (int q = 0; q <= P; ++q) o.v[q] = S.ov[q];
    o.r = S.orank;
    const int64_t wd = S.ov[P + 1];
    const Cands cw = cofacet_cands<P>(c, o.v);
    if (cw.cnt > HT && cw[HT] > wd) {  // the first pass does not reach every candidate above wd
        if (!heavy_apparent_check<P>(c, S)) return -1;
        return heavy_add_coboundary<P>(c, S, B, bcap, o) ? 1 : 0;
    }
    HPROF_T0();
    const int64_t w = (int64_t)threadIdx.x < cw.cnt ? cw[threadIdx.x] : -1;
    bool ok = w >= 0, older = false;
#pragma unroll
    for (int q = 0; q <= P; ++q) ok = ok && (w != o.v[q]);
    uint64_t key = EMPTY;
    if (ok) {
        uint32_t mx = 0;
#pragma unroll
        for (int q = 0; q <= P; ++q) mx = max(mx, c.R(o.v[q], w));
        older = w > wd && mx <= o.r;
        const uint32_t rt = max(o.r, mx);
        ok = rt <= c.thr;
        if (ok) key = row_key<P>(c, o, w, rt);
    }
    if (__syncthreads_or(older)) return -1;
    HPROF_LAP(14);
    if (OVERLAP && cw.cnt <= HT)  // this was the only pass: probe the next pivot's owner during the merge
        return heavy_cob_place_next<P>(c, S, B, bcap, ok, key, self_key, next_kind) ? 1 : 0;
    if (!heavy_cob_place(S, B, bcap, ok, key)) return 0;
    return heavy_add_coboundary<P>(c, S, B, bcap, o, HT) ? 1 : 0;
}

}  // namespace
}  // namespace vr
