// hypha.cu -- persistence pairs of an explicit Z/2 boundary matrix with the
// GPU-scan, clearing and compression phases of HYPHA (paper, arXiv
// 2502.05063, Ch. 4: Algorithms 3-6 for the scan, Algorithm 7 clearing,
// Algorithms 8-9 compression, Algorithm 10 the whole), followed by the
// standard reduction (Algorithm 2) of the columns the scan leaves unstable.
//
// The matrix is the boundary matrix of a filtered simplicial complex, columns
// (and rows) in filtration order, in CSC form with the rows of each column
// ascending.  Notation: low(j) = the largest row of column j.
//
//  GPU scan.  Left[r] = the smallest column with an entry in row r (atomicMin
//    over all entries).  A column whose low is the leftmost entry of its row
//    needs no addition in Algorithm 2 (nothing to its left shares the low): it
//    is stable, Lookup[low(j)] = j, and column low(j) is zeroed (clearing).
//    Empty columns are stable.  The others are collected, in order, as the
//    unstable columns (warp-aggregated append, then a sort to restore order).
//  Clearing (Lemma 4.2.3).  For every nonzero column j, column low(j) is a
//    creator (on a boundary matrix the last facet of a simplex closes a cycle)
//    and reduces to zero: it is marked cleared.
//  Compression (Lemma 4.2.4, Lemma 4.2.5).  A row r can never be a pivot row
//    (and may be dropped from every column) if column r contains the leftmost
//    entry of some row (it must eventually have a pivot), or if row r is the
//    pivot of a stable column all of whose other rows can be dropped.  The
//    other rows of a stable column lie above its pivot, so the rule is a
//    recursion over smaller rows; it is evaluated as a fixed point, one pass
//    over the candidate rows per level.  Then each unstable column (one thread
//    each) walks its rows from the largest down: droppable rows go, and a row
//    that is the pivot of a stable column to its left is cancelled by adding
//    that column (Algorithm 8).
//  Final reduction.  The unstable columns, in order, by Algorithm 2 with the
//    lookup of known pivots; droppable rows are dropped from every column
//    involved.  It is sequential by nature (each column waits for the pivots
//    of the columns before it) and runs as one small block on the device, each
//    addition a merge of sorted rows.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "vr_common.cuh"

namespace vr {
namespace {

constexpr int32_t INF32 = 0x7FFFFFFF;
constexpr uint8_t C_UNKNOWN = 0, C_YES = 1, C_NO = 2;

__device__ __forceinline__ int32_t col_low(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t j) {
    const int64_t a = cp[j], b = cp[j + 1];
    return b > a ? rows[b - 1] : -1;
}

// Algorithm 4: leftmost column of every row; empty columns are stable
__global__ void k_set_leftmost(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t n,
                               int32_t* __restrict__ left, uint8_t* __restrict__ stable) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = cp[j], b = cp[j + 1];
        if (a == b) stable[j] = 1;
        for (int64_t e = a; e < b; ++e) atomicMin(left + rows[e], (int32_t)j);
    }
}

// Algorithm 5: pivots of 0-addition columns; their low columns are cleared
__global__ void k_set_lookup(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t n,
                             const int32_t* __restrict__ left, int32_t* __restrict__ lookup,
                             uint8_t* __restrict__ stable) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = col_low(cp, rows, j);
        if (l >= 0 && left[l] == (int32_t)j) {
            lookup[l] = (int32_t)j;
            stable[j] = 1;
            stable[l] = 1;
        }
    }
}

// Algorithm 7 (Lemma 4.2.3): the low of every nonzero column is a zero column
__global__ void k_clear_lows(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t n,
                             uint8_t* __restrict__ cleared) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = col_low(cp, rows, j);
        if (l >= 0) cleared[l] = 1;
    }
}

// Algorithm 6: the columns neither stable nor cleared, warp-aggregated
__global__ void k_set_unstable(int64_t n, const uint8_t* __restrict__ stable, const uint8_t* __restrict__ cleared,
                               int32_t* __restrict__ u, unsigned long long* __restrict__ nu) {
    const int lane = threadIdx.x & 31;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; b < n;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = b + lane;
        const bool un = j < n && !stable[j] && !cleared[j];
        const uint32_t bl = __ballot_sync(0xffffffffu, un);
        unsigned long long base = 0;
        if (lane == 0 && bl) base = atomicAdd(nu, (unsigned long long)__popc(bl));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (un) u[base + __popc(bl & ((1u << lane) - 1u))] = (int32_t)j;
    }
}

__global__ void k_fill_i32(int32_t* __restrict__ a, int64_t m, int32_t v) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        a[k] = v;
}

// rows that are column indices holding some leftmost entry (Lemma 4.2.5)
__global__ void k_mark_in_left(const int32_t* __restrict__ left, int64_t n, uint8_t* __restrict__ C) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = left[r];
        if (c != INF32) C[c] = C_YES;
    }
}

// Algorithm 9 as a fixed point: a row that is the pivot of a stable column is
// compressible iff every other row of that column is; undecided rows are
// decided once their smaller rows are.  *changed counts decisions this pass.
__global__ void k_compressible_pass(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t n,
                                    const int32_t* __restrict__ lookup, uint8_t* __restrict__ C,
                                    unsigned long long* __restrict__ changed) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (C[r] != C_UNKNOWN) continue;
        const int32_t L = lookup[r];
        if (L < 0) {
            C[r] = C_NO;
            atomicAdd(changed, 1ull);
            continue;
        }
        bool all = true, known = true;
        for (int64_t e = cp[L]; e < cp[L + 1]; ++e) {
            const int32_t k = rows[e];
            if (k == (int32_t)r) continue;
            const uint8_t ck = ((volatile uint8_t*)C)[k];
            if (ck == C_NO) { all = false; break; }
            if (ck == C_UNKNOWN) known = false;
        }
        if (!all) { C[r] = C_NO; atomicAdd(changed, 1ull); }
        else if (known) { C[r] = C_YES; atomicAdd(changed, 1ull); }
    }
}

// Row r may be dropped from column j (compression): it is compressible and
// either no stable column has its pivot in row r (Lemma 4.2.5 row: never a
// pivot row, Lemma 4.2.4) or that stable column L lies left of j (adding L,
// whose other rows are all droppable, would only cancel r; every stable
// column in that recursion lies left of L, since each is the leftmost
// column of its row and L has an entry in that row).
__device__ __forceinline__ bool droppable(const uint8_t* __restrict__ C, const int32_t* __restrict__ lk0, int32_t r,
                                          int32_t j) {
    if (C[r] != C_YES) return false;
    const int32_t L = lk0[r];
    return L < 0 || L < j;
}

// Algorithm 8, one thread per unstable column: walk the rows from the largest
// down; a droppable row goes; a row that is the pivot of a stable column to
// the left is cancelled by adding that column (all of whose other rows are
// smaller).  The column is rewritten into its scratch slot (two halves of
// `cap` rows); if it would not fit, it is left as it was (out_len = -1).
__global__ void k_apply_compression(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows,
                                    const int32_t* __restrict__ u, int64_t nu, const int32_t* __restrict__ lk0,
                                    const uint8_t* __restrict__ C, int32_t* __restrict__ scratch, int64_t cap,
                                    int32_t* __restrict__ out_len, unsigned long long* __restrict__ adds) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nu; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t cid = u[q];
        int32_t* col = scratch + q * 2 * cap;
        int32_t* tmp = col + cap;
        const int64_t a = cp[cid], b = cp[cid + 1];
        int64_t len = b - a;
        if (len > cap) { out_len[q] = -1; continue; }
        for (int64_t e = 0; e < len; ++e) col[e] = rows[a + e];
        bool ok = true;
        unsigned long long na = 0;
        int64_t pos = len - 1;
        while (pos >= 0) {
            const int32_t rid = col[pos];
            if (droppable(C, lk0, rid, cid)) {
                for (int64_t t = pos; t + 1 < len; ++t) col[t] = col[t + 1];
                --len;
                --pos;
                continue;
            }
            const int32_t pc = lk0[rid];
            if (pc >= 0 && pc < cid) {
                // col[0..pos] XOR column pc (its low is rid, so rid cancels), then the rows above
                const int64_t pa = cp[pc], pb = cp[pc + 1];
                int64_t i = 0, k = pa, w = 0;
                while (i <= pos || k < pb) {
                    const int32_t x = i <= pos ? col[i] : INF32, y = k < pb ? rows[k] : INF32;
                    if (w >= cap) { ok = false; break; }
                    if (x == y) { ++i; ++k; continue; }
                    if (x < y) { tmp[w++] = x; ++i; } else { tmp[w++] = y; ++k; }
                }
                if (!ok) break;
                const int64_t above = len - 1 - pos;
                if (w + above > cap) { ok = false; break; }
                for (int64_t t = 0; t < above; ++t) tmp[w + t] = col[pos + 1 + t];
                len = w + above;
                for (int64_t t = 0; t < len; ++t) col[t] = tmp[t];
                pos = w - 1;
                ++na;
                continue;
            }
            --pos;  // kept
        }
        out_len[q] = ok ? (int32_t)len : -1;
        if (ok && na) atomicAdd(adds, na);
    }
}

// Final phase: Algorithm 2 on the unstable columns in order, by one warp.
// A row travels with the first column index from which it is droppable
// (droppable(r, j) <=> j >= t), so dropping needs no further lookup; the
// owner of a pivot row, and where its reduced column lives (the input rows of
// a stable column, or the pool for a column reduced here), is one 16-byte
// record.  Each addition: read the owner record of the working column's low,
// load the owner's rows that column j keeps (one coalesced pass, ballot
// compaction), and merge them into the working column by warp merge path.
struct __align__(8) RowT {
    int32_t r;  // row
    int32_t t;  // the row is droppable for columns j >= t (INF32: never)
};
constexpr int OWN_IN = 4;  // rows kept in the record itself (input columns of dimension <= 2 have at most 3)
struct __align__(16) Owner {
    int64_t off;  // of its rows in `rows_t` or, with POOL_BIT, in `pool`
    int32_t len;
    int32_t col;  // the owning column, -1: none
    RowT in[OWN_IN];  // its rows when len <= OWN_IN: one read per addition
};
constexpr int64_t POOL_BIT = (int64_t)1 << 62;

__global__ void k_drop_from(const uint8_t* __restrict__ C, const int32_t* __restrict__ lk0, int64_t n,
                            int32_t* __restrict__ T) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        T[r] = C[r] != C_YES ? INF32 : (lk0[r] < 0 ? 0 : lk0[r] + 1);  // as droppable(), reading L < 0 || L < j
}

__global__ void k_rows_t(const int32_t* __restrict__ rows, int64_t nnz, const int32_t* __restrict__ T,
                         RowT* __restrict__ rows_t) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        rows_t[e] = RowT{rows[e], T[rows[e]]};
}

// owner records of the pivots the scan found (stable columns)
__global__ void k_owner_init(const int64_t* __restrict__ cp, int64_t n, const int32_t* __restrict__ lk0,
                             const RowT* __restrict__ rows_t, Owner* __restrict__ own) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = lk0[r];
        Owner w{};
        w.col = -1;
        if (o >= 0) {
            w.off = cp[o];
            w.len = (int32_t)(cp[o + 1] - cp[o]);
            w.col = o;
            if (w.len <= OWN_IN)
                for (int i = 0; i < w.len; ++i) w.in[i] = rows_t[w.off + i];
        }
        own[r] = w;
    }
}

// out <- a XOR b for ascending rows without repeats, by one warp; returns the
// length.  Lane L starts at diagonal L * per of the merged sequence (equal rows:
// a's first, and a boundary between equal rows moves before them, so a
// cancelling pair is never split); a first walk counts each lane's cancelling
// pairs, a warp scan turns the counts into output offsets, a second walk writes.
__device__ int warp_xor_merge(const RowT* a, int la, const RowT* b, int lb, RowT* out) {
    const int lane = threadIdx.x & 31;
    const int tot = la + lb;
    const int per = (tot + 31) >> 5;
    const int d = min(tot, lane * per);
    int lo = max(0, d - la), hi = min(d, lb);  // b rows among the first d: largest k with b[k-1] < a[d-k]
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (b[m - 1].r < a[d - m].r) lo = m;
        else hi = m - 1;
    }
    const int k0 = lo;
    int i0 = d - lo;
    if (i0 > 0 && k0 < lb && a[i0 - 1].r == b[k0].r) --i0;
    int i1 = __shfl_down_sync(0xffffffffu, i0, 1), k1 = __shfl_down_sync(0xffffffffu, k0, 1);
    if (lane == 31) {
        i1 = la;
        k1 = lb;
    }
    int c = 0;
    for (int i = i0, k = k0; i < i1 && k < k1;) {
        const int32_t x = a[i].r, y = b[k].r;
        c += x == y;
        i += x <= y;
        k += y <= x;
    }
    int cs = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, cs, o);
        if (lane >= o) cs += t;
    }
    const int ctot = __shfl_sync(0xffffffffu, cs, 31);
    int pos = i0 + k0 - 2 * (cs - c);
    for (int i = i0, k = k0; i < i1 || k < k1;) {
        const int32_t x = i < i1 ? a[i].r : INF32, y = k < k1 ? b[k].r : INF32;
        if (x == y) {
            ++i;
            ++k;
        } else if (x < y) {
            out[pos++] = a[i++];
        } else {
            out[pos++] = b[k++];
        }
    }
    __syncwarp();
    return tot - 2 * ctot;
}

// rows of src[0..len) that column j keeps, appended in order at dst[at..); returns the new end
__device__ __forceinline__ int warp_keep(const RowT* src, int64_t len, int32_t j, RowT* dst, int at) {
    const int lane = threadIdx.x & 31;
    for (int64_t e0 = 0; e0 < len; e0 += 32) {
        const int64_t e = e0 + lane;
        RowT x{INF32, 0};
        bool keep = false;
        if (e < len) {
            x = src[e];
            keep = j < x.t;
        }
        const unsigned bl = __ballot_sync(0xffffffffu, keep);
        if (keep) dst[at + __popc(bl & ((1u << lane) - 1u))] = x;
        at += __popc(bl);
    }
    return at;
}

struct FinalArgs {
    const int64_t* cp;
    const RowT* rows_t;  // the input rows with their drop thresholds
    const int32_t* u;
    int64_t nu;
    const int32_t* scratch;  // compressed slots, converted to RowT pairs (k_slot_rows_t)
    int64_t cap;
    const int32_t* clen;
    Owner* own;          // per row: the owner of that pivot, updated with the new pivots
    RowT* pool;
    int64_t pool_cap;
    RowT* work;          // three working buffers of work_cap rows
    int64_t work_cap;
    int fs;              // rows the shared buffers take (FS; lowered by VR_HYPHA_SHARED_ROWS for tests)
    int32_t* low_out;    // n
    unsigned long long* adds;
    int* err;
};

// In place: the compressed rows of each slot (int32) become RowT pairs, from
// the last one down (pair e covers the int32 entries 2e and 2e+1, all read by then).
__global__ void k_slot_rows_t(int32_t* __restrict__ scratch, int64_t cap, const int32_t* __restrict__ clen,
                              int64_t nu, const int32_t* __restrict__ T) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nu; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t len = clen[q];
        int32_t* col = scratch + q * 2 * cap;
        RowT* out = reinterpret_cast<RowT*>(col);
        for (int32_t e = len - 1; e >= 0; --e) {
            const int32_t r = col[e];
            out[e] = RowT{r, T[r]};
        }
    }
}

constexpr int FT = 32;
constexpr int FS = 4096;  // rows of each shared working buffer (the global ones take longer columns)

// where the rows of unstable column q are: its compressed slot, or its input rows
struct ColSrc {
    const RowT* src;
    int64_t len;
};
__device__ __forceinline__ ColSrc col_src(const FinalArgs& A, int64_t q, int32_t clen, int64_t a, int64_t b) {
    if (clen >= 0) return ColSrc{reinterpret_cast<const RowT*>(A.scratch + q * 2 * A.cap), clen};
    return ColSrc{A.rows_t + a, b - a};
}

// The unstable columns in order.  Their inputs do not depend on the reduction,
// so they are fetched ahead in three stages that never wait on one another:
// while column q is reduced, the first 32 rows of column q+1, the offsets of
// column q+2 and the index of column q+3 are in flight.
__global__ void __launch_bounds__(FT, 1) k_final_reduce(FinalArgs A) {
    extern __shared__ __align__(16) unsigned char fsm[];
    RowT* sw = reinterpret_cast<RowT*>(fsm);  // three buffers of FS rows
    const int lane = threadIdx.x & 31;
    const int64_t nu = A.nu;
    unsigned long long adds = 0;
    int64_t pool_used = 0;
    const RowT none{INF32, 0};
    // prime the pipeline
    int32_t j0 = A.u[0], c0 = A.clen[0];
    ColSrc s0 = col_src(A, 0, c0, c0 < 0 ? A.cp[j0] : 0, c0 < 0 ? A.cp[j0 + 1] : 0);
    RowT r0 = lane < s0.len ? s0.src[lane] : none;
    int32_t j1 = -1, c1 = 0;
    int64_t a1 = 0, b1 = 0;
    if (nu > 1) {
        j1 = A.u[1];
        c1 = A.clen[1];
        if (c1 < 0) {
            a1 = A.cp[j1];
            b1 = A.cp[j1 + 1];
        }
    }
    int32_t j2 = -1, c2 = 0;
    if (nu > 2) {
        j2 = A.u[2];
        c2 = A.clen[2];
    }
    for (int64_t q = 0; q < nu; ++q) {
        // stage loads for the next three columns (consumed in later iterations)
        int32_t j3 = -1, c3 = 0;
        if (q + 3 < nu) {
            j3 = A.u[q + 3];
            c3 = A.clen[q + 3];
        }
        int64_t a2 = 0, b2 = 0;
        if (q + 2 < nu && c2 < 0) {
            a2 = A.cp[j2];
            b2 = A.cp[j2 + 1];
        }
        ColSrc s1{nullptr, 0};
        RowT r1 = none;
        if (q + 1 < nu) {
            s1 = col_src(A, q + 1, c1, a1, b1);
            if (lane < s1.len) r1 = s1.src[lane];
        }
        // reduce column q
        const int32_t j = j0;
        if (s0.len > A.work_cap) {
            if (lane == 0) atomicExch(A.err, DEV_CAPACITY);
            return;
        }
        bool big = s0.len > A.fs;  // the working column and the owner's kept rows in shared memory while they fit
        RowT* w0 = big ? A.work : sw;
        RowT* w1 = big ? A.work + A.work_cap : sw + FS;
        RowT* wb = big ? A.work + 2 * A.work_cap : sw + 2 * FS;
        int len;
        {
            const bool keep = lane < s0.len && j < r0.t;
            const unsigned bl = __ballot_sync(0xffffffffu, keep);
            if (keep) w0[__popc(bl & ((1u << lane) - 1u))] = r0;
            len = __popc(bl);
            if (s0.len > 32) len = warp_keep(s0.src + 32, s0.len - 32, j, w0, len);
        }
        __syncwarp();
        for (;;) {
            if (len == 0) break;
            const int32_t low = w0[len - 1].r;
            const Owner ow = A.own[low];
            if (ow.col < 0 || ow.col >= j) break;  // the pivot is new: j is reduced
            if ((int64_t)len + ow.len > A.work_cap) {
                if (lane == 0) atomicExch(A.err, DEV_CAPACITY);
                return;
            }
            if (!big && len + ow.len > A.fs) {  // move to the global buffers
                for (int e = lane; e < len; e += 32) A.work[e] = w0[e];
                __syncwarp();
                big = true;
                w0 = A.work;
                w1 = A.work + A.work_cap;
                wb = A.work + 2 * A.work_cap;
            }
            int lb;
            if (ow.len <= OWN_IN) {  // the rows came with the record
                RowT x = none;
#pragma unroll
                for (int i = 0; i < OWN_IN; ++i)
                    if (lane == i && i < ow.len) x = ow.in[i];
                const bool keep = lane < ow.len && j < x.t;
                const unsigned bl = __ballot_sync(0xffffffffu, keep);
                if (keep) wb[__popc(bl & ((1u << lane) - 1u))] = x;
                lb = __popc(bl);
            } else {
                const RowT* osrc = (ow.off & POOL_BIT) ? A.pool + (ow.off & ~POOL_BIT) : A.rows_t + ow.off;
                lb = warp_keep(osrc, ow.len, j, wb, 0);
            }
            __syncwarp();
            len = warp_xor_merge(w0, len, wb, lb, w1);
            RowT* t = w0;
            w0 = w1;
            w1 = t;
            ++adds;
        }
        if (len > 0) {
            if (pool_used + len > A.pool_cap) {
                if (lane == 0) atomicExch(A.err, DEV_CAPACITY);
                return;
            }
            for (int e = lane; e < len; e += 32) A.pool[pool_used + e] = w0[e];
            const int32_t low = w0[len - 1].r;
            if (lane == 0) {
                Owner w{};
                w.off = pool_used | POOL_BIT;
                w.len = len;
                w.col = j;
                if (len <= OWN_IN)
                    for (int i = 0; i < len; ++i) w.in[i] = w0[i];
                A.own[low] = w;
                A.low_out[j] = low;
            }
            pool_used += len;
        }
        __syncwarp();
        // advance the pipeline
        j0 = j1;
        s0 = s1;
        r0 = r1;
        j1 = j2;
        c1 = c2;
        a1 = a2;
        b1 = b2;
        j2 = j3;
        c2 = c3;
    }
    if (lane == 0) atomicAdd(A.adds, adds);
}

// lows of the stable nonzero columns (their input lows are final)
__global__ void k_stable_lows(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t n,
                              const uint8_t* __restrict__ stable, const uint8_t* __restrict__ cleared,
                              const int32_t* __restrict__ lookup, int32_t* __restrict__ low_out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = col_low(cp, rows, j);
        low_out[j] = (stable[j] && !cleared[j] && l >= 0 && lookup[l] == (int32_t)j) ? l : -1;
    }
}


__global__ void k_check_rows(const int64_t* __restrict__ cp, const int32_t* __restrict__ rows, int64_t n,
                             int* __restrict__ err) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = cp[j], b = cp[j + 1];
        if (a < 0 || b < a) { atomicExch(err, DEV_BAD_INPUT); continue; }
        for (int64_t e = a; e < b; ++e) {
            const int32_t r = rows[e];
            // rows ascending, strictly above the diagonal (a face comes first)
            if (r < 0 || r >= j || (e > a && rows[e - 1] >= r)) { atomicExch(err, DEV_BAD_INPUT); break; }
        }
    }
}

// CUDA events between the phases, on the call's stream
struct StageTimer {
    cudaStream_t s;
    cudaEvent_t ev[8];
    int k = 0;
    explicit StageTimer(cudaStream_t st) : s(st) { mark(); }
    void mark() {
        if (k < 8 && cudaEventCreate(&ev[k]) == cudaSuccess) cudaEventRecord(ev[k++], s);
    }
    float ms(int i) const {  // between marks i and i+1 (after a synchronisation)
        float t = 0.f;
        if (i + 1 < k && cudaEventElapsedTime(&t, ev[i], ev[i + 1]) != cudaSuccess) t = 0.f;
        return t;
    }
    ~StageTimer() {
        for (int i = 0; i < k; ++i) cudaEventDestroy(ev[i]);
    }
};

unsigned hgrid(int64_t m) {
    int64_t b = (m + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 148 * 16 ? 148 * 16 : b));
}

}  // namespace
}  // namespace vr

extern "C" vr_status vr_hypha_pairs(const int64_t* colptr, const int32_t* rows, int64_t ncols, int64_t nnz,
                                    uint32_t flags, void* stream, int32_t* out_low, vr_hypha_stats* stats) {
    using namespace vr;
    if (ncols < 0 || nnz < 0 || (ncols > 0 && (!colptr || !out_low)) || (nnz > 0 && !rows) ||
        ncols >= (int64_t)INF32 || flags != 0)
        return VR_ERR_INVALID_ARG;
    if (ncols == 0) {
        if (stats) memset(stats, 0, sizeof *stats);
        return VR_OK;
    }
    try {
        cudaStream_t s = (cudaStream_t)stream;
        Workspace ws(s);
        HostScratch hs;
        const int64_t n = ncols;
        int64_t* cp = ws.alloc_n<int64_t>(n + 1);
        int32_t* rw = ws.alloc_n<int32_t>(nnz > 0 ? nnz : 1);
        VR_CUDA(cudaMemcpyAsync(cp, colptr, (n + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
        if (nnz > 0) VR_CUDA(cudaMemcpyAsync(rw, rows, nnz * sizeof(int32_t), cudaMemcpyDefault, s));
        int* err = ws.zeros_n<int>(1);
        k_check_rows<<<hgrid(n), 256, 0, s>>>(cp, rw, n, err);
        int32_t* left = ws.alloc_n<int32_t>(n);
        int32_t* lookup = ws.alloc_n<int32_t>(n);
        uint8_t* stable = ws.zeros_n<uint8_t>(n);
        uint8_t* cleared = ws.zeros_n<uint8_t>(n);
        uint8_t* C = ws.zeros_n<uint8_t>(n);
        k_fill_i32<<<hgrid(n), 256, 0, s>>>(left, n, INF32);
        VR_CUDA(cudaMemsetAsync(lookup, 0xFF, n * sizeof(int32_t), s));
        StageTimer tm(s);
        // ---- GPU scan (Algorithms 3-6) and clearing (Algorithm 7)
        k_set_leftmost<<<hgrid(n), 256, 0, s>>>(cp, rw, n, left, stable);
        k_set_lookup<<<hgrid(n), 256, 0, s>>>(cp, rw, n, left, lookup, stable);
        k_clear_lows<<<hgrid(n), 256, 0, s>>>(cp, rw, n, cleared);
        int32_t* u = ws.alloc_n<int32_t>(n);
        unsigned long long* ctr = ws.zeros_n<unsigned long long>(4);  // [0] nu [1] changed [2] comp adds [3] adds
        k_set_unstable<<<hgrid(n), 256, 0, s>>>(n, stable, cleared, u, ctr);
        VR_CUDA(cudaGetLastError());
        tm.mark();
        VR_CUDA(cudaMemcpyAsync(&hs.p[0], ctr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        int h_err = 0;
        VR_CUDA(cudaMemcpyAsync(&hs.p[1], err, sizeof(int), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        h_err = (int)(hs.p[1] & 0xFFFFFFFF);
        if (h_err) throw Error{VR_ERR_INVALID_ARG};
        const int64_t nu = hs.p[0];
        // the unstable columns in column order (the append is unordered)
        if (nu > 1) {
            uint32_t* key = reinterpret_cast<uint32_t*>(u);
            radix_sort_u32(ws, key, nullptr, nu, 32);
        }
        // ---- compression (Algorithms 8-9)
        int64_t passes = 0;
        if (nu > 0) {
            k_mark_in_left<<<hgrid(n), 256, 0, s>>>(left, n, C);
            for (;;) {
                VR_CUDA(cudaMemsetAsync(ctr + 1, 0, sizeof(unsigned long long), s));
                k_compressible_pass<<<hgrid(n), 256, 0, s>>>(cp, rw, n, lookup, C, ctr + 1);
                VR_CUDA(cudaMemcpyAsync(&hs.p[2], ctr + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
                VR_CUDA(cudaStreamSynchronize(s));
                ++passes;
                if (hs.p[2] == 0) break;
            }
        }
        tm.mark();
        const int64_t cap = 256;  // rows a compressed column may hold in its slot
        int32_t* scratch = ws.alloc_n<int32_t>((size_t)std::max<int64_t>(nu, 1) * 2 * cap);
        int32_t* clen = ws.alloc_n<int32_t>(std::max<int64_t>(nu, 1));
        int32_t* lk0 = ws.alloc_n<int32_t>(n);  // the scan's pivots, before the final phase adds its own
        VR_CUDA(cudaMemcpyAsync(lk0, lookup, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (nu > 0) {
            k_apply_compression<<<hgrid(nu), 256, 0, s>>>(cp, rw, u, nu, lk0, C, scratch, cap, clen, ctr + 2);
            VR_CUDA(cudaGetLastError());
        }
        tm.mark();
        // ---- final reduction of the unstable columns
        int32_t* low_d = ws.alloc_n<int32_t>(n);
        k_stable_lows<<<hgrid(n), 256, 0, s>>>(cp, rw, n, stable, cleared, lookup, low_d);
        if (nu > 0) {
            int32_t* T = ws.alloc_n<int32_t>(n);
            RowT* rows_t = ws.alloc_n<RowT>(std::max<int64_t>(nnz, 1));
            Owner* own = ws.alloc_n<Owner>(n);
            k_drop_from<<<hgrid(n), 256, 0, s>>>(C, lk0, n, T);
            k_rows_t<<<hgrid(nnz), 256, 0, s>>>(rw, nnz, T, rows_t);
            k_owner_init<<<hgrid(n), 256, 0, s>>>(cp, n, lk0, rows_t, own);
            k_slot_rows_t<<<hgrid(nu), 256, 0, s>>>(scratch, cap, clen, nu, T);
            FinalArgs A;
            A.cp = cp; A.rows_t = rows_t; A.u = u; A.nu = nu; A.scratch = scratch; A.cap = cap;
            A.clen = clen; A.own = own;
            A.pool_cap = std::max<int64_t>(nnz * 8, 1 << 20);
            A.pool = ws.alloc_n<RowT>(A.pool_cap);
            A.work_cap = std::max<int64_t>(n, 1 << 16);
            A.work = ws.alloc_n<RowT>(3 * A.work_cap);
            A.low_out = low_d;
            A.adds = ctr + 3;
            A.err = err;
            A.fs = FS;
            if (const char* v = getenv("VR_HYPHA_SHARED_ROWS")) A.fs = (int)std::min<long>(FS, std::max(1L, atol(v)));
            const size_t fsmem = 3 * FS * sizeof(RowT);
            VR_CUDA(cudaFuncSetAttribute(k_final_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
            k_final_reduce<<<1, FT, fsmem, s>>>(A);
            VR_CUDA(cudaGetLastError());
        }
        tm.mark();
        VR_CUDA(cudaMemcpyAsync(out_low, low_d, n * sizeof(int32_t), cudaMemcpyDefault, s));
        VR_CUDA(cudaMemcpyAsync(hs.p + 4, ctr, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaMemcpyAsync(&hs.p[1], err, sizeof(int), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        if ((hs.p[1] & 0xFF) == DEV_CAPACITY) throw Error{VR_ERR_OOM};
        if (hs.p[1] & 0xFF) throw Error{VR_ERR_INTERNAL};
        if (stats) {
            memset(stats, 0, sizeof *stats);
            stats->columns = n;
            stats->unstable = nu;
            stats->compression_passes = passes;
            stats->compression_additions = hs.p[6];
            stats->additions = hs.p[7];
            stats->ms_scan = tm.ms(0);
            stats->ms_compression = tm.ms(1) + tm.ms(2);
            stats->ms_reduce = tm.ms(3);
        }
        return VR_OK;
    } catch (const Error& e) {
        return e.code;
    } catch (const std::bad_alloc&) {
        return VR_ERR_OOM;
    }
}
