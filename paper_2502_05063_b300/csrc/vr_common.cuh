// vr_common.cuh -- internal declarations shared by the libvrgpu translation
// units (device helpers, the per-call workspace and the stage launchers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "vr.h"

namespace vr {

// ---------------------------------------------------------------------------
// status plumbing
// ---------------------------------------------------------------------------
struct Error {
    vr_status code;
};

#define VR_CUDA(expr)                                                        \
    do {                                                                     \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) {                                             \
            vr::set_last_cuda_error(e_, #expr, __FILE__, __LINE__);          \
            throw vr::Error{e_ == cudaErrorMemoryAllocation ? VR_ERR_OOM     \
                                                            : VR_ERR_CUDA}; \
        }                                                                    \
    } while (0)

#define VR_CHECK(cond, status)                                               \
    do {                                                                     \
        if (!(cond)) throw vr::Error{status};                                \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
bool log_enabled();  // VR_LOG=1 in the environment: per-stage timings on stderr

// Device-side error word written by kernels (capacity, input and consistency checks).
enum DeviceError : int {
    DEV_OK = 0,
    DEV_CAPACITY = 1,   // a scratch buffer was too small
    DEV_TIMEOUT = 2,    // reserved: no kernel waits on another, so none writes it
    DEV_INTERNAL = 3,   // a consistency check failed
    DEV_BAD_INPUT = 4,  // NaN / negative distance
};

// ---------------------------------------------------------------------------
// per-call workspace: stream-ordered allocations released together
// ---------------------------------------------------------------------------
class Workspace {
  public:
    explicit Workspace(cudaStream_t s);
    ~Workspace();
    void* alloc(size_t bytes);  // 256-byte aligned, not zeroed
    template <class T>
    T* alloc_n(size_t n) { return static_cast<T*>(alloc(n * sizeof(T) + 16)); }
    template <class T>
    T* zeros_n(size_t n) {
        T* p = alloc_n<T>(n);
        VR_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
        return p;
    }
    void free_all();
    cudaStream_t stream;

  private:
    std::vector<void*> ptrs_;
};

// Pinned host staging buffer for small device->host reads.
struct HostScratch {
    HostScratch();
    ~HostScratch();
    int64_t* p;  // 64 int64 slots
};

// ---------------------------------------------------------------------------
// small helpers usable on host and device
// ---------------------------------------------------------------------------
__host__ __device__ inline int bits_for(uint64_t maxval) {  // bits to hold 0..maxval
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

// Binomial table C(v, k) for v = 0..n, k = 0..K, layout [k][v] (row k is
// contiguous in v), saturating at UINT64_MAX.
struct Binom {
    const uint64_t* t;  // device pointer, (K+1) * (n+1) entries
    int64_t n;
    int K;
    __device__ __forceinline__ uint64_t operator()(int64_t v, int k) const {
        return __ldg(t + (size_t)k * (size_t)(n + 1) + (size_t)v);
    }
};
std::vector<uint64_t> host_binomials(int64_t n, int K);  // same layout on the host

// Decode the q-simplex with index c (eq. 5.6) into ascending vertices v[0..q]:
// v[q] is the largest v with C(v, q+1) <= c, then recurse on the remainder.
template <int Q>
__device__ __forceinline__ void decode_simplex(const Binom& B, uint64_t c, int64_t top, int* v) {
#pragma unroll
    for (int i = Q; i >= 0; --i) {
        // largest x in [i, top] with C(x, i+1) <= c  (binary search)
        int64_t lo = i, hi = top;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (B(mid, i + 1) <= c) lo = mid; else hi = mid - 1;
        }
        v[i] = (int)lo;
        c -= B(lo, i + 1);
        top = lo - 1;
    }
}

// Largest v in [lo, hi] with C(v, k) <= c (C(lo, k) <= c given), for k <= 4,
// from a closed-form estimate: C(v,2) <= c  <=>  v <= (1 + sqrt(1 + 8c)) / 2,
// and C(v,3) ~ (v-1)^3 / 6, C(v,4) ~ (v-1.5)^4 / 24 within one of the float
// root.  C(x, k) and C(x+1, k) are read together, so an exact estimate costs
// one table round trip; otherwise a few checked steps correct it.  Returns
// false if they run out (the caller then searches); *cv receives C(v, k).
template <class BT = Binom>
__device__ __forceinline__ bool binom_root(const BT& B, uint64_t c, int k, int64_t lo, int64_t hi, int64_t& v,
                                           uint64_t& cv) {
    if (k == 1) {  // C(v,1) = v
        v = c < (uint64_t)hi ? (int64_t)c : hi;
        v = v < lo ? lo : v;
        cv = (uint64_t)v;
        return true;
    }
    const float fc = (float)c;
    float est;
    if (k == 2) est = 0.5f * (1.0f + sqrtf(1.0f + 8.0f * fc));
    else if (k == 3) est = cbrtf(6.0f * fc) + 1.0f;
    else est = powf(24.0f * fc, 0.25f) + 1.5f;
    int64_t x = (int64_t)est;
    x = x < lo ? lo : (x > hi ? hi : x);
    uint64_t b0 = B(x, k), b1 = x < hi ? B(x + 1, k) : ~0ull;
    for (int s = 0; s < 6; ++s) {
        if (b0 > c && x > lo) {  // too high
            --x;
            b1 = b0;
            b0 = B(x, k);
        } else if (b1 <= c) {    // too low (x < hi, since b1 is the sentinel at hi)
            ++x;
            b0 = b1;
            b1 = x < hi ? B(x + 1, k) : ~0ull;
        } else {
            v = x;
            cv = b0;
            return b0 <= c || x == lo;
        }
    }
    return false;
}

// The same decoding by a whole (converged) warp: each vertex with k = i+1 <=
// 4 from binom_root, otherwise (or if its correction runs out) by a 32-ary
// search (lane L tests lo + L * step; the tested values C(x, k) grow with
// x, so the passing lanes form a prefix), two dependent table reads per
// vertex for n <= 1024.  Every lane computes and receives the same v.
template <int Q, class BT = Binom>
__device__ __forceinline__ void warp_decode_simplex(const BT& B, uint64_t c, int64_t top, int* v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = Q; i >= 0; --i) {
        int64_t lo = i, hi = top;  // C(lo, i+1) <= c holds throughout
        int64_t r;
        uint64_t cr;
        if (i + 1 <= 4 && binom_root<BT>(B, c, i + 1, lo, hi, r, cr)) {
            v[i] = (int)r;
            c -= cr;
            top = r - 1;
            continue;
        } else {
            while (lo < hi) {
                const int64_t step = (hi - lo + 32) >> 5;  // ceil((hi - lo + 1) / 32)
                const int64_t x = lo + (int64_t)lane * step;
                const bool ok = x <= hi && B(x, i + 1) <= c;
                const int L = 31 - __clz((int)__ballot_sync(0xffffffffu, ok));
                lo += (int64_t)L * step;
                hi = min(hi, lo + step - 1);
            }
        }
        v[i] = (int)lo;
        c -= B(lo, i + 1);
        top = lo - 1;
    }
}

// Diameter ranks: the distance matrix is replaced by the dense rank of each
// entry among the distinct values {0} U {d(i,j)}, so that "diam(a) < diam(b)"
// and "diam(a) == diam(b)" are integer comparisons; ranks map back to the
// float values through a sorted table.  Row-major n x ld, symmetric.
struct RankMatrix {
    const uint32_t* r;
    int64_t n;
    int64_t ld;
    // indices are below 2^31, so one 32x32->64 multiply-add forms the offset
    __device__ __forceinline__ uint32_t operator()(int64_t i, int64_t j) const {
        return __ldg(r + (size_t)(uint32_t)i * (uint32_t)ld + (uint32_t)j);
    }
};

// ---------------------------------------------------------------------------
// stage launchers (host side), one per translation unit
// ---------------------------------------------------------------------------

// dist.cu
void launch_distances(const float* pts, int64_t n, int dim, float* lower_tri, cudaStream_t s);
void launch_check_lower_tri(const float* lower_tri, int64_t m, int* dev_err, cudaStream_t s);

// radix_sort.cu : LSD radix sort, ascending, stable, by the low `bits` bits.
void radix_sort_u64(Workspace& ws, uint64_t* keys, uint64_t* vals, int64_t num, int bits);
void radix_sort_u32(Workspace& ws, uint32_t* keys, uint32_t* vals, int64_t num, int bits);
void scan_u32_exclusive(uint32_t* data, int64_t num, cudaStream_t s);  // in place, total < 2^32

// rank.cu
struct RankInfo {
    uint32_t* rank;       // n x ld
    int64_t ld;
    float* values;        // device, distinct values ascending, values[0] == 0
    int64_t num_values;   // host copy of the count
    const int64_t* num_values_dev;
    uint32_t enclosing_rank;  // rank of R = min_i max_j d(i,j)
};
RankInfo build_ranks(Workspace& ws, const float* lower_tri, int64_t n, HostScratch& hs);
uint32_t threshold_rank(Workspace& ws, const RankInfo& ri, float threshold, HostScratch& hs);
void clamp_ranks(Workspace& ws, const RankInfo& ri, int64_t n, uint32_t thr_rank);  // ranks > thr -> thr + 1

// Device-side records of emitted pairs (ranks, not values).
struct PairRec {
    uint32_t birth_rank;
    uint32_t death_rank;  // UINT32_MAX for essential
    uint64_t birth_cidx;
    int64_t death_cidx;   // -1 for essential
};

// h0.cu : minimum spanning tree (Prim, strict order) + elder-rule pairing.
// Writes n-1 finite pairs and the essential one to out (n records), sets the
// dimension-1 clearing bits of the tree edges.
void launch_h0(const RankMatrix& R, uint32_t thr_rank, PairRec* out, int* out_count,
               uint32_t* clear_bits_dim1, int* dev_err, Workspace& ws);

// apparent.cu : fused filtration construction with clearing (Alg 17/18)
// and apparent-pair search (Lemma 5.3.6) for the p-simplices.
struct ApparentOut {
    uint64_t* nonapparent_keys;   // coboundary-order sort keys of non-apparent columns
    unsigned long long* num_nonapparent;
    uint32_t* clear_next;         // bitmap over (p+1)-simplices (NULL at the top dimension)
    PairRec* zero_pairs;          // apparent pairs, only if keep_zero (else NULL)
    unsigned long long* num_zero_pairs;
    unsigned long long* counters; // [0] above_threshold [1] cleared [2] columns [3] apparent
    int64_t capacity;             // capacity of nonapparent_keys
    int* dev_err;
    // sparse mode: clear_next is indexed by position in this sorted list of the
    // (p+1)-simplex indices of the complex (NULL: indexed by the index itself)
    const uint64_t* next_list = nullptr;
    int64_t next_len = 0;
};
void launch_filtration_apparent(int p, const RankMatrix& R, const Binom& B, uint32_t thr_rank,
                                const uint32_t* clear_bits, int cidx_bits, int rank_bits, uint64_t num_cand,
                                const ApparentOut& o, cudaStream_t s);

// sparse.cu : the complex listed from neighbour lists (sparse / low-threshold mode).
constexpr int SIMPLEX_VSTRIDE = 8;  // vertices stored per listed simplex (uint16, ascending, p+1 used)
struct Neighbours {               // CSR lists of the threshold graph, ascending
    uint32_t* off;                // n + 1
    uint32_t* nbr;
    int64_t num;
};
struct SimplexList {              // simplices of one dimension, by combinatorial index ascending
    uint64_t* cidx;
    uint16_t* verts;              // SIMPLEX_VSTRIDE per simplex
    int64_t len;
};
Neighbours build_neighbours(Workspace& ws, const RankMatrix& R, uint32_t thr, HostScratch& hs);
SimplexList edge_list(Workspace& ws, const RankMatrix& R, const Neighbours& N, HostScratch& hs);
SimplexList next_list(Workspace& ws, const RankMatrix& R, const Binom& B, const Neighbours& N, uint32_t thr,
                      const SimplexList& L, int p, int out_cidx_bits, HostScratch& hs);
void launch_sparse_filtration_apparent(int p, const RankMatrix& R, const Binom& B, const Neighbours& N,
                                       const SimplexList& L, const uint32_t* clear_bits, bool clear_by_pos,
                                       int cidx_bits, int rank_bits, const ApparentOut& o, cudaStream_t s);

// reduce.cu : Z/2 reduction of the non-apparent columns (Algorithm 12).
struct ReduceIn {
    int p;
    RankMatrix R;
    Binom B;
    uint32_t thr_rank;
    int cidx_bits;        // bits of a p-simplex index in the column keys
    int row_cidx_bits;    // bits of a (p+1)-simplex index in the row keys
    int rank_bits;
    const uint64_t* cols; // sorted column keys, num_cols
    int64_t num_cols;
    int mode;             // 0: explicit reduced columns, 1: V (generators), 2: oblivious (Sec. 5.2.9)
    const uint32_t* nb_off = nullptr;  // sparse mode: the threshold graph's CSR lists (cofacets from them)
    const uint32_t* nb = nullptr;
};
struct ReduceOut {
    PairRec* pairs;               // capacity num_cols
    unsigned long long* num_pairs;
    uint32_t* clear_next;         // may be NULL
    const uint64_t* next_list = nullptr;  // sparse mode: clear_next indexed by position in this list
    int64_t next_len = 0;
    unsigned long long* counters; // [0] additions [1] pairs [2] essential
    int* dev_err;
};
void run_reduction(const ReduceIn& in, const ReduceOut& out, bool keep_zero, Workspace& ws,
                   HostScratch& hs);

}  // namespace vr
