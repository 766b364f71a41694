// api.cu -- the C ABI of libvrgpu and the per-dimension driver.
//
// Driver (paper Fig 5.3(b), Sec. 5.3.1, with dimension 0 as in Sec. 5.2.5):
//   distances -> ranks and enclosing radius -> H0 (tree + elder rule) ->
//   for p = 1..dmax:
//     filtration with clearing + apparent pairs (one fused kernel)
//     radix sort of the non-apparent columns into coboundary order
//     Z/2 reduction of those columns (Algorithm 12 schedule in reduce.cu)
//     the pivots of dimension p clear the (p+1)-columns (Sec. 5.2.3)
// Everything after the input copy runs on the caller's stream; the host only
// reads counts to size the next buffers and, at the end, the pairs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vr_common.cuh"

namespace vr {

// ---------------------------------------------------------------------------
// plumbing
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_err, sizeof g_err, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
    if (log_enabled()) fprintf(stderr, "[vr] CUDA error: %s\n", g_err);
}

static void configure_pool_once() {
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t thr = UINT64_MAX;  // keep freed blocks cached between calls
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    });
}

Workspace::Workspace(cudaStream_t s) : stream(s) { configure_pool_once(); }
Workspace::~Workspace() { free_all(); }

void* Workspace::alloc(size_t bytes) {
    void* p = nullptr;
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    VR_CUDA(cudaMallocAsync(&p, bytes, stream));
    ptrs_.push_back(p);
    return p;
}

void Workspace::free_all() {
    for (void* p : ptrs_) cudaFreeAsync(p, stream);
    ptrs_.clear();
}

HostScratch::HostScratch() : p(nullptr) {
    if (cudaMallocHost(&p, 64 * sizeof(int64_t)) != cudaSuccess) {
        p = nullptr;
        throw Error{VR_ERR_OOM};
    }
}
HostScratch::~HostScratch() {
    if (p) cudaFreeHost(p);
}

static HostScratch& host_scratch() {
    static thread_local HostScratch hs;
    return hs;
}

std::vector<uint64_t> host_binomials(int64_t n, int K) {
    std::vector<uint64_t> t((size_t)(K + 1) * (n + 1), 0);
    auto at = [&](int k, int64_t v) -> uint64_t& { return t[(size_t)k * (n + 1) + v]; };
    for (int64_t v = 0; v <= n; ++v) {
        at(0, v) = 1;
        for (int k = 1; k <= K; ++k) {
            if (v == 0) { at(k, v) = 0; continue; }
            uint64_t a = at(k - 1, v - 1), b = at(k, v - 1);
            at(k, v) = (a > UINT64_MAX - b) ? UINT64_MAX : a + b;
        }
    }
    return t;
}

static uint64_t binom_host(int64_t n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) {
        r = r * (unsigned __int128)(n - k + i) / i;
        if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
    }
    return (uint64_t)r;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void check_dev_err(const int* dev_err, cudaStream_t s) {
    int h = 0;
    VR_CUDA(cudaMemcpyAsync(&h, dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaStreamSynchronize(s));
    if (h != DEV_OK && log_enabled()) fprintf(stderr, "[vr] device error %d (site %d)\n", h & 0xFF, h >> 8);
    switch (h & 0xFF) {  // the upper bits name the failing check (DEV_INTERNAL)
        case DEV_OK: return;
        case DEV_CAPACITY: throw Error{VR_ERR_OOM};
        case DEV_TIMEOUT: throw Error{VR_ERR_TIMEOUT};
        case DEV_BAD_INPUT: throw Error{VR_ERR_INVALID_ARG};
        default: throw Error{VR_ERR_INTERNAL};
    }
}

// runtime-q decode for the small result kernels
__device__ void decode_rt(const Binom& B, uint64_t c, int q, int64_t top, int* v) {
    for (int i = q; i >= 0; --i) {
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

// the edge (u > v) of a q-simplex attaining its diameter, ties -> largest C(u,2)+v
__device__ void critical_edge(const RankMatrix& R, const Binom& B, uint64_t cidx, int q, int& cu, int& cv) {
    int v[VR_MAX_DIM + 2];
    decode_rt(B, cidx, q, R.n - 1, v);
    uint32_t best = 0;
    cu = -1; cv = -1;
    for (int i = 1; i <= q; ++i)
        for (int j = 0; j < i; ++j) {
            uint32_t r = R(v[i], v[j]);
            int64_t e = (int64_t)v[i] * (v[i] - 1) / 2 + v[j];
            int64_t be = cu < 0 ? -1 : (int64_t)cu * (cu - 1) / 2 + cv;
            if (cu < 0 || r > best || (r == best && e > be)) { best = r; cu = v[i]; cv = v[j]; }
        }
}

__global__ void k_critical_edges(const PairRec* __restrict__ recs, int64_t num, int p, RankMatrix R, Binom B,
                                 int32_t* __restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < num; k += (int64_t)gridDim.x * blockDim.x) {
        const PairRec r = recs[k];
        int u = -1, v = -1;
        if (p > 0) critical_edge(R, B, r.birth_cidx, p, u, v);
        out[4 * k + 0] = u;
        out[4 * k + 1] = v;
        u = v = -1;
        if (r.death_cidx >= 0) critical_edge(R, B, (uint64_t)r.death_cidx, p + 1, u, v);
        out[4 * k + 2] = u;
        out[4 * k + 3] = v;
    }
}

struct HostPairs {
    std::vector<PairRec> recs;
    std::vector<int32_t> edges;
};

static HostPairs fetch_pairs(Workspace& ws, const PairRec* dev, int64_t num, int p, const RankMatrix& R,
                             const Binom& B, bool want_edges) {
    HostPairs h;
    h.recs.resize((size_t)num);
    if (num == 0) return h;
    VR_CUDA(cudaMemcpyAsync(h.recs.data(), dev, num * sizeof(PairRec), cudaMemcpyDeviceToHost, ws.stream));
    if (want_edges) {
        int32_t* e = ws.alloc_n<int32_t>(4 * num);
        int64_t blocks = (num + 127) / 128;
        if (blocks > 4096) blocks = 4096;
        k_critical_edges<<<(unsigned)blocks, 128, 0, ws.stream>>>(dev, num, p, R, B, e);
        VR_CUDA(cudaGetLastError());
        h.edges.resize((size_t)4 * num);
        VR_CUDA(cudaMemcpyAsync(h.edges.data(), e, 4 * num * sizeof(int32_t), cudaMemcpyDeviceToHost, ws.stream));
    }
    VR_CUDA(cudaStreamSynchronize(ws.stream));
    return h;
}

// ---------------------------------------------------------------------------
// device-resident output: filter, order and convert the records on the device
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool dropped(const PairRec& r, int keep_zero) {
    return !keep_zero && r.death_rank != 0xFFFFFFFFu && r.death_rank == r.birth_rank;
}

__global__ void k_emit_keys1(const PairRec* __restrict__ recs, int64_t num, int keep_zero, uint64_t* __restrict__ keys,
                             uint64_t* __restrict__ idx, unsigned long long* __restrict__ kept) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < num; k += (int64_t)gridDim.x * blockDim.x) {
        const PairRec r = recs[k];
        keys[k] = r.birth_cidx;
        idx[k] = (uint64_t)k;
        if (!dropped(r, keep_zero)) atomicAdd(kept, 1ull);
    }
}

// second (stable) pass: birth rank, then death rank; dropped records last
__global__ void k_emit_keys2(const PairRec* __restrict__ recs, int64_t num, int keep_zero,
                             const uint64_t* __restrict__ idx, uint64_t* __restrict__ keys) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < num; k += (int64_t)gridDim.x * blockDim.x) {
        const PairRec r = recs[idx[k]];
        keys[k] = dropped(r, keep_zero) ? ~0ull : (((uint64_t)r.birth_rank << 32) | r.death_rank);
    }
}

__global__ void k_emit_gather(const PairRec* __restrict__ recs, int64_t cnt, const uint64_t* __restrict__ idx,
                              const float* __restrict__ values, PairRec* __restrict__ sorted,
                              vr_pair* __restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += (int64_t)gridDim.x * blockDim.x) {
        const PairRec r = recs[idx[k]];
        sorted[k] = r;
        vr_pair v;
        v.birth = values[r.birth_rank];
        v.death = r.death_rank == 0xFFFFFFFFu ? __int_as_float(0x7f800000) : values[r.death_rank];
        v.birth_simplex = r.birth_cidx;
        v.death_simplex = r.death_cidx;
        out[k] = v;
    }
}

// Pairs of dimension p as the host path would return them (zero-length ones
// dropped unless keep_zero; sorted by (birth, death, birth simplex)), in
// device memory that outlives the call (stream-ordered allocation on the
// call's stream, released by vr_device_result_free on that stream).
static int64_t device_emit(Workspace& ws, HostScratch& hs, const PairRec* recs, int64_t num, int p,
                           const RankMatrix& R, const Binom& B, const float* values, bool keep_zero,
                           bool want_edges, vr_pair** out, int32_t** edges) {
    cudaStream_t s = ws.stream;
    int64_t cnt = 0;
    if (num > 0) {
        uint64_t* keys = ws.alloc_n<uint64_t>(num);
        uint64_t* idx = ws.alloc_n<uint64_t>(num);
        unsigned long long* kept = ws.zeros_n<unsigned long long>(1);
        const unsigned blocks = (unsigned)std::min<int64_t>((num + 255) / 256, 4096);
        k_emit_keys1<<<blocks, 256, 0, s>>>(recs, num, keep_zero ? 1 : 0, keys, idx, kept);
        VR_CUDA(cudaGetLastError());
        radix_sort_u64(ws, keys, idx, num, 64);
        k_emit_keys2<<<blocks, 256, 0, s>>>(recs, num, keep_zero ? 1 : 0, idx, keys);
        VR_CUDA(cudaGetLastError());
        radix_sort_u64(ws, keys, idx, num, 64);
        VR_CUDA(cudaMemcpyAsync(&hs.p[40], kept, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        cnt = hs.p[40];
        VR_CUDA(cudaMallocAsync((void**)out, (size_t)std::max<int64_t>(cnt, 1) * sizeof(vr_pair), s));
        if (want_edges)
            VR_CUDA(cudaMallocAsync((void**)edges, (size_t)std::max<int64_t>(cnt, 1) * 4 * sizeof(int32_t), s));
        if (cnt > 0) {
            PairRec* sorted = ws.alloc_n<PairRec>(cnt);
            k_emit_gather<<<blocks, 256, 0, s>>>(recs, cnt, idx, values, sorted, *out);
            VR_CUDA(cudaGetLastError());
            if (want_edges) {
                k_critical_edges<<<blocks, 128, 0, s>>>(sorted, cnt, p, R, B, *edges);
                VR_CUDA(cudaGetLastError());
            }
        }
    } else {
        VR_CUDA(cudaMallocAsync((void**)out, sizeof(vr_pair), s));
        if (want_edges) VR_CUDA(cudaMallocAsync((void**)edges, 4 * sizeof(int32_t), s));
    }
    return cnt;
}

// ---------------------------------------------------------------------------
// optional stage log (VR_LOG=1): CUDA-event time of each stage on the stream
// ---------------------------------------------------------------------------
bool log_enabled() {
    static const bool on = getenv("VR_LOG") && getenv("VR_LOG")[0] == '1';
    return on;
}

// CUDA events on the caller's stream around each stage; the durations go to
// vr_result.stats and, with VR_LOG=1, to stderr.
struct StageLog {
    cudaStream_t s;
    std::vector<std::pair<std::string, cudaEvent_t>> ev;
    explicit StageLog(cudaStream_t st) : s(st) { mark("start"); }
    void mark(const std::string& name) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, s);
        ev.emplace_back(name, e);
    }
    cudaEvent_t find(const std::string& name) const {
        for (auto it = ev.rbegin(); it != ev.rend(); ++it)  // the last mark of that name
            if (it->first == name) return it->second;
        return nullptr;
    }
    float between(const std::string& a, const std::string& b) const {  // after a synchronisation
        cudaEvent_t ea = find(a), eb = find(b);
        float ms = 0.0f;
        if (ea && eb && cudaEventElapsedTime(&ms, ea, eb) != cudaSuccess) ms = 0.0f;
        return ms;
    }
    void print() const {
        for (size_t i = 1; i < ev.size(); ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[i - 1].second, ev[i].second);
            fprintf(stderr, "[vr] %-24s %9.3f ms\n", ev[i].first.c_str(), ms);
        }
    }
    ~StageLog() {
        for (auto& e : ev) cudaEventDestroy(e.second);
    }
};

static std::string stage_name(const char* what, int p) { return "dim" + std::to_string(p) + " " + what; }

// ---------------------------------------------------------------------------
// result assembly
// ---------------------------------------------------------------------------
static void fill_dim(vr_result* res, int p, const HostPairs& hp, const std::vector<float>& values, bool keep_zero,
                     bool want_edges) {
    std::vector<int64_t> idx;
    idx.reserve(hp.recs.size());
    for (size_t k = 0; k < hp.recs.size(); ++k) {
        const PairRec& r = hp.recs[k];
        if (r.death_rank != 0xFFFFFFFFu && r.death_rank == r.birth_rank && !keep_zero) continue;
        idx.push_back((int64_t)k);
    }
    auto val = [&](uint32_t rk) { return rk == 0xFFFFFFFFu ? INFINITY : values[rk]; };
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
        const PairRec &x = hp.recs[a], &y = hp.recs[b];
        float xb = val(x.birth_rank), yb = val(y.birth_rank), xd = val(x.death_rank), yd = val(y.death_rank);
        if (xb != yb) return xb < yb;
        if (xd != yd) return xd < yd;
        return x.birth_cidx < y.birth_cidx;
    });
    const int64_t m = (int64_t)idx.size();
    res->count[p] = m;
    res->pairs[p] = (vr_pair*)malloc((size_t)(m > 0 ? m : 1) * sizeof(vr_pair));
    if (!res->pairs[p]) throw Error{VR_ERR_OOM};
    if (want_edges) {
        res->critical_edges[p] = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * 4 * sizeof(int32_t));
        if (!res->critical_edges[p]) throw Error{VR_ERR_OOM};
    }
    for (int64_t k = 0; k < m; ++k) {
        const PairRec& r = hp.recs[idx[k]];
        vr_pair& o = res->pairs[p][k];
        o.birth = val(r.birth_rank);
        o.death = val(r.death_rank);
        o.birth_simplex = r.birth_cidx;
        o.death_simplex = r.death_cidx;
        if (want_edges) memcpy(res->critical_edges[p] + 4 * k, &hp.edges[4 * idx[k]], 4 * sizeof(int32_t));
    }
    res->stats[p].emitted = m;
}

// VR_DEBUG_CHECKS: identities every correct result satisfies, from the
// counters and the emitted pairs.  Obs 3.2.14: each p-simplex of the complex
// is a birth (paired or essential) or the death of a (p-1)-class; here the
// p-simplices within the threshold are the kept columns plus the cleared ones,
// the cleared ones are exactly the death simplices of the (p-1)-pairs
// (Sec. 5.2.3), and every kept column is paired or essential.  Each emitted
// pair has birth <= death, and the pairs are sorted as documented.
static void debug_checks(const vr_result* res, uint32_t flags) {
    for (int p = 0; p <= res->dmax; ++p) {
        const vr_stats& st = res->stats[p];
        if ((flags & VR_APPARENT_ONLY) && p == res->dmax && p >= 1) {  // no reduction in this dimension
            VR_CHECK(st.reduced + st.apparent == st.columns && res->count[p] == 0, VR_ERR_INTERNAL);
            VR_CHECK(st.cleared == res->stats[p - 1].pairs, VR_ERR_INTERNAL);
            VR_CHECK(st.candidates == st.above_threshold + st.cleared + st.columns, VR_ERR_INTERNAL);
            continue;
        }
        VR_CHECK(st.columns == st.pairs + st.essential, VR_ERR_INTERNAL);
        if (p >= 1) {
            VR_CHECK(st.cleared == res->stats[p - 1].pairs, VR_ERR_INTERNAL);
            VR_CHECK(st.candidates == st.above_threshold + st.cleared + st.columns, VR_ERR_INTERNAL);
            VR_CHECK(st.reduced + st.apparent <= st.columns, VR_ERR_INTERNAL);
        }
        for (int64_t k = 0; res->pairs[p] && k < res->count[p]; ++k) {  // host results only
            const vr_pair& a = res->pairs[p][k];
            VR_CHECK(a.birth <= a.death && a.birth >= 0.0f, VR_ERR_INTERNAL);
            VR_CHECK((a.death_simplex < 0) == std::isinf(a.death), VR_ERR_INTERNAL);
            if (k > 0) {
                const vr_pair& b = res->pairs[p][k - 1];
                const bool ordered = b.birth < a.birth || (b.birth == a.birth && (b.death < a.death ||
                                     (b.death == a.death && b.birth_simplex <= a.birth_simplex)));
                VR_CHECK(ordered, VR_ERR_INTERNAL);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the driver
// ---------------------------------------------------------------------------
// Device-resident pairs (vr_barcodes_*_device): per dimension, the sorted
// pairs and critical edges in device memory owned by the caller's result.
struct DevOut {
    vr_pair* pairs[VR_MAX_DIM + 1];
    int32_t* edges[VR_MAX_DIM + 1];
};

__global__ void k_count_essential(const PairRec* __restrict__ recs, int64_t num, unsigned long long* __restrict__ c) {
    unsigned long long k = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < num; i += (int64_t)gridDim.x * blockDim.x)
        k += recs[i].death_rank == 0xFFFFFFFFu;
    if (k) atomicAdd(c, k);
}

static vr_result* compute(Workspace& ws, const float* lower, int64_t n, int dmax, float threshold, uint32_t flags,
                          DevOut* dv = nullptr) {
    HostScratch& hs = host_scratch();
    const bool keep_zero = flags & VR_KEEP_ZERO_LENGTH;
    const bool want_edges = flags & VR_CRITICAL_EDGES;
    vr_result* res = (vr_result*)calloc(1, sizeof(vr_result));
    if (!res) throw Error{VR_ERR_OOM};
    struct Guard {
        vr_result* r;
        ~Guard() { if (r) vr_result_free(r); }
    } guard{res};
    res->dmax = dmax;
    res->n = n;
    res->threshold = threshold;
    if (threshold < 0) {  // Rips_t is empty for t < 0 (eq. 5.3)
        for (int p = 0; p <= dmax; ++p) res->pairs[p] = (vr_pair*)malloc(sizeof(vr_pair));
        guard.r = nullptr;
        return res;
    }
    cudaStream_t s = ws.stream;
    StageLog log(s);
    RankInfo ri = build_ranks(ws, lower, n, hs);
    log.mark("ranks");
    const uint32_t thr = threshold_rank(ws, ri, threshold, hs);
    std::vector<float> values((size_t)ri.num_values);
    VR_CUDA(cudaMemcpyAsync(values.data(), ri.values, ri.num_values * sizeof(float), cudaMemcpyDeviceToHost, s));
    res->threshold = (isinf(threshold) && threshold > 0) ? 0.0f : threshold;
    const RankMatrix R{ri.rank, n, ri.ld};
    // ranks above the threshold collapse to thr + 1, so keys need only its bits
    if ((uint64_t)thr + 1 < (uint64_t)ri.num_values) clamp_ranks(ws, ri, n, thr);
    const int rank_bits = std::max(1, bits_for(std::min<uint64_t>((uint64_t)ri.num_values - 1, (uint64_t)thr + 1)));
    const int K = dmax + 3;
    std::vector<uint64_t> hb = host_binomials(n, K);
    uint64_t* db = ws.alloc_n<uint64_t>(hb.size());
    VR_CUDA(cudaMemcpyAsync(db, hb.data(), hb.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    const Binom B{db, n, K};
    VR_CUDA(cudaStreamSynchronize(s));  // host binomial vector and values copy
    if (isinf(threshold) && threshold > 0) res->threshold = values[thr];

    // every dimension's packed keys must fit before any work starts: a column key
    // holds the diameter rank above the p-simplex index, a row key the rank above
    // the (p+1)-simplex index
    for (int p = 1; p <= dmax; ++p) {
        const uint64_t ncand = binom_host(n, p + 1), nrow = binom_host(n, p + 2);
        const int cb = std::max(1, bits_for(ncand > 0 ? ncand - 1 : 0));
        const int rcb = std::max(1, bits_for(nrow > 0 ? nrow - 1 : 0));
        VR_CHECK(nrow != UINT64_MAX && rank_bits + cb <= 64 && rank_bits + rcb <= 63, VR_ERR_INDEX_OVERFLOW);
    }

    int* dev_err = ws.zeros_n<int>(1);
    unsigned long long* cnt = ws.zeros_n<unsigned long long>(16);

    // ---- dimension 0
    uint32_t* clear = nullptr;
    if (dmax >= 1) clear = ws.zeros_n<uint32_t>((binom_host(n, 2) + 31) / 32 + 1);
    PairRec* p0 = ws.alloc_n<PairRec>(n);
    int* p0n = ws.zeros_n<int>(1);
    launch_h0(R, thr, p0, p0n, clear, dev_err, ws);
    log.mark("h0");
    VR_CUDA(cudaMemcpyAsync(&hs.p[0], p0n, sizeof(int), cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaStreamSynchronize(s));
    {
        const int64_t m0 = (int64_t)(int32_t)(hs.p[0] & 0xFFFFFFFF);
        int64_t ess = 0;
        res->stats[0].candidates = n;
        res->stats[0].columns = n;
        if (dv) {
            unsigned long long* ce = ws.zeros_n<unsigned long long>(1);
            k_count_essential<<<(unsigned)std::min<int64_t>((m0 + 255) / 256 + 1, 1024), 256, 0, s>>>(p0, m0, ce);
            VR_CUDA(cudaGetLastError());
            VR_CUDA(cudaMemcpyAsync(&hs.p[41], ce, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
            ess = hs.p[41];
            res->count[0] = device_emit(ws, hs, p0, m0, 0, R, B, ri.values, keep_zero, want_edges, &dv->pairs[0],
                                        &dv->edges[0]);
            res->stats[0].emitted = res->count[0];
        } else {
            HostPairs hp = fetch_pairs(ws, p0, m0, 0, R, B, want_edges);
            for (auto& r : hp.recs) ess += r.death_rank == 0xFFFFFFFFu;
            fill_dim(res, 0, hp, values, keep_zero, want_edges);
        }
        res->stats[0].pairs = m0 - ess;
        res->stats[0].essential = ess;
    }

    // ---- dimensions 1..dmax
    // sparse mode: the simplices of the complex are listed from neighbour lists
    // (sparse.cu) instead of enumerating every index; clearing bits of dimension
    // p >= 2 are then indexed by position in the list of p-simplices
    const bool sparse = flags & VR_SPARSE;
    Neighbours nb{};
    SimplexList L{}, Lnext{};
    if (sparse && dmax >= 1) {
        nb = build_neighbours(ws, R, thr, hs);
        L = edge_list(ws, R, nb, hs);
    }
    for (int p = 1; p <= dmax; ++p) {
        const uint64_t nall = binom_host(n, p + 1);
        const uint64_t ncand = sparse ? (uint64_t)L.len : nall;
        const uint64_t nrow = binom_host(n, p + 2);
        const int cb = std::max(1, bits_for(nall > 0 ? nall - 1 : 0));
        const int rcb = std::max(1, bits_for(nrow > 0 ? nrow - 1 : 0));
        VR_CHECK(nrow != UINT64_MAX && rank_bits + cb <= 64 && rank_bits + rcb <= 63, VR_ERR_INDEX_OVERFLOW);
        uint32_t* clear_next = nullptr;
        if (sparse && p < dmax) {
            Lnext = next_list(ws, R, B, nb, thr, L, p, rcb, hs);
            clear_next = ws.zeros_n<uint32_t>(((uint64_t)Lnext.len + 31) / 32 + 1);
        } else if (p < dmax) {
            clear_next = ws.zeros_n<uint32_t>((nrow + 31) / 32 + 1);
        }
        VR_CUDA(cudaMemsetAsync(cnt, 0, 16 * sizeof(unsigned long long), s));
        int64_t cap = (int64_t)std::max<uint64_t>(1 << 16, ncand / 16);
        if ((uint64_t)cap > ncand) cap = (int64_t)std::max<uint64_t>(ncand, 1);
        PairRec* zero_pairs = nullptr;
        if (keep_zero) zero_pairs = ws.alloc_n<PairRec>(ncand);
        uint64_t* keys = nullptr;
        for (int attempt = 0; attempt < 2; ++attempt) {
            keys = ws.alloc_n<uint64_t>(cap);
            VR_CUDA(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
            VR_CUDA(cudaMemsetAsync(dev_err, 0, sizeof(int), s));
            ApparentOut ao;
            ao.nonapparent_keys = keys;
            ao.num_nonapparent = cnt + 4;
            ao.clear_next = clear_next;
            ao.zero_pairs = zero_pairs;
            ao.num_zero_pairs = cnt + 5;
            ao.counters = cnt;
            ao.capacity = cap;
            ao.dev_err = dev_err;
            if (sparse && clear_next) {
                ao.next_list = Lnext.cidx;
                ao.next_len = Lnext.len;
            }
            log.mark(stage_name("launch apparent", p));
            if (sparse)
                launch_sparse_filtration_apparent(p, R, B, nb, L, clear, p >= 2, cb, rank_bits, ao, s);
            else
                launch_filtration_apparent(p, R, B, thr, clear, cb, rank_bits, ncand, ao, s);
            log.mark(stage_name("apparent", p));
            VR_CUDA(cudaMemcpyAsync(hs.p, cnt, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
            if (hs.p[4] <= cap) break;
            cap = hs.p[4];  // rerun with room for every non-apparent column
        }
        check_dev_err(dev_err, s);
        vr_stats& st = res->stats[p];
        st.candidates = (int64_t)ncand;
        st.above_threshold = hs.p[0];
        st.cleared = hs.p[1];
        st.columns = hs.p[2];
        st.apparent = hs.p[3];
        const int64_t nna = hs.p[4];
        const int64_t nzero = hs.p[5];
        st.reduced = nna;
        // rank-matrix entries the fused kernel reads: diameters of the candidates,
        // p+1 per examined cofacet, all pairs of t for each facet test
        st.lookups = (int64_t)ncand * (p + 1) * p / 2 + hs.p[6] * (p + 1) + hs.p[7] * (p + 2) * (p + 1) / 2;
        st.cofacets_scanned = hs.p[6];
        if ((flags & VR_APPARENT_ONLY) && p == dmax) {
            // the top dimension stops after the apparent-pair search: its apparent
            // pairs are counted, its non-apparent columns are not reduced
            st.pairs = st.apparent;
            if (dv) {
                device_emit(ws, hs, nullptr, 0, p, R, B, ri.values, keep_zero, want_edges, &dv->pairs[p],
                            &dv->edges[p]);
            } else {
                res->pairs[p] = (vr_pair*)malloc(sizeof(vr_pair));
                if (!res->pairs[p]) throw Error{VR_ERR_OOM};
                if (want_edges) {
                    res->critical_edges[p] = (int32_t*)malloc(4 * sizeof(int32_t));
                    if (!res->critical_edges[p]) throw Error{VR_ERR_OOM};
                }
            }
            res->count[p] = 0;
            log.mark(stage_name("launch sort", p));
            log.mark(stage_name("sort", p));
            log.mark(stage_name("launch reduce", p));
            log.mark(stage_name("reduce", p));
            break;
        }
        log.mark(stage_name("launch sort", p));
        radix_sort_u64(ws, keys, nullptr, nna, rank_bits + cb);
        log.mark(stage_name("sort", p));
        PairRec* pr = ws.alloc_n<PairRec>(nna > 0 ? nna : 1);
        unsigned long long* rc = cnt + 8;  // [8] num_pairs [9] additions [10] pairs [11] essential
        ReduceIn in;
        in.p = p;
        in.R = R;
        in.B = B;
        in.thr_rank = thr;
        in.cidx_bits = cb;
        in.row_cidx_bits = rcb;
        in.rank_bits = rank_bits;
        in.cols = keys;
        in.num_cols = nna;
        in.mode = (flags & VR_REDUCE_V) ? 1 : (flags & VR_REDUCE_OBLIVIOUS) ? 2 : 0;
        if (sparse) {  // coboundaries from the neighbour lists
            in.nb_off = nb.off;
            in.nb = nb.nbr;
        }
        ReduceOut out;
        out.pairs = pr;
        out.num_pairs = rc;
        out.clear_next = clear_next;
        if (sparse && clear_next) {
            out.next_list = Lnext.cidx;
            out.next_len = Lnext.len;
        }
        out.counters = rc + 1;
        out.dev_err = dev_err;
        log.mark(stage_name("launch reduce", p));
        run_reduction(in, out, keep_zero, ws, hs);
        log.mark(stage_name("reduce", p));
        VR_CUDA(cudaMemcpyAsync(hs.p + 8, rc, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        check_dev_err(dev_err, s);  // synchronises
        st.additions = hs.p[9];
        st.pairs = hs.p[10] + st.apparent;
        st.essential = hs.p[11];
        if (dv) {
            const PairRec* src = pr;
            int64_t num = hs.p[8];
            if (keep_zero && nzero > 0) {  // the reduction's pairs, then the apparent ones
                PairRec* cat = ws.alloc_n<PairRec>(num + nzero);
                VR_CUDA(cudaMemcpyAsync(cat, pr, num * sizeof(PairRec), cudaMemcpyDeviceToDevice, s));
                VR_CUDA(cudaMemcpyAsync(cat + num, zero_pairs, nzero * sizeof(PairRec), cudaMemcpyDeviceToDevice, s));
                src = cat;
                num += nzero;
            }
            res->count[p] = device_emit(ws, hs, src, num, p, R, B, ri.values, keep_zero, want_edges, &dv->pairs[p],
                                        &dv->edges[p]);
            st.emitted = res->count[p];
        } else {
            HostPairs hp = fetch_pairs(ws, pr, hs.p[8], p, R, B, want_edges);
            if (keep_zero && nzero > 0) {
                HostPairs hz = fetch_pairs(ws, zero_pairs, nzero, p, R, B, want_edges);
                hp.recs.insert(hp.recs.end(), hz.recs.begin(), hz.recs.end());
                hp.edges.insert(hp.edges.end(), hz.edges.begin(), hz.edges.end());
            }
            fill_dim(res, p, hp, values, keep_zero, want_edges);
        }
        log.mark(stage_name("emit", p));
        clear = clear_next;
        if (sparse) L = Lnext;
    }
    VR_CUDA(cudaStreamSynchronize(s));
    res->stats[0].ms_filtration = log.between("start", "ranks");
    res->stats[0].ms_reduce = log.between("ranks", "h0");
    for (int p = 1; p <= dmax; ++p) {
        res->stats[p].ms_filtration = log.between(stage_name("launch apparent", p), stage_name("apparent", p));
        res->stats[p].ms_sort = log.between(stage_name("launch sort", p), stage_name("sort", p));
        res->stats[p].ms_reduce = log.between(stage_name("launch reduce", p), stage_name("reduce", p));
    }
    if (log_enabled()) log.print();
    if (flags & VR_DEBUG_CHECKS) debug_checks(res, flags);
    guard.r = nullptr;
    return res;
}

static vr_status run_guarded(vr_result** out, const float* data, bool is_points, int64_t n, int32_t amb,
                             int32_t dmax, float threshold, uint32_t flags, void* stream, DevOut* dv = nullptr) {
    if (!out) return VR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!data && n > 1) return VR_ERR_INVALID_ARG;
    if (n < 1 || n > (1 << 16) || dmax < 0 || dmax > VR_MAX_DIM || std::isnan(threshold)) return VR_ERR_INVALID_ARG;
    if (is_points && (amb < 1 || amb > 1024)) return VR_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)(VR_KEEP_ZERO_LENGTH | VR_CRITICAL_EDGES | VR_DEBUG_CHECKS | VR_APPARENT_ONLY |
                            VR_REDUCE_V | VR_REDUCE_OBLIVIOUS | VR_SPARSE))
        return VR_ERR_INVALID_ARG;
    if ((flags & VR_REDUCE_V) && (flags & VR_REDUCE_OBLIVIOUS)) return VR_ERR_INVALID_ARG;
    // simplex indices of dimension dmax+1 must fit 63 bits (checked before any device work)
    if (binom_host(n, dmax + 2) >= (1ull << 63)) return VR_ERR_INDEX_OVERFLOW;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        Workspace ws(s);
        const int64_t m = n * (n - 1) / 2;
        float* lower = ws.alloc_n<float>(m > 0 ? m : 1);
        if (is_points) {
            const float* dpts = data;
            if (!is_device_ptr(data)) {
                float* t = ws.alloc_n<float>(n * amb);
                VR_CUDA(cudaMemcpyAsync(t, data, n * amb * sizeof(float), cudaMemcpyHostToDevice, s));
                dpts = t;
            }
            launch_distances(dpts, n, amb, lower, s);
        } else if (m > 0) {
            if (is_device_ptr(data))
                VR_CUDA(cudaMemcpyAsync(lower, data, m * sizeof(float), cudaMemcpyDeviceToDevice, s));
            else
                VR_CUDA(cudaMemcpyAsync(lower, data, m * sizeof(float), cudaMemcpyHostToDevice, s));
            int* err = ws.zeros_n<int>(1);
            launch_check_lower_tri(lower, m, err, s);
            check_dev_err(err, s);
        }
        *out = compute(ws, lower, n, dmax, threshold, flags, dv);
        VR_CUDA(cudaStreamSynchronize(s));
        return VR_OK;
    } catch (const Error& e) {
        if (*out) { vr_result_free(*out); *out = nullptr; }
        return e.code;
    } catch (const std::bad_alloc&) {
        return VR_ERR_OOM;
    } catch (...) {
        return VR_ERR_INTERNAL;
    }
}

static void free_devout(DevOut& dv, cudaStream_t s) {
    for (int p = 0; p <= VR_MAX_DIM; ++p) {
        if (dv.pairs[p]) cudaFreeAsync(dv.pairs[p], s);
        if (dv.edges[p]) cudaFreeAsync(dv.edges[p], s);
        dv.pairs[p] = nullptr;
        dv.edges[p] = nullptr;
    }
}

static vr_status run_device(vr_device_result** out, const float* data, bool is_points, int64_t n, int32_t amb,
                            int32_t dmax, float threshold, uint32_t flags, void* stream) {
    if (!out) return VR_ERR_INVALID_ARG;
    *out = nullptr;
    DevOut dv;
    memset(&dv, 0, sizeof dv);
    vr_result* r = nullptr;
    vr_status st = run_guarded(&r, data, is_points, n, amb, dmax, threshold, flags, stream, &dv);
    cudaStream_t s = (cudaStream_t)stream;
    if (st != VR_OK) {
        free_devout(dv, s);
        return st;
    }
    vr_device_result* d = (vr_device_result*)calloc(1, sizeof(vr_device_result));
    if (!d) {
        free_devout(dv, s);
        vr_result_free(r);
        return VR_ERR_OOM;
    }
    d->dmax = r->dmax;
    d->n = r->n;
    d->threshold = r->threshold;
    memcpy(d->count, r->count, sizeof d->count);
    memcpy(d->stats, r->stats, sizeof d->stats);
    vr_result_free(r);
    const bool want_edges = flags & VR_CRITICAL_EDGES;
    d->stream = stream;
    for (int p = 0; p <= dmax; ++p) {
        if (!dv.pairs[p] && cudaMallocAsync((void**)&dv.pairs[p], sizeof(vr_pair), s) != cudaSuccess) st = VR_ERR_OOM;
        if (want_edges && !dv.edges[p] && cudaMallocAsync((void**)&dv.edges[p], 4 * sizeof(int32_t), s) != cudaSuccess)
            st = VR_ERR_OOM;
        d->pairs[p] = dv.pairs[p];
        d->critical_edges[p] = want_edges ? dv.edges[p] : nullptr;
    }
    if (st == VR_OK && cudaStreamSynchronize(s) != cudaSuccess) st = VR_ERR_CUDA;
    if (st != VR_OK) {
        free_devout(dv, s);
        free(d);
        return st;
    }
    *out = d;
    return VR_OK;
}

}  // namespace vr

// ---------------------------------------------------------------------------
// exported C ABI
// ---------------------------------------------------------------------------
extern "C" {

vr_status vr_barcodes_points(const float* pts, int64_t n, int32_t ambient_dim, int32_t dmax, float threshold,
                             uint32_t flags, void* stream, vr_result** out) {
    return vr::run_guarded(out, pts, true, n, ambient_dim, dmax, threshold, flags, stream);
}

vr_status vr_barcodes_dists(const float* lower_tri, int64_t n, int32_t dmax, float threshold, uint32_t flags,
                            void* stream, vr_result** out) {
    return vr::run_guarded(out, lower_tri, false, n, 0, dmax, threshold, flags, stream);
}

vr_status vr_barcodes_points_device(const float* pts, int64_t n, int32_t ambient_dim, int32_t dmax, float threshold,
                                    uint32_t flags, void* stream, vr_device_result** out) {
    return vr::run_device(out, pts, true, n, ambient_dim, dmax, threshold, flags, stream);
}

vr_status vr_barcodes_dists_device(const float* lower_tri, int64_t n, int32_t dmax, float threshold, uint32_t flags,
                                   void* stream, vr_device_result** out) {
    return vr::run_device(out, lower_tri, false, n, 0, dmax, threshold, flags, stream);
}

void vr_device_result_free(vr_device_result* r) {
    if (!r) return;
    for (int p = 0; p <= VR_MAX_DIM; ++p) {
        if (r->pairs[p]) cudaFreeAsync(r->pairs[p], (cudaStream_t)r->stream);
        if (r->critical_edges[p]) cudaFreeAsync(r->critical_edges[p], (cudaStream_t)r->stream);
    }
    free(r);
}

void vr_result_free(vr_result* r) {
    if (!r) return;
    for (int p = 0; p <= VR_MAX_DIM; ++p) {
        free(r->pairs[p]);
        free(r->critical_edges[p]);
    }
    free(r);
}

vr_status vr_simplex_vertices(uint64_t cidx, int32_t q, int64_t n, int32_t* out_vertices) {
    if (!out_vertices || q < 0 || q > VR_MAX_DIM + 1 || n < q + 1 || n > (1 << 20)) return VR_ERR_INVALID_ARG;
    if (cidx >= vr::binom_host(n, q + 1)) return VR_ERR_INVALID_ARG;
    int64_t top = n - 1;
    for (int i = q; i >= 0; --i) {
        int64_t x = top;
        while (vr::binom_host(x, i + 1) > cidx) --x;
        out_vertices[i] = (int32_t)x;
        cidx -= vr::binom_host(x, i + 1);
        top = x - 1;
    }
    return VR_OK;
}

const char* vr_status_string(vr_status s) {
    switch (s) {
        case VR_OK: return "ok";
        case VR_ERR_INVALID_ARG: return "invalid argument";
        case VR_ERR_OOM: return "out of memory";
        case VR_ERR_INDEX_OVERFLOW: return "simplex index or sort key overflows 64 bits";
        case VR_ERR_CUDA: return "CUDA runtime error";
        case VR_ERR_TIMEOUT: return "timeout (reserved: no entry point returns it)";
        case VR_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

vr_status vr_distances(const float* pts, int64_t n, int32_t ambient_dim, float* out_lower_tri, void* stream) {
    if (n < 1 || ambient_dim < 1 || ambient_dim > 1024 || (n > 1 && (!pts || !out_lower_tri)))
        return VR_ERR_INVALID_ARG;
    try {
        vr::launch_distances(pts, n, ambient_dim, out_lower_tri, (cudaStream_t)stream);
        VR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return VR_OK;
    } catch (const vr::Error& e) {
        return e.code;
    }
}

vr_status vr_sort_u64(uint64_t* keys, uint64_t* values, int64_t num, int32_t bits, void* stream) {
    if (num < 0 || bits < 0 || bits > 64 || (num > 0 && !keys)) return VR_ERR_INVALID_ARG;
    try {
        vr::Workspace ws((cudaStream_t)stream);
        vr::radix_sort_u64(ws, keys, values, num, bits);
        VR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return VR_OK;
    } catch (const vr::Error& e) {
        return e.code;
    }
}

}  // extern "C"
