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
//      the rest in order by the front/back block engine;
//   6. pairs sorted per cloud and appended to the output.
// A cloud that outgrows a per-block buffer is flagged and recomputed by the
// host through the single-cloud path.
#include <algorithm>
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
constexpr int64_t BACKCAP = 1 << 20;   // back rows of the block engine per cloud (8 MB)
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
    HeavySmem S;
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
        // ---- 1. points and distances (bits of the single-precision formula)
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
        }
        __syncthreads();
        const RankMatrix R{mat, n, BLD};
        // ---- 2. threshold: enclosing radius unless given
        if (threadIdx.x == 0) M.thr = A.thr_inf ? 0xFFFFFFFFu : A.thr_bits;
        __syncthreads();
        if (A.thr_inf) {
            for (int i = wid; i < n; i += HW) {
                uint32_t m = 0;
                for (int j = lane; j < n; j += 32) m = max(m, R(i, j));
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
                        const uint32_t r = R(u, v);
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
            // ---- 3b. warps 1..15: apparent pairs of the edges within the threshold
            unsigned long long c_app = 0, c_cand = 0;
            for (int ch = wid - 1; ch * 32 < ne; ch += HW - 1) {
                const int e = ch * 32 + lane;
                int va = 0, vb = 0;
                uint32_t r = 0;
                bool kept = false;
                if (e < ne) {
                    edge_of(e, va, vb);
                    r = R(va, vb);
                    kept = r <= thr;
                    c_cand += kept;
                }
                uint32_t km = __ballot_sync(0xffffffffu, kept);
                while (km) {
                    const int src = __ffs(km) - 1;
                    km &= km - 1;
                    const int a = __shfl_sync(0xffffffffu, va, src), b = __shfl_sync(0xffffffffu, vb, src);
                    const uint32_t sr = __shfl_sync(0xffffffffu, r, src);
                    const int se = __shfl_sync(0xffffffffu, e, src);
                    int wf = -1;
                    for (int base = n - 1; base >= 0; base -= 32) {
                        const int w = base - lane;
                        const bool ok = w >= 0 && w != a && w != b && R(a, w) <= sr && R(b, w) <= sr;
                        const uint32_t bl = __ballot_sync(0xffffffffu, ok);
                        if (bl) { wf = base - (__ffs(bl) - 1); break; }
                    }
                    // facet t - {x} for a vertex x > wf of s must not keep the diameter
                    bool apparent = wf >= 0;
                    if (apparent && a > wf && R(b, wf) == sr) apparent = false;
                    if (apparent && b > wf && R(a, wf) == sr) apparent = false;
                    if (lane == 0) {
                        if (apparent) ++c_app;
                        else {
                            const int at = atomicAdd(&M.ncols, 1);
                            if (at < CCAP) cols[at] = ((~(uint64_t)sr & 0xFFFFFFFFull) << EDGE_BITS) | (uint64_t)se;
                            else M.overflow = 1;
                        }
                    }
                }
            }
            if (lane == 0) {
                if (c_app) atomicAdd(A.stats + 1, c_app);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c_cand += __shfl_xor_sync(0xffffffffu, c_cand, o);
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
        c.pool_cap = POOLCAP;
        c.rc_ptr = A.rc_off + slot * (int64_t)CCAP;
        c.mode = MODE_EXPLICIT;
        c.rc_len = A.rc_len + slot * (int64_t)CCAP;
        uint32_t* adds_j = A.adds + slot * (int64_t)CCAP;
        for (uint64_t i = threadIdx.x; i < hsz; i += HT) c.hkeys[i] = EMPTY;
        if (threadIdx.x == 0) *c.pool_used = 0;
        __syncthreads();
        // 5a/5b. one round over the columns, one warp each, without additions:
        // it finds every pivot and settles, in order by the prefix-minimum rule,
        // the columns whose pivot has no owner.  The rest go to the block engine
        // (measured faster on these clouds than more warp rounds).
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
        // 5c. the remaining columns in order, each to completion (block engine)
        if (A.prof && threadIdx.x == 0) atomicAdd(A.prof + 8, (unsigned long long)nu);
        unsigned long long adds = 0;
        for (int q = 0; q < nu; ++q) {
            const int j = ucur[q];
            const uint64_t self_key = cols[j];
            Simplex<1> s;
            load_col<1>(c, self_key, s);
            if (threadIdx.x == 0) { S.fsize = 0; S.bsize = 0; S.holes = 0; S.Ks = EMPTY; S.cur = 0; }
            __syncthreads();
            bool ok = heavy_add_coboundary<1>(c, S, back, BACKCAP, s);
            uint64_t key = EMPTY;
            unsigned long long col_adds = 0;
            uint64_t prev = 0;  // pivot before the last addition
            int pre = 0;  // owner kind of the current pivot if probed during the last merge (3: none)
            while (ok) {
                if (++col_adds > (1ull << 22)) { ok = false; break; }  // far beyond any column: flag the cloud
                if (S.fsize == 0 && !heavy_refill<8>(S, back)) { key = EMPTY; break; }
                key = S.buf[S.cur][0];
                // A column finished here keeps no reduced form, so its owner's
                // coboundary D_o stands in for R_o: a valid column operation, but
                // one that may leave the pivot in place and then repeat forever.
                // An unchanged pivot sends the cloud to the single-cloud path.
                if (col_adds > 1 && key == prev) { ok = false; break; }
                prev = key;
                const int kind = pre ? (pre == 3 ? 0 : pre) : heavy_owner_probe<1>(c, S, key, self_key);
                pre = 0;
                if (kind == 0) break;
                if (kind == 1) {
                    const int64_t opos = S.opos;
                    if (c.rc_len[opos]) {
                        ok = heavy_add_stored<1>(c, S, back, BACKCAP, opos);
                    } else {
                        Simplex<1> o;
                        load_col<1>(c, cols[opos], o);
                        ok = heavy_add_coboundary<1>(c, S, back, BACKCAP, o);
                    }
                } else {
                    // the next pivot's owner is probed during the merge (one pass covers
                    // n <= 256): 85.4 -> 80.8 ms on the 4096-cloud batch, 5.55 -> 5.22 ms
                    // on the 256 circles, where one long cocycle column per cloud holds
                    // nearly all the additions
                    const int r = heavy_apparent_add<1, true>(c, S, back, BACKCAP, self_key, &pre);
                    if (r < 0) break;  // the pivot has no owner: the column is complete
                    ok = r > 0;
                }
                ++adds;
                __syncthreads();
            }
            if (!ok) {
                if (threadIdx.x == 0) M.overflow = 1;
                __syncthreads();
                break;
            }
            if (threadIdx.x == 0) {
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
                if (out) h1tmp[M.nh1++] = pr;
            }
            __syncthreads();
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
};

std::mutex g_batch_mutex;
BatchPlan* g_plan = nullptr;
std::map<std::pair<int, int64_t>, int> g_tuned;  // (device, mean-size bucket) -> slots per SM

size_t slot_bytes() {
    return (size_t)BMAXN * BLD * 4 + (size_t)HCAP * 12 +
           (size_t)CCAP * (8 + 8 + 1 + 8 + sizeof(PairRec) + 8 + 4 + 4) + (size_t)BACKCAP * 8 +
           (size_t)HW * STAGE * 8 + (size_t)POOLCAP * 8 + 16 * 256;
}

void free_plan(BatchPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
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
// the first batch of a given mean cloud size and remembered per device.
int tuned_slots(BatchPlan& P, cudaStream_t s, int sms, int64_t bucket) {
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
        const int64_t bucket = total / num_clouds / 32;
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
        // host reads: usage, per-cloud errors
        unsigned long long used[2] = {0, 0};
        VR_CUDA(cudaMemcpyAsync(used, P->args.used, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        std::vector<int32_t> cerr(num_clouds);
        VR_CUDA(cudaMemcpyAsync(cerr.data(), P->args.cloud_err, num_clouds * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
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
            VR_CUDA(cudaMemcpyAsync(cerr.data(), P->args.cloud_err, num_clouds * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
        }
        if (P->args.prof) {
            unsigned long long pr[16], st[4];
            VR_CUDA(cudaMemcpy(pr, P->args.prof, sizeof pr, cudaMemcpyDeviceToHost));
            VR_CUDA(cudaMemcpy(st, P->args.stats, sizeof st, cudaMemcpyDeviceToHost));
            const char* names[8] = {"distances+threshold", "H0 tree + apparent", "H0 output", "clear+sort",
                                    "first pass", "finalize", "block engine", "H1 output"};
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
        VR_CUDA(cudaMemcpyAsync(res->thresholds, P->args.thr_used, num_clouds * sizeof(float), cudaMemcpyDeviceToHost, s));
        for (int p = 0; p <= dmax; ++p)
            VR_CUDA(cudaMemcpyAsync(res->pair_offsets[p], P->off[p], (num_clouds + 1) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, s));
        VR_CUDA(cudaStreamSynchronize(s));
        std::vector<int> bad;
        int codes[8] = {0};
        for (int i = 0; i < num_clouds; ++i)
            if (cerr[i]) { bad.push_back(i); codes[cerr[i] & 7]++; }
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
                    VR_CUDA(cudaStreamSynchronize(s));
                    memcpy(res->pair_offsets[p], off.data(), (num_clouds + 1) * sizeof(int64_t));
                    continue;
                }
            }
            res->pairs[p] = (vr_pair*)malloc(std::max<int64_t>(off[num_clouds], 1) * sizeof(vr_pair));
            if (want_edges)
                res->critical_edges[p] = (int32_t*)malloc(std::max<int64_t>(off[num_clouds], 1) * 4 * sizeof(int32_t));
            if (!res->pairs[p] || (want_edges && !res->critical_edges[p])) throw Error{VR_ERR_OOM};
            if (bad.empty()) {
                VR_CUDA(cudaMemcpyAsync(res->pairs[p], P->pairs[p], off[num_clouds] * sizeof(vr_pair),
                                        cudaMemcpyDeviceToHost, s));
                if (want_edges)
                    VR_CUDA(cudaMemcpyAsync(res->critical_edges[p], P->edges[p], off[num_clouds] * 4 * sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, s));
                VR_CUDA(cudaStreamSynchronize(s));
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
