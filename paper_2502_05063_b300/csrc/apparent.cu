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
//    only the non-apparent columns (about 1% of them) are written out, as
//    packed (rank, index) keys for the later radix sort;
//  * candidates are taken 32 consecutive indices per warp (one per lane,
//    each lane decodes its own simplex from the combinatorial number system
//    of eq. 5.6), and the cofacet search of each kept candidate is
//    warp-cooperative: the lanes test 32 consecutive added vertices w at
//    once (w descending = cofacet index descending), reading row v_i of the
//    symmetric rank matrix at columns w..w-31 -- one coalesced 128-byte load
//    per vertex of s -- and a ballot picks the largest qualifying w;
//  * the facet test needs only the ranks among the p+2 vertices of t, one
//    pair per lane, and a ballot per vertex of s above w.
// Apparent pairs have zero persistence (diam(s) = diam(t)); they are only
// counted, marked in the clearing bitmap of dimension p+1, and written out
// when zero-length pairs are requested.
#include "vr_common.cuh"

namespace vr {

namespace {

// pair index k of a (Q)-vertex set -> (i, j), i > j
__device__ __forceinline__ void pair_of(int k, int& i, int& j) {
    i = 1;
    while (k >= i) { k -= i; ++i; }
    j = k;
}

template <int P>
__global__ void __launch_bounds__(256)
k_filtration_apparent(RankMatrix R, Binom B, uint32_t thr, const uint32_t* __restrict__ clear_bits,
                      int cidx_bits, uint64_t rmask, uint64_t num_cand, ApparentOut o) {
    constexpr int NV = P + 1;                 // vertices of s
    constexpr int NPAIR_T = (P + 2) * (P + 1) / 2;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = R.n;
    unsigned long long c_above = 0, c_cleared = 0, c_kept = 0, c_app = 0, c_scan = 0, c_facet = 0;

    constexpr int NPS = NV * (NV - 1) / 2;    // vertex pairs of s
    constexpr int K_LANE = 32;                 // vertices each lane tests for its own column first
    for (uint64_t chunk = warp; chunk * 32 < num_cand; chunk += nwarps) {
        const uint64_t c = chunk * 32 + lane;
        // the warp decodes its first index once; lane L's index is L more, which
        // in the combinatorial number system (eq. 5.6) adds L to the smallest
        // vertex unless that reaches the next one (then the lane decodes itself)
        int v[NV];
        warp_decode_simplex<P>(B, chunk * 32, n - 1, v);
        v[0] += lane;
        uint32_t pr[NPS > 0 ? NPS : 1];  // ranks of the pairs of s, pair k = (a, b), a > b, in pair_of order
        uint32_t r = 0;
        bool kept = false;
        if (c < num_cand) {
            if (v[0] >= v[1]) decode_simplex<P>(B, c, n - 1, v);
            int k = 0;
#pragma unroll
            for (int a = 1; a < NV; ++a)
#pragma unroll
                for (int b = 0; b < a; ++b) {
                    pr[k] = R(v[a], v[b]);
                    r = max(r, pr[k]);
                    ++k;
                }
            if (r > thr) ++c_above;
            else if (clear_bits && ((__ldg(clear_bits + (c >> 5)) >> (c & 31)) & 1u)) ++c_cleared;
            else { kept = true; ++c_kept; }
        }
        // 1. lane-parallel: each lane tests w = n-1, n-2, ... for its own column
        bool active = kept;
        int64_t wf = -1;
        uint32_t rw[NV];  // ranks R(v[a], wf) at the hit
#pragma unroll
        for (int a = 0; a < NV; ++a) rw[a] = 0;
        int steps = 0;
        for (int step = 0; step < K_LANE; ++step) {
            const int64_t w = n - 1 - step;
            if (w < 0 || !__any_sync(0xffffffffu, active)) break;
            ++steps;
            if (active) {
                bool ok = true;
#pragma unroll
                for (int a = 0; a < NV; ++a) ok = ok && (w != v[a]);
                if (ok) {
                    uint32_t rr[NV];  // row w of the symmetric matrix: lanes with consecutive v[0] read one line
#pragma unroll
                    for (int a = 0; a < NV; ++a) rr[a] = R(w, v[a]);
#pragma unroll
                    for (int a = 0; a < NV; ++a) ok = ok && (rr[a] <= r);
                    if (ok) {
                        wf = w;
                        active = false;
#pragma unroll
                        for (int a = 0; a < NV; ++a) rw[a] = rr[a];
                    }
                }
            }
        }
        if (kept) c_scan += wf >= 0 ? (unsigned long long)(n - wf) : (unsigned long long)steps;
        // 2. columns still open: warp-cooperative search over the remaining vertices
        const int64_t base0 = n - 1 - K_LANE;
        uint32_t rem = __ballot_sync(0xffffffffu, active && base0 >= 0);
        while (rem) {
            const int src = __ffs(rem) - 1;
            rem &= rem - 1;
            int sv[NV];
#pragma unroll
            for (int a = 0; a < NV; ++a) sv[a] = __shfl_sync(0xffffffffu, v[a], src);
            const uint32_t sr = __shfl_sync(0xffffffffu, r, src);
            int64_t hit = -1;
            unsigned long long examined = 0;
            for (int64_t base = base0; base >= 0; base -= 32) {
                const int64_t w = base - lane;
                bool ok = w >= 0;
#pragma unroll
                for (int a = 0; a < NV; ++a) ok = ok && (w != sv[a]);
#pragma unroll
                for (int a = 0; a < NV; ++a) ok = ok && (R(sv[a], w) <= sr);
                const uint32_t bl = __ballot_sync(0xffffffffu, ok);
                if (bl) {
                    hit = base - (__ffs(bl) - 1);
                    examined += base - hit + 1;
                    break;
                }
                examined += base >= 31 ? 32 : base + 1;
            }
            if (lane == src) {
                c_scan += examined;
                if (hit >= 0) {
                    wf = hit;
#pragma unroll
                    for (int a = 0; a < NV; ++a) rw[a] = R(v[a], wf);
                }
            }
        }
        // 3. facet test in registers: a facet t - {v[a]} with v[a] > wf (smaller index
        //    than s) must not keep the diameter; its pairs are the pairs of s without
        //    v[a] and the pairs (wf, v[b]), b != a
        bool apparent = false;
        if (kept && wf >= 0) {
            ++c_facet;
            apparent = true;
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                if (v[a] > wf) {
                    bool keeps = false;
                    int k = 0;
#pragma unroll
                    for (int i = 1; i < NV; ++i)
#pragma unroll
                        for (int j = 0; j < i; ++j) {
                            if (i != a && j != a && pr[k] == r) keeps = true;
                            ++k;
                        }
#pragma unroll
                    for (int bb = 0; bb < NV; ++bb)
                        if (bb != a && rw[bb] == r) keeps = true;
                    if (keeps) apparent = false;
                }
            }
        }
        // 4. outputs
        if (apparent) {
            ++c_app;
            if (o.clear_next || o.zero_pairs) {
                uint64_t ct = 0;  // index of t: wf inserted into the ascending vertices of s
                int k = 0;
                bool placed = false;
#pragma unroll
                for (int a = 0; a < NV; ++a) {
                    if (!placed && wf < v[a]) { ct += B(wf, k + 1); ++k; placed = true; }
                    ct += B(v[a], k + 1);
                    ++k;
                }
                if (!placed) ct += B(wf, k + 1);
                if (o.clear_next) atomicOr(o.clear_next + (ct >> 5), 1u << (ct & 31));
                if (o.zero_pairs) {
                    const unsigned long long at = atomicAdd(o.num_zero_pairs, 1ull);
                    PairRec prc;
                    prc.birth_rank = r; prc.death_rank = r;
                    prc.birth_cidx = c; prc.death_cidx = (int64_t)ct;
                    o.zero_pairs[at] = prc;
                }
            }
        }
        const bool nonapp = kept && !apparent;
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
    // counters
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        c_above += __shfl_xor_sync(0xffffffffu, c_above, off);
        c_cleared += __shfl_xor_sync(0xffffffffu, c_cleared, off);
        c_kept += __shfl_xor_sync(0xffffffffu, c_kept, off);
        c_app += __shfl_xor_sync(0xffffffffu, c_app, off);
        c_scan += __shfl_xor_sync(0xffffffffu, c_scan, off);
        c_facet += __shfl_xor_sync(0xffffffffu, c_facet, off);
    }
    if (lane == 0) {
        if (c_above) atomicAdd(o.counters + 0, c_above);
        if (c_cleared) atomicAdd(o.counters + 1, c_cleared);
        if (c_kept) atomicAdd(o.counters + 2, c_kept);
        if (c_app) atomicAdd(o.counters + 3, c_app);
        if (c_scan) atomicAdd(o.counters + 6, c_scan);
        if (c_facet) atomicAdd(o.counters + 7, c_facet);
    }
}

template <int P>
void launch_p(const RankMatrix& R, const Binom& B, uint32_t thr, const uint32_t* clear_bits, int cidx_bits,
              uint64_t rmask, uint64_t num_cand, const ApparentOut& o, cudaStream_t s) {
    const uint64_t chunks = (num_cand + 31) / 32;
    uint64_t blocks = (chunks + 7) / 8;
    const uint64_t cap = 148ull * 8;  // 8 resident 256-thread blocks per SM
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_filtration_apparent<P><<<(unsigned)blocks, 256, 0, s>>>(R, B, thr, clear_bits, cidx_bits, rmask, num_cand, o);
    VR_CUDA(cudaGetLastError());
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
