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
// strictly decreasing keys, hence distinct pivots.
//
// Phase 1: one warp per column, at most 8 additions (none when there are
// at most four columns per SM), all columns at once.  No column is final
// yet, so every owner is apparent; a column is kept as the list of
// simplices added to it (see reduce_one), and finished columns that needed
// additions store that list, their column of V.  Phase 2:
// one block per remaining column (the front/back engine of
// reduce_device.cuh), state kept across rounds, at most 64 additions per
// round so that finalized pivots reach waiting columns early; a column
// whose pivot belongs to a column finished in phase 2 adds that column's
// reduced form.  The first unfinished column can never be blocked, so every
// round makes progress (it is finalized or gains its additions); if the
// first column overflows its back buffer in a batch of rounds, the remaining
// columns restart in new buffers with at least twice the room (VR_ERR_OOM
// past 2^31 rows) while finished columns keep theirs, with their reduced forms.
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

#include "reduce_device.cuh"

namespace vr {

namespace {

template <int P>
__global__ void __launch_bounds__(RED_WARPS * 32)
k_reduce_round(Ctx c, const uint32_t* __restrict__ U, int64_t u, int budget, uint64_t* __restrict__ cur_key,
               uint8_t* __restrict__ status, uint32_t* __restrict__ adds, unsigned long long* __restrict__ work) {
    __shared__ uint64_t stage_all[RED_WARPS][STAGE];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(work, 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        if ((int64_t)k >= u) break;
        const int64_t j = U[k];
        uint64_t key;
        uint8_t st;
        uint32_t ad;
        reduce_one<P>(c, j, budget, stage_all[wid], key, st, ad);
        if (lane == 0) { cur_key[j] = key; status[j] = st; adds[j] = ad; }
    }
}


// Finalize a round with one block (any multiple of 32 threads): in order,
// column j is final iff complete and its key is below the prefix minimum of
// the earlier unfinished keys; the rest go, in order, to Unext.  If the first
// column overflowed, *first_status becomes ST_OVERFLOW (and stays so until
// the host clears it: rounds are checked in batches).  The round's
// keys, states and addition counts were written by other blocks of the same
// kernel (heavy rounds) or by an earlier kernel, so they are read through L2.
__device__ void finalize_rows(const Ctx& c, const Emit& e, const uint32_t* __restrict__ U, int64_t u,
                              const uint64_t* cur_key, const uint8_t* status, const uint32_t* adds,
                              uint32_t* __restrict__ Unext, unsigned long long* __restrict__ u_next,
                              unsigned long long* __restrict__ first_status, const HeavyState* hv = nullptr,
                              uint32_t* __restrict__ slot_of = nullptr) {
    __shared__ uint64_t wmin[32];
    __shared__ uint32_t wcnt[32];
    __shared__ uint32_t rel_j[1024], rel_s[1024], rel_a[1024];  // windowed: slots released by this chunk
    __shared__ uint32_t rel_n;
    __shared__ unsigned long long rel_off;
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
        const uint64_t key = valid ? __ldcg(cur_key + j) : EMPTY;
        const uint8_t st = valid ? __ldcg(status + j) : ST_COMPLETE;
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
        if (k == 0 && st == ST_OVERFLOW) *first_status = ST_OVERFLOW;  // sticky until the host clears it
        if (fin) finish_column(c, e, j, key, __ldcg(adds + j));
        if (hv && hv->free_slots) {
            // windowed engine: finalized columns give their slots back; in V mode
            // their generators first move to the pool (one column at a time, by
            // the whole block), where later columns read them as R_j
            if (threadIdx.x == 0) rel_n = 0;
            __syncthreads();
            const uint32_t sl = fin ? slot_of[j] : 0xFFFFFFFFu;
            if (sl != 0xFFFFFFFFu) {
                const uint32_t q = atomicAdd(&rel_n, 1u);
                rel_j[q] = j;
                rel_s[q] = sl;
                rel_a[q] = __ldcg(adds + j);
            }
            __syncthreads();
            const uint32_t nrel = rel_n;
            for (uint32_t q = 0; q < nrel; ++q) {
                const uint32_t jj = rel_j[q], ss = rel_s[q];
                if (c.mode == MODE_V && rel_a[q] > 0) {
                    const int64_t len = __ldcg(hv->vlen + ss);
                    if (threadIdx.x == 0) rel_off = atomicAdd(c.pool_used, (unsigned long long)len);
                    __syncthreads();
                    const unsigned long long off = rel_off;
                    const bool fits = (int64_t)(off + len) <= c.pool_cap;
                    const uint64_t* src = hv->V[ss];
                    if (fits)
                        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) c.pool[off + i] = __ldcg(src + i);
                    if (threadIdx.x == 0) {
                        c.rc_ptr[jj] = fits ? (uint64_t)(c.pool + off) : 0;
                        c.rc_len[jj] = fits ? (uint32_t)len : 0u;
                        if (!fits) atomicExch(c.err, DEV_CAPACITY);
                    }
                } else if (threadIdx.x == 0 && c.mode == MODE_V) {
                    c.rc_len[jj] = 0;  // no addition: the column is D_j itself
                }
                if (threadIdx.x == 0) {
                    hv->free_slots[atomicAdd(hv->free_top, 1)] = (int32_t)ss;
                    slot_of[jj] = 0xFFFFFFFFu;
                }
                __syncthreads();
            }
        }
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

__global__ void __launch_bounds__(1024)
k_finalize(Ctx c, Emit e, const uint32_t* __restrict__ U, int64_t u, const uint64_t* __restrict__ cur_key,
           const uint8_t* __restrict__ status, const uint32_t* __restrict__ adds, uint32_t* __restrict__ Unext,
           unsigned long long* __restrict__ u_next, unsigned long long* __restrict__ first_status) {
    finalize_rows(c, e, U, u, cur_key, status, adds, Unext, u_next, first_status);
}


template <int P>
__device__ void heavy_column(const Ctx& c, const uint32_t* __restrict__ U, int64_t k,
                             uint32_t* __restrict__ slot_of, const HeavyState& hs, int budget,
                             uint64_t* __restrict__ cur_key, uint8_t* __restrict__ status,
                             uint32_t* __restrict__ adds_out) {
    extern __shared__ __align__(16) unsigned char hsm[];
    HeavySmem& S = *reinterpret_cast<HeavySmem*>(hsm);
    __shared__ int64_t slot_sh;
    const int64_t j = U[k];
    if (threadIdx.x == 0) {
        int64_t sl = slot_of[j];
        if (sl == 0xFFFFFFFFu) {  // windowed engine: the column enters the window
            const int t = atomicSub(hs.free_top, 1) - 1;
            if (t >= 0) {
                sl = hs.free_slots[t];
                slot_of[j] = (uint32_t)sl;
                hs.init[sl] = 0;
            } else {  // cannot happen (as many slots as window places): leave the column as it was
                atomicAdd(hs.free_top, 1);
                atomicExch(c.err, DEV_INTERNAL | (5 << 8));
                sl = -1;
            }
        }
        slot_sh = sl;
    }
    __syncthreads();
    const int64_t slot = slot_sh;
    if (slot < 0) return;
    if (hs.init[slot] && status[j] == ST_COMPLETE) {
        // complete in an earlier round and waiting to be finalized in order: it
        // changes only if its pivot has since become a finished column's pivot
        // (whether it has an apparent owner never changes), so one probe of the
        // hash stands in for reloading and saving its state
        __shared__ int still;
        const uint64_t key = cur_key[j];
        if (key == EMPTY) return;  // a zero column stays zero
        if (threadIdx.x < 32) {
            const int64_t hp = warp_hash_find(c, c.rcmask - (key & c.rcmask));
            if (threadIdx.x == 0) still = hp < 0;
        }
        __syncthreads();
        if (still) return;
    }
    uint64_t* B = hs.B[slot];
    const int64_t bcap = hs.bcap[slot];
    const uint64_t self_key = c.cols[j];
    Simplex<P> s;
    load_col<P>(c, self_key, s);
    if (threadIdx.x < 20) S.tp[threadIdx.x] = 0;
    __syncthreads();
    uint32_t adds;
    bool ok = true;
    const bool vmode = c.mode == MODE_V;
    uint64_t* V = vmode ? hs.V[slot] : nullptr;
    const int64_t vcap = vmode ? hs.vcap[slot] : 0;
    if (!hs.init[slot]) {
        if (threadIdx.x == 0) { S.fsize = 0; S.bsize = 0; S.holes = 0; S.Ks = EMPTY; S.cur = 0; S.vlen = 0; }
        __syncthreads();
        adds = 0;
        ok = heavy_add_coboundary<P>(c, S, B, bcap, s);
        if (ok && vmode) ok = heavy_v_append1(S, V, vcap, self_key);
    } else {
        if (threadIdx.x == 0) {
            S.fsize = hs.fsize[slot]; S.bsize = hs.bsize[slot]; S.holes = hs.holes[slot]; S.Ks = hs.Ks[slot]; S.cur = 0;
            S.vlen = vmode ? hs.vlen[slot] : 0;
        }
        adds = hs.adds[slot];
        __syncthreads();
        for (int i = threadIdx.x; i < S.fsize; i += HT) S.buf[0][i] = hs.F[slot * FC + i];
        __syncthreads();
    }
    uint64_t key = ok ? EMPTY : 0;  // 0: no consistent state yet, the smallest (always valid) bound
    uint8_t st = ST_COMPLETE;
    int done = 0;
    int pre = 0;  // owner kind of the current pivot if probed during the last merge (3: none)
    long long t0 = clock64(), t_ref = 0, t_look = 0, t_add = 0, n_look = 0;
    const long long t_resume = t0;
    while (ok) {
        long long ta = HCLK();
        if (S.fsize == 0 && !heavy_refill(S, B)) { key = EMPTY; break; }  // zero column
        long long tb = HCLK();
        t_ref += tb - ta;
        key = S.buf[S.cur][0];
        // the owner of this pivot may have been probed during the last merge
        const int kind = pre ? (pre == 3 ? 0 : pre) : heavy_owner_probe<P>(c, S, key, self_key);
        if (pre && threadIdx.x == 0 && key != S.sel) atomicExch(c.err, DEV_INTERNAL | (1 << 8));
        pre = 0;
        long long tc = HCLK();
        t_look += tc - tb;
        ++n_look;
        if (kind == 0) break;  // pivot unknown: complete
        if (done >= budget) {
            if (kind == 2 && !heavy_apparent_check<P>(c, S)) break;  // no owner after all: complete
            st = ST_BUDGET;
            break;
        }
        if (hs.prof && threadIdx.x == 0) S.tp[15] -= clock64();
        if (kind == 1) {
            const int64_t opos = S.opos;
            const uint32_t os = slot_of[opos];
            if (c.mode == MODE_EXPLICIT && os != 0xFFFFFFFFu && hs.init[os] && hs.adds[os] > 0) {
                // owner finished by this engine: add its reduced form, front then back
                ok = heavy_add_multiset(S, B, bcap, hs.F + (int64_t)os * FC, hs.fsize[os]) &&
                     heavy_add_multiset(S, B, bcap, hs.B[os], hs.bsize[os]);
            } else if (c.mode != MODE_OBLIVIOUS && c.rc_len[opos]) {
                // R_o from its generators (column o of V)
                ok = heavy_add_stored<P>(c, S, B, bcap, opos);
                if (ok && vmode)
                    ok = heavy_v_append(S, V, vcap, reinterpret_cast<const uint64_t*>(c.rc_ptr[opos]),
                                        c.rc_len[opos]);
            } else {
                // D_o: the owner needed no addition, or (oblivious) nothing of R_o is kept
                Simplex<P> o;
                load_col<P>(c, c.cols[opos], o);
                ok = heavy_add_coboundary<P>(c, S, B, bcap, o);
                if (ok && vmode) ok = heavy_v_append1(S, V, vcap, c.cols[opos]);
            }
        } else {
            // the probe's candidate s' is overwritten when the merge probes the next pivot
            const uint64_t okey = vmode ? probed_owner_key<P>(c, S) : 0;
            const int r = heavy_apparent_add<P>(c, S, B, bcap, self_key, &pre);
            if (r < 0) {  // s' is not apparent: the pivot has no owner, the column is complete
                if (hs.prof && threadIdx.x == 0) S.tp[15] += clock64();
                break;
            }
            ok = r > 0;
            if (ok && vmode) ok = heavy_v_append1(S, V, vcap, okey);
        }
        ++adds;
        ++done;
        __syncthreads();
        if (hs.prof && threadIdx.x == 0) S.tp[15] += clock64();
        t_add += HCLK() - tc;
    }
    if (hs.prof && threadIdx.x == 0) {
        atomicAdd(hs.prof + 0, (unsigned long long)t_ref);
        atomicAdd(hs.prof + 1, (unsigned long long)t_look);
        atomicAdd(hs.prof + 2, (unsigned long long)t_add);
        atomicAdd(hs.prof + 3, (unsigned long long)(clock64() - t_resume - t_ref - t_look - t_add));
        atomicAdd(hs.prof + 4, (unsigned long long)done);
        atomicAdd(hs.prof + 5, (unsigned long long)n_look);
        atomicMax(hs.prof + 6, (unsigned long long)done);
        atomicMax(hs.prof + 7, (unsigned long long)(clock64() - t_resume));
        const long long tot = clock64() - t_resume;
        if (tot > 500000 && done >= 60)
            printf("[vr] dim%d col %lld: %d adds %lld cycles: refill %lld lookup %lld add %lld | gen %lld sort %lld "
                   "merge %lld multiset %lld (%lld) | refill sample %lld count %lld compact %lld sort %lld (%lld) "
                   "back %lld front %d\n",
                   P, (long long)j, done, tot, t_ref, t_look, t_add, S.tp[0], S.tp[1], S.tp[2], S.tp[3], S.tp[8],
                   S.tp[4], S.tp[5], S.tp[6], S.tp[7], S.tp[9], (long long)S.bsize, S.fsize);
        if (tot > 500000 && done >= 60)
            printf("[vr] dim%d col %lld: head check %lld, wait for merge %lld, spill %lld | owner probe %lld "
                   "apparent test+gen %lld | add total %lld | merge group %lld, merges %lld, mean a %lld b %lld\n",
                   P, (long long)j, S.tp[10], S.tp[11], S.tp[12], S.tp[13], S.tp[14], S.tp[15], S.tp[16], S.tp[19],
                   S.tp[17] / (S.tp[19] ? S.tp[19] : 1), S.tp[18] / (S.tp[19] ? S.tp[19] : 1));
    }
    if (!ok) st = ST_OVERFLOW;  // key holds the last consistent pivot, a valid bound
    for (int i = threadIdx.x; i < S.fsize && ok; i += HT) hs.F[slot * FC + i] = S.buf[S.cur][i];
    if (threadIdx.x == 0) {
        hs.fsize[slot] = S.fsize;
        hs.bsize[slot] = S.bsize;
        hs.holes[slot] = S.holes;
        hs.Ks[slot] = S.Ks;
        hs.adds[slot] = adds;
        if (vmode) hs.vlen[slot] = S.vlen;
        hs.init[slot] = ok ? 1 : 0;  // an overflowed column restarts from scratch
        cur_key[j] = key;
        status[j] = st;
        adds_out[j] = adds;
    }
}

// One round of the block engine: block k reduces column U[k] for k < *d_u
// (the count the previous round left on the device; the grid may be larger),
// and the last block to finish finalizes the round into Unext / *d_unext.
// No block waits for another, so rounds can be queued without the host.
template <int P>
__global__ void __launch_bounds__(HT, 1)
k_reduce_heavy(Ctx c, Emit e, const uint32_t* __restrict__ U, const unsigned long long* __restrict__ d_u,
               uint32_t* __restrict__ slot_of, HeavyState hs, int budget,
               uint64_t* __restrict__ cur_key, uint8_t* __restrict__ status, uint32_t* __restrict__ adds_out,
               uint32_t* __restrict__ Unext, unsigned long long* __restrict__ d_unext,
               unsigned long long* __restrict__ first_status, unsigned int* __restrict__ done) {
    __shared__ int last;
    const int64_t u = (int64_t)*d_u;
    if ((int64_t)blockIdx.x < u) heavy_column<P>(c, U, blockIdx.x, slot_of, hs, budget, cur_key, status, adds_out);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    finalize_rows(c, e, U, u, cur_key, status, adds_out, Unext, d_unext, first_status, &hs, slot_of);
    if (threadIdx.x == 0) *done = 0;  // ready for the next round (launched after this kernel ends)
}

// Slot k for column U[k], with the k-th back buffer of `arena` (bcap rows each).
__global__ void k_assign_slots(const uint32_t* __restrict__ U, int64_t u, uint32_t* __restrict__ slot_of,
                               uint8_t* __restrict__ init, uint64_t* arena, int64_t bcap, uint64_t** B,
                               int64_t* __restrict__ bc, uint64_t* varena, int64_t vcap, uint64_t** V,
                               int64_t* __restrict__ vc) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x) {
        slot_of[U[k]] = (uint32_t)k;
        init[k] = 0;
        B[k] = arena + k * bcap;
        bc[k] = bcap;
        if (varena) {
            V[k] = varena + k * vcap;
            vc[k] = vcap;
        }
    }
}

// Windowed engine: a column outside the window does not run, so no state of
// it may read as complete (its pivot may have gained an owner since phase 1);
// its key stays as a lower bound on its final pivot.
__global__ void k_mark_unsettled(const uint32_t* __restrict__ U, int64_t u, uint8_t* __restrict__ status) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x)
        status[U[k]] = ST_BUDGET;
}

__global__ void k_release_slots(const uint32_t* __restrict__ U, int64_t u, uint32_t* __restrict__ slot_of) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x)
        slot_of[U[k]] = 0xFFFFFFFFu;
}

// Windowed engine: every slot gets its buffers (the k-th of each arena) and
// joins the free list; a regrowth calls it again with larger buffers (every
// held slot restarts its column from scratch).
__global__ void k_window_slots(int64_t nslot, int32_t* __restrict__ free_slots, int32_t* __restrict__ free_top,
                               uint8_t* __restrict__ init, uint64_t* arena, int64_t bcap, uint64_t** B,
                               int64_t* __restrict__ bc, uint64_t* varena, int64_t vcap, uint64_t** V,
                               int64_t* __restrict__ vc, int fresh) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nslot; k += (int64_t)gridDim.x * blockDim.x) {
        init[k] = 0;
        B[k] = arena + k * bcap;
        bc[k] = bcap;
        if (varena) {
            V[k] = varena + k * vcap;
            vc[k] = vcap;
        }
        if (fresh) free_slots[k] = (int32_t)k;
    }
    if (fresh && blockIdx.x == 0 && threadIdx.x == 0) *free_top = (int32_t)nslot;
}

// Regrowth: the unfinished columns U[0..u) restart in the k-th buffer of a
// new arena; finished columns keep their slots, buffers and reduced forms.
__global__ void k_regrow_slots(const uint32_t* __restrict__ U, int64_t u, const uint32_t* __restrict__ slot_of,
                               uint8_t* __restrict__ init, uint64_t* arena, int64_t bcap, uint64_t** B,
                               int64_t* __restrict__ bc, uint64_t* varena, int64_t vcap, uint64_t** V,
                               int64_t* __restrict__ vc) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < u; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t slot = slot_of[U[k]];
        init[slot] = 0;
        B[slot] = arena + k * bcap;
        bc[slot] = bcap;
        if (varena) {
            V[slot] = varena + k * vcap;
            vc[slot] = vcap;
        }
    }
}

__global__ void k_iota(uint32_t* U, int64_t m) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        U[k] = (uint32_t)k;
}

constexpr int64_t HEAVY_WINDOW = 256;  // block-engine columns in flight (V and oblivious modes)

// Rows of the arena the block engine's back buffers share.
int64_t heavy_arena_rows() {
    const char* v = getenv("VR_HEAVY_ARENA_LOG2");
    int lg = v ? atoi(v) : 28;
    lg = lg < 16 ? 16 : (lg > 30 ? 30 : lg);
    return (int64_t)1 << lg;
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
    // Phase 1: one warp per column, at most 8 additions, every column at once.
    {
        const int64_t max_slots = 148 * 4 * RED_WARPS;
        int64_t slots = u < max_slots ? u : max_slots;
        slots = (slots + RED_WARPS - 1) / RED_WARPS * RED_WARPS;
        VR_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s));
        // Phase 1 is a throughput engine for many short columns; with at most
        // four columns per SM the block engine takes every column at once, and
        // warp-engine additions of a column that does not finish here would be
        // redone, so phase 1 then only settles the columns needing no addition.
        int sms = 148;
        {
            int dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        }
        const int p1_budget = u <= 4 * (int64_t)sms ? 0 : 8;
        k_reduce_round<P><<<(unsigned)(slots / RED_WARPS), RED_WARPS * 32, 0, s>>>(c, U, u, p1_budget, cur_key, status,
                                                                                   adds, ctr);
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
    // first unfinished column can never be blocked by an earlier one, so it
    // gains `budget` additions every round until it is finalized.
    int rounds = 0;
    if (u > 0) {
        const size_t smem = sizeof(HeavySmem);
        VR_CUDA(cudaFuncSetAttribute(k_reduce_heavy<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // default mode: a slot per column (finished columns keep R_j in theirs);
        // V and oblivious modes: a window of at most HEAVY_WINDOW columns in order
        const bool windowed = c.mode != MODE_EXPLICIT;
        const int64_t nslot = windowed ? std::min<int64_t>(u, HEAVY_WINDOW) : u;
        int64_t window = nslot;  // slots in circulation (shrinks when the buffers must grow past the caps)
        HeavyState h;
        // back buffers share an arena of 2^28 rows (2 GB; VR_HEAVY_ARENA_LOG2 overrides, for tests)
        const int64_t arena = heavy_arena_rows();
        int64_t bcap = std::max<int64_t>((int64_t)1 << 16, std::min<int64_t>((int64_t)1 << 22, arena / nslot)) & ~(int64_t)15;
        h.F = ws.alloc_n<uint64_t>((size_t)nslot * FC);
        h.B = ws.alloc_n<uint64_t*>(nslot);
        h.bcap = ws.alloc_n<int64_t>(nslot);
        h.Ks = ws.alloc_n<uint64_t>(nslot);
        h.fsize = ws.alloc_n<int32_t>(nslot);
        h.bsize = ws.alloc_n<int64_t>(nslot);
        h.init = ws.alloc_n<uint8_t>(nslot);
        h.adds = ws.alloc_n<uint32_t>(nslot);
        h.holes = ws.alloc_n<int64_t>(nslot);
        h.prof = log_enabled() ? ws.zeros_n<unsigned long long>(8) : nullptr;
        // V mode: each slot's generator list, from an arena of 2^26 entries (grown
        // with the back buffers, up to 2^30 entries in all)
        const bool vmode = c.mode == MODE_V;
        int64_t vcap = std::max<int64_t>((int64_t)1 << 12, std::min<int64_t>((int64_t)1 << 22, ((int64_t)1 << 26) / nslot));
        h.V = vmode ? ws.alloc_n<uint64_t*>(nslot) : nullptr;
        h.vcap = vmode ? ws.alloc_n<int64_t>(nslot) : nullptr;
        h.vlen = vmode ? ws.zeros_n<int64_t>(nslot) : nullptr;
        h.free_slots = windowed ? ws.alloc_n<int32_t>(nslot) : nullptr;
        h.free_top = windowed ? ws.zeros_n<int32_t>(1) : nullptr;
        uint32_t* slot_of = ws.alloc_n<uint32_t>(m);
        VR_CUDA(cudaMemsetAsync(slot_of, 0xFF, m * sizeof(uint32_t), s));  // no slot: phase-1 columns
        if (windowed) {
            k_window_slots<<<(unsigned)((nslot + 255) / 256), 256, 0, s>>>(
                nslot, h.free_slots, h.free_top, h.init, ws.alloc_n<uint64_t>((size_t)nslot * bcap), bcap, h.B,
                h.bcap, vmode ? ws.alloc_n<uint64_t>((size_t)nslot * vcap) : nullptr, vcap, h.V, h.vcap, 1);
            k_mark_unsettled<<<(unsigned)std::min<int64_t>((u + 255) / 256, 4096), 256, 0, s>>>(U, u, status);
        } else
            k_assign_slots<<<(unsigned)((u + 255) / 256), 256, 0, s>>>(
                U, u, slot_of, h.init, ws.alloc_n<uint64_t>((size_t)nslot * bcap), bcap, h.B, h.bcap,
                vmode ? ws.alloc_n<uint64_t>((size_t)nslot * vcap) : nullptr, vcap, h.V, h.vcap);
        int budget = 64;
        // Columns are finalized between rounds only, so a round that runs as
        // long as its longest column would keep columns it unblocks idle; a
        // cap of 64 additions (about 0.3 ms) keeps rounds short.  With at most
        // eight unfinished columns few can be waiting, and longer rounds save
        // launches, state reloads and finalizations (measured on torus500: up to
        // 256 additions, its two long dimension-1 columns 10.0 -> 9.65 ms with the
        // bound at four, dimension 2 8.99 -> 8.85 ms with it at eight; up to 1024,
        // the step 19.70 -> 19.66 ms, three alternating pairs on one GPU).
        constexpr int budget_cap = 64, budget_cap_few = 1024;
        int64_t stalled_adds = 0;  // additions granted to the first column since a column was last finalized
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (h.prof) { VR_CUDA(cudaEventCreate(&ev[0])); VR_CUDA(cudaEventCreate(&ev[1])); }
        // Each round leaves its unfinished count on the device (du[0] / du[1]
        // alternate with U / Un), so rounds are queued `chunk` at a time and
        // the host only looks between chunks; a round queued after the last
        // column finished has nothing to do.  VR_LOG=1 looks after every round.
        unsigned long long* du = ws.zeros_n<unsigned long long>(3);  // counts [0] [1], first status [2]
        unsigned int* done = ws.zeros_n<unsigned int>(1);
        VR_CUDA(cudaMemcpyAsync(du, ctr + 1, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
        int cur = 0;
        const int chunk = log_enabled() ? 1 : 8;
        while (u > 0) {
            const int64_t u0 = u;
            int granted = 0;
            VR_CUDA(cudaMemsetAsync(du + 2, 0, sizeof(unsigned long long), s));
            for (int r = 0; r < chunk; ++r) {
                if (h.prof) {
                    VR_CUDA(cudaMemsetAsync(h.prof + 6, 0, 2 * sizeof(unsigned long long), s));
                    VR_CUDA(cudaEventRecord(ev[0], s));
                }
                k_reduce_heavy<P><<<(unsigned)(windowed ? std::min<int64_t>(u0, window) : u0), HT, smem, s>>>(c, e, U, du + cur, slot_of, h, budget,
                                                                   cur_key, status, adds, Un, du + (cur ^ 1), du + 2,
                                                                   done);
                VR_CUDA(cudaGetLastError());
                if (h.prof) VR_CUDA(cudaEventRecord(ev[1], s));
                uint32_t* t = U; U = Un; Un = t;
                cur ^= 1;
                ++rounds;
                granted += budget;
                const int cap = u0 <= 8 ? budget_cap_few : budget_cap;
                budget = budget < cap ? 2 * budget : cap;
            }
            VR_CUDA(cudaMemcpyAsync(&hs.p[8], du + cur, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaMemcpyAsync(&hs.p[9], du + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            if (h.prof)
                VR_CUDA(cudaMemcpyAsync(&hs.p[24], h.prof + 6, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
            const int64_t un = hs.p[8];
            const int64_t first = hs.p[9];
            if (log_enabled()) {
                float ms = 0.f;
                if (h.prof) VR_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
                fprintf(stderr,
                        "[vr] dim%d block round %d: budget %d bcap %lld: %lld -> %lld unfinished; %.3f ms, "
                        "max additions %lld, max block cycles %lld\n",
                        P, rounds, budget, (long long)bcap, (long long)u0, (long long)un, ms, (long long)hs.p[24],
                        (long long)hs.p[25]);
            }
            const bool stalled = un == u0;
            u = un;
            stalled_adds = stalled ? stalled_adds + granted : 0;
            if (stalled_adds > ((int64_t)1 << 24)) throw Error{VR_ERR_INTERNAL};  // no column can need this many
            if (first == ST_OVERFLOW && u > 0) {
                // the first column (which no other column can block) outgrew its
                // back buffer in this batch: the remaining columns restart from
                // scratch with at least twice the room (the whole arena when
                // that is more), up to 2^31 rows in all
                int64_t held = windowed ? window : u;  // buffers to replace
                const int64_t nb = std::max<int64_t>(2 * bcap, arena / held) & ~(int64_t)15;
                const int64_t nv = vmode ? std::max<int64_t>(2 * vcap, ((int64_t)1 << 26) / held) : 0;
                // windowed: fewer columns in flight rather than failing (the first
                // column, which every round advances, keeps its place)
                while (windowed && held > 1 && ((double)nb * (double)held > (double)((int64_t)1 << 31) ||
                                                (double)nv * (double)held > (double)((int64_t)1 << 30)))
                    held /= 2;
                if ((double)nb * (double)held > (double)((int64_t)1 << 31)) throw Error{VR_ERR_OOM};
                if (vmode && (double)nv * (double)held > (double)((int64_t)1 << 30)) throw Error{VR_ERR_OOM};
                bcap = nb;
                vcap = nv;
                if (log_enabled())
                    fprintf(stderr, "[vr] dim%d regrowth: %lld unfinished columns restart with %lld rows each\n", P,
                            (long long)u, (long long)bcap);
                if (windowed) {
                    const int fresh = held < window ? 1 : 0;
                    if (fresh) {  // a smaller window: every column gives its slot back (all restart anyway),
                                  // and a column left outside it must not read as complete
                        k_release_slots<<<(unsigned)std::min<int64_t>((u + 255) / 256, 4096), 256, 0, s>>>(
                            U, u, slot_of);
                        k_mark_unsettled<<<(unsigned)std::min<int64_t>((u + 255) / 256, 4096), 256, 0, s>>>(
                            U, u, status);
                    }
                    window = held;
                    k_window_slots<<<(unsigned)((window + 255) / 256), 256, 0, s>>>(
                        window, h.free_slots, h.free_top, h.init, ws.alloc_n<uint64_t>((size_t)window * bcap), bcap,
                        h.B, h.bcap, vmode ? ws.alloc_n<uint64_t>((size_t)window * vcap) : nullptr, vcap, h.V,
                        h.vcap, fresh);
                } else
                    k_regrow_slots<<<(unsigned)((u + 255) / 256), 256, 0, s>>>(
                        U, u, slot_of, h.init, ws.alloc_n<uint64_t>((size_t)u * bcap), bcap, h.B, h.bcap,
                        nullptr, vcap, h.V, h.vcap);
                VR_CUDA(cudaGetLastError());
            }
        }
        if (h.prof) {
            VR_CUDA(cudaEventDestroy(ev[0]));
            VR_CUDA(cudaEventDestroy(ev[1]));
            VR_CUDA(cudaMemcpyAsync(&hs.p[16], h.prof, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            VR_CUDA(cudaStreamSynchronize(s));
            unsigned long long hc[4];
            VR_CUDA(cudaMemcpyFromSymbol(hc, g_heavy_counts, sizeof hc));
            fprintf(stderr, "[vr] dim%d block engine: %llu refills, %llu rows to front, %llu rows to back, %llu passes\n", P,
                    hc[0], hc[1], hc[2], hc[3]);
            const unsigned long long zero[4] = {0, 0, 0, 0};
            VR_CUDA(cudaMemcpyToSymbol(g_heavy_counts, zero, sizeof zero));
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
        fprintf(stderr, "[vr] dim%d reduction: %d block rounds, stored generators %lld of %lld\n", P, rounds,
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
    // a warp-engine column stores at most RGEN generators, once; in V mode the
    // block engine's columns store theirs too
    c.pool_cap = in.num_cols * RGEN + (in.mode == 1 ? ((int64_t)1 << 26) : 0);
    c.pool = ws.alloc_n<uint64_t>((size_t)c.pool_cap);
    c.pool_used = ws.zeros_n<unsigned long long>(1);
    c.rc_ptr = ws.alloc_n<uint64_t>((size_t)in.num_cols);
    c.mode = in.mode;
    c.nb_off = in.nb_off;
    c.nb = in.nb;
    c.rc_len = ws.zeros_n<uint32_t>((size_t)in.num_cols);
    Emit e;
    e.pairs = out.pairs;
    e.num_pairs = out.num_pairs;
    e.clear_next = out.clear_next;
    e.counters = out.counters;
    e.keep_zero = keep_zero ? 1 : 0;
    e.next_list = out.next_list;
    e.next_len = out.next_len;
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
