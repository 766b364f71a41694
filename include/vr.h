/*
 * vr.h -- C ABI of libvrgpu: Vietoris-Rips persistence barcodes over Z/2 on
 * NVIDIA B300 (sm_103a).
 *
 * Method: the GPU-accelerated Vietoris-Rips computation of arXiv 2502.05063,
 * Ch. 5 ("Ripser++"): the Rips filtration of eq. 5.3 with the simplex-wise
 * order of Sec. 5.1.4, simplices encoded by the combinatorial number system
 * (eq. 5.6), computed dimension by dimension as cohomology (Sec. 5.2.4) with
 * clearing (Sec. 5.2.3), filtration construction with clearing (Algorithms
 * 17/18), apparent pairs (Def 5.3.4, Lemma 5.3.6, Algorithm 13) and a Z/2
 * reduction of the remaining columns (Algorithm 12); dimension 0 by the
 * minimum spanning tree (Sec. 5.2.5).
 *
 * Conventions shared by every entry point:
 *  - Distances are single precision, d(i,j) = sqrt(sum_k (x_ik - x_jk)^2)
 *    with k ascending and every operation rounded once (no fused
 *    multiply-add), so every birth and death is an entry of that matrix.
 *  - A p-simplex with vertices v_p > ... > v_0 has combinatorial index
 *    cidx = sum_i C(v_i, i+1) (eq. 5.6).
 *  - threshold = +INFINITY means "no threshold": the filtration is truncated
 *    at the enclosing radius R = min_x max_y d(x,y) (Sec. 5.2.12,
 *    Prop 5.2.13), which changes no pair of nonzero persistence.  A finite
 *    threshold keeps the simplices with diam <= threshold (eq. 5.3).
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; host data is copied in on `stream`.  The
 *    library never frees caller memory.  Results are library-allocated host
 *    memory, released with the matching *_free call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    are synchronous with respect to the host: they return after the
 *    results are on the host.
 *  - On error nothing is written to *out (it is set to NULL) and the call
 *    returns a nonzero vr_status; vr_status_string() names it.
 *  - No kernel of the library waits on another thread block: the rounds of
 *    the reduction synchronise at kernel boundaries on the host, so there is
 *    no device-side wait to time out.  VR_ERR_TIMEOUT is reserved and is not
 *    returned by any entry point.
 */
#ifndef VR_H
#define VR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VR_MAX_DIM 6 /* highest homology dimension dmax accepted */

typedef enum {
    VR_OK = 0,
    VR_ERR_INVALID_ARG = 1,     /* bad size, NaN/negative/asymmetric distances, dmax out of range */
    VR_ERR_OOM = 2,             /* a device or host allocation failed                              */
    VR_ERR_INDEX_OVERFLOW = 3,  /* C(n, dmax+2) or a packed sort key does not fit 64 bits           */
    VR_ERR_CUDA = 4,            /* a CUDA runtime call failed (no device, launch failure, ...)      */
    VR_ERR_TIMEOUT = 5,         /* reserved: no entry point returns it (no device-side waits)       */
    VR_ERR_INTERNAL = 6         /* an internal consistency check failed                             */
} vr_status;

/* flags */
#define VR_KEEP_ZERO_LENGTH 0x1u /* also report pairs with death == birth                     */
#define VR_CRITICAL_EDGES   0x2u /* fill vr_result.critical_edges (needed by vr_backward)     */
#define VR_DEBUG_CHECKS     0x4u /* check identities every correct result satisfies before
                                    returning (Obs 3.2.14 counts per dimension: each simplex
                                    within the threshold is a birth or a death; cleared
                                    columns = death simplices one dimension down; birth <=
                                    death; documented pair order); a violation returns
                                    VR_ERR_INTERNAL.  Host-side, after the computation.     */
#define VR_APPARENT_ONLY    0x8u /* top dimension dmax: stop after filtration with clearing and
                                    the apparent-pair search (the quantity of the apparent-
                                    fraction experiment, Sec. 5.6.6): stats[dmax] is filled up
                                    to `reduced` (its non-apparent columns, not reduced),
                                    stats[dmax].pairs counts the apparent pairs, and no pairs
                                    of dimension dmax are returned (count[dmax] = 0).
                                    Dimensions below dmax are computed in full.              */
/* Reduction of the non-apparent columns (Sec. 5.2.9; at most one of the two;
 * the pairs are the same in every mode, only work and memory differ):
 *  default              a column finished with additions keeps its reduced
 *                       column R_j: as its generators (column j of V) when it
 *                       finished in the warp engine, explicitly (sorted front
 *                       and unsorted back) when it finished in the block engine;
 *  VR_REDUCE_V          every such column keeps only V_j, its generators, and a
 *                       later column that adds R_j regenerates sum of D_g
 *                       (the reduction-matrix technique);
 *  VR_REDUCE_OBLIVIOUS  nothing is kept: a pivot owned by column o adds D_o
 *                       (Algorithm 12 as printed, Lemma 5.2.10).               */
#define VR_REDUCE_V         0x10u
#define VR_REDUCE_OBLIVIOUS 0x20u
/* Sparse (low-threshold) mode (Sec. 5.3.12-5.3.13, Algorithm 15; warp-based
 * filtering, Sec. 5.5.3; capacity-driven allocation, Sec. 5.7.2): the
 * simplices within the threshold are listed from the neighbour lists of the
 * threshold graph, dimension by dimension, instead of enumerating all
 * C(n, p+1) indices, and the apparent cofacet of a simplex is searched among
 * the neighbours of its vertex of least degree.  The same pairs as without
 * it; memory and time follow the size of the complex.  In this mode
 * stats[p].candidates counts the listed p-simplices (above_threshold = 0).
 * Meant for thresholds far below the enclosing radius.                        */
#define VR_SPARSE           0x40u

/* One persistence pair of dimension p.  birth = diam(birth simplex),
 * death = diam(death simplex) or +INFINITY for an essential class. */
typedef struct {
    float birth;
    float death;
    uint64_t birth_simplex; /* cidx of the birth p-simplex                         */
    int64_t death_simplex;  /* cidx of the death (p+1)-simplex, -1 if essential    */
} vr_pair;

/* Per-dimension counters (Tables 5.1, 5.4, 5.5 of the paper report the same
 * quantities).  For p = 0 only `candidates` (= n), `pairs`, `essential` and
 * `emitted` are filled. */
typedef struct {
    int64_t candidates;  /* p-simplices enumerated, C(n, p+1)                            */
    int64_t above_threshold; /* candidates with diam > threshold                         */
    int64_t cleared;     /* candidates dropped by the clearing lemma                      */
    int64_t columns;     /* columns of the coboundary matrix after threshold and clearing */
    int64_t apparent;    /* apparent pairs found by the Apparent Pairs Lemma              */
    int64_t reduced;     /* non-apparent columns passed to the Z/2 reduction              */
    int64_t additions;   /* column additions performed by the reduction                   */
    int64_t pairs;       /* persistence pairs of dimension p, zero-length included        */
    int64_t essential;   /* classes that never die                                        */
    int64_t emitted;     /* entries written to vr_result.pairs[p]                          */
    int64_t cofacets_scanned; /* cofacets examined by the apparent-pair search                 */
    int64_t lookups;     /* diameter-rank entries read by the fused filtration/apparent kernel */
    float ms_filtration; /* CUDA-event time of the fused filtration/clearing/apparent kernel
                            (p = 0: diameter ranks and enclosing radius)                      */
    float ms_sort;       /* radix sort of the non-apparent columns (p >= 1)                   */
    float ms_reduce;     /* Z/2 reduction (p = 0: spanning tree and elder rule)               */
} vr_stats;

typedef struct {
    int32_t dmax;                       /* homology dimensions 0..dmax are reported            */
    int64_t n;                          /* number of points                                    */
    float threshold;                    /* threshold actually used (R when none was given)     */
    int64_t count[VR_MAX_DIM + 1];      /* pairs per dimension                                 */
    vr_pair* pairs[VR_MAX_DIM + 1];     /* sorted by (birth, death, birth_simplex)             */
    int32_t* critical_edges[VR_MAX_DIM + 1]; /* if VR_CRITICAL_EDGES: 4 per pair,
                                           (u_b, v_b, u_d, v_d) with u > v the edge attaining the
                                           birth / death diameter (ties: largest C(u,2)+v);
                                           u_d = v_d = -1 for essential pairs; else NULL        */
    vr_stats stats[VR_MAX_DIM + 1];
} vr_result;

/* Barcodes of a point cloud.
 *  pts        float[n][ambient_dim], row-major, host or device.
 *  n          number of points, 1 <= n <= 65536.  C(n, dmax+2) >= 2^63 returns
 *             VR_ERR_INDEX_OVERFLOW before any device work; so does a dimension
 *             whose packed keys (diameter rank above a simplex index, Sec. 5.5.2)
 *             would not fit 64 bits, checked once the distinct distances are
 *             ranked and before the first dimension is computed.
 *  ambient_dim 1..1024.
 *  dmax       0..VR_MAX_DIM.
 *  threshold  see above; must not be NaN.  threshold < 0 gives an empty result.
 *  flags      VR_* flags.
 *  out        receives a vr_result* on success.                              */
vr_status vr_barcodes_points(const float* pts, int64_t n, int32_t ambient_dim, int32_t dmax,
                             float threshold, uint32_t flags, void* stream, vr_result** out);

/* Barcodes of a distance matrix given as its condensed lower triangle:
 * entry (i,j), i > j, at index i(i-1)/2 + j, n(n-1)/2 floats, host or device.
 * Entries must be finite and >= 0 (VR_ERR_INVALID_ARG otherwise).          */
vr_status vr_barcodes_dists(const float* lower_tri, int64_t n, int32_t dmax, float threshold,
                            uint32_t flags, void* stream, vr_result** out);

void vr_result_free(vr_result* r);

/* Device-resident variants (for callers that keep the pairs on the GPU, such
 * as the torch autograd path): the same computation and the same pairs, in
 * the same order, but pairs[p] and critical_edges[p] are DEVICE pointers on
 * the call's device, allocated by the library in stream order on `stream`
 * (cudaMallocAsync) and released by vr_device_result_free in that stream's
 * order (cudaFreeAsync; the stream must still exist then, and work queued on
 * it before the free may still read the arrays); counts, stats and the
 * threshold are on the host.  The arrays are complete when the call returns.
 * The pairs are ordered and filtered on the device; nothing but counts goes
 * to the host.  Arguments and errors as vr_barcodes_points / _dists. */
typedef struct {
    int32_t dmax;
    int64_t n;
    float threshold;
    int64_t count[VR_MAX_DIM + 1];
    vr_pair* pairs[VR_MAX_DIM + 1];            /* device, count[p] entries (at least one allocated) */
    int32_t* critical_edges[VR_MAX_DIM + 1];   /* device, 4 per pair, if VR_CRITICAL_EDGES; else NULL */
    vr_stats stats[VR_MAX_DIM + 1];
    void* stream;                              /* the call's stream (used by the free) */
} vr_device_result;

vr_status vr_barcodes_points_device(const float* pts, int64_t n, int32_t ambient_dim, int32_t dmax,
                                    float threshold, uint32_t flags, void* stream, vr_device_result** out);
vr_status vr_barcodes_dists_device(const float* lower_tri, int64_t n, int32_t dmax, float threshold,
                                   uint32_t flags, void* stream, vr_device_result** out);
void vr_device_result_free(vr_device_result* r);

/* Batched barcodes of many independent clouds (the batched form: one
 * persistent launch over a work queue of clouds).
 *  pts        float[sum n_i][ambient_dim], clouds stored back to back, host or device.
 *  offsets    int64[num_clouds+1], cloud i is rows offsets[i] .. offsets[i+1]-1 (host).
 *  Each cloud must have 1 <= n_i <= VR_BATCH_MAX_N points and dmax must be 0 or 1.
 *  Results: for cloud i, its pairs of dimension p are
 *  pairs[p][pair_offsets[p][i] .. pair_offsets[p][i+1]-1], sorted as above.  */
#define VR_BATCH_MAX_N 256
typedef struct {
    int32_t num_clouds;
    int32_t dmax;
    int64_t* pair_offsets[2];           /* int64[num_clouds+1] per dimension            */
    vr_pair* pairs[2];
    int32_t* critical_edges[2];         /* 4 per pair if VR_CRITICAL_EDGES, else NULL;
                                           rows of the packed `pts` array (not cloud-local) */
    float* thresholds;                  /* float[num_clouds]: threshold used per cloud  */
    int32_t recomputed;                 /* clouds that outgrew a per-block buffer of the
                                           persistent launch and were computed by the
                                           single-cloud path instead (same results)     */
} vr_batch_result;

vr_status vr_barcodes_batched(const float* pts, const int64_t* offsets, int32_t num_clouds,
                              int32_t ambient_dim, int32_t dmax, float threshold, uint32_t flags,
                              void* stream, vr_batch_result** out);
void vr_batch_result_free(vr_batch_result* r);

/* Device-resident variant of vr_barcodes_batched: the same pairs in the same
 * order; pairs[p] and critical_edges[p] are device pointers (allocated and,
 * by vr_batch_device_result_free, released in the order of `stream`, as for
 * vr_device_result), pair_offsets and thresholds host arrays.  The device
 * arrays are written in the order of `stream` and the call returns without
 * waiting for those copies: read them on `stream`, or after an event or
 * synchronization on it. */
typedef struct {
    int32_t num_clouds;
    int32_t dmax;
    int64_t* pair_offsets[2];           /* host, int64[num_clouds+1] per dimension        */
    vr_pair* pairs[2];                  /* device                                          */
    int32_t* critical_edges[2];         /* device, 4 per pair if VR_CRITICAL_EDGES, else NULL */
    float* thresholds;                  /* host, float[num_clouds]                          */
    void* stream;                       /* the call's stream (used by the free)             */
    int32_t recomputed;                 /* as in vr_batch_result                            */
} vr_batch_device_result;

vr_status vr_barcodes_batched_device(const float* pts, const int64_t* offsets, int32_t num_clouds,
                                     int32_t ambient_dim, int32_t dmax, float threshold, uint32_t flags,
                                     void* stream, vr_batch_device_result** out);
void vr_batch_device_result_free(vr_batch_device_result* r);

/* Backward pass: d loss / d pts given d loss / d (birth, death) of the pairs
 * of a forward result computed with VR_CRITICAL_EDGES.  Each finite value is
 * the length of its critical edge (u, v), so it contributes
 * g * (x_u - x_v) / |x_u - x_v| to point u and the negative to point v.
 *  pts        float[n][ambient_dim], device pointer.
 *  edges      int32[num][4] (u_b, v_b, u_d, v_d), device pointer (-1 = no edge).
 *  grad_birth, grad_death  float[num], device pointers.
 *  grad_pts   float[n][ambient_dim], device pointer, accumulated into (+=).
 * An edge endpoint outside 0..n-1 (other than -1) returns VR_ERR_INVALID_ARG;
 * that edge contributes nothing, the valid edges still accumulate.
 * The forward result is passed as its critical-edge array (not as the
 * vr_result) so that edges kept on the device by the torch path, and the
 * packed edges of a batched result, use this same entry point.           */
vr_status vr_backward(const float* pts, int64_t n, int32_t ambient_dim, const int32_t* edges,
                      int64_t num, const float* grad_birth, const float* grad_death,
                      float* grad_pts, void* stream);

/* Vertices of the q-simplex with combinatorial index cidx among n points,
 * written in ascending order to out_vertices[0..q].  Host-only arithmetic. */
vr_status vr_simplex_vertices(uint64_t cidx, int32_t q, int64_t n, int32_t* out_vertices);

const char* vr_status_string(vr_status s);

/* ------------------------------------------------------------------------
 * Stage entry points, exposed so each step can be checked on its own.
 * All pointers are device pointers; all run on `stream` and synchronise it.
 * ---------------------------------------------------------------------- */

/* Distance step: condensed lower triangle of the single-precision formula. */
vr_status vr_distances(const float* pts, int64_t n, int32_t ambient_dim, float* out_lower_tri,
                       void* stream);

/* Radix sort of num 64-bit keys in place by their low `bits` bits (ascending,
 * stable), values (may be NULL) permuted alongside.                          */
vr_status vr_sort_u64(uint64_t* keys, uint64_t* values, int64_t num, int32_t bits, void* stream);

/* Allocation-free variant of vr_sort_u64.  The paper has no counterpart: it
 * exists for callers that must not allocate device memory during the call --
 * code running under a fixed, pre-reserved device-memory budget (a serving
 * process that partitions the GPU up front, a host whose allocator must not
 * be re-entered from a library).  It sorts the same way as vr_sort_u64 (same
 * kernels, same results) but takes its scratch from a static device array
 * that every GPU loading the library keeps until the process exits.
 *  num        at most VR_SORT_NOALLOC_MAX_KEYS; larger sizes return
 *             VR_ERR_INVALID_ARG and touch nothing.
 *  keys, values  device pointers, as in vr_sort_u64 (values may be NULL).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array: calls whose
 * work overlaps on the GPU (several streams or host threads) race and must be
 * serialised by the caller.  Every call synchronises `stream` before it
 * returns (the sort is finished on return), so no call of it may be made
 * while `stream` is being captured into a CUDA graph.                       */
/* Persistence pairs of an explicit boundary matrix: HYPHA (Ch. 4, Algorithm
 * 10) -- the GPU scan for leftmost entries and 0-addition columns
 * (Algorithms 3-6), clearing (Algorithm 7, Lemma 4.2.3), compression
 * (Algorithms 8-9, Lemmas 4.2.4-4.2.5), then the standard reduction
 * (Algorithm 2) of the columns that remain, all on the device.
 *  colptr   int64[ncols+1], rows int32[nnz]: the Z/2 boundary matrix of a
 *           filtered simplicial complex in CSC form, columns (and rows) in
 *           filtration order, the rows of each column ascending and below
 *           the column (faces come first); host or device memory.
 *           Clearing and compression rely on it being a boundary matrix.
 *  flags    must be 0.
 *  out_low  int32[ncols], host or device: the pivot row of each column of
 *           the fully reduced matrix (low(R_j)), -1 for a zero column; the
 *           pairs (low(R_j), j) are the persistence pairs (Thm 3.2.20).
 *  stats    may be NULL.
 * A malformed matrix (rows out of order, a row not below its column)
 * returns VR_ERR_INVALID_ARG.                                              */
typedef struct {
    int64_t columns;
    int64_t unstable;               /* columns neither stable (0-addition) nor cleared     */
    int64_t compression_passes;     /* fixed-point passes of the compressible-row search   */
    int64_t compression_additions;  /* stable columns added during compression            */
    int64_t additions;              /* column additions of the final reduction             */
    float ms_scan;                  /* GPU scan and clearing                               */
    float ms_compression;
    float ms_reduce;
} vr_hypha_stats;
vr_status vr_hypha_pairs(const int64_t* colptr, const int32_t* rows, int64_t ncols, int64_t nnz, uint32_t flags,
                         void* stream, int32_t* out_low, vr_hypha_stats* stats);

/* Read-bandwidth probe for the roofline denominators (the paper has no
 * counterpart).  Streams a zeroed device buffer of `bytes` bytes `iters`
 * times with 16-byte loads that bypass L1, on `stream`, and writes the read
 * bandwidth in GB/s (10^9 bytes per second, CUDA-event timed, after one
 * untimed pass) to *out_gbs.  A buffer well inside the 126 MB L2 measures
 * L2 read bandwidth; one far larger measures HBM read bandwidth.  The buffer
 * is allocated and freed on `stream`; nothing else is touched.
 *  bytes      2^20 .. 2^36;  iters 1 .. 100000.                             */
vr_status vr_probe_read_gbs(int64_t bytes, int32_t iters, void* stream, double* out_gbs);

#define VR_SORT_NOALLOC_MAX_KEYS (1 << 18)
vr_status vr_sort_u64_noalloc(uint64_t* keys, uint64_t* values, int64_t num, int32_t bits, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VR_H */
