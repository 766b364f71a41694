// radix_sort.cu -- least-significant-digit radix sort on packed integer keys.
//
// The filtration must be put in coboundary order, decreasing diameter then
// increasing combinatorial index (Algorithm 18, Sec. 5.5.2 of the paper);
// the keys packed by the callers make that order the ascending order of an
// unsigned integer, and only the significant low bits are sorted.
//
// Up to 4096 keys: one block, a bitonic network on (key, index) pairs in
// shared memory (k_small_sort), the same stable order in one launch; up to
// 32768: chunks of 4096 so sorted, then each key placed by searching the
// other chunks (two launches).
// Otherwise one pass per 8-bit digit, three kernels per pass, no inter-block waits:
//   1. k_hist    per-tile digit histogram, stored digit-major
//   2. k_scan    exclusive scan of the (digit, tile) counts in one block
//   3. k_scatter stable scatter: a tile is walked in index order, ranks of
//                equal digits inside a warp come from __match_any_sync, the
//                offsets of earlier warps and rounds from shared counters.
#include <mutex>

#include "vr_common.cuh"

namespace vr {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                       // items per thread
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;     // 4096 keys per tile
constexpr int RS_BINS = 256;

// The digit of a pass: 8 bits, fewer in the last pass when `bits` is not a
// multiple of 8 (the bits above `bits` take no part in the order).
inline uint32_t digit_mask(int bits, int shift) {
    return bits - shift >= 8 ? 0xFFu : ((1u << (bits - shift)) - 1u);
}

template <class K>
__global__ void k_hist(const K* __restrict__ keys, int64_t num, int shift, uint32_t dmask, uint32_t* __restrict__ hist,
                       int64_t tiles) {
    __shared__ uint32_t bins[RS_BINS];
    for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) bins[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t idx = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (idx < num) atomicAdd(&bins[(uint32_t)(keys[idx] >> shift) & dmask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) hist[(int64_t)b * tiles + blockIdx.x] = bins[b];
}

// Exclusive scan of cnt[0..len) in place, one block of 1024 threads.
__global__ void k_scan(uint32_t* __restrict__ cnt, int64_t len) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < len; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        uint32_t x = idx < len ? cnt[idx] : 0;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            uint32_t ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += y;
            }
            warp_tot[lane] = ti - t;  // exclusive over warps
        }
        __syncthreads();
        uint32_t c0 = carry;
        if (idx < len) cnt[idx] = c0 + warp_tot[wid] + incl - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_tot[wid] + incl;
        __syncthreads();
    }
}

template <class K, class V, bool HAS_V>
__global__ void k_scatter(const K* __restrict__ kin, const V* __restrict__ vin, K* __restrict__ kout,
                          V* __restrict__ vout, int64_t num, int shift, uint32_t dmask,
                          const uint32_t* __restrict__ offs,
                          int64_t tiles) {
    __shared__ uint32_t base_off[RS_BINS];         // global start of each digit for this tile
    __shared__ uint32_t running[RS_BINS];          // items of each digit already placed
    __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];   // this round: items per warp and digit
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) {
        base_off[b] = offs[(int64_t)b * tiles + blockIdx.x];
        running[b] = 0;
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][b] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t idx = base + (int64_t)r * RS_THREADS + threadIdx.x;
        bool valid = idx < num;
        K key = valid ? kin[idx] : (K)0;
        V val = (HAS_V && valid) ? vin[idx] : (V)0;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & dmask) : (uint32_t)(RS_BINS + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t lrank = __popc(peers & lt_mask);
        if (valid && lrank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x) {
            uint32_t acc = running[b];
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = wcnt[w][b];
                wcnt[w][b] = acc;  // becomes the warp's offset for this round
                acc += c;
            }
            running[b] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = base_off[d] + wcnt[wid][d] + lrank;
            kout[pos] = key;
            if (HAS_V) vout[pos] = val;
        }
        __syncthreads();
        for (int b = threadIdx.x; b < RS_BINS; b += blockDim.x)
            for (int w = 0; w < RS_WARPS; ++w) wcnt[w][b] = 0;
        __syncthreads();
    }
}

// Up to SMALL_MAX keys: one block sorts (masked key, input index) pairs in
// shared memory with a bitonic network -- the index breaks ties, so the order
// is the stable one the radix passes give -- and the values follow through
// the indices.  One launch instead of three per 8-bit digit.
constexpr int SMALL_MAX = 4096;  // larger inputs: the radix passes were faster (measured at 11K and 16K keys)
constexpr int SMALL_THREADS = 1024;

template <class K, class V, bool HAS_V>
__global__ void __launch_bounds__(SMALL_THREADS)
k_small_sort(K* __restrict__ keys, V* __restrict__ vals, int num, int len, K mask) {
    extern __shared__ __align__(16) unsigned char sm[];
    K* a = reinterpret_cast<K*>(sm);
    uint32_t* ix = reinterpret_cast<uint32_t*>(a + len);
    for (int i = threadIdx.x; i < len; i += SMALL_THREADS) {
        a[i] = i < num ? keys[i] : ~(K)0;  // padding sorts last: its indices are the largest
        ix[i] = (uint32_t)i;
    }
    __syncthreads();
    const int half = len >> 1;
    for (int k = 2; k <= len; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < half; p += SMALL_THREADS) {
                const int i = 2 * p - (p & (j - 1));
                const K x = a[i], y = a[i + j];
                const uint32_t xi = ix[i], yi = ix[i + j];
                const K xm = xi < (uint32_t)num ? (x & mask) : ~(K)0;
                const K ym = yi < (uint32_t)num ? (y & mask) : ~(K)0;
                const bool gt = xm > ym || (xm == ym && xi > yi);
                if (gt == ((i & k) == 0)) {
                    a[i] = y; a[i + j] = x;
                    ix[i] = yi; ix[i + j] = xi;
                }
            }
            __syncthreads();
        }
    V v[SMALL_MAX / SMALL_THREADS];
    if (HAS_V) {
#pragma unroll
        for (int r = 0; r < SMALL_MAX / SMALL_THREADS; ++r) {
            const int i = r * SMALL_THREADS + threadIdx.x;
            if (i < num) v[r] = vals[ix[i]];
        }
    }
    __syncthreads();  // every value is read before any is written
    for (int i = threadIdx.x; i < num; i += SMALL_THREADS) keys[i] = a[i];
    if (HAS_V) {
#pragma unroll
        for (int r = 0; r < SMALL_MAX / SMALL_THREADS; ++r) {
            const int i = r * SMALL_THREADS + threadIdx.x;
            if (i < num) vals[i] = v[r];
        }
    }
}

// Up to CHUNKED_MAX keys: chunks of SMALL_MAX are sorted by one block each
// (same order as k_small_sort: masked key, then input index), then every key
// finds its place by searching the other chunks -- two launches.
constexpr int CHUNKED_MAX = 8 * SMALL_MAX;

template <class K>
__global__ void __launch_bounds__(SMALL_THREADS)
k_chunk_sort(const K* __restrict__ keys, int num, K mask, K* __restrict__ ck, uint32_t* __restrict__ ci) {
    __shared__ K a[SMALL_MAX];
    __shared__ uint32_t ix[SMALL_MAX];
    const int base = blockIdx.x * SMALL_MAX;
    const int cnt = min(SMALL_MAX, num - base);
    for (int i = threadIdx.x; i < SMALL_MAX; i += SMALL_THREADS) {
        a[i] = i < cnt ? (keys[base + i] & mask) : ~(K)0;
        ix[i] = (uint32_t)(base + i);  // padding: indices past num, sorted last
    }
    __syncthreads();
    constexpr int half = SMALL_MAX >> 1;
    for (int k = 2; k <= SMALL_MAX; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < half; p += SMALL_THREADS) {
                const int i = 2 * p - (p & (j - 1));
                const K x = a[i], y = a[i + j];
                const uint32_t xi = ix[i], yi = ix[i + j];
                const bool gt = x > y || (x == y && xi > yi);
                if (gt == ((i & k) == 0)) {
                    a[i] = y; a[i + j] = x;
                    ix[i] = yi; ix[i + j] = xi;
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < cnt; i += SMALL_THREADS) {
        ck[base + i] = a[i];
        ci[base + i] = ix[i];
    }
}

// Key t of chunk c (rank r in it) goes to r plus the keys of the other chunks
// before it in (masked key, index) order.
template <class K, class V, bool HAS_V>
__global__ void k_chunk_place(const K* __restrict__ keys, const V* __restrict__ vals, int num,
                              const K* __restrict__ ck, const uint32_t* __restrict__ ci, K* __restrict__ kout,
                              V* __restrict__ vout) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= num) return;
    const int c = t / SMALL_MAX, r = t % SMALL_MAX;
    const K x = ck[t];
    const uint32_t xi = ci[t];
    const int nch = (num + SMALL_MAX - 1) / SMALL_MAX;
    int pos = r;
    for (int c2 = 0; c2 < nch; ++c2) {
        if (c2 == c) continue;
        const int b = c2 * SMALL_MAX, n2 = min(SMALL_MAX, num - b);
        int q = 0;  // keys of chunk c2 before (x, xi), by fixed steps
        for (int st = 1 << (31 - __clz(n2)); st > 0; st >>= 1) {
            const int u = q + st;
            if (u <= n2) {
                const K y = ck[b + u - 1];
                if (y < x || (y == x && ci[b + u - 1] < xi)) q = u;
            }
        }
        pos += q;
    }
    kout[pos] = keys[xi];
    if (HAS_V) vout[pos] = vals[xi];
}

template <class K, class V, bool HAS_V>
void radix_sort_impl(Workspace& ws, K* keys, V* vals, int64_t num, int bits) {
    if (num <= 1 || bits <= 0) return;
    VR_CHECK(num < (int64_t)UINT32_MAX, VR_ERR_INVALID_ARG);
    if (num <= SMALL_MAX) {
        int len = 1;
        while (len < num) len <<= 1;
        const size_t smem = (size_t)len * (sizeof(K) + sizeof(uint32_t));
        const K mask = bits >= (int)(8 * sizeof(K)) ? ~(K)0 : (K)((((K)1) << bits) - 1);
        VR_CUDA(cudaFuncSetAttribute(k_small_sort<K, V, HAS_V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(SMALL_MAX * (sizeof(K) + sizeof(uint32_t)))));
        k_small_sort<K, V, HAS_V><<<1, SMALL_THREADS, smem, ws.stream>>>(keys, vals, (int)num, len, mask);
        VR_CUDA(cudaGetLastError());
        return;
    }
    if (num <= CHUNKED_MAX) {
        const K mask = bits >= (int)(8 * sizeof(K)) ? ~(K)0 : (K)((((K)1) << bits) - 1);
        const int nch = (int)((num + SMALL_MAX - 1) / SMALL_MAX);
        K* ck = ws.alloc_n<K>(num);
        uint32_t* ci = ws.alloc_n<uint32_t>(num);
        K* kout = ws.alloc_n<K>(num);
        V* vout = HAS_V ? ws.alloc_n<V>(num) : nullptr;
        k_chunk_sort<K><<<nch, SMALL_THREADS, 0, ws.stream>>>(keys, (int)num, mask, ck, ci);
        k_chunk_place<K, V, HAS_V><<<(unsigned)((num + 255) / 256), 256, 0, ws.stream>>>(keys, vals, (int)num, ck, ci,
                                                                                          kout, vout);
        VR_CUDA(cudaGetLastError());
        VR_CUDA(cudaMemcpyAsync(keys, kout, num * sizeof(K), cudaMemcpyDeviceToDevice, ws.stream));
        if (HAS_V) VR_CUDA(cudaMemcpyAsync(vals, vout, num * sizeof(V), cudaMemcpyDeviceToDevice, ws.stream));
        return;
    }
    const int64_t tiles = (num + RS_TILE - 1) / RS_TILE;
    K* kalt = ws.alloc_n<K>(num);
    V* valt = HAS_V ? ws.alloc_n<V>(num) : nullptr;
    uint32_t* hist = ws.alloc_n<uint32_t>(tiles * RS_BINS);
    K* kin = keys; K* kout = kalt;
    V* vin = vals; V* vout = valt;
    const int passes = (bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = ps * 8;
        const uint32_t dmask = digit_mask(bits, shift);
        k_hist<K><<<(unsigned)tiles, RS_THREADS, 0, ws.stream>>>(kin, num, shift, dmask, hist, tiles);
        k_scan<<<1, 1024, 0, ws.stream>>>(hist, tiles * RS_BINS);
        k_scatter<K, V, HAS_V><<<(unsigned)tiles, RS_THREADS, 0, ws.stream>>>(kin, vin, kout, vout, num, shift,
                                                                               dmask, hist, tiles);
        VR_CUDA(cudaGetLastError());
        K* tk = kin; kin = kout; kout = tk;
        V* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys) {
        VR_CUDA(cudaMemcpyAsync(keys, kin, num * sizeof(K), cudaMemcpyDeviceToDevice, ws.stream));
        if (HAS_V) VR_CUDA(cudaMemcpyAsync(vals, vin, num * sizeof(V), cudaMemcpyDeviceToDevice, ws.stream));
    }
}

}  // namespace

void radix_sort_u64(Workspace& ws, uint64_t* keys, uint64_t* vals, int64_t num, int bits) {
    if (vals) radix_sort_impl<uint64_t, uint64_t, true>(ws, keys, vals, num, bits);
    else radix_sort_impl<uint64_t, uint64_t, false>(ws, keys, nullptr, num, bits);
}

void scan_u32_exclusive(uint32_t* data, int64_t num, cudaStream_t s) {
    if (num <= 0) return;
    k_scan<<<1, 1024, 0, s>>>(data, num);
    VR_CUDA(cudaGetLastError());
}

void radix_sort_u32(Workspace& ws, uint32_t* keys, uint32_t* vals, int64_t num, int bits) {
    if (vals) radix_sort_impl<uint32_t, uint32_t, true>(ws, keys, vals, num, bits);
    else radix_sort_impl<uint32_t, uint32_t, false>(ws, keys, nullptr, num, bits);
}

}  // namespace vr

// ---------------------------------------------------------------------------
// Allocation-free variant of the sort (vr_sort_u64_noalloc).
//
// For callers that cannot allocate device memory while they run -- code
// working inside a fixed, pre-reserved device-memory budget (a serving
// process that partitions the GPU up front, a host application whose
// allocator must not be re-entered from a library call) -- the ping-pong
// key/value buffers and the digit histogram come from this file-scope
// device array instead of cudaMallocAsync.  Every GPU that loads the library
// holds the array until the process exits.  Host code cannot use the array's
// name as a device address: the address is fetched with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on it.
// All calls share the array, so calls whose work overlaps on the GPU (other
// streams, other host threads) race and must be serialised by the caller.
// Nothing in it needs to start at zero: every pass rewrites the histogram
// and both buffers before reading them.
// ---------------------------------------------------------------------------
namespace vr {
namespace {

constexpr int64_t NOALLOC_MAX_KEYS = (int64_t)1 << 18;  // 262,144 keys: about 4.3 MB of scratch
constexpr int64_t NOALLOC_TILES = (NOALLOC_MAX_KEYS + RS_TILE - 1) / RS_TILE;

struct NoAllocScratch {
    uint64_t keys[NOALLOC_MAX_KEYS];
    uint64_t vals[NOALLOC_MAX_KEYS];
    uint32_t hist[NOALLOC_TILES * RS_BINS];
};

static __device__ __align__(256) NoAllocScratch g_sort_scratch;

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
NoAllocScratch* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_sort_scratch on the current device (set-up on first use).
NoAllocScratch* noalloc_scratch() {
    int dev = 0;
    VR_CUDA(cudaGetDevice(&dev));
    VR_CHECK(dev >= 0 && dev < NOALLOC_MAX_DEVICES, VR_ERR_CUDA);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        VR_CUDA(cudaGetSymbolAddress(&p, g_sort_scratch));
        g_noalloc_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    return g_noalloc_addr[dev];
}

template <bool HAS_V>
void sort_passes_noalloc(NoAllocScratch* sc, uint64_t* keys, uint64_t* vals, int64_t num, int bits,
                         cudaStream_t s) {
    const int64_t tiles = (num + RS_TILE - 1) / RS_TILE;
    uint64_t* kin = keys; uint64_t* kout = sc->keys;
    uint64_t* vin = vals; uint64_t* vout = sc->vals;
    const int passes = (bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = ps * 8;
        const uint32_t dmask = digit_mask(bits, shift);
        k_hist<uint64_t><<<(unsigned)tiles, RS_THREADS, 0, s>>>(kin, num, shift, dmask, sc->hist, tiles);
        k_scan<<<1, 1024, 0, s>>>(sc->hist, tiles * RS_BINS);
        k_scatter<uint64_t, uint64_t, HAS_V><<<(unsigned)tiles, RS_THREADS, 0, s>>>(kin, vin, kout, vout, num, shift,
                                                                                   dmask, sc->hist, tiles);
        VR_CUDA(cudaGetLastError());
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint64_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys) {
        VR_CUDA(cudaMemcpyAsync(keys, kin, num * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (HAS_V) VR_CUDA(cudaMemcpyAsync(vals, vin, num * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace

}  // namespace vr

extern "C" vr_status vr_sort_u64_noalloc(uint64_t* keys, uint64_t* values, int64_t num, int32_t bits, void* stream) {
    if (num < 0 || bits < 0 || bits > 64 || (num > 0 && !keys)) return VR_ERR_INVALID_ARG;
    if (num > vr::NOALLOC_MAX_KEYS) return VR_ERR_INVALID_ARG;  // larger than the static scratch
    try {
        cudaStream_t s = (cudaStream_t)stream;
        if (num > 1 && bits > 0) {
            vr::NoAllocScratch* sc = vr::noalloc_scratch();
            if (values) vr::sort_passes_noalloc<true>(sc, keys, values, num, bits, s);
            else vr::sort_passes_noalloc<false>(sc, keys, nullptr, num, bits, s);
        }
        VR_CUDA(cudaStreamSynchronize(s));
        return VR_OK;
    } catch (const vr::Error& e) {
        return e.code;
    }
}
