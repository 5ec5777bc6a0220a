// Sketch construction on the GPU.
//
//  * oph_build_sketches: OPH / HOPH sketches (Sec. 3.2, Sec. 4.1).  One warp
//    owns one set.  Sets are visited in descending size order (a counting
//    sort by size bucket builds the work list) and striped across all
//    resident warps of one persistent launch.  IDs are read with 128-bit
//    loads; each ID is mapped through the packed psi table (psi value ->
//    bin and offset) that stays resident in L2, and the per-bin minimum is
//    kept in the warp's shared-memory sketch with a read-then-atomicMin.
//    The finished sketch is written group-major ([G][n][k']) with coalesced
//    stores.
//  * minwise_build_sketches: MinWise (Sec. 1), one warp per set, lane t
//    owning the minima of permutations t, t+32, ...; the k permuted values
//    of an ID are contiguous ([D][k] table) so each gather is coalesced.
//  * hoph_synth_ids: counter-based synthetic IDs (benchmark inputs).
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kSketchThreads = 256;
constexpr int kSketchWarps = kSketchThreads / 32;
constexpr int kBuckets = 65;

struct SketchArgs {
    const uint32_t *ids;
    const int64_t *off;
    int64_t n_sets;
    uint32_t *planes;
    int64_t plane_stride;  // n_sets * k'
    uint32_t k, kg;
    const uint32_t *key;   // packed psi table (table path)
    uint32_t key_bits;
    uint64_t D;
    const uint64_t *lo;    // bin bounds (hash path)
    uint64_t ha, hb;
    const int32_t *order;  // size-sorted set indices, or nullptr for 0..n-1
    int32_t *status;
};

// psi(x) = ((a x + b) mod (2^61 - 1)) >> 29 with a Mersenne-prime reduction:
// a x = hi 2^64 + lo == 8 hi + (lo >> 61) + (lo & p)  (mod p).
__device__ __forceinline__ uint32_t hash61(uint64_t x, uint64_t a, uint64_t b) {
    const uint64_t p = (1ull << 61) - 1;
    const uint64_t lo = a * x;
    const uint64_t hi = __umul64hi(a, x);
    uint64_t t = (hi << 3) + (lo >> 61) + (lo & p) + b;
    t = (t & p) + (t >> 61);
    if (t >= p) t -= p;
    return (uint32_t)(t >> 29);
}

template <bool HASH>
__global__ void __launch_bounds__(kSketchThreads) oph_sketch_kernel(const SketchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_lo = reinterpret_cast<uint64_t *>(smem_raw);  // HASH only
    uint32_t *s_sk = reinterpret_cast<uint32_t *>(smem_raw + (HASH ? (a.k + 1) * 8 : 0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *sk = s_sk + (size_t)warp * a.k;
    if (HASH)
        for (uint32_t i = threadIdx.x; i <= a.k; i += blockDim.x) s_lo[i] = a.lo[i];
    for (uint32_t i = lane; i < a.k; i += 32) sk[i] = HOPH_EMPTY_VALUE;
    __syncthreads();

    const uint32_t mask = a.key_bits >= 32 ? 0xFFFFFFFFu : ((1u << a.key_bits) - 1u);
    bool bad = false;
    auto take = [&](uint32_t x) {
        uint32_t bin, off;
        if (HASH) {
            const uint32_t v = hash61(x, a.ha, a.hb);
            uint32_t l = 0, h = a.k;  // lo[l] <= v < lo[h]
            while (h - l > 1) {
                const uint32_t m = (l + h) >> 1;
                if (s_lo[m] <= v) l = m; else h = m;
            }
            bin = l;
            off = (uint32_t)(v - s_lo[l]);
        } else {
            if (x >= a.D) {
                bad = true;
                return;
            }
            const uint32_t key = __ldg(a.key + x);
            bin = (uint32_t)((uint64_t)key >> a.key_bits);
            off = key & mask;
        }
        if (off < sk[bin]) atomicMin(sk + bin, off);
    };

    const int64_t warps_total = (int64_t)gridDim.x * kSketchWarps;
    for (int64_t item = (int64_t)blockIdx.x * kSketchWarps + warp; item < a.n_sets;
         item += warps_total) {
        const int64_t set = a.order ? a.order[item] : item;
        const int64_t beg = a.off[set], end = a.off[set + 1];
        const int64_t n = end - beg;
        const uint32_t *p = a.ids + beg;
        // scalar head up to a 16-byte boundary, 128-bit body, scalar tail
        const int64_t head = (int64_t)min((long long)n, (long long)((4 - ((reinterpret_cast<uintptr_t>(p) >> 2) & 3)) & 3));
        if (lane < head) take(p[lane]);
        const uint4 *p4 = reinterpret_cast<const uint4 *>(p + head);
        const int64_t nvec = (n - head) >> 2;
        int64_t i = lane;
        for (; i + 32 < nvec; i += 64) {
            const uint4 v0 = ldg_nc_v4(p4 + i);
            const uint4 v1 = ldg_nc_v4(p4 + i + 32);
            take(v0.x); take(v0.y); take(v0.z); take(v0.w);
            take(v1.x); take(v1.y); take(v1.z); take(v1.w);
        }
        if (i < nvec) {
            const uint4 v0 = ldg_nc_v4(p4 + i);
            take(v0.x); take(v0.y); take(v0.z); take(v0.w);
        }
        const int64_t tail0 = head + (nvec << 2);
        if (tail0 + lane < n) take(p[tail0 + lane]);
        __syncwarp();
        // group-major store: bin b -> plane b / k', position b % k'
        for (uint32_t b = lane; b < a.k; b += 32) {
            const uint32_t g = b / a.kg, j = b - g * a.kg;
            a.planes[(int64_t)g * a.plane_stride + set * a.kg + j] = sk[b];
            sk[b] = HOPH_EMPTY_VALUE;
        }
        __syncwarp();
    }
    if (bad) hoph_flag(a.status, HOPH_ERR_ID_RANGE);
}

// --- size-bucket work list: bucket = bit length of the set size ------------

__device__ __forceinline__ int size_bucket(int64_t n) { return n <= 0 ? 0 : 64 - __clzll(n); }

__global__ void bucket_hist_kernel(const int64_t *off, int64_t n, uint32_t *hist) {
    __shared__ uint32_t h[kBuckets];
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[size_bucket(off[i + 1] - off[i])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// exclusive prefix over buckets in descending size order (largest first)
__global__ void bucket_base_kernel(const uint32_t *hist, uint32_t *base) {
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            base[b] = run;
            run += hist[b];
        }
    }
}

__global__ void bucket_scatter_kernel(const int64_t *off, int64_t n, const uint32_t *base,
                                      uint32_t *cursor, int32_t *order) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = size_bucket(off[i + 1] - off[i]);
        order[base[b] + atomicAdd(&cursor[b], 1u)] = (int32_t)i;
    }
}

// --- MinWise -----------------------------------------------------------------

struct MinwiseArgs {
    const uint32_t *ids;
    const int64_t *off;
    int64_t n_sets;
    const uint32_t *tab;  // [D][mk]
    uint64_t D;
    uint32_t mk;
    uint32_t *out;        // [n_sets][mk]
    int32_t *status;
};

__global__ void __launch_bounds__(256) minwise_kernel(const MinwiseArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *m = reinterpret_cast<uint32_t *>(smem_raw) + (size_t)warp * a.mk;
    bool bad = false;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t set = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; set < a.n_sets;
         set += warps_total) {
        for (uint32_t t = lane; t < a.mk; t += 32) m[t] = HOPH_EMPTY_VALUE;
        const int64_t beg = a.off[set], end = a.off[set + 1];
        for (int64_t base = beg; base < end; base += 32) {
            const bool have = base + lane < end;
            const uint32_t x = have ? a.ids[base + lane] : 0u;
            const bool ok = have && x < a.D;
            if (have && !ok) bad = true;
            uint32_t okmask = __ballot_sync(0xFFFFFFFFu, ok);
            while (okmask) {
                const int j = __ffs(okmask) - 1;
                okmask &= okmask - 1;
                const uint32_t xj = __shfl_sync(0xFFFFFFFFu, x, j);
                const uint32_t *row = a.tab + (size_t)xj * a.mk;
                for (uint32_t t = lane; t < a.mk; t += 32) {
                    const uint32_t v = __ldg(row + t);
                    if (v < m[t]) m[t] = v;
                }
            }
        }
        for (uint32_t t = lane; t < a.mk; t += 32) a.out[set * a.mk + t] = m[t];
    }
    if (bad) hoph_flag(a.status, HOPH_ERR_ID_RANGE);
}

// --- synthetic IDs -----------------------------------------------------------

__global__ void synth_ids_kernel(uint64_t seed, int64_t first, int64_t n, uint64_t D,
                                 uint32_t kind, const double *cdf, int64_t n_cdf, uint32_t *out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(first + e + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        if (kind == 0) {
            out[e] = (uint32_t)(((z >> 32) * D) >> 32);
        } else {
            const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            int64_t l = 0, h = n_cdf;  // first i with u < cdf[i]
            while (l < h) {
                const int64_t m = (l + h) >> 1;
                if (cdf[m] > u) h = m; else l = m + 1;
            }
            out[e] = (uint32_t)l;
        }
    }
}

int grid_for(hoph_plan *pl, int per_sm) { return pl->num_sms * per_sm; }

}  // namespace

extern "C" {

int oph_build_sketches(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                       int64_t n_sets, uint32_t *d_planes, void *stream) {
    if (!plan || n_sets < 0 || (n_sets > 0 && (!d_offsets || !d_planes))) return HOPH_ERR_PARAM;
    if (n_sets >= (1ll << 31)) return HOPH_ERR_PARAM;
    if (n_sets == 0) return HOPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const hoph_params &P = plan->P;
    SketchArgs a;
    a.ids = d_ids;
    a.off = d_offsets;
    a.n_sets = n_sets;
    a.planes = d_planes;
    a.plane_stride = n_sets * (int64_t)P.k_group;
    a.k = P.k;
    a.kg = P.k_group;
    a.key = plan->d_key;
    a.key_bits = plan->key_bits;
    a.D = P.universe_D;
    a.lo = plan->d_lo;
    a.ha = plan->hash_a;
    a.hb = plan->hash_b;
    a.order = nullptr;
    a.status = plan->d_status;

    const bool hash = P.perm_kind == HOPH_PERM_HASH61;
    const size_t smem = (hash ? (P.k + 1) * 8 : 0) + (size_t)kSketchWarps * P.k * 4;
    int per_sm = 0;
    if (hash) {
        HOPH_CUDA_TRY(cudaFuncSetAttribute(oph_sketch_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HOPH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oph_sketch_kernel<true>,
                                                                    kSketchThreads, smem));
    } else {
        HOPH_CUDA_TRY(cudaFuncSetAttribute(oph_sketch_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HOPH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, oph_sketch_kernel<false>, kSketchThreads, smem));
    }
    if (per_sm < 1) return HOPH_ERR_UNSUPPORTED;
    const int64_t resident = (int64_t)grid_for(plan, per_sm) * kSketchWarps;
    // size-sorted work list once there are several sets per resident warp
    if (n_sets > 2 * resident) {
        const size_t bytes = 3 * kBuckets * sizeof(uint32_t) + (size_t)n_sets * sizeof(int32_t);
        unsigned char *scr = (unsigned char *)hoph_scratch(plan, bytes);
        if (!scr) return HOPH_ERR_NOMEM;
        uint32_t *hist = (uint32_t *)scr, *base = hist + kBuckets, *cursor = base + kBuckets;
        int32_t *order = (int32_t *)(cursor + kBuckets);
        HOPH_CUDA_TRY(cudaMemsetAsync(hist, 0, 3 * kBuckets * sizeof(uint32_t), s));
        const int g = plan->num_sms * 4;
        bucket_hist_kernel<<<g, 256, 0, s>>>(d_offsets, n_sets, hist);
        bucket_base_kernel<<<1, 32, 0, s>>>(hist, base);
        bucket_scatter_kernel<<<g, 256, 0, s>>>(d_offsets, n_sets, base, cursor, order);
        a.order = order;
        plan->launches += 3;
    }
    int64_t blocks = std::min<int64_t>((n_sets + kSketchWarps - 1) / kSketchWarps,
                                       (int64_t)grid_for(plan, per_sm));
    if (hash)
        oph_sketch_kernel<true><<<(unsigned)blocks, kSketchThreads, smem, s>>>(a);
    else
        oph_sketch_kernel<false><<<(unsigned)blocks, kSketchThreads, smem, s>>>(a);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 1;
    return HOPH_OK;
}

int minwise_build_sketches(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                           int64_t n_sets, uint32_t *d_sketches, void *stream) {
    if (!plan || n_sets < 0 || (n_sets > 0 && (!d_offsets || !d_sketches))) return HOPH_ERR_PARAM;
    if (!plan->d_minwise) return HOPH_ERR_PARAM;
    if (n_sets == 0) return HOPH_OK;
    MinwiseArgs a;
    a.ids = d_ids;
    a.off = d_offsets;
    a.n_sets = n_sets;
    a.tab = plan->d_minwise;
    a.D = plan->P.universe_D;
    a.mk = plan->P.minwise_k;
    a.out = d_sketches;
    a.status = plan->d_status;
    const size_t smem = (size_t)8 * a.mk * 4;
    HOPH_CUDA_TRY(
        cudaFuncSetAttribute(minwise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t blocks = std::min<int64_t>((n_sets + 7) / 8, (int64_t)plan->num_sms * 8);
    minwise_kernel<<<(unsigned)blocks, 256, smem, (cudaStream_t)stream>>>(a);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 1;
    return HOPH_OK;
}

int hoph_synth_ids(uint64_t seed, int64_t first, int64_t n_ids, uint64_t D, uint32_t kind,
                   const double *d_cdf, int64_t n_cdf, uint32_t *d_ids, void *stream) {
    if (n_ids < 0 || first < 0 || kind > 1 || (n_ids > 0 && !d_ids)) return HOPH_ERR_PARAM;
    if (kind == 0 && (D == 0 || D > (1ull << 32))) return HOPH_ERR_PARAM;
    if (kind == 1 && (!d_cdf || n_cdf <= 0)) return HOPH_ERR_PARAM;
    if (n_ids == 0) return HOPH_OK;
    int dev = 0, sms = 0;
    HOPH_CUDA_TRY(cudaGetDevice(&dev));
    HOPH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t blocks = std::min<int64_t>((n_ids + 255) / 256, (int64_t)sms * 16);
    synth_ids_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(seed, first, n_ids, D, kind,
                                                                         d_cdf, n_cdf, d_ids);
    HOPH_CUDA_TRY(cudaGetLastError());
    return HOPH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// oph_build_sketches_static: the sketch kernel above with its size-sorted
// work list held in a fixed device array, for callers that must not allocate
// device memory while they sketch (a serving loop running on a fixed memory
// budget owned by its own pool allocator, or a latency-critical path that
// cannot afford the device-wide synchronisation a cudaMalloc / cudaFree may
// bring).  oph_build_sketches itself grows plan scratch on demand.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kStaticMaxSets = 1 << 18;  // sets per call (262,144)
constexpr size_t kStaticWords = 3 * kBuckets + (size_t)kStaticMaxSets;

// Bucket histogram, bucket bases, bucket cursors, then the set order: about
// 1 MiB.  One copy per GPU that loads the library, kept until the process
// exits, shared by every call on that GPU.
static __device__ __align__(256) uint32_t g_static_worklist[kStaticWords];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
uint32_t *g_static_addr[kMaxDevices] = {};

// Device address of g_static_worklist on the current device.  The symbol
// name is only a host-side handle; the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it.
int static_worklist(uint32_t **out) {
    int dev = 0;
    HOPH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return HOPH_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_worklist);
        if (e != cudaSuccess || !p) return hoph_cuda_fail(e);
        g_static_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_static_addr[dev];
    return HOPH_OK;
}

}  // namespace

extern "C" int oph_build_sketches_static(hoph_plan *plan, const uint32_t *d_ids,
                                         const int64_t *d_offsets, int64_t n_sets,
                                         uint32_t *d_planes, void *stream) {
    if (!plan || n_sets < 0 || (n_sets > 0 && (!d_offsets || !d_planes))) return HOPH_ERR_PARAM;
    if (n_sets > kStaticMaxSets) return HOPH_ERR_TOO_LARGE;
    if (n_sets == 0) return HOPH_OK;
    uint32_t *scr = nullptr;
    const int rc = static_worklist(&scr);
    if (rc != HOPH_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const hoph_params &P = plan->P;
    SketchArgs a;
    a.ids = d_ids;
    a.off = d_offsets;
    a.n_sets = n_sets;
    a.planes = d_planes;
    a.plane_stride = n_sets * (int64_t)P.k_group;
    a.k = P.k;
    a.kg = P.k_group;
    a.key = plan->d_key;
    a.key_bits = plan->key_bits;
    a.D = P.universe_D;
    a.lo = plan->d_lo;
    a.ha = plan->hash_a;
    a.hb = plan->hash_b;
    a.status = plan->d_status;
    // the array keeps the previous call's contents: the histogram and the
    // cursors must start at zero (the bases and the order are overwritten)
    uint32_t *hist = scr, *base = hist + kBuckets, *cursor = base + kBuckets;
    int32_t *order = reinterpret_cast<int32_t *>(cursor + kBuckets);
    HOPH_CUDA_TRY(cudaMemsetAsync(hist, 0, kBuckets * sizeof(uint32_t), s));
    HOPH_CUDA_TRY(cudaMemsetAsync(cursor, 0, kBuckets * sizeof(uint32_t), s));
    const int g = plan->num_sms * 4;
    bucket_hist_kernel<<<g, 256, 0, s>>>(d_offsets, n_sets, hist);
    bucket_base_kernel<<<1, 32, 0, s>>>(hist, base);
    bucket_scatter_kernel<<<g, 256, 0, s>>>(d_offsets, n_sets, base, cursor, order);
    a.order = order;

    const bool hash = P.perm_kind == HOPH_PERM_HASH61;
    const size_t smem = (hash ? (P.k + 1) * 8 : 0) + (size_t)kSketchWarps * P.k * 4;
    int per_sm = 0;
    if (hash) {
        HOPH_CUDA_TRY(cudaFuncSetAttribute(oph_sketch_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HOPH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oph_sketch_kernel<true>,
                                                                    kSketchThreads, smem));
    } else {
        HOPH_CUDA_TRY(cudaFuncSetAttribute(oph_sketch_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HOPH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, oph_sketch_kernel<false>, kSketchThreads, smem));
    }
    if (per_sm < 1) return HOPH_ERR_UNSUPPORTED;
    const int64_t blocks = std::min<int64_t>((n_sets + kSketchWarps - 1) / kSketchWarps,
                                             (int64_t)grid_for(plan, per_sm));
    if (hash)
        oph_sketch_kernel<true><<<(unsigned)blocks, kSketchThreads, smem, s>>>(a);
    else
        oph_sketch_kernel<false><<<(unsigned)blocks, kSketchThreads, smem, s>>>(a);
    HOPH_CUDA_TRY(cudaGetLastError());
    return HOPH_OK;
}
