// Sketch construction on the GPU.
//
//  * oph_build_sketches: OPH / HOPH sketches (Sec. 3.2, Sec. 4.1).  Sets are
//    visited in descending size order (a counting sort by size bucket builds
//    the work list); in one persistent launch the sets of >= 2048 IDs get a
//    whole CTA each and the others one warp each, striped across all
//    resident warps.  IDs are read with 128-bit
//    loads; each ID is mapped through the packed psi table (psi value ->
//    bin and offset) that stays resident in L2, and the per-bin minimum is
//    kept in the warp's shared-memory sketch with a shared atomicMin.
//    The finished sketch is written group-major ([G][n][k']) with coalesced
//    stores.
//  * minwise_build_sketches: MinWise (Sec. 1), one warp per set, lane t
//    owning the minima of permutations t, t+32, ...; the k permuted values
//    of an ID are contiguous ([D][k] table) so each gather is coalesced.
//  * hoph_synth_ids: counter-based synthetic IDs (benchmark inputs).
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int kSketchThreads = 256;
constexpr int kSketchWarps = kSketchThreads / 32;
constexpr int kBuckets = 65;
constexpr int kBigBucket = 12;  // sets of >= 2048 IDs (bit length >= 12) get a whole CTA
constexpr int kResidentCtas = 6;  // sketch CTAs per SM (40 registers x 256 threads)
constexpr int64_t kSplitPhases = 16384;  // from this many sets: one launch per phase
constexpr int64_t kSmallList = 4096;     // up to this many sets: the work list in one CTA

// Hash path: psi-space regions of equal-width bins (the whole space for equal
// bins, one per group for a:b); a value's bin is first + floor(o * nb / z),
// computed as the high half of o * magic with magic = floor(2^64 nb / z) + 1:
// o * magic / 2^64 exceeds o nb / z by less than o / 2^64 < 2^-32 <= 1 / z,
// and o nb / z is at most 1 / z below the next integer, so the floor is the
// same.  magic = 0 marks bins of one value (nb = z: the bin is the offset).
struct RegionTable {
    int32_t n;
    uint32_t start[HOPH_MAX_GROUPS];
    uint32_t first[HOPH_MAX_GROUPS];
    uint64_t magic[HOPH_MAX_GROUPS];
};

struct SketchArgs {
    const uint32_t *ids;
    const int64_t *off;
    int64_t n_sets;
    void *planes;          // uint32 or (compact) uint16 [G][n_sets][k']
    int32_t compact;       // uint16 planes
    int64_t plane_stride;  // n_sets * k'
    uint32_t k, kg, G;
    const uint32_t *key;   // packed psi table (table path)
    uint32_t key_bits;
    uint64_t D;
    const uint64_t *lo;    // bin bounds (hash path)
    uint64_t ha, hb;
    const int32_t *order;  // size-sorted set indices, or nullptr for 0..n-1
    const uint32_t *n_big; // items [0, *n_big) of order are sketched a CTA per set
    RegionTable reg;       // hash path: bin regions
    int32_t generate;      // IDs come from the counter generator, not from ids[]
    uint64_t gen_seed;     // generator stream; set i's IDs are elements off[i]..off[i+1]-1
    uint64_t gen_D;        // generated IDs are uniform over 0..gen_D-1
    int32_t *status;
};

// Synthetic ID of element e of stream `seed`: the (e+1)-th SplitMix64 output
// mapped to [0, D) by a multiply-shift of its top 32 bits (hoph_synth_ids kind 0):
// (h D) >> 32 for the top word h, which is h itself for D = 2^32 and the high
// half of the 32 x 32 product h D below it.
__device__ __forceinline__ uint32_t synth_id(uint64_t seed, uint64_t e, uint64_t D) {
    uint64_t z = seed + (e + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const uint32_t h = (uint32_t)(z >> 32);
    return (D >> 32) ? h : __umulhi(h, (uint32_t)D);
}

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

// Bin and offset of a hashed psi-value v: the region containing v (a few
// comparisons against the region starts), then floor(o * nb / z) by the
// region's magic multiplier (the high word of o * magic, as o * (magic >> 32)
// plus the high half of o * (magic & 0xFFFFFFFF)), then the offset from the
// bin's lower bound.
__device__ __forceinline__ uint64_t hash_bin(const RegionTable &t, const uint32_t *s_lo, uint32_t v) {
    int r = 0;
    for (int i = 1; i < t.n; ++i) r += v >= t.start[i];
    const uint32_t o = v - t.start[r];
    const uint64_t m = t.magic[r];
    const uint32_t q =
        m ? (uint32_t)(((uint64_t)o * (uint32_t)(m >> 32) + __umulhi(o, (uint32_t)m)) >> 32) : o;
    const uint32_t bin = t.first[r] + q;
    return ((uint64_t)bin << 32) | (v - s_lo[bin]);
}

// Table path: the IDs below kHotIds (the most frequent words of a
// frequency-ranked vocabulary) are collected as bits of `hot` instead of
// being gathered and applied one by one; kSkipKey marks them, kBadKey an ID
// outside V (no table key reaches either: k 2^key_bits stays below 2^32 for
// the table sizes a plan accepts).
constexpr uint32_t kHotIds = 32;
constexpr uint32_t kSkipKey = 0xFFFFFFFEu;
constexpr uint32_t kBadKey = 0xFFFFFFFFu;

// 1 << x, or 0 for x >= 32 (PTX shl clamps the shift amount to the width)
__device__ __forceinline__ uint32_t bit_or_zero(uint32_t x) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(x));
    return r;
}

// The hot IDs of a set (bits of hm, collected by its warp or CTA), applied
// to its sketch once each by lanes 0..31; one at or beyond D (a universe of
// fewer than 32 IDs) is flagged instead.
__device__ __forceinline__ void apply_hot(const SketchArgs &a, uint32_t *sk, uint32_t hm,
                                          int lane, bool &bad) {
    if (hm >> lane & 1u) {
        if ((uint64_t)lane >= a.D) {
            bad = true;
            return;
        }
        const uint32_t mask = a.key_bits >= 32 ? 0xFFFFFFFFu : ((1u << a.key_bits) - 1u);
        const uint32_t key = __ldg(a.key + lane);
        atomicMin(sk + (key >> a.key_bits), key & mask);
    }
}

// One thread's share of the IDs [p, p+n) (thread t of a group of T threads):
// a scalar head up to a 16-byte boundary, a 128-bit body whose eight table
// gathers are issued before any of their minima is applied, a scalar tail.
// Each ID updates the shared sketch `sk` with an atomicMin (no read first: one
// shared-memory operation per ID instead of a read and, when it improves, an
// atomic).
template <bool HASH, bool WIDE = true>
__device__ __forceinline__ void sketch_ids(const SketchArgs &a, const uint32_t *s_lo,
                                           const RegionTable *s_reg, uint32_t *sk,
                                           const uint32_t *p, int64_t n, int t, int T,
                                           bool &bad, uint32_t &hot) {
    const uint32_t mask = a.key_bits >= 32 ? 0xFFFFFFFFu : ((1u << a.key_bits) - 1u);
    // hash path: psi-value of x as (bin << 32) | offset (bin < k always);
    // table path: the packed table key (bin << key_bits) | offset itself, or
    // all ones for an ID outside V (no table key is all ones: k 2^key_bits
    // stays below 2^32 for the table sizes a plan accepts), so a thread keeps
    // 32 bits per lookup in flight
    using Loc = typename std::conditional<HASH, uint64_t, uint32_t>::type;
    auto locate = [&](uint32_t x) -> Loc {
        if constexpr (HASH) {
            return hash_bin(*s_reg, s_lo, hash61(x, a.ha, a.hb));
        } else {
            // the most frequent IDs of a frequency-ranked vocabulary (x < 32)
            // only set a bit; the set's bits are applied once at its end
            hot |= bit_or_zero(x);
            return x < kHotIds ? kSkipKey : (x < a.D ? __ldg(a.key + x) : kBadKey);
        }
    };
    auto apply = [&](Loc v) {
        if constexpr (HASH) {
            atomicMin(sk + (uint32_t)(v >> 32), (uint32_t)v);
        } else {
            if (v >= kSkipKey) {
                if (v == kBadKey) bad = true;
                return;
            }
            atomicMin(sk + (v >> a.key_bits), v & mask);
        }
    };
    const int64_t head =
        (int64_t)min((long long)n, (long long)((4 - ((reinterpret_cast<uintptr_t>(p) >> 2) & 3)) & 3));
    if (t < head) apply(locate(p[t]));
    const uint4 *p4 = reinterpret_cast<const uint4 *>(p + head);
    const int64_t nvec = (n - head) >> 2;
    int64_t i = t;
    // WIDE: two 128-bit loads (eight lookups) in flight per iteration, else one
    for (; WIDE && i + T < nvec; i += 2 * (int64_t)T) {
        const uint4 v0 = ldg_nc_v4(p4 + i);
        const uint4 v1 = ldg_nc_v4(p4 + i + T);
        const Loc b0 = locate(v0.x), b1 = locate(v0.y), b2 = locate(v0.z), b3 = locate(v0.w);
        const Loc b4 = locate(v1.x), b5 = locate(v1.y), b6 = locate(v1.z), b7 = locate(v1.w);
        apply(b0); apply(b1); apply(b2); apply(b3);
        apply(b4); apply(b5); apply(b6); apply(b7);
    }
    for (; i < nvec; i += T) {
        const uint4 v0 = ldg_nc_v4(p4 + i);
        const Loc b0 = locate(v0.x), b1 = locate(v0.y), b2 = locate(v0.z), b3 = locate(v0.w);
        apply(b0); apply(b1); apply(b2); apply(b3);
        if (WIDE) break;  // the wide loop leaves at most one vector per thread
    }
    const int64_t tail0 = head + (nvec << 2);
    for (int64_t j = tail0 + t; j < n; j += T) apply(locate(p[j]));
}

// As sketch_ids, with the IDs of elements [first, first + n) of the
// generator stream produced in registers instead of loaded.
template <bool HASH>
__device__ __forceinline__ void sketch_generated(const SketchArgs &a, const uint32_t *s_lo,
                                                 const RegionTable *s_reg, uint32_t *sk,
                                                 uint64_t first, int64_t n, int t, int T,
                                                 bool &bad, uint32_t &hot) {
    const uint32_t mask = a.key_bits >= 32 ? 0xFFFFFFFFu : ((1u << a.key_bits) - 1u);
    // as in sketch_ids
    using Loc = typename std::conditional<HASH, uint64_t, uint32_t>::type;
    auto locate = [&](uint32_t x) -> Loc {
        if constexpr (HASH) {
            return hash_bin(*s_reg, s_lo, hash61(x, a.ha, a.hb));
        } else {
            // the most frequent IDs of a frequency-ranked vocabulary (x < 32)
            // only set a bit; the set's bits are applied once at its end
            hot |= bit_or_zero(x);
            return x < kHotIds ? kSkipKey : (x < a.D ? __ldg(a.key + x) : kBadKey);
        }
    };
    auto apply = [&](Loc v) {
        if constexpr (HASH) {
            atomicMin(sk + (uint32_t)(v >> 32), (uint32_t)v);
        } else {
            if (v >= kSkipKey) {
                if (v == kBadKey) bad = true;
                return;
            }
            atomicMin(sk + (v >> a.key_bits), v & mask);
        }
    };
    int64_t j = t;
    for (; j + 3 * (int64_t)T < n; j += 4 * (int64_t)T) {
        const Loc b0 = locate(synth_id(a.gen_seed, first + j, a.gen_D));
        const Loc b1 = locate(synth_id(a.gen_seed, first + j + T, a.gen_D));
        const Loc b2 = locate(synth_id(a.gen_seed, first + j + 2 * T, a.gen_D));
        const Loc b3 = locate(synth_id(a.gen_seed, first + j + 3 * T, a.gen_D));
        apply(b0); apply(b1); apply(b2); apply(b3);
    }
    for (; j < n; j += T) apply(locate(synth_id(a.gen_seed, first + j, a.gen_D)));
}

// group-major store of one finished sketch (bin b -> plane b / k', slot b % k')
// and reset of the shared copy
// (compact planes: offsets < 0xFFFF; the empty marker truncates to 0xFFFF)
template <bool COMPACT>
__device__ __forceinline__ void store_sketch(const SketchArgs &a, uint32_t *sk, int64_t set, int t,
                                             int T) {
    using E = typename std::conditional<COMPACT, uint16_t, uint32_t>::type;
    E *dst = static_cast<E *>(a.planes) + set * a.kg;
    for (uint32_t g = 0; g < a.G; ++g, dst += a.plane_stride, sk += a.kg) {
        for (uint32_t j = t; j < a.kg; j += T) {
            dst[j] = (E)sk[j];
            sk[j] = HOPH_EMPTY_VALUE;
        }
    }
}

// The work list in two phases.  Phase 1 (PHASES & 1): the large sets at its
// head (items [0, *n_big)), a CTA per set, all warps feeding one shared
// sketch.  Phase 2 (PHASES & 2): warp per set over the rest; when both run in
// one launch (small batches), strided so that the CTAs that took a large set
// get the smallest of the remaining sets.  Without a work list (a.n_big null)
// only phase 2 runs, in input order.
template <bool HASH, int PHASES, bool COMPACT>
__global__ void __launch_bounds__(kSketchThreads, (!HASH && PHASES != 3) ? 8 : 6)
    oph_sketch_kernel(const SketchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // HASH only: the bins' lower bounds (below 2^32 for every bin of a universe
    // of at most 2^32 values)
    uint32_t *s_lo = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *s_sk = reinterpret_cast<uint32_t *>(smem_raw + (HASH ? (a.k + 3) / 4 * 16 : 0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ RegionTable s_reg;
    if (HASH) {
        for (uint32_t i = threadIdx.x; i < a.k; i += blockDim.x) s_lo[i] = (uint32_t)a.lo[i];
        if (threadIdx.x == 0) s_reg = a.reg;
    }
    const uint32_t regions = (PHASES & 2) ? kSketchWarps : 1;
    for (uint32_t i = threadIdx.x; i < regions * a.k; i += blockDim.x) s_sk[i] = HOPH_EMPTY_VALUE;
    __syncthreads();
    bool bad = false;
    uint32_t hot = 0;
    const int64_t n_big = a.n_big ? (int64_t)*a.n_big : 0;
    // phase 1 (warp 0's sketch region serves the CTA; store_sketch resets it)
    for (int64_t item = (PHASES & 1) ? blockIdx.x : n_big; item < n_big; item += gridDim.x) {
        const int64_t set = a.order[item];
        const int64_t beg = a.off[set], end = a.off[set + 1];
        if (a.generate)
            sketch_generated<HASH>(a, s_lo, &s_reg, s_sk, (uint64_t)beg, end - beg, threadIdx.x,
                                   blockDim.x, bad, hot);
        else
            sketch_ids<HASH>(a, s_lo, &s_reg, s_sk, a.ids + beg, end - beg, threadIdx.x,
                             blockDim.x, bad, hot);
        if (!HASH) {  // each warp applies the hot IDs its own lanes met
            apply_hot(a, s_sk, __reduce_or_sync(0xFFFFFFFFu, hot), lane, bad);
            hot = 0;
        }
        __syncthreads();
        store_sketch<COMPACT>(a, s_sk, set, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    // phase 2
    if (!(PHASES & 2)) {
        if (bad) hoph_flag(a.status, HOPH_ERR_ID_RANGE);
        return;
    }
    uint32_t *sk = s_sk + (size_t)warp * a.k;
    const int64_t warps_total = (int64_t)gridDim.x * kSketchWarps;
    const int64_t cta = PHASES == 3 ? (int64_t)(gridDim.x - 1 - blockIdx.x) : blockIdx.x;
    for (int64_t item = n_big + cta * kSketchWarps + warp; item < a.n_sets; item += warps_total) {
        const int64_t set = a.order ? a.order[item] : item;
        const int64_t beg = a.off[set], end = a.off[set + 1];
        if (a.generate)
            sketch_generated<HASH>(a, s_lo, &s_reg, sk, (uint64_t)beg, end - beg, lane, 32, bad,
                                   hot);
        else
            sketch_ids<HASH, (HASH || PHASES != 2)>(a, s_lo, &s_reg, sk, a.ids + beg, end - beg,
                                                    lane, 32, bad, hot);
        if (!HASH) {
            apply_hot(a, sk, __reduce_or_sync(0xFFFFFFFFu, hot), lane, bad);
            hot = 0;
        }
        __syncwarp();
        store_sketch<COMPACT>(a, sk, set, lane, 32);
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

// The size bucket from which a set gets a whole CTA: `bits` when given (an
// execution knob), else sets of at least 2,048 IDs and, when warps > 0 (a
// batch sketched in one launch), also more than four times the batch's IDs
// per resident warp.
__device__ __forceinline__ int cta_bucket(const int64_t *off, int64_t n, int64_t warps, int bits) {
    if (bits > 0) return bits;
    int big = kBigBucket;
    if (warps > 0) {
        const uint64_t per_warp = (uint64_t)(off[n] - off[0]) / (uint64_t)warps;
        big = max(big, size_bucket((int64_t)(4 * per_warp)) + 1);
    }
    return big;
}

// exclusive prefix over buckets in descending size order (largest first);
// *n_big = number of sets from the CTA bucket up
__global__ void bucket_base_kernel(const uint32_t *hist, uint32_t *base, uint32_t *n_big,
                                   const int64_t *off, int64_t n, int64_t warps, int bits) {
    if (threadIdx.x == 0) {
        const int big = cta_bucket(off, n, warps, bits);
        uint32_t run = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            if (b == big - 1) *n_big = run;
            base[b] = run;
            run += hist[b];
        }
    }
}

// The three steps above in one CTA, for a batch of at most kSmallList sets
// (a query batch): histogram, prefix and large-set count, scatter.
__global__ void __launch_bounds__(1024) bucket_small_kernel(const int64_t *off, int64_t n,
                                                            uint32_t *n_big, int32_t *order,
                                                            int64_t warps, int bits) {
    __shared__ uint32_t h[kBuckets], cur[kBuckets];
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        atomicAdd(&h[size_bucket(off[i + 1] - off[i])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int big = cta_bucket(off, n, warps, bits);
        uint32_t run = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            if (b == big - 1) *n_big = run;
            cur[b] = run;
            run += h[b];
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        order[atomicAdd(&cur[size_bucket(off[i + 1] - off[i])], 1u)] = (int32_t)i;
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

// Integer-throughput probe: 8 independent chains per thread of one
// operation (KIND 0: 32-bit multiply-add, 1: 64-bit multiply-add, 2: high
// half of a 64-bit product plus an add); the constants come from the thread
// index so nothing folds away.
template <int KIND>
__global__ void __launch_bounds__(256) int_probe_kernel(int64_t iters, uint64_t *sink) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (KIND == 0) {
        uint32_t x[8];
        const uint32_t a = (uint32_t)(t * 2654435761u) | 1u, b = (uint32_t)t ^ 0x9E3779B9u;
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = (uint32_t)t + c;
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
        uint32_t r = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) r ^= x[c];
        sink[t] = r;
    } else {
        uint64_t x[8];
        const uint64_t a = (t * 0x9E3779B97F4A7C15ull) | 1ull, b = t ^ 0xBF58476D1CE4E5B9ull;
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = t + (uint64_t)c;
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = (KIND == 1 ? x[c] * a : __umul64hi(x[c], a)) + b;
        uint64_t r = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) r ^= x[c];
        sink[t] = r;
    }
}

int grid_for(hoph_plan *pl, int per_sm) { return pl->num_sms * per_sm; }

SketchArgs sketch_args(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                       int64_t n_sets, void *d_planes) {
    const hoph_params &P = plan->P;
    SketchArgs a;
    a.ids = d_ids;
    a.off = d_offsets;
    a.n_sets = n_sets;
    a.planes = d_planes;
    a.compact = 0;
    a.plane_stride = n_sets * (int64_t)P.k_group;
    a.k = P.k;
    a.kg = P.k_group;
    a.G = P.k / P.k_group;
    a.key = plan->d_key;
    a.key_bits = plan->key_bits;
    a.D = P.universe_D;
    a.lo = plan->d_lo;
    a.ha = plan->hash_a;
    a.hb = plan->hash_b;
    a.order = nullptr;
    a.n_big = nullptr;
    a.generate = 0;
    a.gen_seed = 0;
    a.gen_D = 0;
    // bin regions of the hash path
    const bool equal = P.a == 0 && P.b == 0;
    a.reg.n = equal ? 1 : (int32_t)plan->G;
    for (int r = 0; r < a.reg.n; ++r) {
        const uint32_t first = equal ? 0 : (uint32_t)r * P.k_group;
        const uint32_t nb = equal ? P.k : P.k_group;
        const uint64_t z = plan->lo[first + nb] - plan->lo[first];
        a.reg.start[r] = (uint32_t)plan->lo[first];
        a.reg.first[r] = first;
        a.reg.magic[r] =
            nb < z ? (uint64_t)(((unsigned __int128)nb << 64) / z) + 1u : 0u;  // z <= 2^32
    }
    a.status = plan->d_status;
    return a;
}

// Size-sorted work list in `wl` (hist, base, cursor: kBuckets words each,
// then n_big, then the order of n_sets entries); hist and cursor are zeroed.
int build_work_list(hoph_plan *plan, const int64_t *d_offsets, int64_t n_sets, uint32_t *wl,
                    SketchArgs &a, cudaStream_t s) {
    uint32_t *hist = wl, *base = hist + kBuckets, *cursor = base + kBuckets;
    uint32_t *n_big = cursor + kBuckets;
    int32_t *order = reinterpret_cast<int32_t *>(n_big + 1);
    a.order = order;
    a.n_big = n_big;
    if (n_sets <= kSmallList) {
        bucket_small_kernel<<<1, 1024, 0, s>>>(
            d_offsets, n_sets, n_big, order,
            (int64_t)plan->num_sms * kResidentCtas * kSketchWarps, plan->exec.sketch_cta_bits);
        HOPH_CUDA_TRY(cudaGetLastError());
        plan->launches += 1;
        return HOPH_OK;
    }
    HOPH_CUDA_TRY(cudaMemsetAsync(hist, 0, kBuckets * sizeof(uint32_t), s));
    HOPH_CUDA_TRY(cudaMemsetAsync(cursor, 0, kBuckets * sizeof(uint32_t), s));
    const int g = plan->num_sms * 4;
    bucket_hist_kernel<<<g, 256, 0, s>>>(d_offsets, n_sets, hist);
    const int64_t warps =
        n_sets >= kSplitPhases ? 0 : (int64_t)plan->num_sms * kResidentCtas * kSketchWarps;
    bucket_base_kernel<<<1, 32, 0, s>>>(hist, base, n_big, d_offsets, n_sets, warps,
                                        plan->exec.sketch_cta_bits);
    bucket_scatter_kernel<<<g, 256, 0, s>>>(d_offsets, n_sets, base, cursor, order);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 3;
    a.order = order;
    a.n_big = n_big;
    return HOPH_OK;
}

template <bool HASH, int PHASES, bool COMPACT>
int launch_phases(hoph_plan *plan, const SketchArgs &a, cudaStream_t s) {
    const uint32_t k = a.k;
    const size_t lo_b = HASH ? (size_t)(k + 3) / 4 * 16 : 0;
    const size_t smem = lo_b + (size_t)((PHASES & 2) ? kSketchWarps : 1) * k * 4;
    auto kern = oph_sketch_kernel<HASH, PHASES, COMPACT>;
    HOPH_CUDA_TRY(hoph_ensure_smem((const void *)kern, (int)smem));
    int per = 0;
    HOPH_CUDA_TRY(hoph_occupancy(&per, (const void *)kern, kSketchThreads, smem));
    if (per < 1) return HOPH_ERR_UNSUPPORTED;
    const int64_t want = PHASES == 1 ? a.n_sets : (a.n_sets + kSketchWarps - 1) / kSketchWarps;
    const int64_t blocks = std::min<int64_t>(want, (int64_t)grid_for(plan, per));
    kern<<<(unsigned)blocks, kSketchThreads, smem, s>>>(a);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 1;
    return HOPH_OK;
}

// The sketch kernel(s) over the work list (or the input order): one launch
// for a small batch; a large one sketches its large sets (a CTA each) with
// the whole GPU first, then the rest.
template <bool HASH, bool COMPACT>
int launch_sketch_kernels(hoph_plan *plan, const SketchArgs &a, cudaStream_t s) {
    if (a.n_big && a.n_sets >= kSplitPhases) {
        const int rc = launch_phases<HASH, 1, COMPACT>(plan, a, s);
        return rc != HOPH_OK ? rc : launch_phases<HASH, 2, COMPACT>(plan, a, s);
    }
    return launch_phases<HASH, 3, COMPACT>(plan, a, s);
}

int launch_sketch(hoph_plan *plan, const SketchArgs &a, cudaStream_t s) {
    const bool hash = plan->P.perm_kind == HOPH_PERM_HASH61;
    if (a.compact)
        return hash ? launch_sketch_kernels<true, true>(plan, a, s)
                    : launch_sketch_kernels<false, true>(plan, a, s);
    return hash ? launch_sketch_kernels<true, false>(plan, a, s)
                : launch_sketch_kernels<false, false>(plan, a, s);
}

constexpr int64_t kWorkListMin = 64;  // below this many sets: identity order, warps only

// oph_build_sketches / oph_build_sketches16
int build_sketches(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                   int64_t n_sets, void *d_planes, bool compact, void *stream) {
    if (!plan || n_sets < 0 || (n_sets > 0 && (!d_offsets || !d_planes))) return HOPH_ERR_PARAM;
    if (n_sets >= (1ll << 31)) return HOPH_ERR_PARAM;
    if (compact && plan->max_width > 0xFFFFu) return HOPH_ERR_UNSUPPORTED;
    if (n_sets == 0) return HOPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SketchArgs a = sketch_args(plan, d_ids, d_offsets, n_sets, d_planes);
    a.compact = compact ? 1 : 0;
    if (n_sets >= kWorkListMin) {
        const size_t bytes = (3 * kBuckets + 1) * sizeof(uint32_t) + (size_t)n_sets * sizeof(int32_t);
        void *p = nullptr;
        const int src = hoph_scratch(plan, bytes, 0, s, &p);
        if (src != HOPH_OK) return src;
        uint32_t *wl = static_cast<uint32_t *>(p);
        const int rc = build_work_list(plan, d_offsets, n_sets, wl, a, s);
        if (rc != HOPH_OK) return rc;
    }
    return launch_sketch(plan, a, s);
}

}  // namespace

extern "C" {

int oph_build_sketches(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                       int64_t n_sets, uint32_t *d_planes, void *stream) {
    return build_sketches(plan, d_ids, d_offsets, n_sets, d_planes, false, stream);
}

int oph_build_sketches16(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                         int64_t n_sets, uint16_t *d_planes, void *stream) {
    return build_sketches(plan, d_ids, d_offsets, n_sets, d_planes, true, stream);
}

int hoph_synth_sketch(hoph_plan *plan, uint64_t seed, uint64_t D, const int64_t *d_offsets,
                      int64_t n_sets, uint32_t *d_planes, void *stream) {
    if (!plan || n_sets < 0 || (n_sets > 0 && (!d_offsets || !d_planes))) return HOPH_ERR_PARAM;
    if (n_sets >= (1ll << 31) || D == 0 || D > (1ull << 32)) return HOPH_ERR_PARAM;
    if (n_sets == 0) return HOPH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SketchArgs a = sketch_args(plan, nullptr, d_offsets, n_sets, d_planes);
    a.generate = 1;
    a.gen_seed = seed;
    a.gen_D = D;
    if (n_sets >= kWorkListMin) {
        const size_t bytes = (3 * kBuckets + 1) * sizeof(uint32_t) + (size_t)n_sets * sizeof(int32_t);
        void *p = nullptr;
        const int src = hoph_scratch(plan, bytes, 0, s, &p);
        if (src != HOPH_OK) return src;
        uint32_t *wl = static_cast<uint32_t *>(p);
        const int rc = build_work_list(plan, d_offsets, n_sets, wl, a, s);
        if (rc != HOPH_OK) return rc;
    }
    return launch_sketch(plan, a, s);
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
    HOPH_CUDA_TRY(hoph_ensure_smem((const void *)minwise_kernel, (int)smem));
    const int64_t blocks = std::min<int64_t>((n_sets + 7) / 8, (int64_t)plan->num_sms * 8);
    minwise_kernel<<<(unsigned)blocks, 256, smem, (cudaStream_t)stream>>>(a);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 1;
    return HOPH_OK;
}

int hoph_int_probe(uint32_t kind, int64_t iters, uint64_t *d_sink, void *stream) {
    if (kind > 2 || iters < 1 || iters > (1ll << 24) || !d_sink) return HOPH_ERR_PARAM;
    int dev = 0, sms = 0;
    HOPH_CUDA_TRY(cudaGetDevice(&dev));
    HOPH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)sms * 8;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0) int_probe_kernel<0><<<grid, 256, 0, s>>>(iters, d_sink);
    else if (kind == 1) int_probe_kernel<1><<<grid, 256, 0, s>>>(iters, d_sink);
    else int_probe_kernel<2><<<grid, 256, 0, s>>>(iters, d_sink);
    HOPH_CUDA_TRY(cudaGetLastError());
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
constexpr size_t kStaticWords = 3 * kBuckets + 1 + (size_t)kStaticMaxSets;

// Bucket histogram, bucket bases, bucket cursors, the large-set count, then
// the set order: about 1 MiB.  One copy per GPU that loads the library, kept until the process
// exits, shared by every call on that GPU.
static __device__ __align__(256) uint32_t g_static_worklist[kStaticWords];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
uint32_t *g_static_addr[kMaxDevices] = {};

// Device address of g_static_worklist on the current device.  The symbol
// name is only a host-side handle; the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it.  That set-up is refused (HOPH_ERR_CAPTURE) while `s` is being captured,
// like every other first-use set-up of the library.  The cached address
// belongs to the device's current context: it is not valid after a
// cudaDeviceReset.
int static_worklist(cudaStream_t s, uint32_t **out) {
    int dev = 0;
    HOPH_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return HOPH_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        if (hoph_capturing(s)) return HOPH_ERR_CAPTURE;
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
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *scr = nullptr;
    const int rc = static_worklist(s, &scr);
    if (rc != HOPH_OK) return rc;
    SketchArgs a = sketch_args(plan, d_ids, d_offsets, n_sets, d_planes);
    // the array keeps the previous call's contents: build_work_list zeroes the
    // histogram and the cursors (the bases, the count and the order are
    // overwritten)
    const int rc2 = build_work_list(plan, d_offsets, n_sets, scr, a, s);
    if (rc2 != HOPH_OK) return rc2;
    return launch_sketch(plan, a, s);
}
