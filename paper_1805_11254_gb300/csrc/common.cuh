// Shared definitions of the GB300 HOPH library: the plan, the exact integer
// decision rule, status reporting, and the inline-PTX helpers (mbarrier,
// TMA bulk tensor copies, bounded waits).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "hoph.h"

#define HOPH_CONTINUE 0
#define HOPH_ACCEPT 1
#define HOPH_REJECT 2

#define HOPH_CUDA_TRY(expr)                                  \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return hoph_cuda_fail(e_);    \
    } while (0)

int hoph_cuda_fail(cudaError_t e);

// Everything the comparison rule needs, by value (kernel argument).
struct DecideParams {
    uint32_t mode;      // HOPH_MODE_*
    uint32_t rule;      // HOPH_EMPTY_*
    uint32_t G;         // groups
    uint32_t kg;        // bins per group (k')
    int64_t tn, td;     // T = tn / td
    int64_t U, L;       // small-probability limits (valid when !always_stop)
    int32_t always_stop;  // eps >= 1: every tail is <= eps
    int32_t literal;      // HOPH_WEIGHT_LITERAL
    int64_t ra, rc;       // r = ra / rc = a / (a + b) (literal weighting)
    uint64_t zsuf[HOPH_MAX_GROUPS + 1];  // zsuf[g] = sum_{j >= g} z_j
    uint64_t z[HOPH_MAX_GROUPS];
};

// Effective bins of a group under the empty-bin rule: k' minus the bins
// empty in both sketches (Eq. 5), minus also those empty in exactly one
// (EITHER), or k' itself (NONE).
__host__ __device__ __forceinline__ int32_t hoph_effective(uint32_t rule, int32_t kg, int32_t both,
                                                           int32_t one) {
    return rule == HOPH_EMPTY_BOTH ? kg - both
         : rule == HOPH_EMPTY_EITHER ? kg - both - one
                                     : kg;
}

// The comparison rule after l of G groups (1 <= l <= G), from the per-group
// matched bins M[j] and effective bins K[j], j < l.  Returns HOPH_ACCEPT,
// HOPH_REJECT or HOPH_CONTINUE.
//
// GOPH (Algorithm 1): the remaining average M_ra = (T(K_c + (G-l)k') - M_c)
// / (G-l) is compared with M_a = T k'; "F(M_ra) <= eps" on the lower tail is
// ceil(M_ra) <= L, i.e. M_ra <= L, and on the upper tail ceil(M_ra) >= U,
// i.e. M_ra > U - 1.  All of it is cross-multiplied into integers.
// HOPH (Algorithm 2, space-weighted): S = sum_{K_j > 0} z_j M_j / K_j is
// kept as Sn / Lam with Lam = prod K_j; P_r = (T Z_all - S) / Z_rem and the
// tests read P_r * k' against L and U - 1.  With literal weighting P_r
// follows Algorithm 2's recursion instead (scaled to integers below).
// After the last group: accept iff the full estimator (Eq. 6 pooled for
// GOPH, Lemma 3 space-weighted for HOPH) is >= T over a non-empty
// denominator.
__host__ __device__ __forceinline__ int hoph_decide(const DecideParams &p, int l,
                                                    const int32_t *M, const int32_t *K) {
    const int64_t tn = p.tn, td = p.td;
    if (p.mode == HOPH_MODE_HOPH) {
        __int128 Sn = 0, Lam = 1;
        int64_t Zd = 0;
        for (int j = 0; j < l; ++j) {
            if (K[j] > 0) {
                Sn = Sn * K[j] + (__int128)p.z[j] * M[j] * Lam;
                Lam *= K[j];
                Zd += (int64_t)p.z[j];
            }
        }
        if (l >= (int)p.G)
            return (Zd > 0 && (__int128)td * Sn >= (__int128)tn * Zd * Lam) ? HOPH_ACCEPT
                                                                            : HOPH_REJECT;
        if (p.literal) {
            // P_j = X_j / (td k' a^{s_j}), s_j = j (j + 1) / 2, from X_0 = tn k':
            // P_j = P_{j-1} (c/a)^j - M_j / k'  <=>  X_j = X_{j-1} c^j - M_j td a^{s_j}
            __int128 X = (__int128)tn * p.kg, As = 1;
            for (int j = 1; j <= l; ++j) {
                __int128 cj = 1, aj = 1;
                for (int i = 0; i < j; ++i) {
                    cj *= p.rc;
                    aj *= p.ra;
                }
                As *= aj;
                X = X * cj - (__int128)M[j - 1] * td * As;
            }
            // P_l k' = X / (td a^{s_l})
            const bool below = X < (__int128)tn * p.kg * As;  // P_l < T
            if (p.always_stop) return below ? HOPH_ACCEPT : HOPH_REJECT;
            if (below) {
                if (X <= (__int128)p.L * td * As) return HOPH_ACCEPT;
            } else {
                if (X > (__int128)(p.U - 1) * td * As) return HOPH_REJECT;
            }
            return HOPH_CONTINUE;
        }
        const int64_t Zrem = (int64_t)p.zsuf[l];
        const __int128 num = (__int128)tn * (Zd + Zrem) * Lam - (__int128)td * Sn;
        const __int128 den = (__int128)td * Zrem * Lam;
        const bool below = (__int128)tn * Zd * Lam < (__int128)td * Sn;  // P_r < T
        if (p.always_stop) return below ? HOPH_ACCEPT : HOPH_REJECT;
        if (below) {
            if (num * (int64_t)p.kg <= (__int128)p.L * den) return HOPH_ACCEPT;
        } else {
            if (num * (int64_t)p.kg > (__int128)(p.U - 1) * den) return HOPH_REJECT;
        }
        return HOPH_CONTINUE;
    }
    // GOPH pooled over groups; OPH_FULL / MINWISE reach here with l == G == 1
    int64_t Mc = 0, Kc = 0;
    for (int j = 0; j < l; ++j) {
        Mc += M[j];
        Kc += K[j];
    }
    if (l >= (int)p.G) return (Kc > 0 && Mc * td >= tn * Kc) ? HOPH_ACCEPT : HOPH_REJECT;
    const int64_t r = (int64_t)p.G - l;
    const int64_t num = tn * (Kc + r * (int64_t)p.kg) - td * Mc;
    const int64_t den = td * r;
    const bool below = tn * Kc - td * Mc < 0;  // M_ra < T k'
    if (p.always_stop) return below ? HOPH_ACCEPT : HOPH_REJECT;
    if (below) {
        if (num <= p.L * den) return HOPH_ACCEPT;
    } else {
        if (num > (p.U - 1) * den) return HOPH_REJECT;
    }
    return HOPH_CONTINUE;
}

// First-pass decision table over the scanned bins: for each effective-bin
// count K in 0..W, pairs with M < rej[K] are rejected, M >= acc[K] accepted,
// the rest continue (the rule is monotone in M for fixed K).
struct FirstPassTable {
    std::vector<uint16_t> rej, acc;
};

struct hoph_plan {
    hoph_params P;
    int device = 0;
    int num_sms = 0;
    uint32_t G = 1;
    std::vector<uint64_t> lo;  // bin lower bounds, k + 1 entries
    uint64_t max_width = 0;    // widest bin (compact planes need <= 65,535)
    uint64_t z[HOPH_MAX_GROUPS] = {};
    DecideParams dp{};
    // psi on the device
    uint32_t *d_key = nullptr;   // packed (bin << key_bits) | offset, D entries
    uint32_t key_bits = 0;
    uint64_t *d_lo = nullptr;    // k + 1 bounds (hash path)
    uint64_t *d_kb = nullptr;    // k + 1 guarded join-key bases lo[w] + w + 1
    uint64_t hash_a = 0, hash_b = 0;
    uint32_t *d_minwise = nullptr;  // [D][minwise_k], psi_t(x) at x * mk + t
    // status word
    int32_t *d_status = nullptr;
    int32_t *h_status = nullptr;  // pinned mirror
    // scratch (lane 0; lanes 1.. serve the other blocks a self-join keeps in
    // flight, each on a stream of the plan's own)
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    static constexpr int kMaxLanes = 8;
    void *lane_scratch[kMaxLanes] = {};
    size_t lane_scratch_bytes[kMaxLanes] = {};
    cudaStream_t lane_stream[kMaxLanes] = {};
    cudaEvent_t lane_event[kMaxLanes] = {};
    cudaEvent_t fork_event = nullptr;
    hoph_exec exec{};
    // optional event timing of hoph_query_batch phases (bench / tooling)
    bool timing = false;
    std::vector<cudaEvent_t> events;  // kTimingMarks per recorded call
    size_t events_used = 0;
    int64_t launches = 0;  // kernels launched by library calls since last read
    // first-pass decision tables per comparison mode (device copies)
    uint16_t *d_table[4] = {nullptr, nullptr, nullptr, nullptr};
    int table_W[4] = {-1, -1, -1, -1};
    bool table_ok[4] = {false, false, false, false};
    std::vector<uint16_t> h_table[4];
};

// timing marks of one hoph_query_batch call: before the index, before the
// filter / dense scan, before the candidate counting, before the sort, end
constexpr int kTimingMarks = 5;

// record timing event `which` (0..kTimingMarks-1) of the current call
// when timing is on
void hoph_timing_mark(hoph_plan *plan, int which, cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device; the attribute is set only when it grows, so calls made
// while a stream is being captured issue no attribute change once warm.
cudaError_t hoph_ensure_smem(const void *func, int bytes);

// cudaOccupancyMaxActiveBlocksPerMultiprocessor, remembered per (kernel,
// device, block size, dynamic shared memory): host time off the launch path
cudaError_t hoph_occupancy(int *blocks, const void *func, int threads, size_t smem);

// grow-only scratch owned by the plan (one per lane, lane 0 for every call
// but a self-join's other blocks in flight): *out = at least `bytes`;
// HOPH_ERR_CAPTURE when it would have to grow while `stream` is being
// captured, HOPH_ERR_NOMEM when the allocation fails
int hoph_scratch(hoph_plan *plan, size_t bytes, int lane, cudaStream_t stream, void **out);

// true while `stream` is being captured into a graph
bool hoph_capturing(cudaStream_t stream);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void hoph_flag(int32_t *status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after `limit_ns` of wall
// time (2 s by default) or when another warp of the CTA raised *abort.
// Returns false on give-up (the caller records HOPH_ERR_TIMEOUT and leaves
// its loop).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  volatile int32_t *abort_flag,
                                                  uint64_t limit_ns = 2000000000ull) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
}

// 3-D tiled TMA load (box {x, y, z} from the tensor map) into shared memory,
// completing on the mbarrier's transaction count.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t x, int32_t y, int32_t z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 4-D tiled TMA load (box from the tensor map) into shared memory.
__device__ __forceinline__ void tma_load_4d(void *smem_dst, const CUtensorMap *map, uint64_t *bar,
                                            int32_t x, int32_t y, int32_t z, int32_t w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w),
        "r"(smem_u32(bar))
        : "memory");
}

// Prefetch a 4-D box of the tensor map into L2 (no shared memory, no barrier).
__device__ __forceinline__ void tma_prefetch_l2_4d(const CUtensorMap *map, int32_t x, int32_t y,
                                                   int32_t z, int32_t w) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w)
                 : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// named barrier among `nthreads` threads (ids 1..15; 0 is __syncthreads)
__device__ __forceinline__ void named_bar_sync(uint32_t id, uint32_t nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint4 ldg_nc_v4(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
