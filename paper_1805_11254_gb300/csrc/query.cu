// Comparison of query sketches against a device-resident collection:
// GOPH (Algorithm 1), (a:b)HOPH (Algorithm 2), plain OPH (Eq. 6) and MinWise.
//
// Two strategies give identical results.
//
// dense  - one persistent launch streams the scanned plane(s) through shared
//          memory (a producer warp issues 3-D TMA tile loads into a ring of
//          mbarrier-guarded stages); for every (query, row) pair, lanes
//          compare 32 bins at a time and __popc of __ballot_sync gives the
//          matched / both-empty / one-empty counts.  Cheap for a handful of
//          queries, ALU-bound for large batches.
// join   - an exact value join for large batches, in three parts:
//          (1) an index of the batch's first-group query values over the
//              keys lo[bin] + value (the value's position in psi-space): a
//              linked list of the queries of every key (one kernel, no
//              scan), and a 2-bit map recording whether an even- and whether
//              an odd-numbered query has the key;
//          (2) a streaming filter: TMA tiles of the first plane, a few lanes
//              per row, every row value looked up in the map in shared
//              memory.  A pair's match count is at most the row's number of
//              hits in the map of the query's parity group, and its
//              denominator at least the row's number of non-empty bins, so a
//              row whose hits in both groups are below the smallest rejection
//              threshold over the denominators it allows is rejected against
//              every query; the other rows are compacted into a candidate
//              list;
//          (3) a counting kernel over the candidates: per-query match counts
//              from the key lists in per-warp shared-memory counters, then the
//              exact first-group decision for each query the row met.
//          It needs "no match => reject" for every possible denominator,
//          checked on the host when the strategy is chosen.
// Pairs that continue after the first group are compacted into per-warp
// shared-memory lists and resolved lane-parallel: each lane gathers only
// its pair's later groups from HBM and applies the exact integer rule group
// by group.  Accepted pairs are appended with an atomic cursor and finally
// sorted by (query, row) by a single-CTA sort, so the output is
// deterministic.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kSurvCap = 32;  // per-warp survivor list (one entry per lane)
constexpr int kMaxW = 1024;   // scanned bins per row
constexpr int kStatWords = 3 * HOPH_MAX_GROUPS + 4;
constexpr uint64_t kMaxJoinKeys = 1ull << 23;  // key space indexing the list heads directly
constexpr uint64_t kDirectMap = 1ull << 19;    // key space indexed directly by the group map
constexpr uint64_t kHashedMapSlots = 1ull << 18;
constexpr int kSmemLimit = 227 * 1024;

struct Survivor {
    int64_t row;
    uint32_t q;
    uint16_t m1, k1;
};

// What every comparison kernel needs to score and finish a pair.
// Sketch planes hold uint32 values, or uint16 offsets in the compact form
// (every bin at most 65,535 values wide, empty marker 0xFFFF); kernels that
// read them are instantiated for both element types E.
template <typename E>
__host__ __device__ constexpr uint32_t empty_of() {
    return (uint32_t)(E)~(E)0;
}

struct PairArgs {
    const void *coll;  // E [G][n_rows][k']
    int64_t cstride;   // elements between collection planes
    const void *qry;   // E [G][n_q][k']
    int64_t qstride;   // elements between query planes
    int64_t n_rows;
    int32_t n_q;
    int32_t kg, Gs, W, G;
    uint32_t rule;
    const uint16_t *thr;  // rej[W+1], acc[W+1], row_min[W+1]
    DecideParams dp;      // rule for the later groups
    hoph_pair *out;
    int64_t cap;
    int64_t self_off;  // >= 0: self-join block, keep row > query, both shifted by it
    unsigned long long *out_count;
    unsigned long long *stat;  // kStatWords counters
    int32_t *status;
};

// stats layout: [0..15] entering, [16..31] accepted, [32..47] rejected,
// [48] later-group sketch bytes, [49] join hits

__host__ __device__ inline uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// MurmurHash3's 32-bit finalizer (Appleby): spreads keys over a power-of-two
// table when the key space is too large to index directly.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Slot of a key in the hashed group map of 2^(32 - shift) slots: the top bits
// of the key times 2^32 / golden ratio (Knuth's multiplicative hashing; two
// instructions per lookup in the filter).
__host__ __device__ __forceinline__ uint32_t map_slot(uint32_t key, uint32_t shift) {
    return (key * 0x9E3779B1u) >> shift;
}

constexpr unsigned long long kNoKey = ~0ull;  // empty slot of the key table
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
constexpr uint32_t kNil = 0xFFFFFFFFu;  // end of a key's query list

// Open-addressing key table (linear probing, at most half full): slot of
// `key`, inserted if absent.  Gives up (kNoSlot) after a full sweep.
__device__ __forceinline__ uint32_t table_insert(unsigned long long *tkey, uint32_t mask,
                                                 uint32_t key) {
    uint32_t slot = mix32(key) & mask;
    for (uint32_t i = 0; i <= mask; ++i) {
        const unsigned long long prev = atomicCAS(tkey + slot, kNoKey, (unsigned long long)key);
        if (prev == kNoKey || prev == (unsigned long long)key) return slot;
        slot = (slot + 1) & mask;
    }
    return kNoSlot;
}

__device__ __forceinline__ uint32_t table_find(const unsigned long long *tkey, uint32_t mask,
                                               uint32_t key) {
    uint32_t slot = mix32(key) & mask;
    for (uint32_t i = 0; i <= mask; ++i) {
        const unsigned long long k = __ldg(tkey + slot);
        if (k == (unsigned long long)key) return slot;
        if (k == kNoKey) return kNoSlot;
        slot = (slot + 1) & mask;
    }
    return kNoSlot;
}

__device__ __forceinline__ void emit_pair(const PairArgs &a, uint32_t q, int64_t row, int groups,
                                          int matches) {
    if (a.self_off >= 0) {  // one unordered pair per (i, j), i < j (checked again here)
        if (row <= (int64_t)q) return;
        q += (uint32_t)a.self_off;
        row += a.self_off;
    }
    const unsigned long long idx = atomicAdd(a.out_count, 1ull);
    if (idx < (unsigned long long)a.cap) {
        hoph_pair p;
        p.row = row;
        p.query = q;
        p.groups = (uint16_t)groups;
        p.matches = (uint16_t)matches;
        a.out[idx] = p;
    }
}

__host__ __device__ __forceinline__ int table_decide(const uint16_t *thr, int W, int m, int K) {
    return m < thr[K] ? HOPH_REJECT : (m >= thr[W + 1 + K] ? HOPH_ACCEPT : HOPH_CONTINUE);
}

// Lane-parallel resolution of the warp's survivor list: lane j finishes
// entry j by comparing the later groups of its pair one at a time.
template <typename E>
__device__ void resolve_survivors(const PairArgs &a, Survivor *list, uint32_t *nsurv,
                                  unsigned long long *s_stats) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const uint32_t n = min(*nsurv, (uint32_t)kSurvCap);
    if ((uint32_t)lane < n) {
        const Survivor sv = list[lane];
        int32_t Ms[HOPH_MAX_GROUPS], Ks[HOPH_MAX_GROUPS];
        Ms[0] = sv.m1;
        Ks[0] = sv.k1;
        int matches = sv.m1;
        for (int l = 2; l <= a.G; ++l) {
            const int g = l - 1;
            const E *rp = static_cast<const E *>(a.coll) + (int64_t)g * a.cstride + sv.row * a.kg;
            const E *qp = static_cast<const E *>(a.qry) + (int64_t)g * a.qstride + (int64_t)sv.q * a.kg;
            int32_t m = 0, both = 0, one = 0;
            for (int b = 0; b < a.kg; ++b) {
                const uint32_t rv = __ldg(rp + b), qv = __ldg(qp + b);
                const bool er = rv == empty_of<E>(), eq = qv == empty_of<E>();
                m += (!eq && rv == qv);
                both += (er && eq);
                one += (er != eq);
            }
            Ms[g] = m;
            Ks[g] = hoph_effective(a.rule, a.kg, both, one);
            matches += m;
            atomicAdd(s_stats + g, 1ull);
            atomicAdd(s_stats + 48, (unsigned long long)a.kg * 2 * sizeof(E));
            const int d = hoph_decide(a.dp, l, Ms, Ks);
            if (d == HOPH_ACCEPT) {
                atomicAdd(s_stats + 16 + g, 1ull);
                emit_pair(a, sv.q, sv.row, l, matches);
                break;
            }
            if (d == HOPH_REJECT) {
                atomicAdd(s_stats + 32 + g, 1ull);
                break;
            }
        }
    }
    __syncwarp();
    if (lane == 0) *nsurv = 0;
    __syncwarp();
}

// Append one survivor from one lane; false if the list is full.
__device__ __forceinline__ bool push_survivor(Survivor *list, uint32_t *nsurv, uint32_t q,
                                              int64_t row, int m1, int k1) {
    const uint32_t slot = atomicAdd(nsurv, 1u);
    if (slot >= (uint32_t)kSurvCap) {
        atomicSub(nsurv, 1u);
        return false;
    }
    Survivor s;
    s.row = row;
    s.q = q;
    s.m1 = (uint16_t)m1;
    s.k1 = (uint16_t)k1;
    list[slot] = s;
    return true;
}

// Fold a CTA's shared counters into the call's global counters.
__device__ __forceinline__ void flush_stats(const unsigned long long *s_stats,
                                            unsigned long long *g_stats, int lane) {
    for (int i = lane; i < kStatWords; i += 32)
        if (s_stats[i]) atomicAdd(g_stats + i, s_stats[i]);
}

// Producer side of a TMA stage ring: lane 0 of the producer warp issues one
// 3-D box load per tile of this CTA, then lets every issued copy land before
// the warp leaves (so no copy targets shared memory of a finished CTA).
__device__ void produce_tiles(const CUtensorMap *map, unsigned char *stages, uint64_t *full,
                              uint64_t *empty, volatile int32_t *abort_flag, int nstages,
                              uint32_t stage_bytes, uint32_t stage_stride, int64_t n_tiles,
                              int R, int32_t *status, bool four_d = false, int prefetch = 0,
                              int boxes = 1) {
    tma_prefetch_desc(map);
    int64_t it = 0;
    // 4-D maps: as each tile is issued, the CTA's tile `prefetch` strides
    // ahead is asked into L2, so more of the stream is in flight than the
    // shared-memory stages hold
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = (int)(it % nstages);
        const uint32_t use = (uint32_t)(it / nstages);
        if (use > 0 && !mbar_wait_bounded(empty + s, (use - 1) & 1, abort_flag)) {
            hoph_flag(status, HOPH_ERR_TIMEOUT);
            *abort_flag = 1;
            break;
        }
        mbar_arrive_expect_tx(full + s, stage_bytes);
        if (four_d) {
            // a tile of R rows as `boxes` boxes of R / boxes rows each
            const int64_t ahead = tile + (int64_t)prefetch * gridDim.x;
            const int br = R / boxes;
            const uint32_t bb = stage_bytes / (uint32_t)boxes;
            for (int b = 0; b < boxes; ++b) {
                if (prefetch > 0 && ahead < n_tiles)
                    tma_prefetch_l2_4d(map, 0, 0, (int32_t)(ahead * R + b * br), 0);
                tma_load_4d(stages + (size_t)s * stage_stride + (size_t)b * bb, map, full + s, 0,
                            0, (int32_t)(tile * R + b * br), 0);
            }
        }
        else
            tma_load_3d(stages + (size_t)s * stage_stride, map, full + s, 0, (int32_t)(tile * R),
                        0);
    }
    const int64_t issued = it;
    for (int64_t j = (issued > nstages ? issued - nstages : 0); j < issued; ++j) {
        const int s = (int)(j % nstages);
        if (!mbar_wait_bounded(full + s, (uint32_t)(j / nstages) & 1, abort_flag)) {
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(full + s, (uint32_t)(j / nstages) & 1) &&
                   global_ns() - t0 < 1000000000ull) {
            }
        }
    }
}

// ===========================================================================
// Dense strategy
// ===========================================================================
struct DenseArgs {
    PairArgs p;
    int32_t use_tma, tile_rows, stages, n_cons;
    int64_t n_tiles;
    uint32_t stage_bytes;   // bytes of one tile (the TMA transaction size)
    uint32_t stage_stride;  // stage_bytes rounded up to 128
};

struct DenseSmem {
    uint32_t bars, abort_flag, thr, toff, qoff, surv, nsurv, stats, stages, total;
};

__host__ __device__ inline DenseSmem dense_smem(const DenseArgs &a) {
    DenseSmem L;
    uint32_t o = 0;
    L.bars = o;       o += 16 * 8;  // full[8], empty[8]
    L.abort_flag = o; o += 16;
    L.thr = o;        o = align_up(o + 3 * (a.p.W + 1) * 2, 16);
    L.toff = o;       o = align_up(o + a.p.W * 4, 16);
    L.qoff = o;       o = align_up(o + a.p.W * 8, 16);
    L.surv = o;       o = align_up(o + a.n_cons * kSurvCap * (uint32_t)sizeof(Survivor), 16);
    L.nsurv = o;      o = align_up(o + a.n_cons * 4, 16);
    L.stats = o;      o = align_up(o + kStatWords * 8, 128);
    L.stages = o;     o += a.stages * a.stage_stride;
    L.total = o;
    return L;
}


// Every (query, row) pair of one tile; lanes over bins.  NCH > 0: the W
// scanned bins fit in NCH 32-bin chunks, and consecutive pairs of a warp
// share the query, whose values and empty masks stay in registers (qv, qem
// of query cur_q) from one tile to the next; NCH = 0: any W, nothing cached.
template <typename E, int NCH>
__device__ __forceinline__ void score_tile_dense(
    const PairArgs &a, int n_cons, const E *tile, int rows_here, int64_t row0,
    const int32_t *s_toff, const int64_t *s_qoff, const uint16_t *s_thr, Survivor *list,
    uint32_t *nsurv, unsigned long long *s_stats, int cw, unsigned long long &acc0,
    uint32_t (&qv)[NCH > 0 ? NCH : 1], uint32_t (&qem)[NCH > 0 ? NCH : 1], int &cur_q,
    const int32_t (&toff)[NCH > 0 ? NCH : 1]) {
    const int lane = threadIdx.x & 31;
    const int nch = (a.W + 31) >> 5;
    constexpr bool cached = NCH > 0;
    // the warp's pairs p = cw, cw + n_cons, ... of the tile in query-major
    // order, as (q, rl) = (p / rows_here, p % rows_here) advanced by steps
    int q = cw / rows_here, rl = cw - q * rows_here;
    for (; q < a.n_q; rl += n_cons) {
        while (rl >= rows_here) {
            rl -= rows_here;
            ++q;
        }
        if (q >= a.n_q) break;
        if (a.self_off >= 0 && row0 + rl <= (int64_t)q) continue;  // pair i >= j of a self-join
        const E *qb = static_cast<const E *>(a.qry) + (int64_t)q * a.kg;
        int m = 0, both = 0, one = 0;
        if constexpr (cached) {
            if (q != cur_q) {
                cur_q = q;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const int w = (c << 5) + lane;
                    const bool valid = w < a.W;
                    qv[c] = valid ? (uint32_t)__ldg(qb + s_qoff[w]) : 0u;
                    qem[c] = __ballot_sync(0xFFFFFFFFu, valid && qv[c] == empty_of<E>());
                }
            }
            const E *tr = tile + rl * a.kg;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int w = (c << 5) + lane;
                const bool valid = w < a.W;
                const uint32_t rv = valid ? (uint32_t)tr[toff[c]] : 0u;
                const uint32_t rem = __ballot_sync(0xFFFFFFFFu, valid && rv == empty_of<E>());
                m += __popc(__ballot_sync(0xFFFFFFFFu,
                                          valid && qv[c] != empty_of<E>() && rv == qv[c]));
                both += __popc(rem & qem[c]);
                one += __popc(rem ^ qem[c]);
            }
        } else {
            for (int c = 0; c < nch; ++c) {
                const int w = (c << 5) + lane;
                const bool valid = w < a.W;
                uint32_t rv = 0, q1 = 0;
                if (valid) {
                    rv = tile[s_toff[w] + rl * a.kg];
                    q1 = __ldg(qb + s_qoff[w]);
                }
                const bool er = rv == empty_of<E>(), eq = q1 == empty_of<E>();
                m += __popc(__ballot_sync(0xFFFFFFFFu, valid && !eq && rv == q1));
                both += __popc(__ballot_sync(0xFFFFFFFFu, valid && er && eq));
                one += __popc(__ballot_sync(0xFFFFFFFFu, valid && er != eq));
            }
        }
        const int K = hoph_effective(a.rule, a.W, both, one);
        const int d = table_decide(s_thr, a.W, m, K);
        if (d == HOPH_ACCEPT) {
            ++acc0;
            if (lane == 0) emit_pair(a, q, row0 + rl, 1, m);
        } else if (d == HOPH_CONTINUE) {
            if (*nsurv >= (uint32_t)kSurvCap) resolve_survivors<E>(a, list, nsurv, s_stats);
            if (lane == 0) push_survivor(list, nsurv, q, row0 + rl, m, K);
            __syncwarp();
        }
    }
}

// Up to 16 warps (15 consumers + the producer, four per SM sub-partition) x
// 112 registers fit the register file; the 8-chunk query cache needs about
// that many.
template <typename E, int NCH>
__global__ void __maxnreg__(112) dense_scan_kernel(const __grid_constant__ DenseArgs a,
                                                   const __grid_constant__ CUtensorMap map) {
    constexpr int NQ = NCH > 0 ? NCH : 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    const DenseSmem L = dense_smem(a);
    const PairArgs &P = a.p;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *empty = full + 8;
    volatile int32_t *abort_flag = reinterpret_cast<volatile int32_t *>(smem + L.abort_flag);
    uint16_t *s_thr = reinterpret_cast<uint16_t *>(smem + L.thr);
    int32_t *s_toff = reinterpret_cast<int32_t *>(smem + L.toff);
    int64_t *s_qoff = reinterpret_cast<int64_t *>(smem + L.qoff);
    Survivor *s_surv = reinterpret_cast<Survivor *>(smem + L.surv);
    uint32_t *s_nsurv = reinterpret_cast<uint32_t *>(smem + L.nsurv);
    unsigned long long *s_stats = reinterpret_cast<unsigned long long *>(smem + L.stats);
    unsigned char *stages = smem + L.stages;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = a.tile_rows;
    for (int i = tid; i < 3 * (P.W + 1); i += blockDim.x) s_thr[i] = P.thr[i];
    for (int w = tid; w < P.W; w += blockDim.x) {
        const int g = w / P.kg, b = w - g * P.kg;
        s_toff[w] = (g * R) * P.kg + b;
        s_qoff[w] = (int64_t)g * P.qstride + b;
    }
    for (int i = tid; i < a.n_cons; i += blockDim.x) s_nsurv[i] = 0;
    for (int i = tid; i < kStatWords; i += blockDim.x) s_stats[i] = 0;
    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, a.n_cons);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == a.n_cons) {
        if (a.use_tma && lane == 0)
            produce_tiles(&map, stages, full, empty, abort_flag, a.stages, a.stage_bytes,
                          a.stage_stride, a.n_tiles, R, P.status);
        return;
    }

    const int cw = warp;
    Survivor *list = s_surv + cw * kSurvCap;
    uint32_t *nsurv = s_nsurv + cw;
    unsigned long long acc0 = 0;
    uint32_t qv[NQ], qem[NQ];  // the warp's current query (cached path)
    int cur_q = -1;
    int32_t toff[NQ];  // tile offsets of this lane's bins (cached path)
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int w = (c << 5) + lane;
        toff[c] = w < P.W ? s_toff[w] : 0;
    }
    int s = 0;        // stage of the current tile
    uint32_t ph = 0;  // its mbarrier phase
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const E *tp = reinterpret_cast<const E *>(stages + (size_t)s * a.stage_stride);
        const int64_t row0 = tile * R;
        const int rows_here = (int)min((long long)R, (long long)(P.n_rows - row0));
        if (a.use_tma) {
            if (!mbar_wait_bounded(full + s, ph, abort_flag)) {
                hoph_flag(P.status, HOPH_ERR_TIMEOUT);
                *abort_flag = 1;
                ok = false;
                break;
            }
        } else {
            // plain cooperative load of the tile ([Gs][R][k'] layout)
            E *dst = reinterpret_cast<E *>(stages);
            const E *src = static_cast<const E *>(P.coll);
            const int per_plane = rows_here * P.kg;
            for (int idx = cw * 32 + lane; idx < P.Gs * per_plane; idx += a.n_cons * 32) {
                const int g = idx / per_plane, rem = idx - g * per_plane;
                dst[g * R * P.kg + rem] = src[(int64_t)g * P.cstride + row0 * P.kg + rem];
            }
            named_bar_sync(1, a.n_cons * 32);
        }
        score_tile_dense<E, NCH>(P, a.n_cons, tp, rows_here, row0, s_toff, s_qoff, s_thr, list, nsurv,
                            s_stats, cw, acc0, qv, qem, cur_q, toff);
        __syncwarp();
        if (a.use_tma) {
            if (lane == 0) mbar_arrive(empty + s);
            if (++s == a.stages) {
                s = 0;
                ph ^= 1u;
            }
        } else {
            named_bar_sync(1, a.n_cons * 32);
        }
    }
    if (ok && *nsurv) resolve_survivors<E>(P, list, nsurv, s_stats);
    if (lane == 0 && acc0) atomicAdd(s_stats + 16, acc0);
    named_bar_sync(1, a.n_cons * 32);
    if (cw == 0) flush_stats(s_stats, P.stat, lane);
}

// ===========================================================================
// Join strategy, part 1: index of the batch's scanned query values
// ===========================================================================
struct IndexArgs {
    const void *qry;     // E [G][n_q][k']
    int64_t qstride;
    int32_t n_q, kg, W, mask_words;
    const uint64_t *binbase;  // key = lo[w] + value
    uint32_t *head;      // [slots]: first entry of the key's list, kNil if none
    uint32_t *next;      // [n_q << wshift]: entry (q << wshift) | w -> next entry
    int32_t wshift;      // bits of a scanned-bin index
    uint32_t *gmap;      // per 16 map slots: an even / an odd query has slot j (bits j, 16 + j; swapped in odd words)
    int32_t map_hashed;  // map slot = map_slot(key, map_shift), else the key itself
    uint32_t map_shift;
    int32_t striped;     // striped map (filter_striped_kernel), else by key
    uint32_t nwb;        // striped map: words per (bin, lane) stack
    int32_t keys_hashed;  // key slot from the key table, else the key itself
    unsigned long long *tkey;
    uint32_t tmask;
    int32_t *status;
    uint32_t *q_emask;   // [n_q][mask_words]
    int32_t *allempty;
    uint32_t *n_allempty;
};

// Striped group map: a warp reads a row of W scanned values as 32-bit words,
// lane l taking words l, l + 32, ...; a bin is filed in the bank (word
// column) of the lane that reads it, and the bins of one lane are stacked.
template <typename E>
__host__ __device__ __forceinline__ uint32_t striped_lane(uint32_t w) {
    return sizeof(E) == 4 ? (w & 31u) : ((w >> 1) & 31u);
}
template <typename E>
__host__ __device__ __forceinline__ uint32_t striped_stack(uint32_t w) {
    return sizeof(E) == 4 ? (w >> 5) : (((w >> 6) << 1) | (w & 1u));
}

// A join batch's state reset in one launch: list heads to kNil, the group
// map and the call's counters to zero (out_count: null when the output
// accumulates over several calls).
__global__ void join_init_kernel(uint32_t *head, int64_t n_head, uint32_t *gmap, int64_t n_gmap,
                                 unsigned long long *st, int n_st, uint32_t *n_allempty,
                                 unsigned long long *n_cand, int64_t *out_count) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t; i < n_head; i += T) head[i] = kNil;
    for (int64_t i = t; i < n_gmap; i += T) gmap[i] = 0u;
    if (t < n_st) st[t] = 0ull;
    if (t == 0) {
        *n_allempty = 0u;
        *n_cand = 0ull;
        if (out_count) *out_count = 0;
    }
}

// warp per query: empty masks, all-empty list, the group map, and the
// queries of every key as a linked list (entry (q << wshift) | w pushed on
// the key's list)
template <typename E>
__global__ void join_count_kernel(const IndexArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= a.n_q) return;
    bool all_empty = true;
    for (int c = 0; c < a.mask_words; ++c) {
        const int w = (c << 5) + lane;
        const bool valid = w < a.W;
        uint32_t v = empty_of<E>();
        if (valid) {
            const int g = w / a.kg, b = w - g * a.kg;
            v = static_cast<const E *>(a.qry)[(int64_t)g * a.qstride + q * a.kg + b];
        }
        const bool e = v == empty_of<E>();
        const uint32_t em = __ballot_sync(0xFFFFFFFFu, valid && e);
        const uint32_t vm = __ballot_sync(0xFFFFFFFFu, valid);
        all_empty = all_empty && em == vm;
        if (lane == 0) a.q_emask[q * a.mask_words + c] = em;
        if (valid && !e) {
            const uint32_t key = (uint32_t)a.binbase[w] + v;
            if (a.striped) {
                // bin w lives in the bank of the lane that reads it (striped_lane),
                // in that lane's stack striped_stack; slot u = v + 1 (0 is the
                // empty bins' guard), word u >> 4 of the stack, the two group
                // bits as below with the halves swapped in odd words
                const uint32_t u = v + 1u;
                const uint32_t word =
                    (striped_stack<E>(w) * a.nwb + (u >> 4)) * 32u + striped_lane<E>(w);
                atomicOr(a.gmap + word,
                         1u << ((u & 15u) + ((((uint32_t)q ^ (u >> 4)) & 1u) << 4)));
            } else {
                const uint32_t mi = a.map_hashed ? map_slot(key, a.map_shift) : key;
                // slot j of word mi >> 4: even-query bit at j and odd-query bit at
                // 16 + j, the halves swapped in odd words, so a right rotation of
                // the word by (mi & 31) brings the even bit to 0 and the odd to 16
                const uint32_t word = mi >> 4;
                atomicOr(a.gmap + word,
                         1u << ((mi & 15u) + ((((uint32_t)q ^ word) & 1u) << 4)));
            }
            const uint32_t slot = a.keys_hashed ? table_insert(a.tkey, a.tmask, key) : key;
            if (slot == kNoSlot) {
                hoph_flag(a.status, HOPH_ERR_CAPACITY);
            } else {
                const uint32_t e = ((uint32_t)q << a.wshift) | (uint32_t)w;
                a.next[e] = atomicExch(a.head + slot, e);
            }
        }
    }
    if (lane == 0 && all_empty) a.allempty[atomicAdd(a.n_allempty, 1u)] = (int32_t)q;
}

// ===========================================================================
// Join strategy, part 2: streaming row filter (one lane per row)
// ===========================================================================
struct FilterArgs {
    int64_t n_rows;
    int32_t kg, Gs, W;
    int32_t tile_rows, n_cons, stages;  // tile_rows = n_cons * 32 / lanes_per_row
    int32_t lanes_per_row;              // W / lanes_per_row bins per lane (16 or 32)
    int64_t n_tiles;
    uint32_t stage_bytes, stage_stride;
    const uint32_t *gmap;     // 2-bit group map over the map slots (16-byte aligned,
                              // zero-padded to a multiple of 4 words)
    uint32_t gmap_words;      // the last word is zero: empty bins look up its slot 0
    uint32_t map_shift;       // hashed map: slot = map_slot(key, map_shift)
    uint32_t nwb;             // striped map: words per (bin, lane) stack
    int32_t boxes;            // TMA boxes per tile (striped: tiles above 256 rows)
    uint32_t stage_align;     // alignment of the stages' offset in shared memory
    const uint64_t *binbase;  // key = lo[w] + value
    const uint16_t *row_min;  // [W + 1]
    int32_t keep_empty;       // rows without a non-empty scanned bin are candidates
    uint32_t *cand;
    unsigned long long *n_cand;
    int32_t *status;
};

// join filter: tiles per CTA prefetched into L2 ahead of the TMA loads
constexpr int kFilterPrefetch = 1;

struct FilterSmem {
    uint32_t bars, abort_flag, row_min, gmap, stages, total;
};

__host__ __device__ inline FilterSmem filter_smem(const FilterArgs &a) {
    FilterSmem L;
    uint32_t o = 0;
    L.bars = o;       o += 16 * 8;
    L.abort_flag = o; o += 16;
    L.row_min = o;    o = align_up(o + (a.W + 1) * 2, 16);
    L.gmap = o;       o = align_up(o + a.gmap_words * 4, a.stage_align);
    L.stages = o;     o += a.stages * a.stage_stride;
    L.total = o;
    return L;
}

// Tiles arrive through a 4-D TMA box {32 bins, k'/32, rows, planes} with the
// 128-byte swizzle: in shared memory each 128-byte line (32 bins of one row)
// holds its 16-byte chunk c at position c ^ (line & 7), so the eight lanes of
// a shared-memory phase, reading the same chunk of eight consecutive lines,
// hit eight different banks.  Lane (r, sub) of a warp owns NPER consecutive
// bins of row r; their psi-space bases stay in registers.  MAXC bounds the
// consumer warps (16, or 31 for narrow rows: more warps hide the map lookups'
// latency at fewer registers per thread).
template <int NPER, bool HASHED, int MAXC, typename E>
__global__ void __launch_bounds__(32 * (MAXC + 1)) filter_kernel(const __grid_constant__ FilterArgs a,
                                                                 const __grid_constant__ CUtensorMap map) {
    constexpr int VPL = 128 / (int)sizeof(E);  // values per 128-byte line
    constexpr int VPC = 16 / (int)sizeof(E);   // values per 16-byte chunk
    extern __shared__ __align__(1024) unsigned char smem[];
    const FilterSmem L = filter_smem(a);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *empty = full + 8;
    volatile int32_t *abort_flag = reinterpret_cast<volatile int32_t *>(smem + L.abort_flag);
    uint16_t *s_rmin = reinterpret_cast<uint16_t *>(smem + L.row_min);
    const uint32_t *s_gmap = reinterpret_cast<const uint32_t *>(smem + L.gmap);
    unsigned char *stages = smem + L.stages;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = a.tile_rows;
    for (int i = tid; i <= a.W; i += blockDim.x) s_rmin[i] = a.row_min[i];
    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, a.n_cons);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == a.n_cons) {
        if (lane == 0)
            produce_tiles(&map, stages, full, empty, abort_flag, a.stages, a.stage_bytes,
                          a.stage_stride, a.n_tiles, R, a.status, true, kFilterPrefetch);
        return;
    }
    {
        // the consumers copy the group map (16-byte pieces; the map is padded
        // to a multiple of four words) while the first tiles are in flight
        const uint4 *src = reinterpret_cast<const uint4 *>(a.gmap);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.gmap);
        const uint32_t n4 = (a.gmap_words + 3) / 4;
        const uint32_t nt = (uint32_t)a.n_cons * 32;
#pragma unroll 4
        for (uint32_t i = tid; i < n4; i += nt) dst[i] = __ldg(src + i);
        named_bar_sync(1, nt);
    }

    const int lpr = a.lanes_per_row;
    const int rpw = 32 / lpr;
    const int r_in = lane / lpr, sub = lane - r_in * lpr;
    const int rl = warp * rpw + r_in;
    const int w0 = sub * NPER;                // first bin of this lane
    const int g = w0 / a.kg;                  // plane of the lane's bins
    const int lpr_row = a.kg / VPL;           // 128-byte lines per row and plane
    // line of (row rl, this lane's bins) within a tile, and the first chunk
    const int line = (g * R + rl) * lpr_row + (w0 - g * a.kg) / VPL;
    const int c0 = (w0 % VPL) / VPC;
    uint32_t kb[NPER];
#pragma unroll
    for (int i = 0; i < NPER; ++i) kb[i] = (uint32_t)a.binbase[w0 + i];

    const uint32_t zero_slot = (a.gmap_words - 1) * 16;
    int s = 0;          // stage of the current tile
    uint32_t ph = 0;    // its mbarrier phase
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const unsigned char *lp = stages + (size_t)s * a.stage_stride + (size_t)line * 128;
        // the swizzle XORs the chunk index with bits 7..9 of the line's address
        const int xr = (int)(smem_u32(lp) >> 7) & 7;
        const int64_t row = tile * R + rl;
        if (!mbar_wait_bounded(full + s, ph, abort_flag)) {
            hoph_flag(a.status, HOPH_ERR_TIMEOUT);
            *abort_flag = 1;
            break;
        }
        // this lane's share: hits = even-group hits | odd-group hits << 16
        // (one map word gives both bits of a key 16 apart), ne = non-empty bins;
        // an empty bin looks up the zero word, so nothing branches
        uint32_t hits = 0, ne = 0;
        if (row < a.n_rows) {
#pragma unroll
            for (int c = 0; c < NPER / VPC; ++c) {
                const uint4 v = *reinterpret_cast<const uint4 *>(lp + (((c0 + c) ^ xr) << 4));
                uint32_t x[VPC];
                if constexpr (VPC == 4) {
                    x[0] = v.x;
                    x[1] = v.y;
                    x[2] = v.z;
                    x[3] = v.w;
                } else {
                    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        x[2 * h] = wv[h] & 0xFFFFu;
                        x[2 * h + 1] = wv[h] >> 16;
                    }
                }
#pragma unroll
                for (int e = 0; e < VPC; ++e) {
                    const bool full_bin = x[e] != empty_of<E>();
                    const uint32_t key = kb[c * VPC + e] + x[e];
                    uint32_t mi = HASHED ? map_slot(key, a.map_shift) : key;
                    // direct map, uint32 values: the empty marker lands on the
                    // bin's guard key (base - 1), which no query sets
                    if (HASHED || sizeof(E) != 4) mi = full_bin ? mi : zero_slot;
                    const uint32_t w = s_gmap[mi >> 4];
                    hits += __funnelshift_r(w, w, mi) & 0x10001u;
                    ne += full_bin;
                }
            }
        }
        for (int o = 1; o < lpr; o <<= 1) {
            hits += __shfl_xor_sync(0xFFFFFFFFu, hits, o);
            ne += __shfl_xor_sync(0xFFFFFFFFu, ne, o);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
        bool pass = false;
        if (sub == 0 && row < a.n_rows) {
            const int h = (int)max(hits & 0xFFFFu, hits >> 16);
            pass = ne == 0 ? (a.keep_empty != 0) : (h >= (int)s_rmin[ne]);
        }
        const uint32_t pm = __ballot_sync(0xFFFFFFFFu, pass);
        if (pm) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.n_cand, (unsigned long long)__popc(pm));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (pass) a.cand[base + __popc(pm & ((1u << lane) - 1u))] = (uint32_t)row;
        }
        if (++s == a.stages) {
            s = 0;
            ph ^= 1u;
        }
    }
}

__device__ __forceinline__ uint32_t umad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Join filter over a striped group map (lanes over bins).  A warp takes 32
// rows at a time; for each, lane l reads 32-bit words l, l + 32, ... of the row
// (NW words, 4 / sizeof(E) values each), so the 32 lanes look up 32 different
// banks of the map and every lookup is one shared-memory wavefront.  A lane
// keeps one packed partial count per row (even-group hits in bits 0-7,
// odd-group hits 16-23; uint32 values: non-empty bins in 8-15; 16-bit values:
// empty low halves in 8-15 and empty high halves in 24-31; W <= 128 keeps each
// below 256) and five butterfly steps (exchange half of the rows with the
// partner lane, add the other half) leave lane r with row r's totals, so every
// lane decides one row.  Tiles come through an unswizzled 4-D box
// {v, k'/v, rows, 1}: row r's values are contiguous; tile_rows is a multiple
// of 32 and the stages start on a multiple of 32 rows' bytes.
template <typename E, int NW>
__global__ void __launch_bounds__(32 * 17, 1) filter_striped_kernel(const __grid_constant__ FilterArgs a,
                                                               const __grid_constant__ CUtensorMap map) {
    constexpr int VPW = 4 / (int)sizeof(E);  // values per 32-bit word
    constexpr int NS = NW * VPW;             // values (map stacks) per lane
    constexpr uint32_t RB = 128u * NW;       // bytes of a row
    extern __shared__ __align__(1024) unsigned char smem[];
    const FilterSmem L = filter_smem(a);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint64_t *empty = full + 8;
    volatile int32_t *abort_flag = reinterpret_cast<volatile int32_t *>(smem + L.abort_flag);
    uint16_t *s_rmin = reinterpret_cast<uint16_t *>(smem + L.row_min);
    unsigned char *stages = smem + L.stages;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = a.tile_rows;
    for (int i = tid; i <= a.W; i += blockDim.x) s_rmin[i] = a.row_min[i];
    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, a.n_cons);
        }
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == a.n_cons) {
        if (lane == 0)
            produce_tiles(&map, stages, full, empty, abort_flag, a.stages, a.stage_bytes,
                          a.stage_stride, a.n_tiles, R, a.status, true, kFilterPrefetch,
                          a.boxes);
        return;
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.gmap);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + L.gmap);
        const uint32_t n4 = (a.gmap_words + 3) / 4;
        const uint32_t nt = (uint32_t)a.n_cons * 32;
#pragma unroll 4
        for (uint32_t i = tid; i < n4; i += nt) dst[i] = __ldg(src + i);
        named_bar_sync(1, nt);
    }
    // offset in shared memory of (stack s, word row 0) in this lane's bank
    uint32_t sbase[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s)
        sbase[s] = L.gmap + ((uint32_t)s * a.nwb * 32u + (uint32_t)lane) * 4u;
    const int keep_empty = a.keep_empty;
    const uint32_t W = (uint32_t)a.W;
    // 1, 8, 128 and 2^16 as values the compiler cannot fold into shifts and
    // adds (the multiply-adds run on the FMA pipe, beside the ALU pipe that
    // the shifts, rotates and masks keep busy)
    const uint32_t one = a.stages > 0 ? 1u : 0u, k8 = one << 3, k128 = one << 7, k64k = one << 16;
    // this lane's word l of row (32-row group base) ^ (j << 7): the group's
    // offset is a multiple of 32 rows' bytes, so OR-ing in the lane's row and
    // word is an addition
    const uint32_t lane_off = (uint32_t)lane * RB | (uint32_t)lane * 4u;

    int s = 0;
    uint32_t ph = 0;
    for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        if (!mbar_wait_bounded(full + s, ph, abort_flag)) {
            hoph_flag(a.status, HOPH_ERR_TIMEOUT);
            *abort_flag = 1;
            break;
        }
        const uint32_t st_off = L.stages + (uint32_t)s * a.stage_stride;
        const int64_t row0 = tile * R;
        const int rows = (int)(a.n_rows - row0 < (int64_t)R ? a.n_rows - row0 : (int64_t)R);
        // groups of 32 rows, dealt round-robin over the warps; rows past the
        // collection's end (a ragged last tile) are looked up but never kept
        for (int r0 = warp * 32; r0 < rows; r0 += a.n_cons * 32) {
            const uint32_t q_off = (st_off + (uint32_t)r0 * RB) | lane_off;
            // acc[j] of lane l counts row r0 + (j ^ l): the butterfly below then
            // always keeps the low half of its slots and sends the high half
            uint32_t acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const unsigned char *rp = smem + (q_off ^ ((uint32_t)j * RB));
                uint32_t t = 0;
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    const uint32_t word = *reinterpret_cast<const uint32_t *>(rp + 128 * i);
                    // slot u = value + 1 (the empty marker wraps to slot 0, the guard);
                    // the word of slot u in its stack is u >> 4, 128 bytes a row
                    if constexpr (VPW == 1) {
                        const uint32_t u = word + 1u;
                        const uint32_t mw = *reinterpret_cast<const uint32_t *>(
                            smem + sbase[i] + ((u & ~15u) << 3));
                        t += (__funnelshift_r(mw, mw, u) & 0x10001u) + (u != 0u ? 0x100u : 0u);
                    } else {
                        // low slot: word + 1 (a carry into the high half is never
                        // read); high slot: word + 2^16, wrapping out of the word.
                        // The rotations read only the low five bits of their amount
                        const uint32_t w1 = umad(word, one, one);
                        const uint32_t w2 = umad(one, k64k, word);
                        const uint32_t m0 = *reinterpret_cast<const uint32_t *>(
                            smem + umad(w1 & 0xFFF0u, k8, sbase[2 * i]));
                        const uint32_t m1 = *reinterpret_cast<const uint32_t *>(
                            smem + umad(w2 >> 20, k128, sbase[2 * i + 1]));
                        t += (__funnelshift_r(m0, m0, w1) & 0x10001u) +
                             (__funnelshift_r(m1, m1, w2 >> 16) & 0x10001u);
                        // empty halves: a stored offset is below 2^15 (a bin has at
                        // most nwb * 16 - 1 <= 32767 values), the empty marker has
                        // bit 15 set; bits 15 and 31 land on 8 and 24
                        t += (word >> 7) & 0x01000100u;
                    }
                }
                acc[j] = t;
            }
            // butterfly: at step o, slot j < o of lane l holds row r0 + (j ^ l), whose
            // partner-lane share sits in the partner's slot j + o (the same row:
            // (j + o) ^ (l ^ o) = j ^ l); after the last step slot 0 is row r0 + l
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
                for (int j = 0; j < o; ++j)
                    acc[j] = umad(__shfl_xor_sync(0xFFFFFFFFu, acc[j + o], o), one, acc[j]);
            }
            const uint32_t tot = acc[0];  // row r0 + lane
            const uint32_t ne =
                VPW == 1 ? (tot >> 8) & 0xFFu : W - (((tot >> 8) & 0xFFu) + (tot >> 24));
            const uint32_t hh = max(tot & 0xFFu, (tot >> 16) & 0xFFu);
            const bool pass = (r0 + lane < rows) &&
                              (ne == 0 ? keep_empty != 0 : hh >= (uint32_t)s_rmin[ne]);
            const uint32_t pm = __ballot_sync(0xFFFFFFFFu, pass);
            if (pm) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.n_cand, (unsigned long long)__popc(pm));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (pass)
                    a.cand[base + __popc(pm & ((1u << lane) - 1u))] = (uint32_t)(row0 + r0 + lane);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
        if (++s == a.stages) {
            s = 0;
            ph ^= 1u;
        }
    }
}

// ===========================================================================
// Join strategy, part 3: per-query counts of the candidate rows
// ===========================================================================
struct CountArgs {
    PairArgs p;
    const uint32_t *cand;
    const unsigned long long *n_cand;
    const uint64_t *binbase;  // key = lo[w] + value
    int32_t keys_hashed;       // key slots from the key table
    const unsigned long long *tkey;
    uint32_t tmask;
    const uint32_t *head;     // key slot -> first entry of its query list
    const uint32_t *next;     // entry -> next entry
    int32_t wshift;           // query of an entry = entry >> wshift
    const uint32_t *q_emask;  // [n_q][mask_words]
    int32_t mask_words;
    const int32_t *allempty;
    const uint32_t *n_allempty;
};

// four warps and about 7 KB of shared memory a CTA (1,024 queries), so that
// a counting CTA fits on an SM beside a running filter CTA of another batch
constexpr int kCountThreads = 128;
constexpr int kCountWarps = kCountThreads / 32;

// a warp's per-query match counters: 8 bits each when a row has fewer than
// 256 scanned bins (a count never exceeds W), else 16
__host__ __device__ inline int count_lg(int W) { return W < 256 ? 2 : 1; }  // log2 per word
__host__ __device__ inline int count_words(int n_q, int W) {
    const int per = 1 << count_lg(W);
    return (n_q + per - 1) / per;
}

struct CountSmem {
    uint32_t thr, woff, counters, rowmask, surv, nsurv, stats, total;
};

__host__ __device__ inline CountSmem count_smem(const CountArgs &a) {
    CountSmem L;
    uint32_t o = 0;
    L.thr = o;      o = align_up(o + 3 * (a.p.W + 1) * 2, 16);
    L.woff = o;     o = align_up(o + a.p.W * 8, 16);
    L.counters = o; o = align_up(o + kCountWarps * count_words(a.p.n_q, a.p.W) * 4, 16);
    L.rowmask = o;  o = align_up(o + kCountWarps * a.mask_words * 4, 16);
    L.surv = o;     o = align_up(o + kCountWarps * kSurvCap * (uint32_t)sizeof(Survivor), 16);
    L.nsurv = o;    o = align_up(o + kCountWarps * 4, 16);
    L.stats = o;    o = align_up(o + kStatWords * 8, 16);
    L.total = o;
    return L;
}

// NCH = 32-bin chunks per row (W <= 32 * NCH).  Each lane keeps its chunks'
// values and list heads in registers between the counting and evaluation
// passes, and the next candidate row's values are loaded while the current
// one is counted.
template <int NCH, typename E>
__global__ void __launch_bounds__(kCountThreads, 6) count_kernel(const __grid_constant__ CountArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const CountSmem L = count_smem(a);
    const PairArgs &P = a.p;
    uint16_t *s_thr = reinterpret_cast<uint16_t *>(smem + L.thr);
    int64_t *s_woff = reinterpret_cast<int64_t *>(smem + L.woff);
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + L.counters);
    uint32_t *s_rowmask = reinterpret_cast<uint32_t *>(smem + L.rowmask);
    Survivor *s_surv = reinterpret_cast<Survivor *>(smem + L.surv);
    uint32_t *s_nsurv = reinterpret_cast<uint32_t *>(smem + L.nsurv);
    unsigned long long *s_stats = reinterpret_cast<unsigned long long *>(smem + L.stats);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cwords = count_words(P.n_q, P.W);
    // counter of query q: bits [csh(q), csh(q) + cbits) of word q >> clg
    const uint32_t clg = (uint32_t)count_lg(P.W), cbits = 32u >> clg;
    const uint32_t cmask = (1u << cbits) - 1u, csel = (1u << clg) - 1u;
    for (int i = tid; i < 3 * (P.W + 1); i += blockDim.x) s_thr[i] = P.thr[i];
    for (int w = tid; w < P.W; w += blockDim.x) {
        const int g = w / P.kg, b = w - g * P.kg;
        s_woff[w] = (int64_t)g * P.cstride + b;
    }
    for (int i = tid; i < kCountWarps * cwords; i += blockDim.x) s_cnt[i] = 0;
    for (int i = tid; i < kCountWarps; i += blockDim.x) s_nsurv[i] = 0;
    for (int i = tid; i < kStatWords; i += blockDim.x) s_stats[i] = 0;
    __syncthreads();

    uint32_t *cnt = s_cnt + warp * cwords;
    uint32_t *rowmask = s_rowmask + warp * a.mask_words;
    Survivor *list = s_surv + warp * kSurvCap;
    uint32_t *nsurv = s_nsurv + warp;
    const uint16_t *row_min = s_thr + 2 * (P.W + 1);
    const int n_allempty = (int)*a.n_allempty;
    // a pair of all-empty scans has M = 0 and K = the rule's effective bins
    const int d00 = table_decide(s_thr, P.W, 0, hoph_effective(P.rule, P.W, P.W, 0));
    const unsigned long long n_cand = *a.n_cand;
    const unsigned long long stride = (unsigned long long)gridDim.x * kCountWarps;
    unsigned long long acc0 = 0, hits = 0;

    int64_t woff[NCH];
    uint32_t kbase[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int w = (c << 5) + lane;
        woff[c] = w < P.W ? s_woff[w] : -1;
        kbase[c] = w < P.W ? (uint32_t)a.binbase[w] : 0u;
    }
    auto load_row = [&](unsigned long long ci, uint32_t *v) {
        const int64_t row = a.cand[ci];
        const E *rb = static_cast<const E *>(P.coll) + row * P.kg;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
            v[c] = woff[c] >= 0 ? (uint32_t)__ldg(rb + woff[c]) : empty_of<E>();
        return row;
    };

    unsigned long long ci = (unsigned long long)blockIdx.x * kCountWarps + warp;
    uint32_t vn[NCH];
    int64_t row_n = ci < n_cand ? load_row(ci, vn) : 0;
    for (; ci < n_cand; ci += stride) {
        uint32_t v[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) v[c] = vn[c];
        const int64_t row = row_n;
        if (ci + stride < n_cand) row_n = load_row(ci + stride, vn);

        int ne = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const bool valid = woff[c] >= 0;
            const bool fullb = valid && v[c] != empty_of<E>();
            const uint32_t em = __ballot_sync(0xFFFFFFFFu, valid && !fullb);
            if (lane == 0 && c < a.mask_words) rowmask[c] = em;
            ne += __popc(__ballot_sync(0xFFFFFFFFu, fullb));
        }
        if (ne == 0) {
            // pairs whose scanned bins are empty on both sides
            if (n_allempty > 0 && d00 != HOPH_REJECT) {
                for (int base = 0; base < n_allempty; base += 32) {
                    if (*nsurv + 32 > (uint32_t)kSurvCap) resolve_survivors<E>(P, list, nsurv, s_stats);
                    const uint32_t q =
                        base + lane < n_allempty ? (uint32_t)a.allempty[base + lane] : 0u;
                    if (base + lane < n_allempty && (P.self_off < 0 || row > (int64_t)q)) {
                        if (d00 == HOPH_ACCEPT) {
                            ++acc0;
                            emit_pair(P, q, row, 1, 0);
                        } else {
                            push_survivor(list, nsurv, q, row, 0, 0);
                        }
                    }
                    __syncwarp();
                }
            }
            continue;
        }
        const int need = row_min[ne];
        // a self-join block pairs a row only with the queries before it
        const uint32_t qlim = P.self_off >= 0 ? (uint32_t)min(row, (int64_t)P.n_q) : (uint32_t)P.n_q;
        // counting pass: the query list of every chunk's key, then counts
        uint32_t f[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            f[c] = kNil;
            if (woff[c] >= 0 && v[c] != empty_of<E>()) {
                const uint32_t key = kbase[c] + v[c];
                const uint32_t slot = a.keys_hashed ? table_find(a.tkey, a.tmask, key) : key;
                if (slot != kNoSlot) f[c] = __ldg(a.head + slot);
            }
        }
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            for (uint32_t e = f[c]; e != kNil; e = __ldg(a.next + e)) {
                const uint32_t q = e >> a.wshift;
                if (q < qlim) {
                    atomicAdd(cnt + (q >> clg), 1u << ((q & csel) * cbits));
                    ++hits;
                }
            }
        }
        __syncwarp();
        // evaluation: each distinct hit query is taken by the first lane that
        // clears its counter; resumable so a full survivor list can drain
        int c = 0;
        uint32_t i = f[0];
        bool done = false;
        while (true) {
            while (!done) {
                // advance to the next (chunk, list entry) of this lane
                if (i == kNil) {
                    if (++c >= NCH) {
                        done = true;
                        break;
                    }
#pragma unroll
                    for (int cc = 0; cc < NCH; ++cc)
                        if (cc == c) i = f[cc];
                    continue;
                }
                // (a query at or past qlim was not counted: m = 0 below)
                const uint32_t q = i >> a.wshift;
                const uint32_t sh = (q & csel) * cbits;
                const uint32_t old = atomicAnd(cnt + (q >> clg), ~(cmask << sh));
                const int m = (int)((old >> sh) & cmask);
                if (m >= need) {
                    int both = 0, one = 0;
                    const uint32_t *qm = a.q_emask + (int64_t)q * a.mask_words;
                    for (int j = 0; j < a.mask_words; ++j) {
                        const uint32_t x = __ldg(qm + j), y = rowmask[j];
                        both += __popc(x & y);
                        one += __popc(x ^ y);
                    }
                    const int K = hoph_effective(P.rule, P.W, both, one);
                    const int d = table_decide(s_thr, P.W, m, K);
                    if (d == HOPH_ACCEPT) {
                        ++acc0;
                        emit_pair(P, q, row, 1, m);
                    } else if (d == HOPH_CONTINUE) {
                        if (!push_survivor(list, nsurv, q, row, m, K)) {
                            atomicAdd(cnt + (q >> clg), (uint32_t)m << sh);  // retry later
                            break;
                        }
                    }
                }
                i = __ldg(a.next + i);
            }
            const bool all_done = __all_sync(0xFFFFFFFFu, done);
            __syncwarp();
            if (*nsurv >= (uint32_t)kSurvCap / 2 || !all_done)
                resolve_survivors<E>(P, list, nsurv, s_stats);
            if (all_done) break;
        }
        __syncwarp();
    }
    if (*nsurv) resolve_survivors<E>(P, list, nsurv, s_stats);
    for (int o = 16; o; o >>= 1) {
        acc0 += __shfl_xor_sync(0xFFFFFFFFu, acc0, o);
        hits += __shfl_xor_sync(0xFFFFFFFFu, hits, o);
    }
    if (lane == 0) {
        if (acc0) atomicAdd(s_stats + 16, acc0);
        if (hits) atomicAdd(s_stats + 49, hits);
    }
    __syncthreads();
    if (warp == 0) flush_stats(s_stats, P.stat, lane);
}

template <int NCH, typename E>
int launch_count(const CountArgs &ca, uint32_t smem, int num_sms, cudaStream_t s) {
    auto kern = count_kernel<NCH, E>;
    HOPH_CUDA_TRY(hoph_ensure_smem((const void *)kern, (int)smem));
    int per = 0;
    HOPH_CUDA_TRY(hoph_occupancy(&per, (const void *)kern, kCountThreads, smem));
    if (per < 1) return HOPH_ERR_UNSUPPORTED;
    kern<<<(unsigned)(num_sms * per), kCountThreads, smem, s>>>(ca);
    HOPH_CUDA_TRY(cudaGetLastError());
    return HOPH_OK;
}

// ===========================================================================
// Deterministic output order: sort the accepted pairs by (query, row)
// ===========================================================================
constexpr int kSortThreads = 1024;
constexpr int kSortSmem = 8192;  // records sorted in shared memory at once (many-CTA sort)
// the one-CTA sort (capacities up to kSortOneCta): runs of 512 records in 8 KB
// and 256 threads, small enough to share an SM with a running filter CTA
constexpr int kSmallSortThreads = 256;
constexpr int kSmallSortRun = 512;

__device__ __forceinline__ unsigned long long pair_key(const hoph_pair &p) {
    return ((unsigned long long)p.query << 40) | (unsigned long long)p.row;
}

__device__ void bitonic_smem(ulonglong2 *v, int m) {
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < m / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const ulonglong2 x = v[lo], y = v[hi];
                if ((x.x > y.x) == up) {
                    v[lo] = y;
                    v[hi] = x;
                }
            }
            __syncthreads();
        }
}

__device__ int64_t lower_bound_key(const ulonglong2 *a, int64_t n, unsigned long long k) {
    int64_t l = 0, h = n;
    while (l < h) {
        const int64_t m = (l + h) >> 1;
        if (a[m].x < k) l = m + 1; else h = m;
    }
    return l;
}

// The call's counters folded into the caller's hoph_stats (one thread).
struct StatsFold {
    const unsigned long long *st;
    const unsigned long long *n_cand;  // null for the dense scan
    int64_t pairs, first_pass_bytes;
    int32_t G, Gs, strategy;
    hoph_stats *out;                   // null: no statistics wanted
};

__device__ void stats_fold(const StatsFold &f) {
    if (!f.out) return;
    const unsigned long long *st = f.st;
    const int64_t pairs = f.pairs;
    const int G = f.G, Gs = f.Gs;
    hoph_stats *out = f.out;
    // atomic: a self-join's blocks in flight fold into the same statistics
    auto add = [](int64_t *dst, int64_t v) {
        if (v) atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)v);
    };
    add(&out->entering[0], pairs);
    const int64_t acc0 = (int64_t)st[16], cont = (Gs < G) ? (int64_t)st[1] : 0;
    add(&out->accepted[0], acc0);
    add(&out->rejected[0], pairs - acc0 - cont);
    for (int g = 1; g < G && Gs < G; ++g) {
        add(&out->entering[g], (int64_t)st[g]);
        add(&out->accepted[g], (int64_t)st[16 + g]);
        add(&out->rejected[g], (int64_t)st[32 + g]);
    }
    add(&out->sketch_bytes, f.first_pass_bytes + (int64_t)st[48]);
    add(&out->join_hits, (int64_t)st[49]);
    if (f.n_cand) add(&out->rows_counted, (int64_t)*f.n_cand);
    out->strategy = f.strategy;
}

__global__ void stats_fold_kernel(const StatsFold f) {
    if (threadIdx.x == 0) stats_fold(f);
}

// Sort the accepted pairs by (query, row); thread 0 also folds the statistics.
__global__ void __launch_bounds__(kSmallSortThreads) sort_pairs_kernel(
    hoph_pair *out, const unsigned long long *count, int64_t cap, ulonglong2 *bufA,
    ulonglong2 *bufB, int32_t *status, const StatsFold f) {
    extern __shared__ __align__(1024) unsigned char smem[];
    ulonglong2 *sv = reinterpret_cast<ulonglong2 *>(smem);
    if (threadIdx.x == 0) stats_fold(f);
    const unsigned long long total = *count;
    if (total > (unsigned long long)cap && threadIdx.x == 0) hoph_flag(status, HOPH_ERR_CAPACITY);
    const int64_t n = (int64_t)min(total, (unsigned long long)cap);
    if (n <= 1) return;
    // sort runs of kSmallSortRun records in shared memory into bufA
    for (int64_t base = 0; base < n; base += kSmallSortRun) {
        const int cnt = (int)min((long long)kSmallSortRun, (long long)(n - base));
        int m = 1;
        while (m < cnt) m <<= 1;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            if (i < cnt) {
                const hoph_pair p = out[base + i];
                sv[i] = make_ulonglong2(pair_key(p),
                                        ((unsigned long long)p.groups << 16) | p.matches);
            } else {
                sv[i] = make_ulonglong2(~0ull, 0ull);
            }
        }
        __syncthreads();
        bitonic_smem(sv, m);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) bufA[base + i] = sv[i];
        __syncthreads();
    }
    // merge sorted runs (keys are unique: rank = own index + rank in the other run)
    ulonglong2 *src = bufA, *dst = bufB;
    for (int64_t run = kSmallSortRun; run < n; run <<= 1) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const int64_t pairbase = (i / (2 * run)) * (2 * run);
            const int64_t a0 = pairbase, a1 = min(pairbase + run, n);
            const int64_t b0 = a1, b1 = min(pairbase + 2 * run, n);
            int64_t pos;
            if (i < a1)
                pos = pairbase + (i - a0) + lower_bound_key(src + b0, b1 - b0, src[i].x);
            else
                pos = pairbase + (i - b0) + lower_bound_key(src + a0, a1 - a0, src[i].x);
            dst[pos] = src[i];
        }
        __syncthreads();
        ulonglong2 *t = src;
        src = dst;
        dst = t;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const ulonglong2 r = src[i];
        hoph_pair p;
        p.query = (uint32_t)(r.x >> 40);
        p.row = (int64_t)(r.x & ((1ull << 40) - 1));
        p.groups = (uint16_t)(r.y >> 16);
        p.matches = (uint16_t)(r.y & 0xFFFFu);
        out[i] = p;
    }
}

// Outputs larger than kSortOneCta records of capacity are sorted by many CTAs
// in a launch sequence (the count is known only on the device, so the host
// launches the passes a full buffer needs and those past the count return at
// once): sort_runs_kernel sorts runs of kSortSmem records in shared memory,
// CTAs striding over the runs; one merge_pass_kernel per doubling of the run
// length merges pairs of sorted runs, every record placed by its rank in the
// other run; sort_finish_kernel writes the result (in bufA or bufB, by the
// parity of the passes that did work) back as hoph_pair records and folds the
// statistics.
constexpr int64_t kSortOneCta = 1 << 16;

__device__ __forceinline__ hoph_pair unpack_pair(const ulonglong2 r) {
    hoph_pair p;
    p.query = (uint32_t)(r.x >> 40);
    p.row = (int64_t)(r.x & ((1ull << 40) - 1));
    p.groups = (uint16_t)(r.y >> 16);
    p.matches = (uint16_t)(r.y & 0xFFFFu);
    return p;
}

__global__ void __launch_bounds__(kSortThreads) sort_runs_kernel(const hoph_pair *out,
                                                                 const unsigned long long *count,
                                                                 int64_t cap, ulonglong2 *bufA) {
    extern __shared__ __align__(1024) unsigned char smem[];
    ulonglong2 *sv = reinterpret_cast<ulonglong2 *>(smem);
    const int64_t n = (int64_t)min(*count, (unsigned long long)cap);
    for (int64_t base = (int64_t)blockIdx.x * kSortSmem; base < n;
         base += (int64_t)gridDim.x * kSortSmem) {
        const int cnt = (int)min((long long)kSortSmem, (long long)(n - base));
        int m = 1;
        while (m < cnt) m <<= 1;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            if (i < cnt) {
                const hoph_pair p = out[base + i];
                sv[i] = make_ulonglong2(pair_key(p),
                                        ((unsigned long long)p.groups << 16) | p.matches);
            } else {
                sv[i] = make_ulonglong2(~0ull, 0ull);
            }
        }
        __syncthreads();
        bitonic_smem(sv, m);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) bufA[base + i] = sv[i];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) merge_pass_kernel(const ulonglong2 *src, ulonglong2 *dst,
                                                         const unsigned long long *count,
                                                         int64_t cap, int64_t run) {
    const int64_t n = (int64_t)min(*count, (unsigned long long)cap);
    if (run >= n) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pairbase = (i / (2 * run)) * (2 * run);
        const int64_t a0 = pairbase, a1 = min(pairbase + run, n);
        const int64_t b0 = a1, b1 = min(pairbase + 2 * run, n);
        const ulonglong2 v = src[i];
        int64_t pos;
        if (i < a1)
            pos = pairbase + (i - a0) + lower_bound_key(src + b0, b1 - b0, v.x);
        else
            pos = pairbase + (i - b0) + lower_bound_key(src + a0, a1 - a0, v.x);
        dst[pos] = v;
    }
}

__global__ void __launch_bounds__(256) sort_finish_kernel(hoph_pair *out,
                                                          const unsigned long long *count,
                                                          int64_t cap, const ulonglong2 *bufA,
                                                          const ulonglong2 *bufB, int32_t *status,
                                                          const StatsFold f) {
    const unsigned long long total = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats_fold(f);
        if (total > (unsigned long long)cap) hoph_flag(status, HOPH_ERR_CAPACITY);
    }
    const int64_t n = (int64_t)min(total, (unsigned long long)cap);
    if (n <= 1) return;
    int passes = 0;
    for (int64_t run = kSortSmem; run < n; run <<= 1) ++passes;
    const ulonglong2 *src = (passes & 1) ? bufB : bufA;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = unpack_pair(src[i]);
}

// ===========================================================================
// Per-pair counts (no early exit): warp per pair, lanes over bins
// ===========================================================================
__global__ void pair_counts_kernel(const uint32_t *qry, int64_t qstride, int64_t n_q,
                                   const uint32_t *coll, int64_t cstride, int64_t n_rows, int kg,
                                   int G, uint16_t *out) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = wid; p < n_q * n_rows; p += nw) {
        const int64_t q = p / n_rows, r = p - q * n_rows;
        for (int g = 0; g < G; ++g) {
            int m = 0, both = 0, one = 0;
            for (int b0 = 0; b0 < kg; b0 += 32) {
                const int b = b0 + lane;
                const bool valid = b < kg;
                const uint32_t qv = valid ? qry[g * qstride + q * kg + b] : 0;
                const uint32_t rv = valid ? coll[g * cstride + r * kg + b] : 0;
                const bool eq = qv == HOPH_EMPTY_VALUE, er = rv == HOPH_EMPTY_VALUE;
                m += __popc(__ballot_sync(0xFFFFFFFFu, valid && !eq && qv == rv));
                both += __popc(__ballot_sync(0xFFFFFFFFu, valid && eq && er));
                one += __popc(__ballot_sync(0xFFFFFFFFu, valid && eq != er));
            }
            if (lane == 0) {
                uint16_t *o = out + (p * G + g) * 3;
                o[0] = (uint16_t)m;
                o[1] = (uint16_t)both;
                o[2] = (uint16_t)one;
            }
        }
    }
}

// ===========================================================================
// Bounded-wait check: the pipeline's wait routine on an mbarrier that no
// thread ever arrives on gives up after `limit_ns` and reports
// HOPH_ERR_TIMEOUT in the status word; nothing faults or hangs.
// ===========================================================================
__global__ void bounded_wait_probe_kernel(uint64_t limit_ns, int32_t *status) {
    __shared__ uint64_t bar;
    __shared__ int32_t abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, &abort_flag, limit_ns))
        hoph_flag(status, HOPH_ERR_TIMEOUT);
}

// ===========================================================================
// Host side
// ===========================================================================
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

CUtensorMapDataType map_type(int esize) {
    return esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
}

// 3-D map over the collection planes (elements of esize bytes): {k', rows,
// planes}, box {k', R, Gs}
bool encode_planes_map(CUtensorMap *map, const void *planes, int esize, int kg, int64_t n_rows,
                       int Gs, int64_t cstride, int R) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    const cuuint64_t gdim[3] = {(cuuint64_t)kg, (cuuint64_t)n_rows, (cuuint64_t)Gs};
    const cuuint64_t gstride[2] = {(cuuint64_t)kg * esize, (cuuint64_t)cstride * esize};
    const cuuint32_t box[3] = {(cuuint32_t)kg, (cuuint32_t)R, (cuuint32_t)Gs};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, map_type(esize), 3, (void *)planes, gdim, gstride, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 4-D swizzled map for the join filter: {v, k'/v, rows, planes}, box
// {v, k'/v, R, Gs} with v = 128 / esize values per 128-byte line, 128-byte
// swizzle (needs k' % v == 0)
bool encode_swizzled_map(CUtensorMap *map, const void *planes, int esize, int kg, int64_t n_rows,
                         int Gs, int64_t cstride, int R, bool swizzle = true) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    const int v = 128 / esize;
    const cuuint64_t gdim[4] = {(cuuint64_t)v, (cuuint64_t)(kg / v), (cuuint64_t)n_rows,
                                (cuuint64_t)Gs};
    const cuuint64_t gstride[3] = {128, (cuuint64_t)kg * esize, (cuuint64_t)cstride * esize};
    const cuuint32_t box[4] = {(cuuint32_t)v, (cuuint32_t)(kg / v), (cuuint32_t)R, (cuuint32_t)Gs};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, map_type(esize), 4, (void *)planes, gdim, gstride, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename E, int NW>
int launch_striped(const FilterArgs &fa, const CUtensorMap &map, uint32_t smem, int num_sms,
                   int ctas_per_sm, cudaStream_t s) {
    if constexpr (sizeof(E) == 2 && NW == 4) {
        return HOPH_ERR_UNSUPPORTED;  // 256 16-bit bins: W <= 128 never gets here
    } else {
        auto kern = filter_striped_kernel<E, NW>;
        HOPH_CUDA_TRY(hoph_ensure_smem((const void *)kern, (int)smem));
        const int threads = 32 * (fa.n_cons + 1);
        int per_sm = 0;
        HOPH_CUDA_TRY(hoph_occupancy(&per_sm, (const void *)kern, threads, smem));
        if (per_sm < 1) return HOPH_ERR_UNSUPPORTED;
        if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
        const int64_t grid = std::min<int64_t>(fa.n_tiles, (int64_t)num_sms * per_sm);
        kern<<<(unsigned)grid, threads, smem, s>>>(fa, map);
        HOPH_CUDA_TRY(cudaGetLastError());
        return HOPH_OK;
    }
}

template <int NPER, bool HASHED, int MAXC, typename E>
int launch_filter_c(const FilterArgs &fa, const CUtensorMap &map, uint32_t smem, int num_sms,
                    int ctas_per_sm, cudaStream_t s) {
    auto kern = filter_kernel<NPER, HASHED, MAXC, E>;
    HOPH_CUDA_TRY(hoph_ensure_smem((const void *)kern, (int)smem));
    const int threads = 32 * (fa.n_cons + 1);
    int per_sm = 0;
    HOPH_CUDA_TRY(hoph_occupancy(&per_sm, (const void *)kern, threads, smem));
    if (per_sm < 1) return HOPH_ERR_UNSUPPORTED;
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    const int64_t grid = std::min<int64_t>(fa.n_tiles, (int64_t)num_sms * per_sm);
    kern<<<(unsigned)grid, threads, smem, s>>>(fa, map);
    HOPH_CUDA_TRY(cudaGetLastError());
    return HOPH_OK;
}

template <int NPER, bool HASHED, typename E>
int launch_filter(const FilterArgs &fa, const CUtensorMap &map, uint32_t smem, int num_sms,
                  int ctas_per_sm, cudaStream_t s) {
    return fa.n_cons > 16
               ? launch_filter_c<NPER, HASHED, 31, E>(fa, map, smem, num_sms, ctas_per_sm, s)
               : launch_filter_c<NPER, HASHED, 16, E>(fa, map, smem, num_sms, ctas_per_sm, s);
}

// First-pass decision table for W scanned bins under `dp` after `l` groups:
// rej[K] / acc[K] for K = 0..W, then row_min[n] for n = 0..W.
bool build_table(const DecideParams &dp, int W, int l, std::vector<uint16_t> &tab) {
    tab.assign(3 * (W + 1), 0);
    for (int K = 0; K <= W; ++K) {
        int rej = K + 1, acc = K + 1;
        for (int m = 0; m <= K; ++m) {
            int32_t M[1] = {m}, Kk[1] = {K};
            const int d = hoph_decide(dp, l, M, Kk);
            if (d != HOPH_REJECT && rej == K + 1) rej = m;
            if (d == HOPH_ACCEPT && acc == K + 1) acc = m;
        }
        // check the monotone shape the table relies on
        for (int m = 0; m <= K; ++m) {
            int32_t M[1] = {m}, Kk[1] = {K};
            const int d = hoph_decide(dp, l, M, Kk);
            const int want = m < rej ? HOPH_REJECT : (m >= acc ? HOPH_ACCEPT : HOPH_CONTINUE);
            if (d != want) return false;
        }
        tab[K] = (uint16_t)rej;
        tab[W + 1 + K] = (uint16_t)acc;
    }
    // row_min[n]: a row with n non-empty scanned bins meets every query with a
    // denominator K >= max(n, 1) (K = W under rule NONE), so a pair below the
    // smallest rejection threshold over those K is rejected whatever the query
    for (int n = 0; n <= W; ++n) {
        int best = W + 1;
        if (dp.rule == HOPH_EMPTY_NONE) {
            best = tab[W];
        } else {
            for (int K = n > 1 ? n : 1; K <= W; ++K) best = best < tab[K] ? best : tab[K];
        }
        tab[2 * (W + 1) + n] = (uint16_t)best;
    }
    return true;
}

// Sort the output by (query, row) and fold the call's statistics: one CTA up
// to kSortOneCta records of capacity, the multi-CTA sequence beyond.
int launch_output_sort(hoph_plan *plan, hoph_pair *d_out, const unsigned long long *count,
                       int64_t cap, ulonglong2 *sortA, ulonglong2 *sortB, const StatsFold &sf,
                       cudaStream_t s, int64_t *launches) {
    if (cap <= kSortOneCta) {
        HOPH_CUDA_TRY(hoph_ensure_smem((const void *)sort_pairs_kernel, kSmallSortRun * 16));
        sort_pairs_kernel<<<1, kSmallSortThreads, kSmallSortRun * 16, s>>>(d_out, count, cap, sortA,
                                                                  sortB, plan->d_status, sf);
        HOPH_CUDA_TRY(cudaGetLastError());
        *launches = 1;
        return HOPH_OK;
    }
    HOPH_CUDA_TRY(hoph_ensure_smem((const void *)sort_runs_kernel, kSortSmem * 16));
    const int64_t runs = (cap + kSortSmem - 1) / kSortSmem;
    sort_runs_kernel<<<(unsigned)std::min<int64_t>(runs, plan->num_sms), kSortThreads,
                       kSortSmem * 16, s>>>(d_out, count, cap, sortA);
    int passes = 0;
    for (int64_t run = kSortSmem; run < cap; run <<= 1, ++passes)
        merge_pass_kernel<<<(unsigned)plan->num_sms * 8, 256, 0, s>>>(
            passes & 1 ? sortB : sortA, passes & 1 ? sortA : sortB, count, cap, run);
    sort_finish_kernel<<<(unsigned)plan->num_sms * 4, 256, 0, s>>>(d_out, count, cap, sortA,
                                                                    sortB, plan->d_status, sf);
    HOPH_CUDA_TRY(cudaGetLastError());
    *launches = passes + 2;
    return HOPH_OK;
}

struct Bump {
    unsigned char *base;
    size_t off = 0;
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

// hoph_query_batch / hoph_query_batch16 over planes of element type E, and
// one block of hoph_self_join: collection planes cstride elements apart
// (n_rows * k' when negative), query planes qstride_in apart (n_queries * k'
// when negative); self_off >= 0 keeps only row > query and shifts both by
// self_off; `first` zeroes the output count, `last` sorts the output; `lane`
// picks the plan's scratch (a self-join's blocks in flight use one each).
template <typename E>
int query_batch_impl(hoph_plan *plan, uint32_t mode, const E *d_query_planes, int64_t n_queries,
                     const E *d_coll_planes, int64_t n_rows, hoph_pair *d_out,
                     int64_t out_capacity, int64_t *d_out_count, hoph_stats *d_stats,
                     void *stream, int64_t cstride_in = -1, int64_t qstride_in = -1,
                     int64_t self_off = -1, bool first = true, bool last = true,
                     int lane = 0) {
    constexpr int ES = (int)sizeof(E);
    if (!plan || !d_out_count || n_queries < 0 || n_rows < 0 || out_capacity < 0)
        return HOPH_ERR_PARAM;
    if (out_capacity > 0 && !d_out) return HOPH_ERR_PARAM;
    if (n_queries > 65535 || n_rows >= (1ll << 40)) return HOPH_ERR_UNSUPPORTED;
    const hoph_params &P = plan->P;
    cudaStream_t s = (cudaStream_t)stream;
    // compact planes hold bin offsets: every bin must fit 16 bits with 0xFFFF
    // left for the empty marker; MinWise values are whole psi-values
    if (ES == 2 && (mode == HOPH_MODE_MINWISE_FULL || plan->max_width > 0xFFFFu))
        return HOPH_ERR_UNSUPPORTED;

    // mode -> scanned planes and the rule of the first pass
    DecideParams dp = plan->dp;
    int kg = (int)P.k_group, G = (int)plan->G, Gs = 1;
    if (mode == HOPH_MODE_GOPH || mode == HOPH_MODE_OPH_FULL) {
        if (P.a != 0) return HOPH_ERR_PARAM;
    } else if (mode == HOPH_MODE_HOPH) {
        if (P.a == 0) return HOPH_ERR_PARAM;
    } else if (mode == HOPH_MODE_MINWISE_FULL) {
        if (!P.minwise_k) return HOPH_ERR_PARAM;
    } else {
        return HOPH_ERR_PARAM;
    }
    DecideParams fp = dp;  // rule of the first pass
    if (mode == HOPH_MODE_OPH_FULL) {
        Gs = G;
        fp.mode = HOPH_MODE_GOPH;
        fp.G = 1;
        fp.kg = P.k;
        G = 1;
    } else if (mode == HOPH_MODE_MINWISE_FULL) {
        kg = (int)P.minwise_k;
        G = 1;
        fp.mode = HOPH_MODE_GOPH;
        fp.G = 1;
        fp.kg = P.minwise_k;
        fp.rule = HOPH_EMPTY_NONE;
    }
    const int W = Gs * kg;
    if (W > kMaxW) return HOPH_ERR_UNSUPPORTED;

    if (n_queries == 0 || n_rows == 0) {
        if (first) HOPH_CUDA_TRY(cudaMemsetAsync(d_out_count, 0, sizeof(int64_t), s));
        return HOPH_OK;
    }
    if (!d_query_planes || !d_coll_planes) return HOPH_ERR_PARAM;

    if (plan->table_W[mode] != W) {
        if (hoph_capturing(s)) return HOPH_ERR_CAPTURE;  // it allocates and copies
        plan->table_ok[mode] = build_table(fp, W, 1, plan->h_table[mode]);
        plan->table_W[mode] = W;
        cudaFree(plan->d_table[mode]);
        plan->d_table[mode] = nullptr;
        if (plan->table_ok[mode]) {
            const size_t b = plan->h_table[mode].size() * 2;
            HOPH_CUDA_TRY(cudaMalloc(&plan->d_table[mode], b));
            HOPH_CUDA_TRY(cudaMemcpy(plan->d_table[mode], plan->h_table[mode].data(), b,
                                     cudaMemcpyHostToDevice));
        }
    }
    if (!plan->table_ok[mode]) return HOPH_ERR_UNSUPPORTED;
    const std::vector<uint16_t> &tab = plan->h_table[mode];

    // (TMA tile coordinates are 32-bit signed: rows beyond 2^31 take the plain loads)
    const bool tma_base_ok = ((kg * ES) % 16 == 0) && kg <= 256 && Gs <= 256 &&
                             n_rows < (1ll << 31) && ((uintptr_t)d_coll_planes & 15) == 0 &&
                             get_encode_fn() != nullptr;

    // join: needs "no match => reject" for every K >= 1, TMA tiles, a rule
    // whose K == 0 pairs are the all-empty ones, and a key space (the psi-space
    // of the scanned bins) whose 2-bit group map fits in shared memory next
    // to two filter stages
    // Key space: the psi-space of the scanned bins.  Up to kDirectMap keys the
    // group map is indexed by key (no false hits); beyond, by a hash into
    // kHashedMapSlots slots (false hits only loosen the filter).  Up to
    // kMaxJoinKeys keys the list heads are indexed by key; beyond, through a
    // key table.
    // A small key space takes the guarded keys lo[w] + w + 1 + value (a key
    // below every bin that no value reaches; the empty marker wraps onto it).
    const uint64_t plain_keys = mode == HOPH_MODE_MINWISE_FULL ? ~0ull : plan->lo[W];
    const bool map_hashed = plain_keys > kDirectMap - W - 1;
    const uint64_t keys = map_hashed ? plain_keys : plain_keys + W + 1;
    const uint64_t *binbase = map_hashed ? plan->d_lo : plan->d_kb;
    const uint64_t map_slots = map_hashed ? kHashedMapSlots : keys;
    uint32_t map_shift = 32;  // hashed map: 32 - log2(kHashedMapSlots)
    while ((1ull << (32 - map_shift)) < kHashedMapSlots) --map_shift;
    const bool keys_hashed = keys > kMaxJoinKeys;
    uint64_t head_slots = keys;
    if (keys_hashed) {
        head_slots = 1024;
        while (head_slots < 2ull * (uint64_t)n_queries * W) head_slots <<= 1;
    }
    bool join_ok = mode != HOPH_MODE_MINWISE_FULL && fp.rule != HOPH_EMPTY_EITHER &&
                   tma_base_ok && kg % (128 / ES) == 0 && W <= 256 && n_queries <= 4096 &&
                   n_rows < (1ll << 32) && head_slots < (1ull << 31) &&
                   map_slots / 4 + 2 * 32 * W * ES + 8 * W + 4096 <= (uint64_t)kSmemLimit;
    for (int K = 1; K <= W && join_ok; ++K) join_ok = tab[K] >= 1;
    int strategy = plan->exec.strategy;
    if (strategy == 1 && !join_ok) return HOPH_ERR_UNSUPPORTED;
    if (strategy < 0) strategy = (join_ok && n_queries >= 16) ? 1 : 0;

    // The striped map (lanes over bins, filter_striped_kernel): one plane,
    // rows of whole 128-byte lines, W <= 128, a direct map of W stacks of
    // nwb words (slot 0 of each the empty guard) that fits next to two
    // stages of 64 rows.  lanes_per_row = 32 asks for it
    uint32_t nwb = 0;
    const int lane_words = W * ES / 128;  // 32-bit words of a row per lane
    if (Gs == 1 && (W * ES) % 128 == 0 && W <= 128 && !map_hashed &&
        (lane_words == 1 || lane_words == 2 || lane_words == 4)) {
        uint64_t maxw = 0;
        for (int w = 0; w < W; ++w) maxw = std::max<uint64_t>(maxw, plan->lo[w + 1] - plan->lo[w]);
        nwb = (uint32_t)((maxw + 1 + 15) / 16);
    }
    const bool striped_ok = nwb > 0 && (ES == 4 || nwb * 16 <= 0x8000) &&
                            (uint64_t)W * nwb * 4 + 2ull * 64 * W * ES + 8 * W + 4096 +
                                    4096ull * lane_words <= (uint64_t)kSmemLimit;
    // (the library's own choice for 16-bit planes, where it is the faster filter)
    const bool striped = strategy == 1 && (plan->exec.lanes_per_row == 32 ||
                                           (plan->exec.lanes_per_row == 0 && ES == 2 && striped_ok));
    if (striped && !striped_ok) return HOPH_ERR_UNSUPPORTED;

    const int mask_words = (W + 31) / 32;
    // group map words (+ the zero word), padded for the filter's 16-byte copy
    const uint64_t gmap_words_used = striped ? (uint64_t)W * nwb : map_slots / 16 + 2;
    const uint64_t gmap_alloc = (gmap_words_used + 3) & ~3ull;
    int wshift = 0;  // bits of a scanned-bin index (join index entries)
    while ((1 << wshift) < W) ++wshift;
    const int64_t qstride = qstride_in >= 0 ? qstride_in : n_queries * (int64_t)kg;
    const int64_t cstride = cstride_in >= 0 ? cstride_in : n_rows * (int64_t)kg;

    // scratch
    Bump bump{nullptr};
    const size_t st_b = kStatWords * 8;
    const size_t cap1 = (size_t)std::max<int64_t>(out_capacity, 1);
    for (int pass = 0; pass < 2; ++pass) {
        bump.off = 0;
        bump.take(st_b);
        if (strategy == 1) {
            bump.take(head_slots * 4);                                   // list heads
            bump.take(((size_t)n_queries << wshift) * 4);               // list links
            bump.take(gmap_alloc * 4);                                  // group map
            bump.take(keys_hashed ? head_slots * 8 : 8);                  // key table
            bump.take((size_t)n_queries * mask_words * 4);              // q_emask
            bump.take((size_t)n_queries * 4 + 4);                       // allempty + count
            bump.take(8);                                               // n_cand
            bump.take((size_t)n_rows * 4);                              // cand
        }
        if (last) {
            bump.take(cap1 * 16);  // sort A
            bump.take(cap1 * 16);  // sort B
        }
        if (pass == 0) {
            void *p = nullptr;
            const int src = hoph_scratch(plan, bump.off, lane, s, &p);
            if (src != HOPH_OK) return src;
            unsigned char *base = static_cast<unsigned char *>(p);
            bump.base = base;
        }
    }
    bump.off = 0;
    unsigned long long *st = (unsigned long long *)bump.take(st_b);
    uint32_t *head = nullptr, *next = nullptr, *gmap = nullptr, *q_emask = nullptr,
             *n_allempty = nullptr, *cand = nullptr;
    int32_t *allempty = nullptr;
    unsigned long long *tkey = nullptr;
    unsigned long long *n_cand = nullptr;
    if (strategy == 1) {
        head = (uint32_t *)bump.take(head_slots * 4);
        next = (uint32_t *)bump.take(((size_t)n_queries << wshift) * 4);
        gmap = (uint32_t *)bump.take(gmap_alloc * 4);
        tkey = (unsigned long long *)bump.take(keys_hashed ? head_slots * 8 : 8);
        q_emask = (uint32_t *)bump.take((size_t)n_queries * mask_words * 4);
        allempty = (int32_t *)bump.take((size_t)n_queries * 4 + 4);
        n_allempty = (uint32_t *)(allempty + n_queries);
        n_cand = (unsigned long long *)bump.take(8);
        cand = (uint32_t *)bump.take((size_t)n_rows * 4);
    }
    ulonglong2 *sortA = last ? (ulonglong2 *)bump.take(cap1 * 16) : nullptr;
    ulonglong2 *sortB = last ? (ulonglong2 *)bump.take(cap1 * 16) : nullptr;

    PairArgs pa;
    pa.coll = d_coll_planes;
    pa.cstride = cstride;
    pa.qry = d_query_planes;
    pa.qstride = qstride;
    pa.n_rows = n_rows;
    pa.n_q = (int32_t)n_queries;
    pa.kg = kg;
    pa.Gs = Gs;
    pa.W = W;
    pa.G = G;
    pa.rule = fp.rule;
    pa.thr = plan->d_table[mode];
    pa.dp = dp;
    pa.out = d_out;
    pa.cap = out_capacity;
    pa.self_off = self_off;
    pa.out_count = reinterpret_cast<unsigned long long *>(d_out_count);
    pa.stat = st;
    pa.status = plan->d_status;

    if (strategy != 1) {  // the join resets its state in join_init_kernel
        if (first) HOPH_CUDA_TRY(cudaMemsetAsync(d_out_count, 0, sizeof(int64_t), s));
        HOPH_CUDA_TRY(cudaMemsetAsync(st, 0, st_b, s));
    }
    hoph_timing_mark(plan, 0, s);
    int64_t launches = 0;

    if (strategy == 1) {
        // ---- join: index
        IndexArgs ia;
        ia.qry = d_query_planes;
        ia.qstride = qstride;
        ia.n_q = (int32_t)n_queries;
        ia.kg = kg;
        ia.W = W;
        ia.mask_words = mask_words;
        ia.binbase = binbase;
        ia.head = head;
        ia.next = next;
        ia.wshift = wshift;
        ia.gmap = gmap;
        ia.map_hashed = map_hashed;
        ia.map_shift = map_shift;
        ia.striped = striped ? 1 : 0;
        ia.nwb = nwb;
        ia.keys_hashed = keys_hashed;
        ia.tkey = tkey;
        ia.tmask = (uint32_t)(head_slots - 1);
        ia.status = plan->d_status;
        ia.q_emask = q_emask;
        ia.allempty = allempty;
        ia.n_allempty = n_allempty;
        join_init_kernel<<<(unsigned)plan->num_sms * 4, 256, 0, s>>>(
            head, (int64_t)head_slots, gmap, (int64_t)gmap_alloc, st, kStatWords,
            n_allempty, n_cand, first ? d_out_count : nullptr);
        if (keys_hashed) HOPH_CUDA_TRY(cudaMemsetAsync(tkey, 0xFF, head_slots * 8, s));
        const unsigned qb = (unsigned)((n_queries * 32 + 255) / 256);
        join_count_kernel<E><<<qb, 256, 0, s>>>(ia);
        HOPH_CUDA_TRY(cudaGetLastError());
        launches += 2;

        // ---- join: streaming row filter
        FilterArgs fa;
        fa.n_rows = n_rows;
        fa.kg = kg;
        fa.Gs = Gs;
        fa.W = W;
        fa.gmap = gmap;
        fa.gmap_words = (uint32_t)gmap_words_used;  // direct / hashed: + a zero word
        fa.map_shift = map_shift;
        fa.nwb = nwb;
        fa.binbase = binbase;
        fa.row_min = pa.thr + 2 * (W + 1);
        const int K0 = hoph_effective(fp.rule, W, W, 0);
        fa.keep_empty = table_decide(tab.data(), W, 0, K0) != HOPH_REJECT;
        fa.cand = cand;
        fa.n_cand = n_cand;
        fa.status = plan->d_status;
        // shape: bins per lane (32 or 16; the striped kernel: lanes over a
        // row's bins, tile_rows rows per tile), consumer warps and stages that
        // fit next to the group map, at least two stages
        int lpr = striped ? 32
                          : (plan->exec.lanes_per_row > 0 ? plan->exec.lanes_per_row
                                                          : std::max(1, W / 32));
        const int nper = W / lpr;
        if (!striped && (W % lpr || (nper != 32 && nper != 16) || lpr > 32))
            return HOPH_ERR_UNSUPPORTED;
        // striped: the stages start on a multiple of 32 rows' bytes (lane l
        // then finds row r0 + (j ^ l) of a group at one XOR off its base)
        fa.stage_align = striped ? 4096u * (uint32_t)lane_words : 1024u;
        const uint32_t fixed = 16 * 8 + 16 + align_up((W + 1) * 2, 16) +
                               align_up(fa.gmap_words * 4, fa.stage_align) + fa.stage_align;
        int n_cons = plan->exec.consumer_warps > 0 ? plan->exec.consumer_warps : 16;
        if (striped) n_cons = std::min(n_cons, 16);
        int stages = plan->exec.stages > 0 ? plan->exec.stages : 3;
        // striped: rows per tile a multiple of 32 (a warp's group), loaded as
        // boxes of at most 256 rows; the default fills a 64 KB stage
        int srows = plan->exec.tile_rows > 0 ? plan->exec.tile_rows : 65536 / (W * ES);
        if (striped) {
            srows = std::min(1024, std::max(32, srows / 32 * 32));
            if (srows > 256) srows = srows / 256 * 256;
            n_cons = std::min(n_cons, srows / 32);
        }
        auto rows_of = [&](int nc) { return striped ? srows : 32 / lpr * nc; };
        auto too_many_rows = [&](int nc) { return striped ? false : rows_of(nc) > 256; };
        auto stage_of = [&](int nc) { return align_up((uint32_t)rows_of(nc) * W * ES, 1024); };
        while (n_cons > 1 && (fixed + (uint32_t)stages * stage_of(n_cons) > (uint32_t)kSmemLimit ||
                              too_many_rows(n_cons))) {
            if (stages > 2) --stages;
            else if (striped && srows > 64) {
                srows = srows > 256 ? srows / 2 / 256 * 256 : srows / 2 / 32 * 32;
                n_cons = std::min(n_cons, srows / 32);
            } else --n_cons;
        }
        if (fixed + (uint32_t)stages * stage_of(n_cons) > (uint32_t)kSmemLimit)
            return HOPH_ERR_UNSUPPORTED;
        fa.lanes_per_row = lpr;
        fa.n_cons = n_cons;
        fa.tile_rows = rows_of(n_cons);
        fa.boxes = striped && fa.tile_rows > 256 ? fa.tile_rows / 256 : 1;
        fa.stages = stages;
        fa.n_tiles = (n_rows + fa.tile_rows - 1) / fa.tile_rows;
        fa.stage_bytes = (uint32_t)fa.tile_rows * W * ES;
        fa.stage_stride = align_up(fa.stage_bytes, 1024);
        CUtensorMap map;
        memset(&map, 0, sizeof map);
        if (!encode_swizzled_map(&map, d_coll_planes, ES, kg, n_rows, Gs, cstride,
                                 fa.tile_rows / fa.boxes, !striped))
            return HOPH_ERR_UNSUPPORTED;
        const FilterSmem FL = filter_smem(fa);
        hoph_timing_mark(plan, 1, s);
        const int cps = plan->exec.ctas_per_sm;
        const int nsm = plan->num_sms;
        const int frc =
            striped ? (lane_words == 1   ? launch_striped<E, 1>(fa, map, FL.total, nsm, cps, s)
                       : lane_words == 2 ? launch_striped<E, 2>(fa, map, FL.total, nsm, cps, s)
                                         : launch_striped<E, 4>(fa, map, FL.total, nsm, cps, s))
            : nper == 32 ? (map_hashed ? launch_filter<32, true, E>(fa, map, FL.total, nsm, cps, s)
                                       : launch_filter<32, false, E>(fa, map, FL.total, nsm, cps, s))
                         : (map_hashed ? launch_filter<16, true, E>(fa, map, FL.total, nsm, cps, s)
                                       : launch_filter<16, false, E>(fa, map, FL.total, nsm, cps, s));
        if (frc != HOPH_OK) return frc;
        hoph_timing_mark(plan, 2, s);

        // ---- join: candidate rows
        CountArgs ca;
        ca.p = pa;
        ca.cand = cand;
        ca.n_cand = n_cand;
        ca.binbase = binbase;
        ca.keys_hashed = keys_hashed;
        ca.tkey = tkey;
        ca.tmask = (uint32_t)(head_slots - 1);
        ca.head = head;
        ca.next = next;
        ca.wshift = wshift;
        ca.q_emask = q_emask;
        ca.mask_words = mask_words;
        ca.allempty = allempty;
        ca.n_allempty = n_allempty;
        const CountSmem CL = count_smem(ca);
        if (CL.total > (uint32_t)kSmemLimit) return HOPH_ERR_UNSUPPORTED;
        const int nch = (W + 31) / 32;
        const int rc = nch <= 1 ? launch_count<1, E>(ca, CL.total, plan->num_sms, s)
                     : nch <= 2 ? launch_count<2, E>(ca, CL.total, plan->num_sms, s)
                     : nch <= 4 ? launch_count<4, E>(ca, CL.total, plan->num_sms, s)
                                : launch_count<8, E>(ca, CL.total, plan->num_sms, s);
        if (rc != HOPH_OK) return rc;
        hoph_timing_mark(plan, 3, s);
        launches += 2;
    } else {
        // ---- dense
        DenseArgs da;
        da.p = pa;
        const int n_cons = plan->exec.consumer_warps > 0 ? plan->exec.consumer_warps : 8;
        if (n_cons > 15) return HOPH_ERR_UNSUPPORTED;
        int R = plan->exec.tile_rows > 0 ? plan->exec.tile_rows : 0;
        if (R == 0) {
            R = (int)std::max<int64_t>(1, std::min<int64_t>(256, 8192 / (W * ES)));
            if (R >= 8) R &= ~7;
        }
        da.n_cons = n_cons;
        da.tile_rows = R;
        da.use_tma = tma_base_ok ? 1 : 0;
        da.stages = tma_base_ok ? (plan->exec.stages > 0 ? plan->exec.stages : 4) : 1;
        da.n_tiles = (n_rows + R - 1) / R;
        da.stage_bytes = (uint32_t)Gs * R * kg * ES;
        da.stage_stride = align_up(da.stage_bytes, 128);
        CUtensorMap map;
        memset(&map, 0, sizeof map);
        if (da.use_tma && !encode_planes_map(&map, d_coll_planes, ES, kg, n_rows, Gs, cstride, R)) {
            da.use_tma = 0;
            da.stages = 1;
        }
        const DenseSmem DL = dense_smem(da);
        if (DL.total > (uint32_t)kSmemLimit) return HOPH_ERR_UNSUPPORTED;
        const int nch = (W + 31) / 32;
        auto dense = nch <= 1   ? dense_scan_kernel<E, 1>
                     : nch <= 2 ? dense_scan_kernel<E, 2>
                     : nch <= 4 ? dense_scan_kernel<E, 4>
                     : nch <= 8 ? dense_scan_kernel<E, 8>
                                : dense_scan_kernel<E, 0>;
        HOPH_CUDA_TRY(hoph_ensure_smem((const void *)dense, (int)DL.total));
        const int threads = 32 * (n_cons + 1);
        int per_sm = 0;
        HOPH_CUDA_TRY(hoph_occupancy(&per_sm, (const void *)dense, threads, DL.total));
        if (per_sm < 1) return HOPH_ERR_UNSUPPORTED;
        if (plan->exec.ctas_per_sm > 0) per_sm = std::min(per_sm, plan->exec.ctas_per_sm);
        const int64_t grid = std::min<int64_t>(da.n_tiles, (int64_t)plan->num_sms * per_sm);
        hoph_timing_mark(plan, 1, s);
        dense<<<(unsigned)grid, threads, DL.total, s>>>(da, map);
        HOPH_CUDA_TRY(cudaGetLastError());
        hoph_timing_mark(plan, 2, s);
        hoph_timing_mark(plan, 3, s);
        launches += 1;
    }

    StatsFold sf;
    sf.st = st;
    sf.n_cand = n_cand;
    // a self-join block compares its queries only with the rows after each
    sf.pairs = n_queries * n_rows - (self_off >= 0 ? n_queries * (n_queries + 1) / 2 : 0);
    sf.first_pass_bytes = (n_rows * (int64_t)W + n_queries * (int64_t)W) * ES;
    sf.G = G;
    sf.Gs = Gs;
    sf.strategy = strategy;
    sf.out = d_stats;
    if (last) {
        int64_t sort_launches = 0;
        const int rc = launch_output_sort(plan, d_out, pa.out_count, out_capacity, sortA, sortB,
                                          sf, s, &sort_launches);
        if (rc != HOPH_OK) return rc;
        launches += sort_launches - 1;
    } else if (d_stats) {
        stats_fold_kernel<<<1, 32, 0, s>>>(sf);
    } else {
        --launches;  // nothing to fold
    }
    HOPH_CUDA_TRY(cudaGetLastError());
    hoph_timing_mark(plan, 4, s);
    plan->launches += launches + 1;
    return HOPH_OK;
}

template <typename E>
int self_join_impl(hoph_plan *plan, uint32_t mode, const E *d_planes, int64_t n_rows,
                   int64_t batch, hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                   hoph_stats *d_stats, void *stream, int64_t part = 0, int64_t parts = 1) {
    if (!plan || !d_out_count || n_rows < 0 || batch < 1 || batch > 4096 || out_capacity < 0 ||
        parts < 1 || part < 0 || part >= parts)
        return HOPH_ERR_PARAM;
    if (out_capacity > 0 && !d_out) return HOPH_ERR_PARAM;
    if (mode == HOPH_MODE_MINWISE_FULL) return HOPH_ERR_UNSUPPORTED;
    if (n_rows >= (1ll << 32)) return HOPH_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    HOPH_CUDA_TRY(cudaMemsetAsync(d_out_count, 0, sizeof(int64_t), s));
    if (n_rows < 2) return HOPH_OK;
    if (!d_planes) return HOPH_ERR_PARAM;
    const int64_t kg = plan->P.k_group;
    const int64_t cstride = n_rows * kg;
    const int64_t n_blocks = (n_rows - 1 + batch - 1) / batch;
    // this call's blocks: part, part + parts, ...
    const int64_t my_blocks = n_blocks > part ? (n_blocks - part + parts - 1) / parts : 0;
    if (my_blocks == 0) return HOPH_OK;
    const int want = plan->exec.join_lanes > 0 ? plan->exec.join_lanes : 8;
    const int lanes = (int)std::min<int64_t>(std::min(want, (int)hoph_plan::kMaxLanes), my_blocks);
    // blocks in flight: block b runs on lane b % lanes, each lane a stream and
    // a scratch of the plan's own, forked from and joined back to `stream`
    if (lanes > 1) {
        for (int i = 0; i < lanes; ++i)
            if (!plan->lane_stream[i] && hoph_capturing(s)) return HOPH_ERR_CAPTURE;
        for (int i = 0; i < lanes; ++i) {
            if (!plan->lane_stream[i])
                HOPH_CUDA_TRY(cudaStreamCreateWithFlags(&plan->lane_stream[i], cudaStreamNonBlocking));
            if (!plan->lane_event[i])
                HOPH_CUDA_TRY(cudaEventCreateWithFlags(&plan->lane_event[i], cudaEventDisableTiming));
        }
        if (!plan->fork_event)
            HOPH_CUDA_TRY(cudaEventCreateWithFlags(&plan->fork_event, cudaEventDisableTiming));
        HOPH_CUDA_TRY(cudaEventRecord(plan->fork_event, s));
        for (int i = 0; i < lanes; ++i)
            HOPH_CUDA_TRY(cudaStreamWaitEvent(plan->lane_stream[i], plan->fork_event, 0));
    }
    int rc = HOPH_OK;
    for (int64_t i = 0; i < my_blocks && rc == HOPH_OK; ++i) {
        const int64_t blk = part + i * parts;
        const int64_t q0 = blk * batch;
        const int64_t nb = std::min(batch, n_rows - 1 - q0);
        const int lane = (int)(i % lanes);
        cudaStream_t ls = lanes > 1 ? plan->lane_stream[lane] : s;
        // rows q0 .. n_rows-1 against queries q0 .. q0+nb-1, both read in place
        const E *bp = d_planes + q0 * kg;
        rc = query_batch_impl<E>(plan, mode, bp, nb, bp, n_rows - q0, d_out, out_capacity,
                                 d_out_count, d_stats, ls, cstride, cstride, q0, false, false,
                                 lane);
    }
    if (lanes > 1) {  // join every lane back, also after an error
        for (int i = 0; i < lanes; ++i) {
            HOPH_CUDA_TRY(cudaEventRecord(plan->lane_event[i], plan->lane_stream[i]));
            HOPH_CUDA_TRY(cudaStreamWaitEvent(s, plan->lane_event[i], 0));
        }
    }
    if (rc != HOPH_OK) return rc;
    // one sort of all blocks' pairs (lane 0's scratch is free again here)
    const size_t cap1 = (size_t)std::max<int64_t>(out_capacity, 1);
    void *sp = nullptr;
    const int src = hoph_scratch(plan, 2 * cap1 * 16, 0, s, &sp);
    if (src != HOPH_OK) return src;
    ulonglong2 *sortA = static_cast<ulonglong2 *>(sp);
    StatsFold none{};
    int64_t sort_launches = 0;
    const int rc2 = launch_output_sort(plan, d_out,
                                       reinterpret_cast<const unsigned long long *>(d_out_count),
                                       out_capacity, sortA, sortA + cap1, none, s, &sort_launches);
    if (rc2 != HOPH_OK) return rc2;
    plan->launches += sort_launches;
    return HOPH_OK;
}

}  // namespace

extern "C" {

int hoph_query_batch(hoph_plan *plan, uint32_t mode, const uint32_t *d_query_planes,
                     int64_t n_queries, const uint32_t *d_coll_planes, int64_t n_rows,
                     hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                     hoph_stats *d_stats, void *stream) {
    return query_batch_impl<uint32_t>(plan, mode, d_query_planes, n_queries, d_coll_planes, n_rows,
                                      d_out, out_capacity, d_out_count, d_stats, stream);
}

int hoph_query_batch16(hoph_plan *plan, uint32_t mode, const uint16_t *d_query_planes,
                       int64_t n_queries, const uint16_t *d_coll_planes, int64_t n_rows,
                       hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                       hoph_stats *d_stats, void *stream) {
    return query_batch_impl<uint16_t>(plan, mode, d_query_planes, n_queries, d_coll_planes,
                                      n_rows, d_out, out_capacity, d_out_count, d_stats, stream);
}


int hoph_self_join(hoph_plan *plan, uint32_t mode, const uint32_t *d_planes, int64_t n_rows,
                   int64_t batch, hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                   hoph_stats *d_stats, void *stream) {
    return self_join_impl<uint32_t>(plan, mode, d_planes, n_rows, batch, d_out, out_capacity,
                                    d_out_count, d_stats, stream);
}

int hoph_self_join16(hoph_plan *plan, uint32_t mode, const uint16_t *d_planes, int64_t n_rows,
                     int64_t batch, hoph_pair *d_out, int64_t out_capacity,
                     int64_t *d_out_count, hoph_stats *d_stats, void *stream) {
    return self_join_impl<uint16_t>(plan, mode, d_planes, n_rows, batch, d_out, out_capacity,
                                    d_out_count, d_stats, stream);
}

int hoph_self_join_part(hoph_plan *plan, uint32_t mode, const void *d_planes,
                        uint32_t value_bytes, int64_t n_rows, int64_t batch, int64_t part,
                        int64_t parts, hoph_pair *d_out, int64_t out_capacity,
                        int64_t *d_out_count, hoph_stats *d_stats, void *stream) {
    if (value_bytes == 4)
        return self_join_impl<uint32_t>(plan, mode, static_cast<const uint32_t *>(d_planes),
                                        n_rows, batch, d_out, out_capacity, d_out_count, d_stats,
                                        stream, part, parts);
    if (value_bytes == 2)
        return self_join_impl<uint16_t>(plan, mode, static_cast<const uint16_t *>(d_planes),
                                        n_rows, batch, d_out, out_capacity, d_out_count, d_stats,
                                        stream, part, parts);
    return HOPH_ERR_PARAM;
}

int hoph_check_bounded_wait(hoph_plan *plan, uint64_t limit_ns, void *stream) {
    if (!plan || limit_ns == 0 || limit_ns > 2000000000ull) return HOPH_ERR_PARAM;
    bounded_wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(limit_ns, plan->d_status);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 1;
    return HOPH_OK;
}

int hoph_pair_counts(hoph_plan *plan, const uint32_t *d_query_planes, int64_t n_queries,
                     const uint32_t *d_coll_planes, int64_t n_rows, uint16_t *d_counts,
                     void *stream) {
    if (!plan || n_queries < 0 || n_rows < 0) return HOPH_ERR_PARAM;
    if (n_queries == 0 || n_rows == 0) return HOPH_OK;
    if (!d_query_planes || !d_coll_planes || !d_counts) return HOPH_ERR_PARAM;
    const int kg = (int)plan->P.k_group, G = (int)plan->G;
    const int64_t pairs = n_queries * n_rows;
    const int64_t blocks = std::min<int64_t>((pairs * 32 + 255) / 256, (int64_t)plan->num_sms * 32);
    pair_counts_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        d_query_planes, n_queries * kg, n_queries, d_coll_planes, n_rows * kg, n_rows, kg, G,
        d_counts);
    HOPH_CUDA_TRY(cudaGetLastError());
    plan->launches += 1;
    return HOPH_OK;
}

}  // extern "C"
