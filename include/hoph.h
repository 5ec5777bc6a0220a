/*
 * hoph.h - C ABI of the GB300 library for One Permutation Hashing (OPH),
 * group-based OPH (GOPH) and hierarchical (a:b) OPH (HOPH) near-duplicate
 * detection, with MinWise as the baseline.
 *
 * Method: Zhang et al., "Hierarchical One Permutation Hashing: Efficient
 * Multimedia Near Duplicate Detection" (arXiv 1805.11254).  Section,
 * equation and algorithm numbers are the paper's.
 *
 * Conventions for every entry point
 *   - Device pointers ("d_" prefix) are CUDA device memory owned by the
 *     caller.  The library never frees or reallocates caller memory.
 *   - `stream` is a cudaStream_t passed as void*.  Work is enqueued on it
 *     and the call returns without synchronising, except where stated.
 *   - Return value: HOPH_OK (0) or a negative HOPH_ERR_* code.  Argument
 *     errors are returned before anything is enqueued.  Errors found on the
 *     device (an ID >= D, a full output buffer, a bounded wait that gave up)
 *     are recorded in the plan's device status word; hoph_sync_status()
 *     synchronises the stream and returns and clears that word.
 *   - A plan owns its permutation table, bin layout, decision thresholds and
 *     scratch memory.  Calls that use one plan must be ordered on one stream
 *     (they share its scratch); use one plan per concurrent stream.
 *   - The scratch grows on demand (a call that needs more synchronises the
 *     device and reallocates it).  A CUDA graph captured from calls on a
 *     plan keeps the scratch addresses of its capture, so before capturing,
 *     make one uncaptured call of the largest shape the plan will serve;
 *     after that no call of a shape up to it grows the scratch.  A call that
 *     would grow the scratch (or build a decision table, or create the
 *     self-join's streams) while its stream is being captured returns
 *     HOPH_ERR_CAPTURE before enqueuing anything.
 */
#ifndef HOPH_H
#define HOPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HOPH_OK 0
#define HOPH_ERR_PARAM (-1)       /* invalid argument or parameter set       */
#define HOPH_ERR_ID_RANGE (-2)    /* an input ID was >= D (element skipped)  */
#define HOPH_ERR_CAPACITY (-3)    /* more accepted pairs than out_capacity   */
#define HOPH_ERR_TIMEOUT (-4)     /* a bounded device wait gave up           */
#define HOPH_ERR_CUDA (-5)        /* a CUDA runtime call failed              */
#define HOPH_ERR_NOMEM (-6)       /* host or device allocation failed        */
#define HOPH_ERR_UNSUPPORTED (-7) /* valid parameters this build cannot run  */
#define HOPH_ERR_TOO_LARGE (-8)   /* input exceeds a fixed-size scratch area  */
#define HOPH_ERR_CAPTURE (-9)     /* the call would (re)allocate plan memory
                                     while its stream is being captured      */

/* ---- enumerations ------------------------------------------------------ */
/* comparison modes of hoph_query_batch */
#define HOPH_MODE_OPH_FULL 0     /* Eq. 6 over all k bins, no early exit       */
#define HOPH_MODE_GOPH 1         /* Algorithm 1, equal groups of k' bins       */
#define HOPH_MODE_HOPH 2         /* Algorithm 2, (a:b) hierarchical groups     */
#define HOPH_MODE_MINWISE_FULL 3 /* MinWise: matching minima / k >= T          */

/* how psi is realised */
#define HOPH_PERM_TABLE 0  /* explicit Fisher-Yates table of D entries       */
#define HOPH_PERM_HASH61 1 /* ((a x + b) mod (2^61 - 1)) >> 29, D = 2^32     */

/* which bins count in a group's denominator K_j */
#define HOPH_EMPTY_BOTH 0   /* drop bins empty in both sketches (Eq. 5)     */
#define HOPH_EMPTY_EITHER 1 /* drop bins empty in either sketch             */
#define HOPH_EMPTY_NONE 2   /* keep all k' bins (Algorithms 1-2 literally)  */

/* HOPH remaining-requirement rule */
#define HOPH_WEIGHT_SPACE 0   /* groups weighted by their share of V (a:b) */
#define HOPH_WEIGHT_LITERAL 1 /* Algorithm 2's recursion, r = a / (a + b)  */

#define HOPH_MAX_GROUPS 16
#define HOPH_EMPTY_VALUE 0xFFFFFFFFu /* the empty-bin marker in a sketch */
#define HOPH_EMPTY_VALUE16 0xFFFFu     /* the same in a compact (uint16) sketch */

/*
 * Method parameters (Sec. 3.1-4.1 and Table 1).
 *   universe_D  size of the vocabulary V; IDs are 0..D-1.  1 <= D <= 2^32.
 *               HOPH_PERM_HASH61 requires D = 2^32.
 *   k           bins per sketch; k_group (k') bins per group; k % k' == 0,
 *               G = k / k' <= HOPH_MAX_GROUPS.
 *   a, b        (a:b)HOPH split of the space (Sec. 4.1); a = b = 0 gives the
 *               equal bins of OPH / GOPH (Sec. 3.2-3.3).  Every HOPH group
 *               must hold at least k' values of V.
 *   perm_kind   HOPH_PERM_TABLE or HOPH_PERM_HASH61.
 *   minwise_k   number of MinWise permutations to build (0 = none); table t
 *               is the Fisher-Yates table of seed + t.
 *   seed        seed of psi.
 *   thr_num/thr_den  the similarity threshold T as an exact fraction
 *               (0 < T <= 1, thr_den <= 65535).
 *   epsilon     the error tolerance of Definition 1, 0 <= eps.
 *   empty_rule  HOPH_EMPTY_*.
 *   weighting   how HOPH turns the groups compared so far into the remaining
 *               requirement P_r (Algorithm 2).  HOPH_WEIGHT_SPACE: P_r =
 *               (T Z_all - sum_j z_j M_j / K_j) / Z_rem over the groups' space
 *               sizes z_j.  HOPH_WEIGHT_LITERAL: Algorithm 2 as printed,
 *               P <- (P - (M_l / k') r^l) / r^l from P = T with r = a / (a + b)
 *               (matched bins over k', empty bins ignored); exact only if the
 *               integers of the scaled recursion fit in 120 bits, else
 *               hoph_plan_create returns HOPH_ERR_PARAM.  Either way the last
 *               group ends with the space-weighted estimator of Lemma 3 >= T.
 *               GOPH / OPH (a = b = 0) ignore it.
 */
typedef struct {
    uint64_t universe_D;
    uint32_t k;
    uint32_t k_group;
    uint32_t a, b;
    uint32_t perm_kind;
    uint32_t minwise_k;
    uint64_t seed;
    uint32_t thr_num, thr_den;
    double epsilon;
    uint32_t empty_rule;
    uint32_t weighting;
} hoph_params;

/* One accepted (query, row) pair (the result set O of Algorithms 1-2). */
typedef struct {
    int64_t row;      /* collection row index                          */
    uint32_t query;   /* query index                                   */
    uint16_t groups;  /* groups compared before the decision           */
    uint16_t matches; /* matched bins over those groups                */
} hoph_pair;

/* Optional per-call statistics, accumulated (the caller zeroes it). */
typedef struct {
    int64_t entering[HOPH_MAX_GROUPS]; /* pairs still open when group g starts */
    int64_t accepted[HOPH_MAX_GROUPS]; /* pairs accepted after group g         */
    int64_t rejected[HOPH_MAX_GROUPS]; /* pairs rejected after group g         */
    int64_t sketch_bytes;              /* sketch bytes read from HBM (model)   */
    int64_t join_hits;                 /* (row value, query) matches counted   */
    int64_t strategy;                  /* 0 dense scan, 1 value join            */
    int64_t rows_counted;              /* join: rows that passed the row filter */
} hoph_stats;

/* Read-only facts about a plan (for tests and tooling). */
typedef struct {
    uint32_t groups;                    /* G                                  */
    uint32_t key_bits;                  /* packed psi table: bits of offset   */
    int64_t upper_limit;                /* U = min{j : P(X >= j) <= eps}      */
    int64_t lower_limit;                /* L = max{j : P(X < j) <= eps}       */
    uint64_t group_size[HOPH_MAX_GROUPS]; /* z_g, the values of V in group g  */
    uint64_t max_bin_width;             /* widest bin (compact planes: <= 65535) */
} hoph_plan_info;

/* Execution knobs (never change results).  0 = library default. */
typedef struct {
    int32_t strategy;        /* -1 auto, 0 dense, 1 value join            */
    int32_t tile_rows;       /* rows per shared-memory tile               */
    int32_t consumer_warps;  /* scoring warps per CTA (dense <= 15, join filter <= 31) */
    int32_t ctas_per_sm;     /* resident CTAs per SM for the scan         */
    int32_t stages;          /* TMA pipeline depth                        */
    int32_t lanes_per_row;   /* join filter: lanes sharing one row (1-8);
                              * 32: a whole warp per row over a group map
                              * striped across the banks by bin (one
                              * scanned plane whose rows are 128, 256 or
                              * 512 bytes, W <= 128; tile_rows then sets
                              * the rows per tile, a multiple of 32);
                              * 0: the library's choice (32 for 16-bit
                              * planes where it applies, else W / 32)   */
    int32_t sketch_cta_bits; /* sketch: sets whose size has at least this
                              * many bits get a whole CTA, the rest a warp;
                              * 0 = library choice, 64 = warps only      */
    int32_t join_lanes;      /* hoph_self_join: blocks in flight at once,
                              * each on a stream and scratch of the plan's
                              * own (1-8; 0 = library choice, 8)         */
} hoph_exec;

typedef struct hoph_plan hoph_plan;

/*
 * Create a plan: validate the parameters, build psi (Sec. 3.2; Fisher-Yates
 * over D driven by SplitMix64(seed), or the 2-universal hash), the bin
 * layout (Sec. 3.2 equal bins or Sec. 4.1 a:b groups), the packed psi ->
 * (bin, offset) table in device memory, the MinWise tables if requested,
 * and the exact integer decision thresholds derived from the binomial tails
 * of Definition 1 (Eq. 10-11).  Synchronous; uses the current CUDA device.
 * *out receives the plan (NULL on error).
 */
int hoph_plan_create(const hoph_params *params, hoph_plan **out);

/* As hoph_plan_create, with psi given as a host table of D entries
 * (host_perm[x] = psi(x), a permutation of 0..D-1).  Copied; the caller
 * keeps ownership of host_perm. */
int hoph_plan_create_with_perm(const hoph_params *params, const uint32_t *host_perm,
                               hoph_plan **out);

/* Free a plan and everything it owns (synchronises the device). */
void hoph_plan_destroy(hoph_plan *plan);

/* Copy read-only facts about a plan into *out. */
int hoph_plan_get_info(const hoph_plan *plan, hoph_plan_info *out);

/* Set execution knobs (exec = NULL restores the defaults). */
int hoph_plan_set_exec(hoph_plan *plan, const hoph_exec *exec);

/*
 * The small-probability limits of Definition 1 for X ~ Bin(k', T) (Table 2's
 * two tails, Eq. 10-11), exactly: *U = min{j : P(X >= j) <= eps} and
 * *L = max{j : P(X < j) <= eps}, j in 0..k'+1, with T = thr_num / thr_den
 * and eps a double taken at its exact binary value.  The tails are compared
 * with eps in integer arithmetic (td^k' P(X = i) is an integer), so an eps
 * equal to a tail, or one ulp from it, is decided exactly.  These are the
 * limits every plan's decisions use (hoph_plan_info.upper_limit /
 * lower_limit).  Host only: no device, no allocation visible to the caller.
 *   k_group   k', 1..65535; thr_num 1..thr_den; thr_den 1..65535;
 *   epsilon   finite, >= 0.
 * Returns HOPH_OK, or HOPH_ERR_PARAM for arguments out of range or a NULL
 * output pointer (outputs untouched then).
 */
int hoph_small_probability_limits(uint32_t k_group, uint32_t thr_num, uint32_t thr_den,
                                  double epsilon, int64_t *U, int64_t *L);

/*
 * OPH / HOPH sketches of n_sets sets (Sec. 3.2 "One Permutation Hashing",
 * Sec. 4.1 construction): for every bin, the smallest psi-value of the set
 * that falls in it minus the bin's lower bound, or HOPH_EMPTY_VALUE.
 *   d_ids       uint32 IDs of all sets back to back (duplicates allowed).
 *   d_offsets   int64[n_sets + 1]; set i is d_ids[d_offsets[i] .. d_offsets[i+1]).
 *   d_planes    uint32[G][n_sets][k'] output, group-major: plane g holds
 *               bins g*k' .. (g+1)*k'-1 of every set.
 * IDs >= D are skipped and flag HOPH_ERR_ID_RANGE in the status word.
 */
int oph_build_sketches(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                       int64_t n_sets, uint32_t *d_planes, void *stream);

/*
 * MinWise sketches (Sec. 1, the baseline): d_sketches[n_sets][minwise_k],
 * entry t = min over the set of psi_t(x); HOPH_EMPTY_VALUE for an empty set.
 * Needs a plan created with minwise_k > 0.  Same input layout as above.
 */
int minwise_build_sketches(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                           int64_t n_sets, uint32_t *d_sketches, void *stream);

/*
 * Compare every query with every collection row and return the similar
 * pairs (Algorithm 1 for HOPH_MODE_GOPH, Algorithm 2 for HOPH_MODE_HOPH,
 * Eq. 6 over all bins for HOPH_MODE_OPH_FULL, MinWise for
 * HOPH_MODE_MINWISE_FULL).
 *   d_query_planes  uint32[G][n_queries][k'] (MinWise: [n_queries][minwise_k]).
 *   d_coll_planes   uint32[G][n_rows][k']    (MinWise: [n_rows][minwise_k]).
 *   d_out           hoph_pair[out_capacity]; receives the accepted pairs
 *                   sorted by (query, row).
 *   d_out_count     int64 on the device; receives the number of accepted
 *                   pairs.  If it exceeds out_capacity, only out_capacity
 *                   pairs (an unspecified subset) are written, the status
 *                   word gets HOPH_ERR_CAPACITY, and the call can be repeated
 *                   with a larger buffer.
 *   d_stats         nullable; hoph_stats accumulated on the device.
 * Mode GOPH and OPH_FULL need an equal-bin plan (a = b = 0); mode HOPH an
 * (a:b) plan; MINWISE_FULL a plan with minwise_k > 0.
 * Plane pointers must be 16-byte aligned.  Every stored value must be one the
 * sketch functions of this plan can produce (an offset below its bin's width,
 * or HOPH_EMPTY_VALUE): the value join indexes shared-memory tables by the
 * values without a bounds check, so other values are undefined behaviour.
 */
int hoph_query_batch(hoph_plan *plan, uint32_t mode, const uint32_t *d_query_planes,
                     int64_t n_queries, const uint32_t *d_coll_planes, int64_t n_rows,
                     hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                     hoph_stats *d_stats, void *stream);

/*
 * Compact sketches: a bin's stored value is its minimum's offset from the
 * bin's lower bound (Sec. 3.2 and 4.1 re-index each bin so the stored value
 * is as small as possible), so when every bin of the plan is at most 65,535
 * values wide (hoph_plan_info.max_bin_width) the offsets fit in 16 bits,
 * with HOPH_EMPTY_VALUE16 (0xFFFF) for an empty bin.  Same layout and the
 * same values as the uint32 planes, half the bytes; decisions and output
 * identical to oph_build_sketches + hoph_query_batch.
 *   oph_build_sketches16   as oph_build_sketches, d_planes uint16[G][n_sets][k'].
 *   hoph_query_batch16     as hoph_query_batch over uint16 planes; modes
 *                          GOPH, HOPH and OPH_FULL.
 * Both return HOPH_ERR_UNSUPPORTED for a plan with a bin wider than 65,535
 * values (and the query for mode MINWISE_FULL, whose values are whole
 * psi-values).  The value join needs k' to be a multiple of 64 here (32 for
 * uint32 planes); other shapes use the dense scan.
 */
int oph_build_sketches16(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                         int64_t n_sets, uint16_t *d_planes, void *stream);
int hoph_query_batch16(hoph_plan *plan, uint32_t mode, const uint16_t *d_query_planes,
                       int64_t n_queries, const uint16_t *d_coll_planes, int64_t n_rows,
                       hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                       hoph_stats *d_stats, void *stream);

/*
 * All near-duplicate pairs inside one collection (Sec. 3.1 states the task
 * over a single dataset: every pair of its items): every pair of rows
 * (i, j), i < j, that the rule of `mode` accepts, as hoph_pair {query = i,
 * row = j, groups, matches}, sorted by (i, j).
 *   d_planes    uint32[G][n_rows][k'] sketches (as for hoph_query_batch).
 *   batch       rows taken as queries per block (1..4096): block b compares
 *               rows b*batch .. b*batch+batch-1 with rows b*batch .. n_rows-1,
 *               so about n_rows^2 / 2 pairs are compared in all.
 *   d_out, out_capacity, d_out_count, d_stats   as for hoph_query_batch; the
 *               statistics cover exactly the pairs i < j (entering[0] sums to
 *               n_rows (n_rows - 1) / 2): a block skips the pairs i >= j
 *               among its own rows before counting or deciding them.
 * Modes GOPH, HOPH and OPH_FULL (not MinWise).  A block reads its query
 * planes in place (no copy).  Up to exec.join_lanes blocks (default 8) are
 * in flight at once, each on a stream and a scratch buffer the plan owns,
 * forked from `stream` and joined back to it before the final sort, so the
 * call stays ordered on `stream` (and can be captured into a graph).  The
 * first call with more than one lane creates those streams: make it outside
 * a stream capture.  n_rows < 2^32.
 */
int hoph_self_join(hoph_plan *plan, uint32_t mode, const uint32_t *d_planes, int64_t n_rows,
                   int64_t batch, hoph_pair *d_out, int64_t out_capacity, int64_t *d_out_count,
                   hoph_stats *d_stats, void *stream);

/*
 * hoph_self_join over compact planes (uint16[G][n_rows][k'] from
 * oph_build_sketches16: each bin's minimum as its offset from the bin's lower
 * bound, HOPH_EMPTY_VALUE16 for an empty bin; Sec. 3.2 / 4.1).  Same
 * arguments, pairs, statistics and errors as hoph_self_join on the uint32
 * planes of the same sets; HOPH_ERR_UNSUPPORTED as for hoph_query_batch16.
 */
int hoph_self_join16(hoph_plan *plan, uint32_t mode, const uint16_t *d_planes, int64_t n_rows,
                     int64_t batch, hoph_pair *d_out, int64_t out_capacity,
                     int64_t *d_out_count, hoph_stats *d_stats, void *stream);

/*
 * One part of a self-join split over `parts` callers (one per GPU, each
 * holding the whole collection): blocks part, part + parts, part + 2 parts,
 * ... of the blocks hoph_self_join would run (block b: rows b*batch ..
 * b*batch+batch-1 as queries against the rows from b*batch on).  The parts'
 * pairs are disjoint, each part's sorted by (query, row); their union in that
 * order is hoph_self_join's output and the sum of their statistics its
 * statistics.  Dealing blocks round-robin gives each part about the same
 * number of pair comparisons.
 *   d_planes     uint32 (value_bytes 4) or compact uint16 (value_bytes 2)
 *                planes [G][n_rows][k'].
 *   part, parts  0 <= part < parts, else HOPH_ERR_PARAM.
 * Other arguments and errors as hoph_self_join / hoph_self_join16.
 */
int hoph_self_join_part(hoph_plan *plan, uint32_t mode, const void *d_planes,
                        uint32_t value_bytes, int64_t n_rows, int64_t batch, int64_t part,
                        int64_t parts, hoph_pair *d_out, int64_t out_capacity,
                        int64_t *d_out_count, hoph_stats *d_stats, void *stream);

/*
 * oph_build_sketches without any device allocation.  The paper has no
 * counterpart: this serves callers that may not allocate device memory
 * during the call, such as a serving loop whose device memory is owned by
 * its own pool allocator, or a latency-critical path that cannot take the
 * device-wide synchronisation a cudaMalloc / cudaFree may cause.
 * Same arguments, output and error behaviour as oph_build_sketches (and
 * bit-identical sketches); the plan must already exist.
 *   - n_sets is limited to 262,144 per call; larger inputs return
 *     HOPH_ERR_TOO_LARGE before anything is enqueued.
 *   - The size-sorted work list lives in a fixed ~1 MiB device array inside
 *     the library, present on every GPU that loads it until the process
 *     exits.  The first call on each device looks up that array's device
 *     address (cudaGetSymbolAddress, with the device current); make that
 *     first call before any stream capture (during one it returns
 *     HOPH_ERR_CAPTURE and enqueues nothing).  The address is kept for the
 *     device's context: it is not valid after a cudaDeviceReset.
 *   - Every call on a device shares the one array: calls whose work overlaps
 *     on the GPU (other streams, other host threads) race and corrupt each
 *     other's work list.  Order such calls on one stream.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 */
int oph_build_sketches_static(hoph_plan *plan, const uint32_t *d_ids, const int64_t *d_offsets,
                              int64_t n_sets, uint32_t *d_planes, void *stream);

/*
 * Per-pair, per-group bin counts (Eq. 2-5) of every (query, row) pair with
 * no early exit: d_counts[n_queries][n_rows][G][3] uint16 holding
 * (matched bins, bins empty in both, bins empty in exactly one).
 */
int hoph_pair_counts(hoph_plan *plan, const uint32_t *d_query_planes, int64_t n_queries,
                     const uint32_t *d_coll_planes, int64_t n_rows, uint16_t *d_counts,
                     void *stream);

/*
 * Seeded synthetic IDs on the device (benchmark inputs, no method
 * arithmetic): element e (0 <= e < n_ids) receives
 *   h = SplitMix64 output number e+1 of the stream seeded with `seed`,
 *   kind 0: ((h >> 32) * D) >> 32 (uniform over 0..D-1);
 *   kind 1: the first index i with u < d_cdf[i], u = (h >> 11) * 2^-53
 *           (inverse-CDF sampling from the float64 table d_cdf[n_cdf]).
 */
int hoph_synth_ids(uint64_t seed, int64_t first, int64_t n_ids, uint64_t D, uint32_t kind,
                   const double *d_cdf, int64_t n_cdf, uint32_t *d_ids, void *stream);

/*
 * Optional phase timing of hoph_query_batch (for benchmarks; no paper
 * counterpart).  While enabled, every call records CUDA events on its stream
 * around four phases: (0) the join-index build, (1) the streaming pass over
 * the first plane (join filter or dense scan), (2) the join's counting of
 * candidate rows, (3) the sort and statistics kernels.
 * hoph_plan_read_timing waits for the last event, writes the summed
 * milliseconds of the four phases to ms[0..3], the number of recorded calls
 * to *calls and the number of kernels launched by library calls on this plan
 * to *launches (both nullable), then resets the counters.
 */
int hoph_plan_enable_timing(hoph_plan *plan, int enable);
int hoph_plan_read_timing(hoph_plan *plan, double *ms, int64_t *calls, int64_t *launches);

/* The four phase times of the most recently recorded call, without resetting
 * anything: for a call captured in a CUDA graph, its events are recorded
 * again by every replay, so this reads the latest replay (after waiting for
 * it).  HOPH_ERR_PARAM if no call has been recorded. */
int hoph_plan_peek_timing(hoph_plan *plan, double *ms);

/*
 * Failure-path check of the bounded device waits (no paper counterpart):
 * launches one warp that runs the pipeline's mbarrier wait on a barrier no
 * thread ever completes, with a limit of limit_ns (1 ns .. 2 s).  The wait
 * gives up and records HOPH_ERR_TIMEOUT in the plan's status word, which
 * hoph_sync_status then returns; the CUDA context stays usable.
 */
int hoph_check_bounded_wait(hoph_plan *plan, uint64_t limit_ns, void *stream);

/*
 * Sketches of synthetic sets whose IDs are generated inside the kernel and
 * never stored (benchmark inputs of any size; same sketches as
 * hoph_synth_ids followed by oph_build_sketches): set i holds the kind-0 IDs
 * (uniform over 0..D-1) of elements d_offsets[i] .. d_offsets[i+1]-1 of the
 * generator stream `seed`.  Output layout and errors as oph_build_sketches.
 */
int hoph_synth_sketch(hoph_plan *plan, uint64_t seed, uint64_t D, const int64_t *d_offsets,
                      int64_t n_sets, uint32_t *d_planes, void *stream);

/*
 * Integer-throughput probe (benchmark tooling; no paper counterpart): the
 * measured peak that ALU-bound sketching (the hashed permutation's 61-bit
 * arithmetic) is compared with.  A grid of (SMs x 8) CTAs of 256 threads;
 * every thread runs `iters` rounds of 8 independent dependency chains of
 * one operation:
 *   kind 0: x = x * a + b, 32-bit (multiply-add);
 *   kind 1: x = x * a + b, 64-bit (low half of a 64 x 64 product);
 *   kind 2: x = mulhi(x, a) + b, 64-bit (high half of a 64 x 64 product).
 * Operations per launch = 8 * iters * (SMs x 8 x 256).  d_sink (uint64,
 * one per thread of the grid: SMs x 2048 entries) receives the chains'
 * final values so no work is dropped.  iters in 1..2^24, kind in 0..2;
 * HOPH_ERR_PARAM otherwise.  Asynchronous on `stream`.
 */
int hoph_int_probe(uint32_t kind, int64_t iters, uint64_t *d_sink, void *stream);

/* Synchronise `stream`, then return and clear the plan's device status word
 * (HOPH_OK if no device-side error was recorded). */
int hoph_sync_status(hoph_plan *plan, void *stream);

/* Text for a status code (static storage). */
const char *hoph_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HOPH_H */
