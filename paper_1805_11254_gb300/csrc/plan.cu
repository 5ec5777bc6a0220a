// Plan creation: parameter validation, psi (Sec. 3.2), the bin layout
// (Sec. 3.2 equal bins, Sec. 4.1 a:b groups), the packed psi table, the
// MinWise tables, and the small-probability limits of Definition 1.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"

int hoph_cuda_fail(cudaError_t e) {
    (void)e;
    cudaGetLastError();  // clear a sticky-free error so later calls are not poisoned
    return HOPH_ERR_CUDA;
}

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): seeds the Fisher-Yates shuffle.
struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// psi over {0..D-1}: Fisher-Yates from the identity, i = D-1 down to 1,
// swap with j = next() mod (i+1).
void fisher_yates(uint64_t D, uint64_t seed, uint32_t *out) {
    for (uint64_t i = 0; i < D; ++i) out[i] = (uint32_t)i;
    SplitMix g{seed};
    for (uint64_t i = D - 1; i >= 1; --i) {
        const uint64_t j = g.next() % (i + 1);
        std::swap(out[i], out[j]);
    }
}

const uint64_t kP61 = (1ull << 61) - 1;

int ceil_log2(uint64_t v) {
    int b = 0;
    while ((1ull << b) < v) ++b;
    return b;
}

// Bounds of the k bins.  Equal bins (a = b = 0): lo_j = ceil(j D / k).
// (a:b): G - 1 splits give floor(rem a / (a + b)) to the next group, the
// last group keeps the remainder; group g's k' bins start at
// s_g + ceil(i z_g / k').
bool build_layout(const hoph_params &p, std::vector<uint64_t> &lo, uint64_t *z) {
    const uint32_t k = p.k, kg = p.k_group, G = k / kg;
    lo.assign(k + 1, 0);
    if (p.a == 0 && p.b == 0) {
        if (p.universe_D < k) return false;
        for (uint32_t j = 0; j <= k; ++j)
            lo[j] = (uint64_t)(((unsigned __int128)j * p.universe_D + k - 1) / k);
    } else {
        uint64_t rem = p.universe_D, start = 0;
        for (uint32_t g = 0; g < G; ++g) {
            const uint64_t zg =
                (g + 1 < G) ? (uint64_t)(((unsigned __int128)rem * p.a) / ((uint64_t)p.a + p.b))
                            : rem;
            if (zg < kg) return false;
            for (uint32_t i = 0; i < kg; ++i)
                lo[(size_t)g * kg + i] = start + ((uint64_t)i * zg + kg - 1) / kg;
            start += zg;
            rem -= zg;
        }
        lo[k] = p.universe_D;
    }
    for (uint32_t g = 0; g < G; ++g) z[g] = lo[(size_t)(g + 1) * kg] - lo[(size_t)g * kg];
    return true;
}

// Exact small-probability limits (Definition 1 with the two tails of
// Eq. 11): X ~ Bin(k', T), U = min{j : P(X >= j) <= eps},
// L = max{j : P(X < j) <= eps}.  With T = tn/td in lowest terms and
// s = td - tn, A_i = C(k', i) tn^i s^(k'-i) = td^k' P(X = i) is an integer,
// so "tail <= eps" is the integer comparison  sum A_i <= mant 2^e td^k'
// with eps = mant 2^e exactly (mant < 2^53).  Non-negative integers are
// little-endian vectors of 32-bit limbs.
namespace big {
typedef std::vector<uint32_t> Num;

void trim(Num &a) {
    while (!a.empty() && a.back() == 0) a.pop_back();
}
void mul_small(Num &a, uint32_t m) {
    if (m == 0) {
        a.clear();
        return;
    }
    uint64_t carry = 0;
    for (uint32_t &l : a) {
        const uint64_t v = (uint64_t)l * m + carry;
        l = (uint32_t)v;
        carry = v >> 32;
    }
    if (carry) a.push_back((uint32_t)carry);
}
// a /= d; the callers only divide where the quotient is exact
void div_small(Num &a, uint32_t d) {
    uint64_t r = 0;
    for (size_t i = a.size(); i-- > 0;) {
        const uint64_t v = (r << 32) | a[i];
        a[i] = (uint32_t)(v / d);
        r = v % d;
    }
    trim(a);
}
void add(Num &a, const Num &b) {
    if (a.size() < b.size()) a.resize(b.size(), 0);
    uint64_t carry = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        const uint64_t v = (uint64_t)a[i] + (i < b.size() ? b[i] : 0u) + carry;
        a[i] = (uint32_t)v;
        carry = v >> 32;
    }
    if (carry) a.push_back((uint32_t)carry);
}
Num shl(const Num &a, uint32_t bits) {
    if (a.empty()) return a;
    const uint32_t w = bits / 32, r = bits % 32;
    Num out(a.size() + w + 1, 0);
    for (size_t i = 0; i < a.size(); ++i) {
        out[i + w] |= a[i] << r;
        if (r) out[i + w + 1] |= a[i] >> (32 - r);
    }
    trim(out);
    return out;
}
int cmp(const Num &a, const Num &b) {  // both trimmed
    if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
    for (size_t i = a.size(); i-- > 0;)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}
Num pow_small(uint32_t base, uint32_t e) {
    Num a{1};
    for (uint32_t i = 0; i < e; ++i) mul_small(a, base);
    trim(a);
    return a;
}
}  // namespace big

// x <= eps * td^k' with eps = mant 2^e2, given rhs = mant td^k'
struct EpsBound {
    big::Num rhs;
    int e2 = 0;
    bool le(const big::Num &x) const {
        if (e2 >= 0) return big::cmp(x, big::shl(rhs, (uint32_t)e2)) <= 0;
        return big::cmp(big::shl(x, (uint32_t)(-e2)), rhs) <= 0;
    }
};

uint32_t gcd32(uint32_t a, uint32_t b) {
    while (b) {
        const uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

void small_probability_limits(uint32_t kg, int64_t tn64, int64_t td64, double eps, int64_t *U,
                              int64_t *L, int32_t *always) {
    *always = eps >= 1.0;
    const uint32_t g = gcd32((uint32_t)tn64, (uint32_t)td64);
    const uint32_t tn = (uint32_t)tn64 / g, td = (uint32_t)td64 / g, s = td - tn;
    if (s == 0) {  // T = 1: X = k' always
        *U = eps >= 1.0 ? 0 : (int64_t)kg + 1;
        *L = eps >= 1.0 ? (int64_t)kg + 1 : (int64_t)kg;
        return;
    }
    EpsBound bound;
    if (eps > 0.0) {
        int e = 0;
        const double f = frexp(eps, &e);  // eps = f 2^e, f in [0.5, 1)
        uint64_t mant = (uint64_t)ldexp(f, 53);
        bound.e2 = e - 53;
        while (!(mant & 1)) {
            mant >>= 1;
            ++bound.e2;
        }
        // rhs = mant td^k'
        big::Num t = big::pow_small(td, kg), lo_part = t;
        big::mul_small(lo_part, (uint32_t)mant);
        big::Num hi_part = t;
        big::mul_small(hi_part, (uint32_t)(mant >> 32));
        hi_part = big::shl(hi_part, 32);
        big::add(lo_part, hi_part);
        big::trim(lo_part);
        bound.rhs = lo_part;
    }  // eps = 0: rhs stays 0, only a zero tail qualifies
    // U: upper tails from the top, A_k' = tn^k', A_{i-1} = A_i i s / ((k'-i+1) tn);
    // {j : P(X >= j) <= eps} is [U, k'+1]
    {
        big::Num A = big::pow_small(tn, kg), up;
        int64_t u = 0;
        for (int64_t j = kg; j >= 0; --j) {
            big::add(up, A);
            big::trim(up);
            if (!bound.le(up)) {
                u = j + 1;
                break;
            }
            if (j > 0) {
                big::mul_small(A, (uint32_t)j * s);
                big::div_small(A, (uint32_t)(kg - j + 1) * tn);
            }
        }
        *U = u;
    }
    // L: lower tails from the bottom, A_0 = s^k', A_{i+1} = A_i (k'-i) tn / ((i+1) s);
    // {j : P(X < j) <= eps} is [0, L]
    {
        big::Num A = big::pow_small(s, kg), low;
        int64_t l = (int64_t)kg + 1;
        for (int64_t j = 1; j <= (int64_t)kg + 1; ++j) {
            big::add(low, A);  // low = P(X < j) td^k'
            big::trim(low);
            if (!bound.le(low)) {
                l = j - 1;
                break;
            }
            if (j <= (int64_t)kg) {
                big::mul_small(A, (uint32_t)(kg - j + 1) * tn);
                big::div_small(A, (uint32_t)j * s);
            }
        }
        *L = l;
    }
}

// The literal recursion's integers (hoph_decide) stay below 2^120 for every
// group at which it decides (l < G): |X_j| <= |X_{j-1}| c^j + k' td a^{s_j}.
bool literal_fits(const DecideParams &dp) {
    const long double lim = ldexpl(1.0L, 120);
    long double X = (long double)dp.tn * dp.kg, As = 1.0L;
    for (uint32_t j = 1; j < dp.G; ++j) {
        const long double cj = powl((long double)dp.rc, (long double)j);
        As *= powl((long double)dp.ra, (long double)j);
        X = X * cj + (long double)dp.kg * dp.td * As;
        if (X >= lim || (long double)dp.kg * 65536.0L * dp.td * As >= lim) return false;
    }
    return true;
}

int validate(const hoph_params &p) {
    if (p.universe_D == 0 || p.universe_D > (1ull << 32)) return HOPH_ERR_PARAM;
    if (p.k == 0 || p.k_group == 0 || p.k % p.k_group) return HOPH_ERR_PARAM;
    if (p.k > 65535) return HOPH_ERR_PARAM;
    if (p.k / p.k_group > HOPH_MAX_GROUPS) return HOPH_ERR_PARAM;
    if ((p.a == 0) != (p.b == 0)) return HOPH_ERR_PARAM;
    if (p.thr_den == 0 || p.thr_den > 65535 || p.thr_num == 0 || p.thr_num > p.thr_den)
        return HOPH_ERR_PARAM;
    if (!(p.epsilon >= 0.0) || !isfinite(p.epsilon)) return HOPH_ERR_PARAM;
    if (p.empty_rule > HOPH_EMPTY_NONE) return HOPH_ERR_PARAM;
    if (p.weighting > HOPH_WEIGHT_LITERAL) return HOPH_ERR_PARAM;
    if (p.perm_kind == HOPH_PERM_TABLE) {
        if (p.universe_D > (1ull << 30)) return HOPH_ERR_UNSUPPORTED;
    } else if (p.perm_kind == HOPH_PERM_HASH61) {
        if (p.universe_D != (1ull << 32)) return HOPH_ERR_PARAM;
        if (p.minwise_k) return HOPH_ERR_UNSUPPORTED;
    } else {
        return HOPH_ERR_PARAM;
    }
    if (p.minwise_k > 4096 || (uint64_t)p.minwise_k * p.universe_D > (1ull << 31))
        return HOPH_ERR_UNSUPPORTED;
    // exact HOPH decisions need products of up to G effective-bin counts to
    // stay inside __int128 next to T's denominator and the space sizes
    if (p.a != 0 && 58 + (p.k / p.k_group) * ceil_log2((uint64_t)p.k_group + 1) > 126)
        return HOPH_ERR_UNSUPPORTED;
    return HOPH_OK;
}

void plan_free(hoph_plan *pl) {
    if (!pl) return;
    for (cudaEvent_t e : pl->events) cudaEventDestroy(e);
    for (int m = 0; m < 4; ++m) cudaFree(pl->d_table[m]);
    cudaFree(pl->d_key);
    cudaFree(pl->d_lo);
    cudaFree(pl->d_kb);
    cudaFree(pl->d_minwise);
    cudaFree(pl->d_status);
    cudaFree(pl->d_scratch);
    for (int i = 0; i < hoph_plan::kMaxLanes; ++i) {
        cudaFree(pl->lane_scratch[i]);
        if (pl->lane_stream[i]) cudaStreamDestroy(pl->lane_stream[i]);
        if (pl->lane_event[i]) cudaEventDestroy(pl->lane_event[i]);
    }
    if (pl->fork_event) cudaEventDestroy(pl->fork_event);
    if (pl->h_status) cudaFreeHost(pl->h_status);
    delete pl;
}

int plan_create(const hoph_params *params, const uint32_t *host_perm, hoph_plan **out) {
    if (!out) return HOPH_ERR_PARAM;
    *out = nullptr;
    if (!params) return HOPH_ERR_PARAM;
    const hoph_params p = *params;
    int rc = validate(p);
    if (rc) return rc;
    if (host_perm && p.perm_kind != HOPH_PERM_TABLE) return HOPH_ERR_PARAM;

    hoph_plan *pl = new (std::nothrow) hoph_plan();
    if (!pl) return HOPH_ERR_NOMEM;
    pl->P = p;
    pl->G = p.k / p.k_group;
    if (!build_layout(p, pl->lo, pl->z)) {
        delete pl;
        return HOPH_ERR_PARAM;
    }
    uint64_t max_width = 0;
    for (uint32_t j = 0; j < p.k; ++j) max_width = std::max(max_width, pl->lo[j + 1] - pl->lo[j]);
    if (max_width >= (1ull << 32)) {  // an offset could collide with the empty marker
        delete pl;
        return HOPH_ERR_PARAM;
    }
    pl->max_width = max_width;

    // decision parameters shared by GOPH / HOPH
    DecideParams &dp = pl->dp;
    dp.mode = (p.a == 0) ? HOPH_MODE_GOPH : HOPH_MODE_HOPH;
    dp.rule = p.empty_rule;
    dp.G = pl->G;
    dp.kg = p.k_group;
    dp.tn = p.thr_num;
    dp.td = p.thr_den;
    small_probability_limits(p.k_group, p.thr_num, p.thr_den, p.epsilon, &dp.U, &dp.L,
                             &dp.always_stop);
    dp.literal = p.weighting == HOPH_WEIGHT_LITERAL && p.a != 0;
    dp.ra = p.a;
    dp.rc = (int64_t)p.a + p.b;
    if (dp.literal && !literal_fits(dp)) {
        delete pl;
        return HOPH_ERR_PARAM;
    }
    dp.zsuf[pl->G] = 0;
    for (int g = (int)pl->G - 1; g >= 0; --g) {
        dp.z[g] = pl->z[g];
        dp.zsuf[g] = dp.zsuf[g + 1] + pl->z[g];
    }

    cudaError_t e = cudaGetDevice(&pl->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(pl->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&pl->h_status, sizeof(int32_t));
    if (e != cudaSuccess) {
        plan_free(pl);
        return hoph_cuda_fail(e);
    }

    if (p.perm_kind == HOPH_PERM_TABLE) {
        const uint64_t D = p.universe_D;
        std::vector<uint32_t> perm;
        const uint32_t *psi = host_perm;
        if (!psi) {
            try {
                perm.resize(D);
            } catch (...) {
                plan_free(pl);
                return HOPH_ERR_NOMEM;
            }
            fisher_yates(D, p.seed, perm.data());
            psi = perm.data();
        }
        // packed key: (bin << key_bits) | (psi(x) - lo[bin])
        const int bin_bits = ceil_log2(p.k);
        pl->key_bits = 32 - bin_bits;
        if (pl->key_bits < 32 && max_width > (1ull << pl->key_bits)) {
            plan_free(pl);
            return HOPH_ERR_UNSUPPORTED;
        }
        std::vector<uint32_t> key(D);
        std::vector<uint8_t> seen(host_perm ? D : 0, 0);
        for (uint64_t x = 0; x < D; ++x) {
            const uint64_t v = psi[x];
            if (v >= D || (host_perm && seen[v]++)) {  // not a permutation of 0..D-1
                plan_free(pl);
                return HOPH_ERR_PARAM;
            }
            const uint32_t bin = (uint32_t)(std::upper_bound(pl->lo.begin(), pl->lo.end(), v) -
                                            pl->lo.begin() - 1);
            key[x] = (uint32_t)(((uint64_t)bin << pl->key_bits) | (v - pl->lo[bin]));
        }
        e = cudaMalloc(&pl->d_key, D * sizeof(uint32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(pl->d_key, key.data(), D * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && p.minwise_k) {
            const uint32_t mk = p.minwise_k;
            std::vector<uint32_t> tab((size_t)D * mk), one(D);
            for (uint32_t t = 0; t < mk; ++t) {
                fisher_yates(D, p.seed + t, one.data());
                for (uint64_t x = 0; x < D; ++x) tab[(size_t)x * mk + t] = one[x];
            }
            e = cudaMalloc(&pl->d_minwise, tab.size() * sizeof(uint32_t));
            if (e == cudaSuccess)
                e = cudaMemcpy(pl->d_minwise, tab.data(), tab.size() * sizeof(uint32_t),
                               cudaMemcpyHostToDevice);
        }
    } else {
        // 2-universal hash parameters from the seed: a = 1 + next() mod (p-1), b = next() mod p
        SplitMix g{p.seed};
        pl->hash_a = 1 + g.next() % (kP61 - 1);
        pl->hash_b = g.next() % kP61;
    }
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_lo, (p.k + 1) * sizeof(uint64_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_lo, pl->lo.data(), (p.k + 1) * sizeof(uint64_t),
                       cudaMemcpyHostToDevice);
    // join keys with a guard key below every bin: kb[w] = lo[w] + w + 1
    std::vector<uint64_t> kb(p.k + 1);
    for (uint32_t w = 0; w <= p.k; ++w) kb[w] = pl->lo[w] + w + 1;
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_kb, (p.k + 1) * sizeof(uint64_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_kb, kb.data(), (p.k + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        plan_free(pl);
        return hoph_cuda_fail(e);
    }
    pl->exec.strategy = -1;
    *out = pl;
    return HOPH_OK;
}

}  // namespace

cudaError_t hoph_ensure_smem(const void *func, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> set_to;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int &cur = set_to[std::make_pair(func, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

cudaError_t hoph_occupancy(int *blocks, const void *func, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> known;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_tuple(func, dev, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = known.find(key);
        if (it != known.end()) {
            *blocks = it->second;
            return cudaSuccess;
        }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, func, threads, smem);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    known[key] = *blocks;
    return cudaSuccess;
}

bool hoph_capturing(cudaStream_t stream) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

int hoph_scratch(hoph_plan *plan, size_t bytes, int lane, cudaStream_t stream, void **out) {
    void *&buf = lane > 0 ? plan->lane_scratch[lane] : plan->d_scratch;
    size_t &have = lane > 0 ? plan->lane_scratch_bytes[lane] : plan->scratch_bytes;
    *out = buf;
    if (bytes <= have) return HOPH_OK;
    // growing would free memory a captured graph may already point at
    if (hoph_capturing(stream)) return HOPH_ERR_CAPTURE;
    size_t want = std::max(bytes, have * 2);
    want = (want + 255) & ~(size_t)255;
    if (buf) {
        cudaDeviceSynchronize();  // a previous launch may still read the old buffer
        cudaFree(buf);
        buf = nullptr;
        have = 0;
    }
    *out = nullptr;
    if (cudaMalloc(&buf, want) != cudaSuccess) {
        cudaGetLastError();
        return HOPH_ERR_NOMEM;
    }
    have = want;
    *out = buf;
    return HOPH_OK;
}

void hoph_timing_mark(hoph_plan *plan, int which, cudaStream_t s) {
    if (!plan->timing) return;
    const size_t idx = plan->events_used + (size_t)which;
    while (plan->events.size() <= idx) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        plan->events.push_back(e);
    }
    // while a stream is captured, only an "external" record becomes an event
    // node of the graph (a plain record would turn into a dependency edge)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cudaGetLastError();
    if (cap == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(plan->events[idx], s, cudaEventRecordExternal);
    else
        cudaEventRecord(plan->events[idx], s);
    if (which == kTimingMarks - 1) plan->events_used += kTimingMarks;
}

extern "C" {

int hoph_plan_enable_timing(hoph_plan *plan, int enable) {
    if (!plan) return HOPH_ERR_PARAM;
    plan->timing = enable != 0;
    plan->events_used = 0;
    plan->launches = 0;
    return HOPH_OK;
}

int hoph_plan_read_timing(hoph_plan *plan, double *ms, int64_t *calls, int64_t *launches) {
    if (!plan || !ms) return HOPH_ERR_PARAM;
    for (int i = 0; i < kTimingMarks - 1; ++i) ms[i] = 0.0;
    const size_t n = plan->events_used / kTimingMarks;
    if (n) HOPH_CUDA_TRY(cudaEventSynchronize(plan->events[plan->events_used - 1]));
    for (size_t c = 0; c < n; ++c)
        for (int i = 0; i < kTimingMarks - 1; ++i) {
            float t = 0.f;
            HOPH_CUDA_TRY(cudaEventElapsedTime(&t, plan->events[kTimingMarks * c + i],
                                               plan->events[kTimingMarks * c + i + 1]));
            ms[i] += t;
        }
    if (calls) *calls = (int64_t)n;
    if (launches) *launches = plan->launches;
    plan->events_used = 0;
    plan->launches = 0;
    return HOPH_OK;
}

int hoph_plan_peek_timing(hoph_plan *plan, double *ms) {
    if (!plan || !ms) return HOPH_ERR_PARAM;
    if (plan->events_used < (size_t)kTimingMarks) return HOPH_ERR_PARAM;
    const size_t b = plan->events_used - kTimingMarks;
    HOPH_CUDA_TRY(cudaEventSynchronize(plan->events[b + kTimingMarks - 1]));
    for (int i = 0; i < kTimingMarks - 1; ++i) {
        float t = 0.f;
        HOPH_CUDA_TRY(cudaEventElapsedTime(&t, plan->events[b + i], plan->events[b + i + 1]));
        ms[i] = t;
    }
    return HOPH_OK;
}

int hoph_plan_create(const hoph_params *params, hoph_plan **out) {
    return plan_create(params, nullptr, out);
}

int hoph_small_probability_limits(uint32_t k_group, uint32_t thr_num, uint32_t thr_den,
                                  double epsilon, int64_t *U, int64_t *L) {
    if (!U || !L || k_group == 0 || k_group > 65535 || thr_den == 0 || thr_den > 65535 ||
        thr_num == 0 || thr_num > thr_den || !(epsilon >= 0.0) || !isfinite(epsilon))
        return HOPH_ERR_PARAM;
    int32_t always = 0;
    small_probability_limits(k_group, thr_num, thr_den, epsilon, U, L, &always);
    return HOPH_OK;
}

int hoph_plan_create_with_perm(const hoph_params *params, const uint32_t *host_perm,
                               hoph_plan **out) {
    if (!host_perm) return HOPH_ERR_PARAM;
    return plan_create(params, host_perm, out);
}

void hoph_plan_destroy(hoph_plan *plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    plan_free(plan);
}

int hoph_plan_get_info(const hoph_plan *plan, hoph_plan_info *out) {
    if (!plan || !out) return HOPH_ERR_PARAM;
    memset(out, 0, sizeof *out);
    out->groups = plan->G;
    out->key_bits = plan->key_bits;
    out->upper_limit = plan->dp.always_stop ? 0 : plan->dp.U;
    out->lower_limit = plan->dp.always_stop ? (int64_t)plan->P.k_group + 1 : plan->dp.L;
    for (uint32_t g = 0; g < plan->G; ++g) out->group_size[g] = plan->z[g];
    out->max_bin_width = plan->max_width;
    return HOPH_OK;
}

int hoph_plan_set_exec(hoph_plan *plan, const hoph_exec *exec) {
    if (!plan) return HOPH_ERR_PARAM;
    if (!exec) {
        memset(&plan->exec, 0, sizeof plan->exec);
        plan->exec.strategy = -1;
        return HOPH_OK;
    }
    if (exec->strategy < -1 || exec->strategy > 1 || exec->tile_rows < 0 ||
        exec->tile_rows > 256 || exec->consumer_warps < 0 || exec->consumer_warps > 31 ||
        exec->ctas_per_sm < 0 || exec->ctas_per_sm > 8 || exec->stages < 0 || exec->stages > 8 ||
        (exec->lanes_per_row != 0 && exec->lanes_per_row != 1 && exec->lanes_per_row != 2 &&
         exec->lanes_per_row != 4 && exec->lanes_per_row != 8 && exec->lanes_per_row != 32) ||
        exec->sketch_cta_bits < 0 || exec->sketch_cta_bits > 64 || exec->join_lanes < 0 ||
        exec->join_lanes > hoph_plan::kMaxLanes)
        return HOPH_ERR_PARAM;
    plan->exec = *exec;
    return HOPH_OK;
}

int hoph_sync_status(hoph_plan *plan, void *stream) {
    if (!plan) return HOPH_ERR_PARAM;
    cudaStream_t s = (cudaStream_t)stream;
    HOPH_CUDA_TRY(cudaMemcpyAsync(plan->h_status, plan->d_status, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, s));
    HOPH_CUDA_TRY(cudaMemsetAsync(plan->d_status, 0, sizeof(int32_t), s));
    HOPH_CUDA_TRY(cudaStreamSynchronize(s));
    return *plan->h_status;
}

const char *hoph_status_string(int status) {
    switch (status) {
        case HOPH_OK: return "ok";
        case HOPH_ERR_PARAM: return "invalid argument or parameter set";
        case HOPH_ERR_ID_RANGE: return "an input ID was >= D";
        case HOPH_ERR_CAPACITY: return "more accepted pairs than the output capacity";
        case HOPH_ERR_TIMEOUT: return "a bounded device wait gave up";
        case HOPH_ERR_CUDA: return "a CUDA runtime call failed";
        case HOPH_ERR_NOMEM: return "allocation failed";
        case HOPH_ERR_UNSUPPORTED: return "parameters not supported by this build";
        case HOPH_ERR_TOO_LARGE: return "input larger than the fixed scratch of this entry point";
        case HOPH_ERR_CAPTURE:
            return "the call needs new plan memory while its stream is captured (make one "
                   "uncaptured call of the largest shape first)";
        default: return "unknown status";
    }
}

}  // extern "C"
