// pa_api.cu -- plans and the C ABI entry points (pa_plan, pa_hash, ...).
//
// Step 0 of Algorithm 1 (Sec. 4, Table 3) is the parameter rule implemented
// in choose_gamma(): gamma is the smallest Mersenne prime exponent >= r +
// margin (or the caller's exponent), k = ceil(n / gamma).  The rest of this
// file sizes the two weighted cyclic transforms (Eq. 2 modulo 2^gamma - 1 and
// the exact product of Eq. 4), builds their root-of-unity and weight tables
// on the host, and enqueues the kernels of pa_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

#include "../../include/pa_gb300.h"
#include "pa_internal.h"

using namespace pa;

// Exponents of the known Mersenne primes (the public list cited in Sec. 3.1).
static const uint32_t kMersenneExponents[] = {
    2,        3,        5,        7,        13,       17,       19,       31,       61,        89,       107,
    127,      521,      607,      1279,     2203,     2281,     3217,     4253,     4423,      9689,     9941,
    11213,    19937,    21701,    23209,    44497,    86243,    110503,   132049,   216091,    756839,   859433,
    1257787,  1398269,  2976221,  3021377,  6972593,  13466917, 20996011, 24036583, 25964951,  30402457, 32582657,
    37156667, 42643801, 43112609, 57885161, 74207281, 77232917, 82589933, 136279841};

static int choose_gamma(uint64_t r, const pa_params *p, uint32_t *gamma) {
    const uint32_t margin = p ? p->gamma_margin : 128u;
    const uint32_t want = p ? p->gamma : 0u;
    for (uint32_t g : kMersenneExponents) {
        if (want) {
            if (g == want) {
                if ((uint64_t)g <= r) return PA_ERR_INVALID;
                *gamma = g;
                return PA_OK;
            }
        } else if ((uint64_t)g >= r + (margin ? margin : 1u)) {
            *gamma = g;
            return PA_OK;
        }
    }
    return PA_ERR_INVALID;
}

// Smallest N = 2^l whose digits keep every convolution coefficient below q:
// digits are < 2^b with b = ceil(G / N); a coefficient of the weighted cyclic
// convolution is a sum of N products per operand pair, each doubled at most
// once by the weight ratio, so it is < 2 K N (2^b - 1)^2, plus one digit of c.
static int choose_len(uint64_t G, uint64_t K, uint32_t *logN) {
    for (uint32_t l = 0; l <= PA_MAX_LOGN; l++) {
        const uint64_t N = 1ULL << l;
        const uint64_t b = (G + N - 1) >> l;
        if (b > 31) continue;
        const unsigned __int128 m = ((unsigned __int128)1 << b) - 1;
        const unsigned __int128 bound = (unsigned __int128)2 * K * N * m * m + m;
        if (bound < GL_Q) {
            *logN = l;
            return PA_OK;
        }
    }
    return PA_ERR_UNSUPPORTED;
}

// ------------------------------------------------------- device memory --

static std::atomic<long long> g_fail_skip{0}, g_fail_count{0};

bool pa::alloc_fail_injected() {
    if (g_fail_count.load() <= 0) return false;
    if (g_fail_skip.load() > 0) {
        g_fail_skip--;
        return false;
    }
    g_fail_count--;
    return true;
}

int DevAlloc::init(bool stream_ordered) {
    async = stream_ordered;
    if (!stream && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        stream = nullptr;
        cudaGetLastError();
        return PA_ERR_CUDA;
    }
    return PA_OK;
}

void *DevAlloc::take(size_t b, int *err) {
    if (*err) return nullptr;
    void *p = nullptr;
    const size_t nb = b ? b : 8;
    // stream-ordered: the allocation is waited for on the private stream, so the
    // buffer is usable from any stream when take() returns
    const bool fail = alloc_fail_injected() ||
                      (async ? (cudaMallocAsync(&p, nb, stream) != cudaSuccess ||
                                cudaStreamSynchronize(stream) != cudaSuccess)
                             : cudaMalloc(&p, nb) != cudaSuccess);
    if (fail) {
        cudaGetLastError();  // an allocation failure must not read as a later launch's error
        *err = PA_ERR_NOMEM;
        return nullptr;
    }
    ptrs.push_back(p);
    bytes += b;
    return p;
}

void DevAlloc::upload(void *dst, const void *src, size_t b, int *err) {
    if (*err || !b) return;
    if (cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, stream) != cudaSuccess) *err = PA_ERR_CUDA;
}

int DevAlloc::sync() { return cudaStreamSynchronize(stream) == cudaSuccess ? PA_OK : PA_ERR_CUDA; }

void DevAlloc::release() {
    for (void *p : ptrs) {
        if (async)
            cudaFreeAsync(p, stream);
        else
            cudaFree(p);
    }
    ptrs.clear();
    bytes = 0;
    if (stream) cudaStreamDestroy(stream);  // resources go once its pending frees have run
    stream = nullptr;
}

namespace {

// F_q has generator 7; omega_N = 7^((q-1)/N).  2 has order 192, so
// 2 = rho^u with rho = 7^((q-1)/192); theta_N = 7^(u (q-1)/(192 N)) then
// satisfies theta_N^N = 2 for every N dividing 2^26.
static const u64 kGen = 7;

u64 root_of_unity(uint32_t logN) { return gl_pow(kGen, (GL_Q - 1) >> logN); }

u64 root_of_two(uint32_t logN) {
    const u64 rho = gl_pow(kGen, (GL_Q - 1) / 192);
    u64 acc = 1;
    uint32_t u = 0;
    for (uint32_t i = 1; i < 192; i++) {
        acc = gl_mul(acc, rho);
        if (acc == 2) {
            u = i;
            break;
        }
    }
    const unsigned __int128 e = (unsigned __int128)u * (((GL_Q - 1) / 192) >> logN);
    return gl_pow(kGen, (u64)(e % (GL_Q - 1)));
}

std::vector<u64> powers(u64 base, size_t count, u64 scale = 1) {
    std::vector<u64> v(count ? count : 1);
    u64 x = scale;
    for (size_t i = 0; i < v.size(); i++) {
        v[i] = x;
        x = gl_mul(x, base);
    }
    return v;
}

}  // namespace

struct pa_plan_s {
    uint64_t n, r, k;
    uint32_t gamma;
    bool mh_only = false;   // modular-arithmetic hash over the whole key (gamma = n, k = 0)
    bool toeplitz = false;  // Toeplitz-hashing comparison scheme (three-prime plan in p3)
    P3Plan *p3 = nullptr;   // three-prime backend (pa_p3.cu): owns its own workspace
    Xform mmh, mh;
    DevAlloc mem;           // every device buffer and table of the plan
    // workspace
    u64 *Y = nullptr;       // operand spectra (and the un-weighted coefficients)
    u64 *S = nullptr;       // accumulated spectra
    u64 *ybuf = nullptr;    // MMH value, gamma bits
    u64 *tbuf = nullptr;    // b*y + c, 2 gamma bits
    u64 *H = nullptr;
    unsigned char *cstate = nullptr, *cta_state = nullptr, *cta_cin = nullptr;
    int *flags = nullptr;   // [0] reload, [1] y all-ones, [2] t all-ones, [3] -, [4..4+k) slice counters
    size_t flags_bytes = 0;
    uint64_t ws_bytes = 0;
    // seed reuse (pa_seed_prepare): stored spectra of a_1..a_k and b, seed copy
    u64 *spec_a = nullptr, *spec_b = nullptr, *seed_copy = nullptr;
    bool prepared = false;
    // host-buffer entry points: two staging slots (key | seed | out | status),
    // a copy stream, per-group "landed" events and per-slot "free" events
    struct Staging {
        u64 *dkey = nullptr, *dseed = nullptr, *dout = nullptr;
        int *dstatus = nullptr;
        int *hstatus = nullptr;  // pinned
        std::vector<cudaEvent_t> ready;
        cudaEvent_t free_ev = nullptr;  // the slot's key and seed have been consumed
        cudaEvent_t out_ev = nullptr;   // the slot's output and status have been copied out
        bool used = false;
    } stage[2];
    int next_stage = 0;
    cudaStream_t copy_stream = nullptr;
    ~pa_plan_s() {
        for (auto &st : stage) {
            for (cudaEvent_t e : st.ready)
                if (e) cudaEventDestroy(e);
            if (st.free_ev) cudaEventDestroy(st.free_ev);
            if (st.out_ev) cudaEventDestroy(st.out_ev);
            if (st.hstatus) cudaFreeHost(st.hstatus);
        }
        if (copy_stream) cudaStreamDestroy(copy_stream);
        if (p3) p3_plan_destroy(p3);
        mem.release();
    }
    void *alloc(size_t bytes, int *err) {
        void *p = mem.take(bytes, err);
        if (p) ws_bytes += bytes;
        return p;
    }
};

// Default four-step split and column tile for a length 2^l transform.
static void default_geometry(uint32_t l, u32 *logR, u32 *tc) {
    *logR = std::min(l / 2, PA_MAX_LOGR);
    u32 t = 8;
    while (t > 1 && ((uint64_t)1 << *logR) * t > 4096) t >>= 1;
    while (t > (1u << (l - *logR))) t >>= 1;
    *tc = t;
}

// Geometry is valid for the kernels: R <= 2^11, C <= 8192, tile R * tc <= 4096, tc <= C.
static bool geometry_ok(uint32_t l, u32 logR, u32 tc) {
    if (logR > PA_MAX_LOGR || logR > l) return false;
    const u32 logC = l - logR;
    if (logC > 13) return false;
    return tc >= 1 && tc <= 8 && (tc & (tc - 1)) == 0 && tc <= (1u << logC) && ((uint64_t)1 << logR) * tc <= 4096;
}

static int build_xform(pa_plan_t *pl, Xform &X, uint64_t G, uint64_t K, u32 logR_sel = ~0u, u32 tc_sel = 0,
                       DevAlloc *sink = nullptr) {
    uint32_t l;
    int rc = choose_len(G, K, &l);
    if (rc) return rc;
    u32 logR, tc;
    default_geometry(l, &logR, &tc);
    if (logR_sel != ~0u) {
        if (!geometry_ok(l, logR_sel, tc_sel)) return PA_ERR_INVALID;
        logR = logR_sel;
        tc = tc_sel;
    }
    DevAlloc &tabs = sink ? *sink : pl->mem;
    X.N = 1ULL << l;
    X.G = G;
    X.K = (u32)K;
    X.logN = l;
    X.logR = logR;
    X.logC = l - X.logR;
    X.R = 1u << X.logR;
    X.C = 1u << X.logC;
    X.hb = (l + 1) / 2;
    X.tc = tc;
    const u64 w = root_of_unity(l), wi = gl_inv(w);
    const u64 th = root_of_two(l), thi = gl_inv(th);
    const u64 ninv = gl_inv(X.N % GL_Q);
    const u64 wR = gl_pow(w, X.C), wC = gl_pow(w, X.R);
    int err = PA_OK;
    auto up = [&](const std::vector<u64> &v) -> const u64 * {
        void *d = tabs.take(v.size() * sizeof(u64), &err);
        tabs.upload(d, v.data(), v.size() * sizeof(u64), &err);
        return (const u64 *)d;
    };
    X.twR = up(powers(wR, X.R));
    X.itwR = up(powers(gl_inv(wR), X.R));
    X.twC = up(powers(wC, X.C));
    X.itwC = up(powers(gl_inv(wC), X.C));
    const size_t nlo = (size_t)1 << X.hb, nhi = (size_t)(X.N >> X.hb);
    X.ipw_lo = up(powers(w, nlo));
    X.ipw_hi = up(powers(gl_pow(w, nlo), nhi));
    X.iipw_lo = up(powers(wi, nlo));
    X.iipw_hi = up(powers(gl_pow(wi, nlo), nhi));
    X.wt_lo = up(powers(th, nlo));
    X.wt_hi = up(powers(gl_pow(th, nlo), nhi));
    X.iwt_lo = up(powers(thi, nlo));
    X.iwt_hi = up(powers(gl_pow(thi, nlo), nhi, ninv));
    // column-pass weights: theta^beta_r and theta^beta_r / 2, beta_r = (-G C r) mod N
    {
        std::vector<u64> cw(2 * (size_t)X.R);
        const u64 half = gl_inv(2);
        for (u32 r = 0; r < X.R; r++) {
            const u64 beta = (0ULL - G * X.C * (u64)r) & (X.N - 1);
            cw[r] = gl_pow(th, beta);
            cw[X.R + r] = gl_mul(cw[r], half);
        }
        X.colw = up(cw);
    }
    if (err) return err;
    {
        void *d = tabs.take(X.N * sizeof(u64), &err);
        if (err) return err;
        X.coltw = (const u64 *)d;
        // on the plan's private stream: building a plan waits for nothing else on the device
        if (launch_fill_coltw(X, (u64 *)d, tabs.stream) || tabs.sync() != PA_OK) return PA_ERR_CUDA;
    }
    return err;
}

// ------------------------------------------------------------ autotuner --
// For a transform shape (G, K, N) the tuner times every valid four-step split
// log2 R in {d - 1, d, d + 1} (d = the default) and column tile width in
// {1, 2, 4, 8} on the plan's own workspace (forward column pass, row pass with
// the multiply-accumulate, inverse column pass; one warm-up, best of three)
// and keeps the fastest.  Results are cached per process.
static std::mutex g_tune_mu;
static std::map<std::tuple<uint64_t, uint64_t, uint32_t>, std::pair<u32, u32>> g_tune_cache;
// Measured backend of tuned AUTO plans, per (gamma, k): PA_BACKEND_GOLDILOCKS or PA_BACKEND_P3.
static std::map<std::pair<uint32_t, uint64_t>, uint32_t> g_backend_cache;

// Device time of one pa_hash on the plan (synthetic key and seed, best of
// three after a warm-up, private stream); -1 on failure.
static float time_plan_ms(pa_plan_t *pl) {
    const uint64_t kw = (pl->n + 63) / 64, sw = ((pl->k + 2) * (uint64_t)pl->gamma + 63) / 64;
    DevAlloc scratch;
    int err = scratch.init(pl->mem.async);
    uint64_t *buf = (uint64_t *)scratch.take((kw + sw + (pl->r + 63) / 64 + 1) * 8, &err);
    if (err) return -1.f;
    cudaStream_t s = scratch.stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = -1.f;
    if (!cudaMemsetAsync(buf, 0x5A, (kw + sw) * 8, s) && !cudaEventCreate(&e0) && !cudaEventCreate(&e1)) {
        for (int rep = 0; rep < 4; rep++) {
            if (cudaEventRecord(e0, s) || pa_hash(pl, buf, buf + kw, buf + kw + sw, nullptr, s) ||
                cudaEventRecord(e1, s) || cudaEventSynchronize(e1)) {
                best = -1.f;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best < 0 || ms < best)) best = ms;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    scratch.sync();
    return best;
}

static int tune_geometry(pa_plan_t *pl, int stage, uint64_t G, uint64_t K, uint32_t l, u32 *logR_out, u32 *tc_out);

// Device bytes of a plan's workspace (shared by pa_plan and the server's admission).
struct WsSizes {
    uint64_t Y, S, ybuf, tbuf, H, cstate, cta, flags, tables;
    uint64_t total() const { return Y + S + ybuf + tbuf + H + cstate + 2 * cta + flags + tables; }
};
static WsSizes ws_sizes(uint32_t gamma, uint64_t k, uint64_t N1, uint64_t N2) {
    WsSizes z;
    const uint64_t Nmax = std::max(N1, N2);
    z.Y = std::max<uint64_t>(2 * k * N1, 2 * N2) * 8;
    z.S = Nmax * 8;
    z.ybuf = ((gamma + 63) / 64 + 2) * 8;
    z.tbuf = ((2ULL * gamma + 63) / 64 + 2) * 8;
    const uint64_t nch = std::max<uint64_t>(Nmax / PA_CARRY_D, 1);
    z.H = nch * 8;
    z.cstate = nch;
    z.cta = nch / PA_CARRY_T + 1;
    z.flags = (4 + k) * sizeof(int);
    // tables of both transforms: a bound for every geometry the tuner may pick
    auto table_words = [](uint64_t N) {
        uint32_t l = 0;
        while ((1ULL << l) < N) l++;
        const uint64_t Rmax = 1ULL << std::min<uint32_t>(l / 2 + 1, PA_MAX_LOGR);
        const uint64_t Cmax = N >> (std::min<uint32_t>(l / 2, PA_MAX_LOGR) > 0 ? std::min<uint32_t>(l / 2, PA_MAX_LOGR) - 1 : 0);
        const uint32_t hb = (l + 1) / 2;
        return 4 * Rmax + 2 * Cmax + 4 * ((1ULL << hb) + (N >> hb)) + N;
    };
    z.tables = (table_words(N1) + table_words(N2)) * 8;
    return z;
}

// Backend of a plan.  PA_BACKEND_AUTO takes the three-prime transforms where
// they are feasible and their Eq. 2 transform is no longer than the Goldilocks
// one (measured 1.3x faster at 2.6e8 bits), or twice as long but at most 2^20
// (measured 1.7x faster at 1e7 bits: T = 2^17 against N = 2^16); else
// Goldilocks (e.g. 1e9 bits: 2^24 against 2^23, measured 0.7x).
static int choose_backend(uint32_t gamma, uint64_t k, const pa_params *params, uint32_t l1, int *backend) {
    const uint32_t want = params ? params->backend : PA_BACKEND_AUTO;
    if (want > PA_BACKEND_P3) return PA_ERR_INVALID;
    uint32_t t1 = 0, t2 = 0;
    const bool p3ok = p3_feasible(gamma, k, &t1, &t2) == PA_OK;
    if (want == PA_BACKEND_P3) {
        if (!p3ok) return PA_ERR_UNSUPPORTED;
        *backend = PA_BACKEND_P3;
    } else if (want == PA_BACKEND_GOLDILOCKS) {
        *backend = PA_BACKEND_GOLDILOCKS;
    } else {
        const bool p3_better = t1 <= l1 || (t1 == l1 + 1 && t1 <= 20);
        *backend = (p3ok && p3_better) ? PA_BACKEND_P3 : PA_BACKEND_GOLDILOCKS;
    }
    return PA_OK;
}

// Step 0 and the plan's device memory; stream_ordered: every allocation and
// table fill on the plan's private stream with cudaMallocAsync (server plans).
int pa::plan_create(uint64_t n_bits, uint64_t r_bits, const pa_params *params, bool stream_ordered,
                    pa_plan_t **out) {
    if (!out || n_bits == 0 || r_bits == 0) return PA_ERR_INVALID;
    *out = nullptr;
    if (params) {
        for (uint32_t v : params->reserved)
            if (v) return PA_ERR_INVALID;
    }
    uint32_t gamma;
    int rc = choose_gamma(r_bits, params, &gamma);
    if (rc) return rc;
    if (prepare_kernels()) return PA_ERR_CUDA;
    pa_plan_t *pl = new (std::nothrow) pa_plan_s();
    if (!pl) return PA_ERR_NOMEM;
    if ((rc = pl->mem.init(stream_ordered))) {
        delete pl;
        return rc;
    }
    pl->n = n_bits;
    pl->r = r_bits;
    pl->gamma = gamma;
    pl->k = (n_bits + gamma - 1) / gamma;
    if (pl->k > 65535) {  // operand pairs index gridDim.y of the column pass
        delete pl;
        return PA_ERR_UNSUPPORTED;
    }
    uint32_t l1, l2;
    if ((rc = choose_len(gamma, pl->k, &l1)) || (rc = choose_len(2ULL * gamma, 1, &l2))) {
        delete pl;
        return rc;
    }
    int backend = PA_BACKEND_GOLDILOCKS;
    if ((rc = choose_backend(gamma, pl->k, params, l1, &backend))) {
        delete pl;
        return rc;
    }
    if (params && params->tune && params->backend == PA_BACKEND_AUTO &&
        p3_feasible(gamma, pl->k, nullptr, nullptr) == PA_OK) {
        // tuned AUTO plan: the backend is the one measured faster for this (gamma, k)
        const auto key = std::make_pair(gamma, pl->k);
        uint32_t chosen = 0;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_backend_cache.find(key);
            if (it != g_backend_cache.end()) chosen = it->second;
        }
        const uint64_t k = pl->k;
        delete pl;
        pa_params pp = *params;
        if (chosen) {
            pp.backend = chosen;
            return plan_create(n_bits, r_bits, &pp, stream_ordered, out);
        }
        pa_plan_t *cand[2] = {nullptr, nullptr};
        float ms[2] = {-1.f, -1.f};
        const uint32_t be[2] = {PA_BACKEND_P3, PA_BACKEND_GOLDILOCKS};
        for (int c = 0; c < 2; c++) {
            pp.backend = be[c];
            if (plan_create(n_bits, r_bits, &pp, stream_ordered, &cand[c]) == PA_OK) ms[c] = time_plan_ms(cand[c]);
        }
        int win = -1;
        for (int c = 0; c < 2; c++)
            if (cand[c] && ms[c] >= 0 && (win < 0 || ms[c] < ms[win])) win = c;
        for (int c = 0; c < 2; c++)
            if (c != win && cand[c]) pa_plan_destroy(cand[c]);
        if (win < 0) return cand[0] || cand[1] ? PA_ERR_CUDA : PA_ERR_NOMEM;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_backend_cache[std::make_pair(gamma, k)] = be[win];
        }
        *out = cand[win];
        return PA_OK;
    }
    if (backend == PA_BACKEND_P3) {
        if ((rc = p3_plan_create(n_bits, r_bits, gamma, pl->k, stream_ordered, &pl->p3))) {
            delete pl;
            return rc;
        }
        uint64_t t1 = 0, t2 = 0, ws = 0;
        p3_plan_query(pl->p3, &t1, &t2, &ws);
        pl->mmh.N = t1;
        pl->mh.N = t2;
        pl->ws_bytes = ws;
        *out = pl;
        return PA_OK;
    }
    const WsSizes z = ws_sizes(gamma, pl->k, 1ULL << l1, 1ULL << l2);
    int err = PA_OK;
    pl->Y = (u64 *)pl->alloc(z.Y, &err);
    pl->S = (u64 *)pl->alloc(z.S, &err);
    pl->ybuf = (u64 *)pl->alloc(z.ybuf, &err);
    pl->tbuf = (u64 *)pl->alloc(z.tbuf, &err);
    pl->H = (u64 *)pl->alloc(z.H, &err);
    pl->cstate = (unsigned char *)pl->alloc(z.cstate, &err);
    pl->cta_state = (unsigned char *)pl->alloc(z.cta, &err);
    pl->cta_cin = (unsigned char *)pl->alloc(z.cta, &err);
    pl->flags_bytes = z.flags;
    pl->flags = (int *)pl->alloc(z.flags, &err);
    if (err) {
        delete pl;
        return err;
    }
    const bool tune = params && params->tune;
    for (int stage = 0; stage < 2 && !rc; stage++) {
        Xform &X = stage ? pl->mh : pl->mmh;
        const uint64_t G = stage ? 2ULL * gamma : gamma, K = stage ? 1 : pl->k;
        u32 logR = ~0u, tc = 0;
        if (tune) rc = tune_geometry(pl, stage, G, K, stage ? l2 : l1, &logR, &tc);
        if (!rc) rc = build_xform(pl, X, G, K, logR, tc);
        X.stage = (u32)stage;
    }
    if (rc) {
        delete pl;
        return rc;
    }
    pl->ws_bytes = pl->mem.bytes;  // workspace and tables
    *out = pl;
    return PA_OK;
}

extern "C" {

int pa_plan(uint64_t n_bits, uint64_t r_bits, const pa_params *params, pa_plan_t **out) {
    return pa::plan_create(n_bits, r_bits, params, false, out);
}

// Comparison scheme: the modular-arithmetic hash over the whole key (Eq. 4
// with alpha = n, beta = r), one exact n x n-bit product.
int pa_mh_plan(uint64_t n_bits, uint64_t r_bits, pa_plan_t **out) {
    if (!out || n_bits == 0 || r_bits == 0 || r_bits > n_bits || n_bits > 0xFFFFFFFFULL) return PA_ERR_INVALID;
    *out = nullptr;
    uint32_t l2;
    int rc = choose_len(2 * n_bits, 1, &l2);
    if (rc) return rc;
    if (prepare_kernels()) return PA_ERR_CUDA;
    pa_plan_t *pl = new (std::nothrow) pa_plan_s();
    if (!pl) return PA_ERR_NOMEM;
    if ((rc = pl->mem.init(false))) {
        delete pl;
        return rc;
    }
    pl->mh_only = true;
    pl->n = n_bits;
    pl->r = r_bits;
    pl->gamma = (uint32_t)n_bits;
    pl->k = 0;
    const WsSizes z = ws_sizes(pl->gamma, 0, 1, 1ULL << l2);
    int err = PA_OK;
    pl->Y = (u64 *)pl->alloc(z.Y, &err);
    pl->S = (u64 *)pl->alloc(z.S, &err);
    pl->ybuf = (u64 *)pl->alloc(z.ybuf, &err);
    pl->tbuf = (u64 *)pl->alloc(z.tbuf, &err);
    pl->H = (u64 *)pl->alloc(z.H, &err);
    pl->cstate = (unsigned char *)pl->alloc(z.cstate, &err);
    pl->cta_state = (unsigned char *)pl->alloc(z.cta, &err);
    pl->cta_cin = (unsigned char *)pl->alloc(z.cta, &err);
    pl->flags_bytes = z.flags;
    pl->flags = (int *)pl->alloc(z.flags, &err);
    if (!err) err = build_xform(pl, pl->mh, 2 * n_bits, 1);
    pl->mh.stage = 1;
    pl->mmh = pl->mh;
    pl->mmh.N = 0;
    if (err) {
        delete pl;
        return err;
    }
    pl->ws_bytes = pl->mem.bytes;
    *out = pl;
    return PA_OK;
}

// Comparison scheme: Toeplitz hashing, z = T x over GF(2) (Sec. 1, Table 1),
// output blocks / key segments of 2^block_log bits (0: automatic).
int pa_toeplitz_plan(uint64_t n_bits, uint64_t r_bits, uint32_t block_log, pa_plan_t **out) {
    if (!out || n_bits == 0 || r_bits == 0 || r_bits > n_bits) return PA_ERR_INVALID;
    *out = nullptr;
    if (block_log == 0) {
        block_log = 6;
        while (block_log < 22 && (1ULL << block_log) < r_bits) block_log++;
    }
    if (block_log < 6 || block_log > 22) return PA_ERR_INVALID;
    pa_plan_t *pl = new (std::nothrow) pa_plan_s();
    if (!pl) return PA_ERR_NOMEM;
    int rc = pl->mem.init(false);
    if (!rc) rc = p3_toeplitz_create(n_bits, r_bits, block_log, &pl->p3);
    if (rc) {
        delete pl;
        return rc;
    }
    pl->toeplitz = true;
    pl->n = n_bits;
    pl->r = r_bits;
    pl->gamma = 0;
    uint64_t rb = 0, seg = 0, blk = 0, t1 = 0, t2 = 0, ws = 0;
    p3_toeplitz_query(pl->p3, &rb, &seg, &blk);
    p3_plan_query(pl->p3, &t1, &t2, &ws);
    pl->k = seg;
    pl->mmh.N = t1;
    pl->mh.N = 0;
    pl->ws_bytes = ws;
    *out = pl;
    return PA_OK;
}

int pa_plan_info_get(const pa_plan_t *pl, pa_plan_info *info) {
    if (!pl || !info) return PA_ERR_INVALID;
    memset(info, 0, sizeof(*info));
    if (pl->toeplitz) {
        info->n_bits = pl->n;
        info->r_bits = pl->r;
        info->k = pl->k;
        info->key_words = (pl->n + 63) / 64;
        info->seed_words = (pl->n + pl->r - 1 + 63) / 64;
        info->out_words = (pl->r + 63) / 64;
        info->mmh_len = pl->mmh.N;
        info->workspace_bytes = pl->ws_bytes;
        info->backend = PA_BACKEND_P3;
        return PA_OK;
    }
    info->n_bits = pl->n;
    info->r_bits = pl->r;
    info->gamma = pl->gamma;
    info->k = pl->k;
    info->key_words = (pl->n + 63) / 64;
    info->seed_words = ((pl->k + 2) * pl->gamma + 63) / 64;
    info->out_words = (pl->r + 63) / 64;
    info->mmh_len = pl->mmh.N;
    info->mh_len = pl->mh.N;
    info->workspace_bytes = pl->ws_bytes;
    info->backend = pl->p3 ? PA_BACKEND_P3 : PA_BACKEND_GOLDILOCKS;
    return PA_OK;
}

int pa_batch_drop_plan(pa_plan_t *pl);

int pa_plan_destroy(pa_plan_t *pl) {
    if (!pl) return PA_ERR_INVALID;
    pa_batch_drop_plan(pl);
    cudaDeviceSynchronize();
    delete pl;
    return PA_OK;
}

}  // extern "C"

void pa::plan_destroy_idle(pa_plan_t *pl) {
    if (!pl) return;
    pa_batch_drop_plan(pl);
    delete pl;
}

// Eq. 2 (MMH): y = sum_i a_i x_i mod 2^gamma - 1, written to y (canonical after
// the optional zero fix-up when `canonical` is set).
static int enqueue_mmh(pa_plan_t *pl, const u64 *key, const u64 *seed, u64 *y, bool canonical, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int e;
    if ((e = cudaMemsetAsync(pl->flags, 0, pl->flags_bytes, s))) return e;
    Operands ops;
    ops.pair0 = 0;
    ops.key = key;
    ops.seed = seed;
    ops.y = nullptr;
    ops.y_zero = nullptr;
    ops.reload = pl->flags;
    ops.n = pl->n;
    ops.gamma = pl->gamma;
    ops.k = pl->k;
    ops.mode = 0;
    const Xform &X = pl->mmh;
    if ((e = launch_fwd_col(X, ops, (int)pl->k, pl->Y, stream))) return e;
    if ((e = launch_row_mac(X, pl->Y, pl->S, stream))) return e;
    if ((e = launch_inv_col(X, pl->S, pl->Y, nullptr, 0, 0, stream))) return e;
    CarryDev cd;
    cd.N = X.N;
    cd.G = X.G;
    cd.logN = X.logN;
    cd.nchunks = X.N / PA_CARRY_D;
    cd.H = pl->H;
    cd.state = pl->cstate;
    cd.cta_state = pl->cta_state;
    cd.cta_cin = pl->cta_cin;
    cd.allones = pl->flags + 1;
    const u64 ywords = (pl->gamma + 63) / 64;
    if ((e = launch_carry(X, cd, pl->Y, y, ywords, stream))) return e;
    if (canonical && (e = launch_canonical_zero(pl->flags + 1, y, ywords, stream))) return e;
    return 0;
}

// Eq. 4 (MH): out = ((b y + c) mod 2^gamma) >> (gamma - r).
static int enqueue_mh(pa_plan_t *pl, const u64 *seed, u64 *out, int *status, void *stream) {
    int e;
    Operands ops;
    ops.pair0 = 0;
    ops.key = nullptr;
    ops.seed = seed;
    ops.y = pl->ybuf;
    ops.y_zero = pl->flags + 1;
    ops.reload = pl->flags;
    ops.n = pl->n;
    ops.gamma = pl->gamma;
    ops.k = pl->k;
    ops.mode = 1;
    const Xform &X = pl->mh;
    if ((e = launch_fwd_col(X, ops, 1, pl->Y, stream))) return e;
    if ((e = launch_row_mac(X, pl->Y, pl->S, stream))) return e;
    if ((e = launch_inv_col(X, pl->S, pl->Y, seed, (pl->k + 1) * (u64)pl->gamma, pl->gamma, stream))) return e;
    CarryDev cd;
    cd.N = X.N;
    cd.G = X.G;
    cd.logN = X.logN;
    cd.nchunks = X.N / PA_CARRY_D;
    cd.H = pl->H;
    cd.state = pl->cstate;
    cd.cta_state = pl->cta_state;
    cd.cta_cin = pl->cta_cin;
    cd.allones = pl->flags + 2;
    if ((e = launch_carry(X, cd, pl->Y, pl->tbuf, (2ULL * pl->gamma + 63) / 64, stream))) return e;
    if ((e = launch_extract(pl->tbuf, pl->gamma, pl->r, pl->flags, pl->k, out, status, stream))) return e;
    return 0;
}

static int cuda_rc(int e) { return e ? PA_ERR_CUDA : PA_OK; }

static CarryDev carry_dev(pa_plan_t *pl, const Xform &X, int *allones) {
    CarryDev cd;
    cd.N = X.N;
    cd.G = X.G;
    cd.logN = X.logN;
    cd.nchunks = X.N / PA_CARRY_D;
    cd.H = pl->H;
    cd.state = pl->cstate;
    cd.cta_state = pl->cta_state;
    cd.cta_cin = pl->cta_cin;
    cd.allones = allones;
    return cd;
}

extern "C" {

int pa_hash(pa_plan_t *pl, const uint64_t *key, const uint64_t *seed, uint64_t *out, int *status, void *stream) {
    if (!pl || !key || !seed || !out) return PA_ERR_INVALID;
    if (pl->toeplitz) {
        int e = p3_toeplitz_hash(pl->p3, (const u64 *)key, (const u64 *)seed, (u64 *)out, stream);
        if (!e && status) e = cudaMemsetAsync(status, 0, sizeof(int), (cudaStream_t)stream);
        return cuda_rc(e);
    }
    if (pl->mh_only) {
        // Eq. 4 with alpha = n: the key itself is the MH input y
        cudaStream_t s = (cudaStream_t)stream;
        int e = cudaMemsetAsync(pl->flags, 0, pl->flags_bytes, s);
        if (!e) e = cudaMemcpyAsync(pl->ybuf, key, ((pl->n + 63) / 64) * 8, cudaMemcpyDeviceToDevice, s);
        if (!e) e = enqueue_mh(pl, (const u64 *)seed, (u64 *)out, status, stream);
        return cuda_rc(e);
    }
    if (pl->p3) {
        return cuda_rc(p3_enqueue_hash(pl->p3, (const u64 *)key, (const u64 *)seed, (u64 *)out, status, stream));
    }
    int e = enqueue_mmh(pl, (const u64 *)key, (const u64 *)seed, pl->ybuf, false, stream);
    if (!e) e = enqueue_mh(pl, (const u64 *)seed, (u64 *)out, status, stream);
    return cuda_rc(e);
}

int pa_debug_mmh(pa_plan_t *pl, const uint64_t *key, const uint64_t *seed, uint64_t *y, int *status, void *stream) {
    if (!pl || !key || !seed || !y) return PA_ERR_INVALID;
    if (pl->mh_only || pl->toeplitz) return PA_ERR_INVALID;
    if (pl->p3) {
        int e = p3_enqueue_mmh(pl->p3, (const u64 *)key, (const u64 *)seed, (u64 *)y, true, stream);
        if (!e && status)
            e = cudaMemcpyAsync(status, p3_flags(pl->p3), sizeof(int), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
        return cuda_rc(e);
    }
    int e = enqueue_mmh(pl, (const u64 *)key, (const u64 *)seed, (u64 *)y, true, stream);
    if (!e && status) e = cudaMemcpyAsync(status, pl->flags, sizeof(int), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return cuda_rc(e);
}

// Host buffers.  Key and seed are copied on the plan's copy stream in a few
// groups of slices; the column pass of a group starts as soon as its slices
// have landed.  Two staging slots alternate, so the copies of one call overlap
// the transforms of the previous call on the same stream.
// Pairs per column launch (about a third of the k pairs) and the number of
// launches (every group non-empty).
static uint64_t host_group_size(uint64_t k) { return (k + 2) / 3; }
static int host_groups(uint64_t k) { return (int)((k + host_group_size(k) - 1) / host_group_size(k)); }

int pa_hash_host_async(pa_plan_t *pl, const uint64_t *key, const uint64_t *seed, uint64_t *out, int *status,
                       void *stream) {
    if (!pl || !key || !seed || !out) return PA_ERR_INVALID;
    if (pl->mh_only || pl->toeplitz) return PA_ERR_INVALID;
    const uint64_t kw = (pl->n + 63) / 64, sw = ((pl->k + 2) * pl->gamma + 63) / 64, ow = (pl->r + 63) / 64;
    const uint64_t g = pl->gamma, k = pl->k;
    const int ng = host_groups(k);
    const uint64_t per = host_group_size(k);
    cudaStream_t s = (cudaStream_t)stream;
    if (!pl->copy_stream && cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking)) return PA_ERR_CUDA;
    auto &st = pl->stage[pl->next_stage];
    pl->next_stage ^= 1;
    if (!st.dkey) {
        // each resource once; the slot counts as set up (dkey) only when all exist,
        // so a call after a failed setup completes it instead of using a partial slot
        if (!st.dseed) {
            int err = PA_OK;
            void *d = pl->alloc((kw + sw + ow + 1) * 8, &err);
            if (err) return err;
            st.dseed = (u64 *)d + kw;
        }
        if (!st.hstatus && (alloc_fail_injected() || cudaMallocHost(&st.hstatus, sizeof(int)) != cudaSuccess)) {
            st.hstatus = nullptr;
            cudaGetLastError();
            return PA_ERR_NOMEM;
        }
        st.ready.resize(ng + 1, nullptr);
        for (auto &ev : st.ready)
            if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                ev = nullptr;
                return PA_ERR_CUDA;
            }
        if (!st.free_ev && cudaEventCreateWithFlags(&st.free_ev, cudaEventDisableTiming) != cudaSuccess) {
            st.free_ev = nullptr;
            return PA_ERR_CUDA;
        }
        if (!st.out_ev && cudaEventCreateWithFlags(&st.out_ev, cudaEventDisableTiming) != cudaSuccess) {
            st.out_ev = nullptr;
            return PA_ERR_CUDA;
        }
        st.dout = st.dseed + sw;
        st.dstatus = (int *)(st.dout + ow);
        st.dkey = st.dseed - kw;
    }
    int e = 0;
    // the slot's previous inputs must have been consumed before they are
    // overwritten, and its previous output and status copied out before the
    // kernels (on `stream`, possibly another stream than last time) rewrite them
    if (st.used) e = cudaStreamWaitEvent(pl->copy_stream, st.free_ev, 0);
    if (st.used && !e) e = cudaStreamWaitEvent(s, st.out_ev, 0);
    auto copy_words = [&](u64 *dst, const uint64_t *src, uint64_t w0, uint64_t w1) {
        if (w1 > w0 && !e)
            e = cudaMemcpyAsync(dst + w0, src + w0, (w1 - w0) * 8, cudaMemcpyHostToDevice, pl->copy_stream);
    };
    for (int q = 0; q < ng && !e; q++) {
        const uint64_t i0 = q * per, i1 = std::min(k, i0 + per);
        const uint64_t b0 = i0 * g, b1k = std::min(pl->n, i1 * g), b1s = i1 * g;
        copy_words(st.dkey, key, b0 / 64, std::min(kw, (b1k + 63) / 64));
        copy_words(st.dseed, seed, b0 / 64, std::min(sw, (b1s + 63) / 64));
        if (!e) e = cudaEventRecord(st.ready[q], pl->copy_stream);
    }
    copy_words(st.dseed, seed, (k * g) / 64, sw);  // b and c
    if (!e) e = cudaEventRecord(st.ready[ng], pl->copy_stream);
    if (pl->p3) {
        // three-prime plans start once the whole key and seed have landed
        if (!e) e = cudaStreamWaitEvent(s, st.ready[ng], 0);
        for (int q = 0; q < ng && !e; q++) e = cudaStreamWaitEvent(s, st.ready[q], 0);
        if (!e) e = p3_enqueue_hash(pl->p3, st.dkey, st.dseed, st.dout, st.dstatus, stream);
        if (!e) e = cudaEventRecord(st.free_ev, s);
        if (!e) e = cudaMemcpyAsync(out, st.dout, ow * 8, cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(status ? status : st.hstatus, st.dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaEventRecord(st.out_ev, s);
        if (e) return PA_ERR_CUDA;
        st.used = true;
        return PA_OK;
    }
    if (!e) e = cudaMemsetAsync(pl->flags, 0, pl->flags_bytes, s);
    Operands ops;
    ops.pair0 = 0;
    ops.key = st.dkey;
    ops.seed = st.dseed;
    ops.y = nullptr;
    ops.y_zero = nullptr;
    ops.reload = pl->flags;
    ops.n = pl->n;
    ops.gamma = pl->gamma;
    ops.k = pl->k;
    ops.mode = 0;
    for (int q = 0; q < ng && !e; q++) {
        const uint64_t i0 = q * per, i1 = std::min(k, i0 + per);
        e = cudaStreamWaitEvent(s, st.ready[q], 0);
        ops.pair0 = (u32)i0;
        if (!e) e = launch_fwd_col(pl->mmh, ops, (int)(i1 - i0), pl->Y, stream);
    }
    if (!e) e = launch_row_mac(pl->mmh, pl->Y, pl->S, stream);
    if (!e) e = launch_inv_col(pl->mmh, pl->S, pl->Y, nullptr, 0, 0, stream);
    if (!e) e = launch_carry(pl->mmh, carry_dev(pl, pl->mmh, pl->flags + 1), pl->Y, pl->ybuf, (g + 63) / 64, stream);
    if (!e) e = cudaStreamWaitEvent(s, st.ready[ng], 0);
    if (!e) e = enqueue_mh(pl, st.dseed, st.dout, st.dstatus, stream);
    if (!e) e = cudaEventRecord(st.free_ev, s);
    if (!e) e = cudaMemcpyAsync(out, st.dout, ow * 8, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(status ? status : st.hstatus, st.dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaEventRecord(st.out_ev, s);
    if (e) return PA_ERR_CUDA;
    st.used = true;
    return PA_OK;
}

int pa_hash_host(pa_plan_t *pl, const uint64_t *key, const uint64_t *seed, uint64_t *out, void *stream) {
    if (!pl) return PA_ERR_INVALID;
    auto &st = pl->stage[pl->next_stage];
    int rc = pa_hash_host_async(pl, key, seed, out, nullptr, stream);
    if (rc) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream)) return PA_ERR_CUDA;
    return *st.hstatus ? PA_RELOAD : PA_OK;
}

// Seed reuse: transform a_1..a_k (Eq. 2) and b (Eq. 4) once and keep their
// spectra in the plan; pa_hash_prepared then transforms only the key slices
// and y.  The plan keeps a copy of the seed (c is read from it).
int pa_seed_prepare(pa_plan_t *pl, const uint64_t *seed, void *stream) {
    if (!pl || !seed) return PA_ERR_INVALID;
    if (pl->mh_only || pl->toeplitz) return PA_ERR_INVALID;
    if (pl->p3) {
        const int e = p3_seed_prepare(pl->p3, (const u64 *)seed, stream);  // PA_ERR_* (< 0) or a CUDA error
        return e < 0 ? e : cuda_rc(e);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t sw = ((pl->k + 2) * pl->gamma + 63) / 64;
    if (!pl->spec_a || !pl->spec_b || !pl->seed_copy) {  // first call, or a retry after a failed allocation
        int err = PA_OK;
        if (!pl->spec_a) pl->spec_a = (u64 *)pl->alloc(pl->k * pl->mmh.N * 8, &err);
        if (!pl->spec_b) pl->spec_b = (u64 *)pl->alloc(pl->mh.N * 8, &err);
        if (!pl->seed_copy) pl->seed_copy = (u64 *)pl->alloc(sw * 8, &err);
        if (err) return err;
    }
    pl->prepared = false;
    int e = cudaMemcpyAsync(pl->seed_copy, seed, sw * 8, cudaMemcpyDeviceToDevice, s);
    Operands ops;
    ops.pair0 = 0;
    ops.key = nullptr;
    ops.seed = pl->seed_copy;
    ops.y = nullptr;
    ops.y_zero = nullptr;
    ops.reload = pl->flags;
    ops.n = pl->n;
    ops.gamma = pl->gamma;
    ops.k = pl->k;
    ops.mode = 2;  // a_i
    if (!e) e = launch_fwd_col_single(pl->mmh, ops, (int)pl->k, pl->Y, stream);
    if (!e) e = launch_row_store(pl->mmh, pl->Y, pl->spec_a, stream);
    ops.mode = 4;  // b
    if (!e) e = launch_fwd_col_single(pl->mh, ops, 1, pl->Y, stream);
    if (!e) e = launch_row_store(pl->mh, pl->Y, pl->spec_b, stream);
    if (e) return PA_ERR_CUDA;
    pl->prepared = true;
    return PA_OK;
}

int pa_hash_prepared(pa_plan_t *pl, const uint64_t *key, uint64_t *out, int *status, void *stream) {
    if (!pl || !key || !out) return PA_ERR_INVALID;
    if (pl->toeplitz) return PA_ERR_INVALID;
    if (pl->p3) {
        if (!p3_prepared(pl->p3)) return PA_ERR_INVALID;
        return cuda_rc(p3_hash_prepared(pl->p3, (const u64 *)key, (u64 *)out, status, stream));
    }
    if (!pl->prepared) return PA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int e = cudaMemsetAsync(pl->flags, 0, pl->flags_bytes, s);
    Operands ops;
    ops.pair0 = 0;
    ops.key = (const u64 *)key;
    ops.seed = pl->seed_copy;
    ops.y = pl->ybuf;
    ops.y_zero = pl->flags + 1;
    ops.reload = pl->flags;
    ops.n = pl->n;
    ops.gamma = pl->gamma;
    ops.k = pl->k;
    // Eq. 2 with stored spectra of a_i
    ops.mode = 3;  // x_i
    if (!e) e = launch_fwd_col_single(pl->mmh, ops, (int)pl->k, pl->Y, stream);
    if (!e) e = launch_row_prepared(pl->mmh, pl->Y, pl->spec_a, pl->S, stream);
    if (!e) e = launch_inv_col(pl->mmh, pl->S, pl->Y, nullptr, 0, 0, stream);
    if (!e) e = launch_carry(pl->mmh, carry_dev(pl, pl->mmh, pl->flags + 1), pl->Y, pl->ybuf, (pl->gamma + 63) / 64, stream);
    // Eq. 4 with the stored spectrum of b
    ops.mode = 5;  // y
    if (!e) e = launch_fwd_col_single(pl->mh, ops, 1, pl->Y, stream);
    if (!e) e = launch_row_prepared(pl->mh, pl->Y, pl->spec_b, pl->S, stream);
    if (!e) e = launch_inv_col(pl->mh, pl->S, pl->Y, pl->seed_copy, (pl->k + 1) * (u64)pl->gamma, pl->gamma, stream);
    if (!e) e = launch_carry(pl->mh, carry_dev(pl, pl->mh, pl->flags + 2), pl->Y, pl->tbuf, (2ULL * pl->gamma + 63) / 64, stream);
    if (!e) e = launch_extract(pl->tbuf, pl->gamma, pl->r, pl->flags, pl->k, (u64 *)out, status, stream);
    return cuda_rc(e);
}

const char *pa_status_string(int code) {
    switch (code) {
        case PA_OK: return "ok";
        case PA_RELOAD: return "reload: a key slice equals 2^gamma - 1";
        case PA_ERR_INVALID: return "invalid argument";
        case PA_ERR_NOMEM: return "out of memory";
        case PA_ERR_CUDA: return "CUDA error";
        case PA_ERR_TIMEOUT: return "timeout";
        case PA_ERR_BUDGET: return "job exceeds the HBM budget";
        case PA_ERR_CANCELLED: return "cancelled";
        case PA_ERR_UNSUPPORTED: return "unsupported size";
        case PA_ERR_BUSY: return "busy / not ready";
        default: return "unknown";
    }
}

const char *pa_version(void) { return "pa_gb300 0.1 (sm_103a)"; }

}  // extern "C"

static int tune_geometry(pa_plan_t *pl, int stage, uint64_t G, uint64_t K, uint32_t l, u32 *logR_out, u32 *tc_out) {
    const auto key = std::make_tuple(G, K, l);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *logR_out = it->second.first;
            *tc_out = it->second.second;
            return PA_OK;
        }
    }
    u32 dR, dtc;
    default_geometry(l, &dR, &dtc);
    // synthetic operands: a fixed bit pattern as key and seed
    const uint64_t words = std::max<uint64_t>((pl->n + 63) / 64, ((pl->k + 2) * pl->gamma + 63) / 64) + 2;
    DevAlloc scratch;
    int aerr = scratch.init(pl->mem.async);
    void *src = scratch.take(words * 8, &aerr);
    if (aerr) return aerr;
    cudaStream_t s = scratch.stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PA_OK;
    if (cudaMemsetAsync(src, 0xA5, words * 8, s) || cudaEventCreate(&e0) || cudaEventCreate(&e1) ||
        cudaMemsetAsync(pl->flags, 0, pl->flags_bytes, s))
        rc = PA_ERR_CUDA;
    float best = 1e30f;
    u32 bestR = dR, besttc = dtc;
    for (int dr = -1; dr <= 1 && !rc; dr++) {
        if ((int)dR + dr < 0) continue;
        const u32 logR = (u32)((int)dR + dr);
        for (u32 tc : {1u, 2u, 4u, 8u}) {
            if (!geometry_ok(l, logR, tc)) continue;
            DevAlloc tmp;
            Xform X;
            if (tmp.init(pl->mem.async) || build_xform(pl, X, G, K, logR, tc, &tmp)) continue;
            X.stage = (u32)stage;
            Operands ops;
            ops.pair0 = 0;
            ops.key = (const u64 *)src;
            ops.seed = (const u64 *)src;
            ops.y = (const u64 *)src;
            ops.y_zero = pl->flags + 1;
            ops.reload = pl->flags;
            ops.n = pl->n;
            ops.gamma = pl->gamma;
            ops.k = pl->k;
            ops.mode = stage;
            float t_min = 1e30f;
            for (int rep = 0; rep < 4 && !rc; rep++) {
                int e = cudaEventRecord(e0, s);
                if (!e) e = launch_fwd_col(X, ops, (int)K, pl->Y, s);
                if (!e) e = launch_row_mac(X, pl->Y, pl->S, s);
                if (!e) e = launch_inv_col(X, pl->S, pl->Y, nullptr, 0, 0, s);
                if (!e) e = cudaEventRecord(e1, s);
                if (!e) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e) rc = PA_ERR_CUDA;
                if (rep > 0) t_min = std::min(t_min, ms);
            }
            if (!rc && t_min < best) {
                best = t_min;
                bestR = logR;
                besttc = tc;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!rc && scratch.sync()) rc = PA_ERR_CUDA;
    scratch.release();
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_pair(bestR, besttc);
    }
    *logR_out = bestR;
    *tc_out = besttc;
    return PA_OK;
}

// Step-0 parameters and transform lengths for (n, r), host arithmetic only.
int pa::choose_params(uint64_t n_bits, uint64_t r_bits, const pa_params *params, uint32_t *gamma, uint64_t *k,
                      uint32_t *log_mmh, uint32_t *log_mh) {
    if (n_bits == 0 || r_bits == 0) return PA_ERR_INVALID;
    int rc = choose_gamma(r_bits, params, gamma);
    if (rc) return rc;
    *k = (n_bits + *gamma - 1) / *gamma;
    if ((rc = choose_len(*gamma, *k, log_mmh))) return rc;
    return choose_len(2ULL * *gamma, 1, log_mh);
}

extern "C" {

// Workspace bytes pa_plan would allocate for (n, r), without allocating.
int pa_plan_estimate_bytes(uint64_t n_bits, uint64_t r_bits, const pa_params *params, uint64_t *bytes) {
    if (!bytes || n_bits == 0 || r_bits == 0) return PA_ERR_INVALID;
    uint32_t gamma, l1, l2;
    int rc = choose_gamma(r_bits, params, &gamma);
    if (rc) return rc;
    const uint64_t k = (n_bits + gamma - 1) / gamma;
    if ((rc = choose_len(gamma, k, &l1)) || (rc = choose_len(2ULL * gamma, 1, &l2))) return rc;
    int backend = PA_BACKEND_GOLDILOCKS;
    if ((rc = choose_backend(gamma, k, params, l1, &backend))) return rc;
    *bytes = backend == PA_BACKEND_P3 ? p3_plan_bytes(gamma, k) : ws_sizes(gamma, k, 1ULL << l1, 1ULL << l2).total();
    return PA_OK;
}

// Field constants for host-side checks: omega_N (order N) and theta_N (theta^N = 2).
int pa_field_constants(uint32_t log_n, uint64_t *omega, uint64_t *theta) {
    if (log_n > 26 || !omega || !theta) return PA_ERR_INVALID;
    *omega = root_of_unity(log_n);
    *theta = root_of_two(log_n);
    return PA_OK;
}

// Device F_q arithmetic check: out[3i..3i+2] = a+b, a-b, a*b (canonical).
int pa_selftest_field(const uint64_t *a, const uint64_t *b, uint64_t *out, uint64_t n, void *stream) {
    if (!a || !b || !out) return PA_ERR_INVALID;
    return launch_selftest_field((const u64 *)a, (const u64 *)b, (u64 *)out, n, stream) ? PA_ERR_CUDA : PA_OK;
}

// Four-step geometry of a plan's transform (stage 0: Eq. 2, 1: Eq. 4).
int pa_plan_geometry(const pa_plan_t *pl, int stage, uint32_t *log_r, uint32_t *log_c, uint32_t *tile_cols) {
    if (!pl || !log_r || !log_c || !tile_cols || stage < 0 || stage > 1) return PA_ERR_INVALID;
    if (pl->p3) {
        const Geo3 *G3 = p3_stage(pl->p3, stage);
        *log_r = G3->logR;
        *log_c = G3->logC;
        *tile_cols = G3->tc;
        return PA_OK;
    }
    const Xform &X = stage ? pl->mh : pl->mmh;
    *log_r = X.logR;
    *log_c = X.logC;
    *tile_cols = X.tc;
    return PA_OK;
}

// Tuning results across processes: one line per entry,
//   "geometry G K logN logR tile"   (four-step split of a Goldilocks transform)
//   "backend gamma k choice"        (measured backend of tuned AUTO plans)
int pa_tune_cache_save(const char *path) {
    if (!path) return PA_ERR_INVALID;
    FILE *f = fopen(path, "w");
    if (!f) return PA_ERR_INVALID;
    int n = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &kv : g_tune_cache) {
            fprintf(f, "geometry %llu %llu %u %u %u\n", (unsigned long long)std::get<0>(kv.first),
                    (unsigned long long)std::get<1>(kv.first), std::get<2>(kv.first), kv.second.first, kv.second.second);
            n++;
        }
        for (auto &kv : g_backend_cache) {
            fprintf(f, "backend %u %llu %u\n", kv.first.first, (unsigned long long)kv.first.second, kv.second);
            n++;
        }
    }
    return fclose(f) == 0 ? n : PA_ERR_INVALID;
}

int pa_tune_cache_load(const char *path) {
    if (!path) return PA_ERR_INVALID;
    FILE *f = fopen(path, "r");
    if (!f) return PA_ERR_INVALID;
    char line[256];
    int n = 0, bad = 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    while (fgets(line, sizeof line, f)) {
        unsigned long long G, K, k;
        unsigned l, logR, tc, gamma, choice;
        if (sscanf(line, "geometry %llu %llu %u %u %u", &G, &K, &l, &logR, &tc) == 5) {
            if (!geometry_ok(l, logR, tc)) {
                bad = 1;
                continue;
            }
            g_tune_cache[std::make_tuple((uint64_t)G, (uint64_t)K, (uint32_t)l)] = std::make_pair(logR, tc);
            n++;
        } else if (sscanf(line, "backend %u %llu %u", &gamma, &k, &choice) == 3) {
            if (choice != PA_BACKEND_GOLDILOCKS && choice != PA_BACKEND_P3) {
                bad = 1;
                continue;
            }
            g_backend_cache[std::make_pair((uint32_t)gamma, (uint64_t)k)] = choice;
            n++;
        } else if (line[0] != '\n' && line[0] != '#') {
            bad = 1;
        }
    }
    fclose(f);
    return bad ? PA_ERR_INVALID : n;
}

// Failure injection for tests: of the library's next device (and pinned host)
// allocations, let `skip` succeed, then fail `count` with PA_ERR_NOMEM.
int pa_debug_fail_allocs(uint32_t skip, uint32_t count) {
    g_fail_skip = skip;
    g_fail_count = count;
    return PA_OK;
}

// Digit split chosen for a modulus of G bits and K operand pairs.
int pa_transform_len(uint64_t G, uint64_t K, uint32_t *log_n) {
    if (!log_n || G == 0 || K == 0) return PA_ERR_INVALID;
    return choose_len(G, K, log_n);
}

}  // extern "C"
