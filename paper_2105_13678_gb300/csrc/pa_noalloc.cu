// pa_noalloc.cu -- pa_hash_noalloc: Algorithm 1 for small blocks without any
// device memory allocation.
//
// Some callers cannot call cudaMalloc: code that runs while device memory is
// owned by another allocator or pool, code with a hard latency budget where an
// allocation (which may synchronise the device) is not allowed, or code that
// must not grow the process's device footprint after start-up.  For them this
// entry point runs the same kernels as pa_plan + pa_hash, but every
// intermediate buffer and every root-of-unity/weight table lives in one
// file-scope __device__ array of PA_NOALLOC_SCRATCH_BYTES (16 MiB).  That
// array is part of the library image: every GPU that loads the library holds
// it until the process exits.  The caller passes only the inputs and outputs.
//
// Host code never dereferences the array's name (on the host it is only a
// stand-in for the symbol); the device address is obtained with
// cudaGetSymbolAddress on the first call made while that device is current
// (and again after the device's context has been re-created, e.g. by
// cudaDeviceReset), and cached.  Every call shares the array and leaves its contents
// behind; the parts that must start at zero are cleared on the stream by each
// call.  Calls whose work overlaps on the GPU (different streams without
// ordering, or several host threads) race on the shared array.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pa_gb300.h"
#include "gl_device.cuh"
#include "pa_internal.h"

using namespace pa;

namespace {

constexpr unsigned long long kScratchBytes = PA_NOALLOC_SCRATCH_BYTES;
constexpr unsigned long long kScratchWords = kScratchBytes / 8;

}  // namespace

static __device__ __align__(256) unsigned long long g_pa_noalloc_scratch[kScratchWords];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mu;
// Per device: the array's device address and the context it was looked up
// in.  A device reset (cudaDeviceReset) or a re-created primary context loads
// a new copy of the module, so the address is looked up again whenever the
// current context differs from the one recorded.
unsigned long long *g_scratch_dev[kMaxDevices];
void *g_scratch_ctx[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void **);

void *current_context() {
    static CtxGetCurrentFn fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)f;
        cudaGetLastError();
        looked_up = true;
    }
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

int scratch_address(unsigned long long **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PA_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    void *ctx = current_context();  // null until the runtime has bound a context to this thread
    if (!g_scratch_dev[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pa_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PA_ERR_CUDA;
        }
        g_scratch_dev[dev] = (unsigned long long *)p;
        g_scratch_ctx[dev] = current_context();
    }
    *out = g_scratch_dev[dev];
    return PA_OK;
}

struct TableJob {
    u64 *dst;
    u64 base, scale;
    u32 count;
};
struct TableJobs {
    TableJob t[26];
};

// Table y of the batch: dst[i] = scale * base^i for i < count.
__global__ void k_fill_tables(TableJobs J) {
    const TableJob tj = J.t[blockIdx.y];
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < tj.count; i += gridDim.x * blockDim.x) {
        u64 r = tj.scale, b = tj.base;
        for (u32 e = i; e; e >>= 1) {
            if (e & 1) r = gd_mul(r, b);
            b = gd_mul(b, b);
        }
        tj.dst[i] = gd_canon(r);
    }
}

// Bump allocator over the static array (offsets only; nothing is allocated).
struct Carve {
    unsigned long long *base;
    unsigned long long used = 0;  // words
    bool overflow = false;
    u64 *take(unsigned long long words) {
        words = (words + 31) & ~31ULL;  // 256-byte alignment
        if (used + words > kScratchWords) {
            overflow = true;
            return nullptr;
        }
        u64 *p = (u64 *)(base + used);
        used += words;
        return p;
    }
};

// Same geometry as a plan's transform; tables are carved from the scratch and
// described in `jobs` for k_fill_tables.
void geometry_and_tables(Xform &X, uint64_t G, uint64_t K, uint32_t l, u32 stage, Carve &cv, TableJobs &jobs,
                         int &nj) {
    X.N = 1ULL << l;
    X.G = G;
    X.K = (u32)K;
    X.stage = stage;
    X.logN = l;
    X.logR = l / 2 < PA_MAX_LOGR ? l / 2 : PA_MAX_LOGR;
    X.logC = l - X.logR;
    X.R = 1u << X.logR;
    X.C = 1u << X.logC;
    X.hb = (l + 1) / 2;
    u32 tc = 8;
    while (tc > 1 && (uint64_t)X.R * tc > 4096) tc >>= 1;
    while (tc > X.C) tc >>= 1;
    X.tc = tc;
    u64 w = 0, th = 0;
    pa_field_constants(l, (uint64_t *)&w, (uint64_t *)&th);
    const u64 wi = gl_inv(w), thi = gl_inv(th), ninv = gl_inv(X.N % GL_Q);
    const u64 wR = gl_pow(w, X.C), wC = gl_pow(w, X.R);
    const u32 nlo = 1u << X.hb, nhi = (u32)(X.N >> X.hb);
    auto add = [&](const u64 *&dst, u64 base, u32 count, u64 scale) {
        if (count == 0) count = 1;
        u64 *p = cv.take(count);
        dst = p;
        jobs.t[nj++] = TableJob{p, base, scale, count};
    };
    add(X.twR, wR, X.R, 1);
    add(X.itwR, gl_inv(wR), X.R, 1);
    add(X.twC, wC, X.C, 1);
    add(X.itwC, gl_inv(wC), X.C, 1);
    add(X.ipw_lo, w, nlo, 1);
    add(X.ipw_hi, gl_pow(w, nlo), nhi, 1);
    add(X.iipw_lo, wi, nlo, 1);
    add(X.iipw_hi, gl_pow(wi, nlo), nhi, 1);
    add(X.wt_lo, th, nlo, 1);
    add(X.wt_hi, gl_pow(th, nlo), nhi, 1);
    add(X.iwt_lo, thi, nlo, 1);
    add(X.iwt_hi, gl_pow(thi, nlo), nhi, ninv);
    // column weights theta^beta_r (and / 2) are filled by k_fill_colw; coltw by launch_fill_coltw
    X.colw = cv.take(2 * (unsigned long long)X.R);
    X.coltw = cv.take(X.N);
}

// colw[r] = theta^beta_r, colw[R + r] = theta^beta_r / 2, beta_r = (-G C r) mod N.
__global__ void k_fill_colw(Xform X, u64 theta, u64 half) {
    u64 *out = const_cast<u64 *>(X.colw);
    for (u32 r = blockIdx.x * blockDim.x + threadIdx.x; r < X.R; r += gridDim.x * blockDim.x) {
        const u64 beta = (0ULL - X.G * X.C * (u64)r) & (X.N - 1);
        u64 v = 1, b = theta;
        for (u64 e = beta; e; e >>= 1) {
            if (e & 1) v = gd_mul(v, b);
            b = gd_mul(b, b);
        }
        out[r] = gd_canon(v);
        out[X.R + r] = gd_canon(gd_mul(v, half));
    }
}

}  // namespace

extern "C" int pa_hash_noalloc(uint64_t n_bits, uint64_t r_bits, const pa_params *params, const uint64_t *key,
                               const uint64_t *seed, uint64_t *out, int *status, void *stream) {
    if (!key || !seed || !out || n_bits == 0 || r_bits == 0) return PA_ERR_INVALID;
    if (params) {
        for (uint32_t v : params->reserved)
            if (v) return PA_ERR_INVALID;
        if (params->backend > PA_BACKEND_P3) return PA_ERR_INVALID;
        if (params->backend == PA_BACKEND_P3) return PA_ERR_UNSUPPORTED;  // Goldilocks transforms only
    }
    uint32_t gamma, l1, l2;
    uint64_t k;
    int rc = choose_params(n_bits, r_bits, params, &gamma, &k, &l1, &l2);
    if (rc) return rc;
    if (k > 65535) return PA_ERR_UNSUPPORTED;

    unsigned long long *base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
    Carve cv;
    cv.base = base;
    TableJobs jobs;
    int nj = 0;
    Xform X1, X2;
    geometry_and_tables(X1, gamma, k, l1, 0, cv, jobs, nj);
    geometry_and_tables(X2, 2ULL * gamma, 1, l2, 1, cv, jobs, nj);
    const uint64_t N1 = X1.N, N2 = X2.N, Nmax = N1 > N2 ? N1 : N2;
    const uint64_t nch = Nmax / PA_CARRY_D ? Nmax / PA_CARRY_D : 1;
    u64 *Y = cv.take(2 * k * N1 > 2 * N2 ? 2 * k * N1 : 2 * N2);
    u64 *S = cv.take(Nmax);
    u64 *ybuf = cv.take((gamma + 63) / 64 + 2);
    u64 *tbuf = cv.take((2ULL * gamma + 63) / 64 + 2);
    u64 *H = cv.take(nch);
    unsigned char *cstate = (unsigned char *)cv.take((nch + 7) / 8);
    unsigned char *cta_state = (unsigned char *)cv.take((nch / PA_CARRY_T + 1 + 7) / 8);
    unsigned char *cta_cin = (unsigned char *)cv.take((nch / PA_CARRY_T + 1 + 7) / 8);
    const size_t flag_bytes = (4 + k) * sizeof(int);
    int *flags = (int *)cv.take((flag_bytes + 7) / 8);
    if (cv.overflow) return PA_ERR_UNSUPPORTED;  // block too large for the static scratch

    cudaStream_t s = (cudaStream_t)stream;
    if (prepare_kernels()) return PA_ERR_CUDA;
    k_fill_tables<<<dim3(16, nj), 256, 0, s>>>(jobs);
    int e = (int)cudaGetLastError();
    const u64 half = gl_inv(2);
    for (Xform *X : {&X1, &X2}) {
        u64 w = 0, th = 0;
        pa_field_constants(X->logN, (uint64_t *)&w, (uint64_t *)&th);
        if (!e) {
            k_fill_colw<<<8, 256, 0, s>>>(*X, th, half);
            e = (int)cudaGetLastError();
        }
        if (!e) e = launch_fill_coltw(*X, const_cast<u64 *>(X->coltw), stream);
    }
    if (!e) e = cudaMemsetAsync(flags, 0, flag_bytes, s);

    Operands ops;
    ops.pair0 = 0;
    ops.key = (const u64 *)key;
    ops.seed = (const u64 *)seed;
    ops.y = ybuf;
    ops.y_zero = flags + 1;
    ops.reload = flags;
    ops.n = n_bits;
    ops.gamma = gamma;
    ops.k = k;
    CarryDev cd;
    cd.H = H;
    cd.state = cstate;
    cd.cta_state = cta_state;
    cd.cta_cin = cta_cin;

    // Eq. 2 (MMH): y = sum a_i x_i mod 2^gamma - 1
    ops.mode = 0;
    if (!e) e = launch_fwd_col(X1, ops, (int)k, Y, stream);
    if (!e) e = launch_row_mac(X1, Y, S, stream);
    if (!e) e = launch_inv_col(X1, S, Y, nullptr, 0, 0, stream);
    cd.N = X1.N;
    cd.G = X1.G;
    cd.logN = X1.logN;
    cd.nchunks = X1.N / PA_CARRY_D;
    cd.allones = flags + 1;
    if (!e) e = launch_carry(X1, cd, Y, ybuf, (gamma + 63) / 64, stream);
    // Eq. 4 (MH): out = ((b y + c) mod 2^gamma) >> (gamma - r)
    ops.mode = 1;
    if (!e) e = launch_fwd_col(X2, ops, 1, Y, stream);
    if (!e) e = launch_row_mac(X2, Y, S, stream);
    if (!e) e = launch_inv_col(X2, S, Y, (const u64 *)seed, (k + 1) * (u64)gamma, gamma, stream);
    cd.N = X2.N;
    cd.G = X2.G;
    cd.logN = X2.logN;
    cd.nchunks = X2.N / PA_CARRY_D;
    cd.allones = flags + 2;
    if (!e) e = launch_carry(X2, cd, Y, tbuf, (2ULL * gamma + 63) / 64, stream);
    if (!e) e = launch_extract(tbuf, gamma, r_bits, flags, k, (u64 *)out, status, stream);
    return e ? PA_ERR_CUDA : PA_OK;
}
