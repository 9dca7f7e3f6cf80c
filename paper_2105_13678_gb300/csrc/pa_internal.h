// pa_internal.h -- shared definitions of the GB300 MMH-MH library (not part of the ABI).
//
// Arithmetic model.  Every large product of Algorithm 1 is an exact cyclic
// convolution computed with a number-theoretic transform over the prime
//   q = 2^64 - 2^32 + 1  ("Goldilocks"),
// using the irrational-base discrete weighted transform (Crandall and Fagin,
// Math. Comp. 62 (1994)): a G-bit operand is cut into N digits, digit j
// holding bits [s_j, s_{j+1}) with s_j = ceil(G j / N), and digit j is
// multiplied by the weight theta^((-G j) mod N) where theta^N = 2 in F_q.  The
// cyclic convolution of the weighted digits, un-weighted, then equals the
// product modulo 2^G - 1.  With G = gamma this is exactly the reduction mod
// the Mersenne prime p of Eq. 2; with G = 2 gamma it is the exact product b*y
// needed by Eq. 4 (b*y + c < 2^(2 gamma) - 1).  theta exists for N <= 2^26
// because 2 has multiplicative order 192 in F_q.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

struct pa_params;
struct pa_plan_s;

#if defined(__CUDACC__)
#define PA_HD __host__ __device__ __forceinline__
#else
#define PA_HD inline
#endif

namespace pa {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u64 GL_Q = 0xFFFFFFFF00000001ULL;  // 2^64 - 2^32 + 1
constexpr u64 GL_EPS = 0xFFFFFFFFULL;        // 2^64 mod q

// a, b canonical (< q) -> canonical sum.
PA_HD u64 gl_add(u64 a, u64 b) {
    u64 s = a + b;
    if (s < a) s += GL_EPS;  // wrapped: add 2^64 mod q (result is then < q)
    if (s >= GL_Q) s -= GL_Q;
    return s;
}

PA_HD u64 gl_sub(u64 a, u64 b) {
    u64 d = a - b;
    if (a < b) d -= GL_EPS;  // wrapped: subtract 2^64 mod q, i.e. add q
    return d;
}

// (hi * 2^64 + lo) mod q, canonical.  2^64 = 2^32 - 1 and 2^96 = -1 (mod q).
PA_HD u64 gl_reduce128(u64 lo, u64 hi) {
    u64 hh = hi >> 32, hl = hi & 0xFFFFFFFFULL;
    u64 t = lo - hh;
    if (lo < hh) t -= GL_EPS;
    u64 u = (hl << 32) - hl;
    u64 r = t + u;
    if (r < u) r += GL_EPS;
    if (r >= GL_Q) r -= GL_Q;
    return r;
}

PA_HD u64 gl_mul(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
    return gl_reduce128(a * b, __umul64hi(a, b));
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    return gl_reduce128((u64)p, (u64)(p >> 64));
#endif
}

inline u64 gl_pow(u64 b, u64 e) {
    u64 r = 1;
    while (e) {
        if (e & 1) r = gl_mul(r, b);
        b = gl_mul(b, b);
        e >>= 1;
    }
    return r;
}

inline u64 gl_inv(u64 a) { return gl_pow(a, GL_Q - 2); }

// ------------------------------------------------------------------ plans --

// Device memory of one plan (pa_api.cu).  Plans made by pa_plan allocate with
// cudaMalloc; plans made by the server allocate stream-ordered
// (cudaMallocAsync / cudaFreeAsync on the plan's private stream), so that
// building or dropping one never waits for other work on the device.  Table
// uploads and fills run on the private stream and are waited for on it alone.
struct DevAlloc {
    cudaStream_t stream = nullptr;  // private, non-blocking
    bool async = false;
    std::vector<void *> ptrs;
    uint64_t bytes = 0;
    int init(bool stream_ordered);                            // PA_OK or PA_ERR_CUDA
    void *take(size_t b, int *err);                           // sets *err = PA_ERR_NOMEM on failure
    void upload(void *dst, const void *src, size_t b, int *err);  // host -> device on `stream`
    int sync();                                               // wait for `stream`; PA_OK or PA_ERR_CUDA
    void release();                                           // free every allocation
    ~DevAlloc() { release(); }
};
// Host-side failure injection for tests (pa_debug_fail_allocs): true when the
// allocation about to be made must fail.
bool alloc_fail_injected();

// One weighted cyclic transform of length N = R * C over F_q.  All tables are
// device pointers owned by the plan.
struct Xform {
    u64 N;       // transform length (power of two)
    u64 G;       // the modulus is 2^G - 1; digit j holds bits [s_j, s_{j+1})
    u32 logN, logR, logC, R, C;
    u32 hb;      // split of the two-level tables: e = hi * 2^hb + lo
    u32 tc;      // columns per CTA tile in the column passes
    u32 K;       // operand pairs accumulated in the transform domain
    u32 stage;   // 0: MMH (Eq. 2), 1: MH (Eq. 4); used for trace names
    const u64 *twR, *itwR;           // omega_R^e, omega_R^-e, e < R
    const u64 *twC, *itwC;           // omega_C^e, omega_C^-e, e < C
    const u64 *ipw_lo, *ipw_hi;      // omega_N^e (two-level), e < N
    const u64 *iipw_lo, *iipw_hi;    // omega_N^-e
    const u64 *wt_lo, *wt_hi;        // theta^e
    const u64 *iwt_lo, *iwt_hi;      // theta^-e / N
    // Column-pass tables.  With j = r C + c, (-G j) mod N = (beta_r + alpha_c) mod N,
    // beta_r = (-G C r) mod N, alpha_c = (-G c) mod N, so the weight is
    // theta^beta_r * theta^alpha_c / 2^[beta_r + alpha_c >= N].  The row factor
    // (and the halving) is applied before the column transform, the column
    // factor after it, merged with the inter-pass twiddle:
    const u64 *colw;                 // [0, R): theta^beta_r; [R, 2R): theta^beta_r / 2
    const u64 *coltw;                // N entries, [r][c]: omega_N^(c bitrev_R(r)) theta^alpha_c
};

// Where the digits of operand o come from.
struct Operands {
    const u64 *key;     // Eq. 2 key, n bits
    const u64 *seed;    // (k+2) gamma bits: a_1..a_k, b, c
    const u64 *y;       // Eq. 4 input (MMH value), gamma bits
    const int *y_zero;  // if *y_zero != 0, y is p itself and reads as 0
    int *reload;        // reload flag + per-slice all-ones counters (Algorithm 1)
    u64 n, gamma, k;
    int mode;           // pairs: 0 MMH (x_i, a_i), 1 MH (y, b), 6 Toeplitz (x_J, w_IJ);
                        // single: 2 a_i, 3 x_i, 4 b, 5 y
    u32 pair0;          // first pair / operand handled by the launch (blockIdx.y offset)
    // Toeplitz (mode 6): key segments of rb bits; the seed, shifted up by rb
    // zero bits, holds seed_bits bits; the windows of output block blk
    u64 rb = 0, seed_bits = 0;
    u32 blk = 0;
};

// Carry resolution of N digits (value mod 2^G - 1, end-around carry).
struct CarryDev {
    u64 N, G;             // digit geometry of the transform: s_j = ceil(G j / N)
    u32 logN;
    u32 ub = 0;           // nonzero: uniform digits, s_j = min(j ub, G) (three-prime backend)
    int linear;           // 0: ring mod 2^G - 1 over all N digits; 1: digits [0, nchunks * D) only,
                          //    carry out of the top dropped (the low half of an exact product)
    u64 nchunks;          // digits / PA_CARRY_D
    u64 *H;               // chunk carry-outs (multi-bit), nchunks
    unsigned char *state; // chunk G/P state, nchunks
    unsigned char *cta_state, *cta_cin;
    int *allones;         // set when the resolved value is 2^G - 1 (== 0)
};

// One stage of the three-prime backend (pa_p3.cu): linear convolution of
// digit vectors of M = T/2 digits of b bits, transform length T = R * C, over
// the primes p[0..2] (< 2^28 for T <= 2^21, else < 2^30; 2^logT | p - 1).  Twiddle tables hold
// (w, floor(w 2^32 / p)) pairs; device pointers owned by the plan.
struct Geo3 {
    u64 T, M;        // transform length, digit slots per operand (T / 2)
    u64 nd;          // digits holding operand bits: ceil(G / b)
    u64 G;           // gamma: operand bits, and the modulus 2^G - 1 (Eq. 2) or 2^G (Eq. 4)
    u64 p01;         // p0 p1
    u32 logT, logR, logC, R, C, tc, b, K, stage;
    u32 head;                   // 2^head p < 2^32 for all three primes (lazy-reduction headroom)
    u32 p[3], pinv[3];          // primes and p^-1 mod 2^32
    uint2 scale[3], red[3];     // 2^32 / T mod p; (1, floor(2^32 / p))
    uint2 c12, p0m2, c3;        // p0^-1 mod p1; p0 mod p2; (p0 p1)^-1 mod p2
    // Round twiddle tables: for round rd of the length-R (C) transform, entry
    // rof[rd] + lo (2^NS - 1) + q holds the q-th twiddle (stage by stage) of
    // the task with offset lo: omega^(+-(lo + jj stride) 2^(s0 + sg)).
    const uint2 *twR[3], *itwR[3];
    const uint2 *twC[3], *itwC[3];
    u32 rofR[6], rofC[6];
    u32 rof4R;      // forward R table: offset of the 4-stage first round (15 twiddles per lo), 0: none
    u32 rof4Ri;     // inverse R table: the same 4-stage round with inverse twiddles, 0: none
    const uint2 *ctw[3], *ictw[3];  // T entries, [r][c]: omega_T^(+-c bitrev_R(r))
    // R = 2^10: the forward ctw of the last column round (rows 8 g + m, m < 8)
    // as A[g][c] = omega_T^(c bitrev_7(g)) (128 C entries) times
    // B[c][m] = omega_T^(128 c bitrev_3(m)) (8 C entries)
    const uint2 *ctwA[3], *ctwB[3];
};

constexpr u32 PA_CARRY_D = 8;      // digits per thread chunk
constexpr u32 PA_CARRY_T = 256;    // threads per CTA in the carry kernels
constexpr u32 PA_COL_T = 256;      // threads per CTA in the column passes
constexpr u32 PA_MAX_LOGN = 24;    // largest transform the kernels implement
constexpr u32 PA_MAX_LOGR = 11;    // column length cap (smem tile R x tc)

// Plans (pa_api.cu).  stream_ordered: allocations and table fills on the
// plan's private stream (cudaMallocAsync), for the server.
int plan_create(uint64_t n_bits, uint64_t r_bits, const ::pa_params *params, bool stream_ordered,
                ::pa_plan_s **out);
// Destroy a plan none of whose work is pending (no device synchronisation).
void plan_destroy_idle(::pa_plan_s *pl);

// Step-0 parameters (pa_api.cu): gamma, k and log2 of both transform lengths.
int choose_params(uint64_t n_bits, uint64_t r_bits, const struct pa_params *params, uint32_t *gamma, uint64_t *k,
                  uint32_t *log_mmh, uint32_t *log_mh);

// Tracing (pa_trace.cu): event pair around a launch when enabled.
void *trace_begin(const char *name, u32 stage, void *stream);
void trace_end(void *token, void *stream);

// Programmatic dependent launch.  Kernels of a stream sequence are launched
// with programmatic stream serialization: the next grid may be scheduled while
// the previous one drains (each CTA signals once its stores are issued), and
// it waits at pdl_wait() -- before touching any memory -- until the previous
// grid has completed and its writes are visible.  Launched without the
// attribute, both are no-ops.
#if defined(__CUDACC__)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// Every launch goes through TRACED(): when tracing is on (pa_trace_enable) and
// the stream is not being captured, a CUDA event pair is recorded on the
// launching stream around the kernel.
#define TRACED(name, stage, stream, launch)                      \
    do {                                                         \
        void *tr_ = trace_begin((name), (stage), (stream));      \
        launch;                                                  \
        trace_end(tr_, (stream));                                \
    } while (0)

// Kernel launch wrappers (pa_kernels.cu).  All return a cudaError_t as int.
int prepare_kernels();
int launch_fwd_col(const Xform &X, const Operands &S, int num_pairs, u64 *Y, void *stream);
int launch_row_mac(const Xform &X, const u64 *Y, u64 *S, void *stream);
int launch_fwd_col_single(const Xform &X, const Operands &S, int num_operands, u64 *Y, void *stream);
int launch_row_store(const Xform &X, const u64 *Y, u64 *Spec, void *stream);
int launch_row_prepared(const Xform &X, const u64 *Y, const u64 *Spec, u64 *S, void *stream);
int launch_inv_col(const Xform &X, const u64 *S, u64 *Z, const u64 *add_src, u64 add_base,
                   u64 add_len, void *stream);
int launch_carry(const Xform &X, const CarryDev &cd, u64 *z, u64 *out_bits, u64 out_words,
                 void *stream);
// General form: cd.nchunks chunks of PA_CARRY_D digits (any count; ndigits
// digits for the single-thread path), ring or linear per cd.linear; parallel
// when there are enough chunks and every chunk spans at least 64 bits.
int launch_carry_chunks(const CarryDev &cd, u64 ndigits, bool wide_chunks, u32 stage, u64 *z, u64 *out_bits,
                        u64 out_words, void *stream, bool zeroed = false, bool pdl = false);
int launch_extract(const u64 *t, u64 gamma, u64 r, const int *reload, u64 k, u64 *out,
                   int *status, void *stream, bool pdl = false);
int launch_canonical_zero(const int *flag, u64 *y, u64 words, void *stream, bool pdl = false);
int launch_selftest_field(const u64 *a, const u64 *b, u64 *out, u64 n, void *stream);
int launch_fill_coltw(const Xform &X, u64 *coltw, void *stream);

// Three-prime backend launchers (pa_p3.cu).
int p3_prepare_kernels();
int p3_launch_fwd_col(const Geo3 &X, const Operands &S, int pairs, u32 *Y, void *stream, bool pair = true);
int p3_launch_row_mac(const Geo3 &X, const u32 *Y, u32 *S3, void *stream, int mode = 0, u32 *spec = nullptr);
int p3_launch_inv_col(const Geo3 &X, u32 *S3, u64 *zero_out, u64 zero_words, void *stream);
int p3_launch_digits(const Geo3 &X, const u32 *S3, u64 *z, u64 npad, const u64 *c_src, u64 c_base, u64 *zero_out,
                     u64 zero_words, void *stream);
int p3_launch_fill_ctw(u32 logR, u32 logC, u32 h, const u32 *lo, const u32 *hi, u32 p, uint2 *out, void *stream);

// Three-prime plans (pa_p3.cu).
struct P3Plan;
// Toeplitz-hashing PA (the comparison scheme): z = T x over GF(2) as block
// products on 1-bit digits, output blocks of 2^rb_log bits.
int p3_toeplitz_create(uint64_t n, uint64_t r, uint32_t rb_log, P3Plan **out);
int p3_toeplitz_hash(P3Plan *pl, const u64 *key, const u64 *seed, u64 *out, void *stream);
void p3_toeplitz_query(const P3Plan *pl, uint64_t *rb, uint64_t *segments, uint64_t *blocks);
int p3_feasible(uint32_t gamma, uint64_t k, uint32_t *logT_mmh, uint32_t *logT_mh);
uint64_t p3_plan_bytes(uint32_t gamma, uint64_t k);
int p3_plan_create(uint64_t n, uint64_t r, uint32_t gamma, uint64_t k, bool stream_ordered, P3Plan **out);
void p3_plan_destroy(P3Plan *pl);
void p3_plan_query(const P3Plan *pl, uint64_t *len_mmh, uint64_t *len_mh, uint64_t *ws_bytes);
const Geo3 *p3_stage(const P3Plan *pl, int stage);
int p3_enqueue_mmh(P3Plan *pl, const u64 *key, const u64 *seed, u64 *y, bool canonical, void *stream);
int p3_enqueue_hash(P3Plan *pl, const u64 *key, const u64 *seed, u64 *out, int *status, void *stream);
// Seed reuse: spectra of a_1..a_k and b (and a seed copy) kept in the plan.
int p3_seed_prepare(P3Plan *pl, const u64 *seed, void *stream);
int p3_hash_prepared(P3Plan *pl, const u64 *key, u64 *out, int *status, void *stream);
bool p3_prepared(const P3Plan *pl);
int *p3_flags(P3Plan *pl);
size_t p3_flags_bytes(const P3Plan *pl);

}  // namespace pa
