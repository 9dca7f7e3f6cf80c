// pa_kernels.cu -- sm_103a kernels of the MMH-MH privacy-amplification hash.
//
// Data path of one block (Algorithm 1, Sec. 3.1), all integer arithmetic:
//   k_fwd_col   unpack gamma-bit slices into weighted digits, column NTTs of
//               the four-step transform, inter-pass twiddles       (Eq. 2/4 inputs)
//   k_row_mac   row NTTs of each operand pair, transform-domain
//               multiply-accumulate sum_i A_i * X_i, inverse row NTTs (Eq. 2)
//   k_inv_col   inverse column NTTs, un-weighting, 1/N, (+ c for Eq. 4)
//   k_carry_*   exact carry resolution of the digit vector modulo 2^G - 1
//               (the Mersenne reduction of Sec. 3.1 happens here as an
//               end-around carry)
//   k_extract   z = bits [gamma - r, gamma) of b*y + c              (Eq. 4)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "gl_device.cuh"
#include "pa_internal.h"

namespace pa {

// ------------------------------------------------------------- helpers --

__device__ __forceinline__ u32 pidx(u32 i) { return i + (i >> 4); }  // 1 pad word per 16

__device__ __forceinline__ u32 bitrev(u32 x, u32 bits) { return bits ? (__brev(x) >> (32 - bits)) : 0u; }

__device__ __forceinline__ u64 tbl2(const u64 *__restrict__ lo, const u64 *__restrict__ hi, u64 e, u32 hb) {
    return gd_mul(__ldg(lo + (e & ((1ULL << hb) - 1))), __ldg(hi + (e >> hb)));
}

__device__ __forceinline__ u64 digit_start(u64 G, u64 j, u64 N, u32 logN) { return (G * j + N - 1) >> logN; }

// nb in [1, 63] bits starting at absolute bit position pos.
__device__ __forceinline__ u64 read_bits(const u64 *__restrict__ src, u64 pos, u32 nb) {
    const u64 wi = pos >> 6;
    const u32 sh = (u32)(pos & 63);
    u64 v = __ldg(src + wi) >> sh;
    if (sh + nb > 64) v |= __ldg(src + wi + 1) << (64 - sh);
    return v & ((1ULL << nb) - 1);
}

// nb in [0, 31] bits starting at absolute bit position pos, read as 32-bit
// words (the second word only when the bits cross into it).
__device__ __forceinline__ u32 read_bits32(const u64 *__restrict__ src, u64 pos, u32 nb) {
    const u32 *s32 = reinterpret_cast<const u32 *>(src);
    const u64 wi = pos >> 5;
    const u32 sh = (u32)(pos & 31);
    const u32 lo = __ldg(s32 + wi);
    const u32 hi = (sh + nb > 32) ? __ldg(s32 + wi + 1) : 0u;
    return __funnelshift_r(lo, hi, sh) & ((1u << nb) - 1u);
}

// Rounds of the in-place transforms.  A round covers stages s0 .. s0+NS-1 of
// a length-L transform (omega_L = 7^((q-1)/L)) on the 2^NS elements
// base + m*stride, lo = base mod stride.  Stage s pairs (i, i + L/2^(s+1))
// with twiddle omega_L^((i mod L/2^(s+1)) * 2^s) (Gentleman-Sande DIF).
// In the final round of a transform stride = 1 and lo = 0, so its twiddles
// are the constants omega_8^k: omega_8 = omega_L^(L/8) = -2^24 for every L
// (2^96 = -1), so omega_8^k = (-1)^k 2^(24k) and the sign swaps the operands
// of the difference.

// Round rd of a length-2^l transform: the first round takes the 1..3 leftover
// stages and every later round 3, so the final round is a full radix-8 round.
__device__ __forceinline__ u32 round_ns(u32 l, u32 rd) { return rd ? 3u : l - 3u * ((l + 2) / 3 - 1); }
__device__ __forceinline__ u32 round_s0(u32 l, u32 rd) { return rd ? round_ns(l, 0) + 3u * (rd - 1) : 0u; }

// x * 2^(24 k), k = 0..3 (2^72 = 2^40 - 2^8 mod q).
__device__ __forceinline__ u64 mul_p24(u64 x, int k) {
    if (k == 1) return gd_mul(x, 1ULL << 24);
    if (k == 2) return gd_mul(x, 1ULL << 48);
    if (k == 3) return gd_mul(x, 0x000000FFFFFFFF00ULL);
    return x;
}

// x * omega_8^k, k = 0..3.
__device__ __forceinline__ u64 mul_w8(u64 x, int k) {
    if (k == 1) return gd_mul(x, 0xFFFFFFFEFF000001ULL);
    if (k == 3) return gd_mul(x, 0xFFFFFEFF00000101ULL);
    return mul_p24(x, k);
}

template <int NS, bool LAST, bool HZ = false>
__device__ __forceinline__ void dif_regs(u64 (&v)[8], u32 s0, u32 lo, u32 stride, const u64 *__restrict__ tw) {
#pragma unroll
    for (int sg = 0; sg < NS; sg++) {
        const int half = 1 << (NS - 1 - sg);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (m & half) continue;
            const u64 a = v[m], b = v[m + half];
            const int k = (m & (half - 1)) * (4 / half);  // LAST: twiddle omega_8^k
            if (HZ && sg == 0) {
                // upper half of the group is zero: (a, 0) -> (a, a w)
                if (LAST) {
                    v[m + half] = mul_w8(a, k);
                } else {
                    const u32 e = (lo + (u32)(m & (half - 1)) * stride) << s0;
                    v[m + half] = gd_mul(a, __ldg(tw + e));
                }
                continue;
            }
            v[m] = gd_add(a, b);
            if (LAST) {
                v[m + half] = mul_p24((k & 1) ? gd_sub(b, a) : gd_sub(a, b), k);
            } else {
                const u32 e = (lo + (u32)(m & (half - 1)) * stride) << (s0 + sg);
                v[m + half] = gd_mul(gd_sub(a, b), __ldg(tw + e));
            }
        }
    }
}

// Inverse of dif_regs up to a factor 2 per stage (decimation in time,
// stages in reverse order, inverse twiddles; in the final round
// omega_8^-k = (-1)^(k+1) 2^(24 (4-k)) for k = 1..3).
template <int NS, bool LAST, bool HO = false>
__device__ __forceinline__ void dit_regs(u64 (&v)[8], u32 s0, u32 lo, u32 stride, const u64 *__restrict__ itw) {
#pragma unroll
    for (int sg = NS - 1; sg >= 0; sg--) {
        const int half = 1 << (NS - 1 - sg);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (m & half) continue;
            const u64 a = v[m];
            u64 b = v[m + half];
            bool neg = false;
            if (LAST) {
                const int k = (m & (half - 1)) * (4 / half);
                if (k) b = mul_p24(b, 4 - k);
                neg = k == 2;
            } else {
                const u32 e = (lo + (u32)(m & (half - 1)) * stride) << (s0 + sg);
                b = gd_mul(b, __ldg(itw + e));
            }
            v[m] = neg ? gd_sub(a, b) : gd_add(a, b);
            if (!(HO && sg == 0)) v[m + half] = neg ? gd_add(a, b) : gd_sub(a, b);  // HO: upper outputs unused
        }
    }
}

// ------------------------------------------------------------- operands --

struct OpDesc {
    const u64 *src;
    u64 base, len;  // operand = bits [base, base + len) of src, zero above len
    int force_odd, check_ones, zero;
};

// Algorithm 1 slices and the seed layout.  Pair i of the MMH stage is
// (x_{i+1}, a_{i+1}): key slice i and seed slice i.  The MH stage has the
// single pair (y, b) with b forced odd.
__device__ __forceinline__ void pair_desc(const Operands &S, u32 i, OpDesc &dx, OpDesc &da) {
    dx.force_odd = da.force_odd = 0;
    dx.check_ones = da.check_ones = 0;
    dx.zero = da.zero = 0;
    if (S.mode == 0) {
        dx.src = S.key;
        dx.base = (u64)i * S.gamma;
        const u64 rem = S.n - dx.base;
        dx.len = rem < S.gamma ? rem : S.gamma;
        dx.check_ones = 1;
        da.src = S.seed;
        da.base = (u64)i * S.gamma;
        da.len = S.gamma;
    } else {
        dx.src = S.y;
        dx.base = 0;
        dx.len = S.gamma;
        dx.zero = (*S.y_zero != 0);
        da.src = S.seed;
        da.base = S.k * S.gamma;
        da.len = S.gamma;
        da.force_odd = 1;
    }
}

// Single operands (seed preparation and prepared hashing): mode 2 = a_{i+1},
// 3 = x_{i+1}, 4 = b (forced odd), 5 = y.
__device__ __forceinline__ void single_desc(const Operands &S, u32 i, OpDesc &d) {
    d.force_odd = 0;
    d.check_ones = 0;
    d.zero = 0;
    d.src = S.seed;
    d.len = S.gamma;
    if (S.mode == 2) {
        d.base = (u64)i * S.gamma;
    } else if (S.mode == 3) {
        d.src = S.key;
        d.base = (u64)i * S.gamma;
        const u64 rem = S.n - d.base;
        d.len = rem < S.gamma ? rem : S.gamma;
        d.check_ones = 1;
    } else if (S.mode == 4) {
        d.base = S.k * S.gamma;
        d.force_odd = 1;
    } else {
        d.src = S.y;
        d.base = 0;
        d.zero = (*S.y_zero != 0);
    }
}

__device__ __forceinline__ u32 op_digit(const OpDesc &d, u64 j, u64 slo, u64 shi, bool &ones) {
    const u64 hi = shi < d.len ? shi : d.len;
    const u32 nb = slo < hi ? (u32)(hi - slo) : 0u;
    u32 dig = read_bits32(d.src, d.base + (slo < hi ? slo : 0), nb);
    ones = ones && (shi <= d.len) && (dig == ((1u << (u32)(shi - slo)) - 1u));
    if (d.force_odd && j == 0) dig |= 1u;
    if (d.zero) dig = 0;
    return dig;
}

// Digits j = r C + c of both operands of a pair, times the row part of the
// weight theta^((-G j) mod N) (the column part is applied after the column
// transform, inside coltw).
// (-G C r) mod N and (-G c) mod N in 32-bit arithmetic (N divides 2^32).
__device__ __forceinline__ u32 gcmodn(const Xform &X) { return (u32)((X.G * X.C) & (X.N - 1)); }
__device__ __forceinline__ u32 alpha_of(const Xform &X, u32 c) { return (0u - (u32)X.G * c) & (u32)(X.N - 1); }

template <bool PAIR>
__device__ __forceinline__ void weighted_pair(const Xform &X, const OpDesc &dx, const OpDesc &da, u32 r, u32 c,
                                              u32 alpha_c, u32 gcm, u64 &wx, u64 &wa, bool &ones) {
    const u64 j = (u64)r * X.C + c;
    const u64 gj = X.G * j;
    const u64 slo = (gj + X.N - 1) >> X.logN;
    const u64 shi = (gj + X.G + X.N - 1) >> X.logN;
    const u32 gx = op_digit(dx, j, slo, shi, ones);
    const u32 beta_r = (0u - gcm * r) & (u32)(X.N - 1);
    const u64 w = __ldg(X.colw + r + (beta_r + alpha_c >= (u32)X.N ? X.R : 0));
    wx = gx ? gd_mul_small(gx, w) : 0;
    if (PAIR) {
        bool dummy = true;
        const u32 ga = op_digit(da, j, slo, shi, dummy);
        wa = ga ? gd_mul_small(ga, w) : 0;
    }
}

// ------------------------------------------------------ forward columns --

#define PA_DISPATCH_NS(ns, call_tmpl)  \
    do {                               \
        if ((ns) == 3) {               \
            call_tmpl(3);              \
        } else if ((ns) == 2) {        \
            call_tmpl(2);              \
        } else {                       \
            call_tmpl(1);              \
        }                              \
    } while (0)


// LL, TC: log2 R and the tile width when fixed at compile time (0: read from X).
template <int NS, bool PAIR, bool FIRST, bool LAST, bool HZ, int LL, int TC>
__device__ __forceinline__ void fwd_col_round(const Xform &X, const OpDesc &dx, const OpDesc &da,
                                              u64 *__restrict__ smx, u64 *__restrict__ sma, u64 *__restrict__ Yx,
                                              u64 *__restrict__ Ya, u32 c0, u32 s0, bool &ones) {
    const u32 l = LL ? (u32)LL : X.logR, tc = TC ? (u32)TC : X.tc;
    const u32 gcm = gcmodn(X);
    const u32 sh = l - s0 - NS, stride = 1u << sh;
    const u32 ntask = ((1u << l) >> NS) * tc;
    const u32 logtc = TC ? (u32)__builtin_ctz(TC) : (u32)(__ffs(tc) - 1);
    for (u32 task = threadIdx.x; task < ntask; task += blockDim.x) {
        const u32 c = task & (tc - 1), g = task >> logtc;
        const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
        const u32 alpha_c = alpha_of(X, c0 + c);
        u64 vx[8], va[8];
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            const u32 r = base + m * stride;
            if (HZ && m >= (1 << (NS - 1))) {  // rows >= R/2: digits j >= N/2 are zero
                vx[m] = 0;
                va[m] = 0;
            } else if (FIRST) {
                weighted_pair<PAIR>(X, dx, da, r, c0 + c, alpha_c, gcm, vx[m], va[m], ones);
            } else {
                vx[m] = smx[pidx(r * tc + c)];
                if (PAIR) va[m] = sma[pidx(r * tc + c)];
            }
        }
        dif_regs<NS, LAST, HZ>(vx, s0, lo, stride, X.twR);
        if (PAIR) dif_regs<NS, LAST, HZ>(va, s0, lo, stride, X.twR);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            const u32 r = base + m * stride;
            if (LAST) {
                // position r holds column frequency bitrev(r): omega_N^(c k_r) theta^alpha_c
                const u64 t = __ldg(X.coltw + (u64)r * X.C + c0 + c);
                Yx[(u64)r * X.C + c0 + c] = gd_mul(vx[m], t);
                if (PAIR) Ya[(u64)r * X.C + c0 + c] = gd_mul(va[m], t);
            } else {
                smx[pidx(r * tc + c)] = vx[m];
                if (PAIR) sma[pidx(r * tc + c)] = va[m];
            }
        }
    }
}

// One CTA: a tile of tc columns of operand pair blockIdx.y (PAIR), written to
// Y[i] and Y[K + i], or of the single operand blockIdx.y, written to Y[i].
template <bool PAIR, int LL, int TC>
__global__ void __launch_bounds__(PA_COL_T, 3) k_fwd_col(Xform X, Operands S, u64 *__restrict__ Y) {
    pdl_wait();
    extern __shared__ u64 sm[];
    const u32 tc = TC ? (u32)TC : X.tc, c0 = blockIdx.x * tc, i = blockIdx.y + S.pair0;
    OpDesc dx, da;
    if (PAIR)
        pair_desc(S, i, dx, da);
    else
        single_desc(S, i, dx);
    u64 *Yx = Y + (u64)i * X.N, *Ya = Y + (u64)(X.K + i) * X.N;
    u64 *smx = sm, *sma = sm + pidx(X.R * tc);
    bool ones = true;
    const u32 l = LL ? (u32)LL : X.logR;
    if (l == 0) {
        for (u32 c = threadIdx.x; c < tc; c += blockDim.x) {
            u64 wx, wa;
            weighted_pair<PAIR>(X, dx, da, 0, c0 + c, alpha_of(X, c0 + c), gcmodn(X), wx, wa, ones);
            const u64 t = __ldg(X.coltw + c0 + c);
            Yx[c0 + c] = gd_mul(wx, t);
            if (PAIR) Ya[c0 + c] = gd_mul(wa, t);
        }
    } else {
        const u32 nr = (l + 2) / 3;
        // Eq. 4 stage: y, b < 2^gamma, so digits j >= N/2 (rows >= R/2) are zero
        const bool hz = X.stage == 1;
#pragma unroll(LL > 0 ? 8 : 1)
        for (u32 rd = 0; rd < nr; rd++) {
            const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
            const bool first = rd == 0, last = rd == nr - 1;
#define PA_FWD_COL(NSV)                                                                     \
    do {                                                                                    \
        if (first && hz && last)                                                            \
            fwd_col_round<NSV, PAIR, true, true, true, LL, TC>(X, dx, da, smx, sma, Yx, Ya, c0, s0, ones); \
        else if (first && hz)                                                               \
            fwd_col_round<NSV, PAIR, true, false, true, LL, TC>(X, dx, da, smx, sma, Yx, Ya, c0, s0, ones); \
        else if (first && last)                                                             \
            fwd_col_round<NSV, PAIR, true, true, false, LL, TC>(X, dx, da, smx, sma, Yx, Ya, c0, s0, ones);   \
        else if (first)                                                                     \
            fwd_col_round<NSV, PAIR, true, false, false, LL, TC>(X, dx, da, smx, sma, Yx, Ya, c0, s0, ones);  \
        else if (last)                                                                      \
            fwd_col_round<NSV, PAIR, false, true, false, LL, TC>(X, dx, da, smx, sma, Yx, Ya, c0, s0, ones);  \
        else                                                                                \
            fwd_col_round<NSV, PAIR, false, false, false, LL, TC>(X, dx, da, smx, sma, Yx, Ya, c0, s0, ones); \
    } while (0)
            PA_DISPATCH_NS(ns, PA_FWD_COL);
#undef PA_FWD_COL
            __syncthreads();
        }
    }
    pdl_trigger();
    if (dx.check_ones) {
        // Algorithm 1 reload rule: slice i is all ones iff every CTA of the slice saw only ones.
        const int all = __syncthreads_and(ones ? 1 : 0);
        if (threadIdx.x == 0 && all) {
            int *cnt = S.reload + 4 + i;
            if (atomicAdd(cnt, 1) + 1 == (int)gridDim.x) atomicExch(S.reload, 1);
        }
    }
}

// --------------------------------------------------- rows + MAC (Eq. 2) --
//
// Row modes: ROW_PAIRS transforms both rows of each pair (x_i, a_i) and
// accumulates their product; ROW_STORE transforms rows of K single operands and
// stores the spectra (seed preparation); ROW_PREPARED transforms the rows of
// x_i and multiplies them with stored spectra.  Spectra are stored at the
// in-place positions of the last forward round.

enum { ROW_PAIRS = 0, ROW_STORE = 1, ROW_PREPARED = 2 };

template <int NS, int ACC, int MODE, bool LAST, int LL>
__device__ __forceinline__ void row_fwd_round(const Xform &X, const u64 *__restrict__ xrow,
                                              const u64 *__restrict__ arow, u64 *__restrict__ smx,
                                              u64 *__restrict__ sma, u64 *__restrict__ spec, u32 s0, bool first,
                                              u64 (&acc)[ACC]) {
    const u32 l = LL ? (u32)LL : X.logC, sh = l - s0 - NS, stride = 1u << sh, ngroups = (1u << l) >> NS;
#pragma unroll
    for (int t = 0; t < (ACC >> NS); t++) {
        const u32 g = threadIdx.x + t * blockDim.x;
        if (g < ngroups) {
            const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
            u64 vx[8], va[8];
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) {
                const u32 idx = base + m * stride;
                vx[m] = first ? __ldg(xrow + idx) : smx[pidx(idx)];
                if (MODE == ROW_PAIRS) va[m] = first ? __ldg(arow + idx) : sma[pidx(idx)];
            }
            dif_regs<NS, LAST>(vx, s0, lo, stride, X.twC);
            if (MODE == ROW_PAIRS) dif_regs<NS, LAST>(va, s0, lo, stride, X.twC);
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) {
                const u32 idx = base + m * stride;
                if (LAST) {
                    if (MODE == ROW_PAIRS)
                        acc[t * (1 << NS) + m] = gd_add(acc[t * (1 << NS) + m], gd_mul(vx[m], va[m]));
                    else if (MODE == ROW_PREPARED)
                        acc[t * (1 << NS) + m] = gd_add(acc[t * (1 << NS) + m], gd_mul(vx[m], __ldg(spec + idx)));
                    else
                        spec[idx] = vx[m];
                } else {
                    smx[pidx(idx)] = vx[m];
                    if (MODE == ROW_PAIRS) sma[pidx(idx)] = va[m];
                }
            }
        }
    }
}

template <int NS, int ACC, bool LAST, int LL>
__device__ __forceinline__ void row_inv_round(const Xform &X, u64 *__restrict__ sm, u64 *__restrict__ Srow, u32 row,
                                              u32 s0, bool to_global, const u64 (&acc)[ACC]) {
    const u32 l = LL ? (u32)LL : X.logC, sh = l - s0 - NS, stride = 1u << sh, ngroups = (1u << l) >> NS;
    const u32 kr = bitrev(row, X.logR);
#pragma unroll
    for (int t = 0; t < (ACC >> NS); t++) {
        const u32 g = threadIdx.x + t * blockDim.x;
        if (g < ngroups) {
            const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
            u64 v[8];
#pragma unroll
            for (int m = 0; m < (1 << NS); m++)
                v[m] = LAST ? acc[t * (1 << NS) + m] : sm[pidx(base + m * stride)];
            dit_regs<NS, LAST>(v, s0, lo, stride, X.itwC);
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) {
                const u32 idx = base + m * stride;
                if (to_global) {
                    const u64 e = (u64)idx * kr;  // omega_N^(-c * k_r)
                    Srow[idx] = gd_mul(v[m], tbl2(X.iipw_lo, X.iipw_hi, e, X.hb));
                } else {
                    sm[pidx(idx)] = v[m];
                }
            }
        }
    }
}

// One CTA per row; blockDim = C / ACC threads, each owning ACC accumulators.
// Y holds the column-pass output; Spec the stored spectra (ROW_STORE writes
// them, ROW_PREPARED reads them); S receives the inverse-row output.
template <int ACC, int MODE, int LL>
__global__ void __launch_bounds__(512, ACC == 8 ? 2 : 1)
    k_row_mac(Xform X, const u64 *__restrict__ Y, u64 *__restrict__ Spec, u64 *__restrict__ S) {
    pdl_wait();
    extern __shared__ u64 sm[];
    const u32 l = LL ? (u32)LL : X.logC, C = 1u << l, row = blockIdx.x;
    const u64 N = X.N;
    u64 *smx = sm, *sma = sm + pidx(C);
    if (l == 0) {
        if (threadIdx.x == 0) {
            u64 s = 0;
            for (u32 i = 0; i < X.K; i++) {
                const u64 x = Y[(u64)i * N + row];
                if (MODE == ROW_PAIRS) s = gd_add(s, gd_mul(x, Y[(u64)(X.K + i) * N + row]));
                if (MODE == ROW_PREPARED) s = gd_add(s, gd_mul(x, Spec[(u64)i * N + row]));
                if (MODE == ROW_STORE) Spec[(u64)i * N + row] = x;
            }
            if (MODE != ROW_STORE) S[row] = s;
        }
        return;
    }
    u64 acc[ACC];
#pragma unroll
    for (int m = 0; m < ACC; m++) acc[m] = 0;
    const u32 nr = (l + 2) / 3;
    for (u32 i = 0; i < X.K; i++) {
        const u64 *xrow = Y + (u64)i * N + (u64)row * C;
        const u64 *arow = Y + (u64)(X.K + i) * N + (u64)row * C;
        u64 *spec = Spec + (u64)i * N + (u64)row * C;
#pragma unroll(LL > 0 ? 8 : 1)
        for (u32 rd = 0; rd < nr; rd++) {
            const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
            const bool first = rd == 0, last = rd == nr - 1;
#define PA_ROW_FWD(NSV)                                                                       \
    do {                                                                                      \
        if (last)                                                                             \
            row_fwd_round<NSV, ACC, MODE, true, LL>(X, xrow, arow, smx, sma, spec, s0, first, acc);  \
        else                                                                                      \
            row_fwd_round<NSV, ACC, MODE, false, LL>(X, xrow, arow, smx, sma, spec, s0, first, acc); \
    } while (0)
            PA_DISPATCH_NS(ns, PA_ROW_FWD);
#undef PA_ROW_FWD
            __syncthreads();
        }
    }
    if (MODE == ROW_STORE) return;
    u64 *Srow = S + (u64)row * C;
#pragma unroll(LL > 0 ? 8 : 1)
    for (int rd = (int)nr - 1; rd >= 0; rd--) {
        const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
        const bool from_acc = rd == (int)nr - 1, to_global = rd == 0;
#define PA_ROW_INV(NSV)                                                        \
    do {                                                                       \
        if (from_acc)                                                          \
            row_inv_round<NSV, ACC, true, LL>(X, smx, Srow, row, s0, to_global, acc);  \
        else                                                                       \
            row_inv_round<NSV, ACC, false, LL>(X, smx, Srow, row, s0, to_global, acc); \
    } while (0)
        PA_DISPATCH_NS(ns, PA_ROW_INV);
#undef PA_ROW_INV
        __syncthreads();
    }
    pdl_trigger();
}

// ------------------------------------------------------ inverse columns --

template <int NS, bool LASTSTAGE, bool TOGLOBAL, bool HO, int LL, int TC>
__device__ __forceinline__ void inv_col_round(const Xform &X, const u64 *__restrict__ Sg, u64 *__restrict__ sm,
                                              u64 *__restrict__ Z, u32 c0, u32 s0,
                                              const u64 *__restrict__ add_src, u64 add_base, u64 add_len) {
    const u32 l = LL ? (u32)LL : X.logR, tc = TC ? (u32)TC : X.tc;
    const u32 sh = l - s0 - NS, stride = 1u << sh;
    const u32 ntask = ((1u << l) >> NS) * tc;
    const u32 logtc = TC ? (u32)__builtin_ctz(TC) : (u32)(__ffs(tc) - 1);
    for (u32 task = threadIdx.x; task < ntask; task += blockDim.x) {
        const u32 c = task & (tc - 1), g = task >> logtc;
        const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
        u64 v[8];
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            const u32 r = base + m * stride;
            v[m] = LASTSTAGE ? __ldg(Sg + (u64)r * X.C + c0 + c) : sm[pidx(r * tc + c)];
        }
        dit_regs<NS, LASTSTAGE, HO>(v, s0, lo, stride, X.itwR);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            const u32 r = base + m * stride;
            if (HO && m >= (1 << (NS - 1))) continue;  // rows >= R/2 hold bits >= gamma: unused
            if (TOGLOBAL) {
                const u64 j = (u64)r * X.C + c0 + c;
                const u64 e = (0ULL - X.G * j) & (X.N - 1);
                u64 z = gd_canon(gd_mul(v[m], tbl2(X.iwt_lo, X.iwt_hi, e, X.hb)));
                if (add_src) {
                    const u64 slo = digit_start(X.G, j, X.N, X.logN);
                    u64 shi = digit_start(X.G, j + 1, X.N, X.logN);
                    if (shi > add_len) shi = add_len;
                    if (slo < shi) z += read_bits(add_src, add_base + slo, (u32)(shi - slo));
                }
                Z[j] = z;
            } else {
                sm[pidx(r * tc + c)] = v[m];
            }
        }
    }
}

template <int LL, int TC>
__global__ void __launch_bounds__(PA_COL_T) k_inv_col(Xform X, const u64 *__restrict__ Sg, u64 *__restrict__ Z,
                                                      const u64 *__restrict__ add_src, u64 add_base, u64 add_len) {
    pdl_wait();
    extern __shared__ u64 sm[];
    const u32 tc = TC ? (u32)TC : X.tc, c0 = blockIdx.x * tc;
    const u32 l = LL ? (u32)LL : X.logR;
    if (l == 0) {
        for (u32 c = threadIdx.x; c < tc; c += blockDim.x) {
            const u64 j = c0 + c;
            const u64 e = (0ULL - X.G * j) & (X.N - 1);
            u64 z = gd_canon(gd_mul(Sg[j], tbl2(X.iwt_lo, X.iwt_hi, e, X.hb)));
            if (add_src) {
                const u64 slo = digit_start(X.G, j, X.N, X.logN);
                u64 shi = digit_start(X.G, j + 1, X.N, X.logN);
                if (shi > add_len) shi = add_len;
                if (slo < shi) z += read_bits(add_src, add_base + slo, (u32)(shi - slo));
            }
            Z[j] = z;
        }
        return;
    }
    const u32 nr = (l + 2) / 3;
    // Eq. 4 stage: only t mod 2^gamma is needed, i.e. digits j < N/2 (rows < R/2)
    const bool ho = X.stage == 1;
#pragma unroll(LL > 0 ? 8 : 1)
    for (int rd = (int)nr - 1; rd >= 0; rd--) {
        const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
        const bool first = rd == (int)nr - 1, last = rd == 0;
#define PA_INV_COL(NSV)                                                                       \
    do {                                                                                      \
        if (last && ho && first)                                                              \
            inv_col_round<NSV, true, true, true, LL, TC>(X, Sg, sm, Z, c0, s0, add_src, add_base, add_len); \
        else if (last && ho)                                                                  \
            inv_col_round<NSV, false, true, true, LL, TC>(X, Sg, sm, Z, c0, s0, add_src, add_base, add_len); \
        else if (first && last)                                                               \
            inv_col_round<NSV, true, true, false, LL, TC>(X, Sg, sm, Z, c0, s0, add_src, add_base, add_len);   \
        else if (first)                                                                       \
            inv_col_round<NSV, true, false, false, LL, TC>(X, Sg, sm, Z, c0, s0, add_src, add_base, add_len);  \
        else if (last)                                                                        \
            inv_col_round<NSV, false, true, false, LL, TC>(X, Sg, sm, Z, c0, s0, add_src, add_base, add_len);  \
        else                                                                                  \
            inv_col_round<NSV, false, false, false, LL, TC>(X, Sg, sm, Z, c0, s0, add_src, add_base, add_len); \
    } while (0)
        PA_DISPATCH_NS(ns, PA_INV_COL);
#undef PA_INV_COL
        __syncthreads();
    }
    pdl_trigger();
}

// ---------------------------------------------------------------- carry --
//
// Digits z_j (< 2^64) at bit offsets s_j = ceil(G j / N) represent
// V = sum_j z_j 2^(s_j); the result is V mod (2^G - 1) as G packed bits, with
// the carry out of bit G-1 wrapping to bit 0 (2^G == 1).  Thread t owns the
// 16-digit chunk t.  Phase A: chunk carry-outs H_t with zero carry-in, then
// the chunk's bits with carry-in H_{t-1}; the 1-bit carry that adding H_{t-1}
// may still produce is summarised as generate / propagate.  Phase B: one warp
// resolves the CTA-level generate/propagate chain around the ring.  Phase C:
// every chunk receiving a carry increments its bit range.

__device__ __forceinline__ u64 cd_start(const CarryDev &cd, u64 j) {
    if (cd.ub) {
        const u64 s = j * cd.ub;
        return s < cd.G ? s : cd.G;
    }
    return digit_start(cd.G, j, cd.N, cd.logN);
}

__device__ __forceinline__ u32 digit_bits(const CarryDev &cd, u64 j) { return (u32)(cd_start(cd, j + 1) - cd_start(cd, j)); }

__device__ __forceinline__ u64 chunk_carry_out(const CarryDev &cd, const u64 *__restrict__ z, u64 t) {
    const u64 j0 = t * PA_CARRY_D;
    unsigned __int128 acc = 0;
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) {
        acc += __ldg(z + j0 + d);
        acc >>= digit_bits(cd, j0 + d);
    }
    return (u64)acc;
}

__global__ void __launch_bounds__(PA_CARRY_T) k_carry_a(CarryDev cd, const u64 *__restrict__ z, u64 *__restrict__ y) {
    pdl_wait();
    __shared__ u64 Hs[PA_CARRY_T];
    __shared__ u64 Hprev;
    __shared__ unsigned wg[PA_CARRY_T / 32], wp[PA_CARRY_T / 32];
    const u64 t = (u64)blockIdx.x * PA_CARRY_T + threadIdx.x;
    const bool act = t < cd.nchunks;  // the last CTA may hold fewer chunks; the rest propagate
    const u64 j0 = act ? t * PA_CARRY_D : 0;
    u64 zz[PA_CARRY_D];
    u32 bd[PA_CARRY_D];
    const ulonglong2 *z2 = reinterpret_cast<const ulonglong2 *>(z + j0);  // j0 is a multiple of 8
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D / 2; d++) {
        const ulonglong2 w = __ldg(z2 + d);
        zz[2 * d] = w.x;
        zz[2 * d + 1] = w.y;
    }
    u64 s = cd_start(cd, j0);
    const u64 s_begin = s;
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) {
        const u64 s1 = cd_start(cd, j0 + d + 1);
        bd[d] = (u32)(s1 - s);
        s = s1;
    }
    unsigned __int128 acc = 0;
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) {
        acc += zz[d];
        acc >>= bd[d];
    }
    const u64 Ht = (u64)acc;
    Hs[threadIdx.x] = Ht;
    if (threadIdx.x == 0)
        Hprev = t ? chunk_carry_out(cd, z, t - 1) : (cd.linear ? 0 : chunk_carry_out(cd, z, cd.nchunks - 1));
    __syncthreads();
    const u64 Hin = threadIdx.x ? Hs[threadIdx.x - 1] : Hprev;

    acc = Hin;
    bool ones = true;
    u64 wi = s_begin >> 6, wv = 0;
    u32 bo = (u32)(s_begin & 63);
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) {
        acc += zz[d];
        const u64 mask = (1ULL << bd[d]) - 1;
        const u64 bits = (u64)acc & mask;
        ones = ones && (bits == mask);
        acc >>= bd[d];
        wv |= bits << bo;
        const u32 nb = bo + bd[d];
        if (nb >= 64) {
            if (act) atomicOr(y + wi, wv);
            wi++;
            wv = (nb > 64) ? (bits >> (64 - bo)) : 0;
            bo = nb - 64;
        } else {
            bo = nb;
        }
    }
    if (bo && act) atomicOr(y + wi, wv);
    const bool g = act && (u64)acc != Ht;  // acc == H_t + (carry from adding H_{t-1})
    const bool p = !act || (!g && ones);
    if (act) cd.state[t] = (unsigned char)((g ? 1 : 0) | (p ? 2 : 0));

    const unsigned gm = __ballot_sync(0xFFFFFFFFu, g), pm = __ballot_sync(0xFFFFFFFFu, p);
    if ((threadIdx.x & 31) == 0) {
        wg[threadIdx.x >> 5] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wp[threadIdx.x >> 5] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned G = 0, P = 1;
        for (u32 w = 0; w < PA_CARRY_T / 32; w++) {
            G = wg[w] | (wp[w] & G);
            P = wp[w] & P;
        }
        cd.cta_state[blockIdx.x] = (unsigned char)(G | (P << 1));
    }
}

// Carry into every CTA range, closed around the ring: each of 1024 threads
// folds a run of CTA states, a two-level ballot scan gives every run its
// carry-in, and each thread walks its run.  The carry out of the top (with no
// carry in) wraps to bit 0; if every range propagates, the value is all ones
// and no carry is taken.
__global__ void __launch_bounds__(1024) k_carry_b(CarryDev cd, u32 nctas) {
    pdl_wait();
    __shared__ unsigned wG[32], wP[32], wcin[32];
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 per = (nctas + 1023) / 1024;
    const u32 b0 = min(tid * per, nctas), b1 = min(b0 + per, nctas);
    unsigned G = 0, P = 1;
    for (u32 b = b0; b < b1; b++) {
        const unsigned st = cd.cta_state[b];
        G = (st & 1) | (((st >> 1) & 1) & G);
        P = ((st >> 1) & 1) & P;
    }
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, G), pm = __ballot_sync(0xFFFFFFFFu, P);
    if (lane == 0) {
        wG[warp] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wP[warp] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned g2 = __ballot_sync(0xFFFFFFFFu, wG[lane]), p2 = __ballot_sync(0xFFFFFFFFu, wP[lane]);
        const u64 a = g2 | p2;
        const unsigned ewrap = cd.linear ? 0u : (unsigned)((a + g2) >> 32);
        const u64 sum = a + g2 + ewrap;
        wcin[lane] = (unsigned)(((sum ^ a ^ g2) >> lane) & 1);
        if (lane == 0) *cd.allones = 1;
    }
    __syncthreads();
    const u64 a = gm | pm, sum = a + gm + wcin[warp];
    unsigned c = (unsigned)(((sum ^ a ^ gm) >> lane) & 1);
    for (u32 b = b0; b < b1; b++) {
        cd.cta_cin[b] = (unsigned char)c;
        const unsigned st = cd.cta_state[b];
        c = (st & 1) | (((st >> 1) & 1) & c);
    }
}

__global__ void __launch_bounds__(PA_CARRY_T) k_carry_c(CarryDev cd, u64 *__restrict__ y) {
    pdl_wait();
    __shared__ unsigned wg[PA_CARRY_T / 32], wp[PA_CARRY_T / 32];
    const u64 t = (u64)blockIdx.x * PA_CARRY_T + threadIdx.x;
    const bool act = t < cd.nchunks;
    const unsigned st = act ? cd.state[t] : 2u;
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, st & 1), pm = __ballot_sync(0xFFFFFFFFu, (st >> 1) & 1);
    const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wg[warp] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wp[warp] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    unsigned cw = cd.cta_cin[blockIdx.x];
    for (u32 w = 0; w < warp; w++) cw = wg[w] | (wp[w] & cw);
    const u64 a = gm | pm, sum = a + gm + cw;
    const bool e = ((sum ^ a ^ gm) >> lane) & 1;

    const u64 j0 = t * PA_CARRY_D;
    const u64 s_lo = act ? cd_start(cd, j0) : 0;
    const u64 s_hi = act ? cd_start(cd, j0 + PA_CARRY_D) : 0;
    bool fin_ones = true, flipping = e;
    for (u64 wi = s_lo >> 6; (wi << 6) < s_hi; wi++) {
        const u64 wb = wi << 6;
        u64 m = ~0ULL;
        if (s_lo > wb) m &= ~0ULL << (s_lo - wb);
        if (s_hi < wb + 64) m &= (1ULL << (s_hi - wb)) - 1;
        const u64 orig = y[wi] & m;
        u64 flip = 0;
        if (flipping) {
            const u64 zeros = ~orig & m;
            if (zeros) {
                const u32 pos = __ffsll((long long)zeros) - 1;
                flip = m & ((2ULL << pos) - 1);
                flipping = false;
            } else {
                flip = m;
            }
            atomicXor(y + wi, flip);
        }
        fin_ones = fin_ones && (((orig ^ flip) & m) == m);
    }
    const int all = __syncthreads_and(fin_ones ? 1 : 0);
    if (threadIdx.x == 0 && !all) *cd.allones = 0;
}

// Small digit vectors: one CTA.  Thread t < runs owns the digits
// [t D, (t + 1) D) (the top thread also the rest up to ndigits); the host
// chooses D so that every run spans >= 64 bits.  Pass 1: each run's carry-out
// H_t with zero carry-in.  Pass 2: run t with carry-in H_{t-1} (H of the top
// run around the ring, 0 when linear) leaves a 1-bit carry at most (H < 2^64
// <= 2^width), summarised as generate / propagate; a two-level ballot scan
// gives every run its 1-bit carry-in (end-around for the ring).  Pass 3: each
// run writes its bits with carry-in H_{t-1} + c_t.  runs == 1 (values of a
// few dozen bits): thread 0 folds the carry around the ring until it is 0.
__device__ __forceinline__ void run_bits(const CarryDev &cd, const u64 *__restrict__ z, u64 j0, u64 j1,
                                         unsigned __int128 cin, bool write, u64 *__restrict__ y, u64 *cout,
                                         bool *ones) {
    unsigned __int128 acc = cin;
    bool all = true;
    u64 s = cd_start(cd, j0);
    u64 wi = s >> 6, wv = 0;
    u32 bo = (u32)(s & 63);
    for (u64 j = j0; j < j1; j++) {
        const u64 s1 = cd_start(cd, j + 1);
        const u32 bd = (u32)(s1 - s);
        s = s1;
        acc += __ldg(z + j);
        if (bd == 0) continue;
        const u64 mask = bd >= 64 ? ~0ULL : (1ULL << bd) - 1;
        const u64 bits = (u64)acc & mask;
        all = all && (bits == mask);
        acc >>= bd;
        if (write) {
            wv |= bits << bo;
            const u32 nb = bo + bd;
            if (nb >= 64) {
                atomicOr(y + wi, wv);
                wi++;
                wv = (nb > 64) ? (bits >> (64 - bo)) : 0;
                bo = nb - 64;
            } else {
                bo = nb;
            }
        }
    }
    if (write && bo) atomicOr(y + wi, wv);
    *cout = (u64)acc;
    *ones = all;
}

__global__ void __launch_bounds__(1024) k_carry_one(CarryDev cd, u64 ndigits, u64 D, u32 runs, const u64 *__restrict__ z,
                                                    u64 *__restrict__ y) {
    pdl_wait();
    __shared__ u64 Hs[1024];
    __shared__ unsigned wG[32], wP[32], wcin[32];
    const u32 t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool act = t < runs;
    const u64 j0 = act ? (u64)t * D : 0, j1 = act ? (t + 1 == runs ? ndigits : j0 + D) : 0;
    if (runs == 1) {
        if (t != 0) return;
        // the ring value is low(V + c) for the fixed point c = carry-out(V + c)
        // (then V = low + c (2^G - 1)); c grows monotonically from 0 and each
        // step shrinks the remaining difference by 2^width, so it settles fast
        u64 c = 0, h = 0;
        bool ones = true;
        for (int pass = 0; pass < 80 && !cd.linear; pass++) {
            run_bits(cd, z, 0, ndigits, c, false, y, &h, &ones);
            if (h == c) break;
            c = h;
        }
        run_bits(cd, z, 0, ndigits, c, true, y, &h, &ones);
        *cd.allones = ones ? 1 : 0;
        return;
    }
    u64 H = 0;
    bool ones = true;
    if (act) run_bits(cd, z, j0, j1, 0, false, y, &H, &ones);
    Hs[t] = H;
    __syncthreads();
    const u64 Hin = !act ? 0 : (t ? Hs[t - 1] : (cd.linear ? 0 : Hs[runs - 1]));
    u64 out = 0;
    bool g = false, p = true;
    if (act) {
        run_bits(cd, z, j0, j1, Hin, false, y, &out, &ones);
        g = out != H;  // out == H_t + (carry out of adding H_{t-1})
        p = !g && ones;
    }
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, g), pm = __ballot_sync(0xFFFFFFFFu, p);
    if (lane == 0) {
        wG[warp] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wP[warp] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned g2 = __ballot_sync(0xFFFFFFFFu, wG[lane]), p2 = __ballot_sync(0xFFFFFFFFu, wP[lane]);
        const u64 a = g2 | p2;
        const unsigned ewrap = cd.linear ? 0u : (unsigned)((a + g2) >> 32);
        const u64 sum = a + g2 + ewrap;
        wcin[lane] = (unsigned)(((sum ^ a ^ g2) >> lane) & 1);
    }
    __syncthreads();
    const u64 a = gm | pm, sum = a + gm + wcin[warp];
    const unsigned c = (unsigned)(((sum ^ a ^ gm) >> lane) & 1);
    bool fin = true;
    if (act) run_bits(cd, z, j0, j1, (unsigned __int128)Hin + c, true, y, &out, &fin);
    const int all = __syncthreads_and(fin ? 1 : 0);
    if (t == 0) *cd.allones = all;
}

// -------------------------------------------------------------- extract --

// Eq. 4: out = bits [gamma - r, gamma) of t = b*y + c; zero on reload.
__global__ void k_extract(const u64 *__restrict__ t, u64 gamma, u64 r, const int *__restrict__ reload,
                          u64 *__restrict__ out, int *status) {
    pdl_wait();
    const u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 nw = (r + 63) >> 6;
    const bool rl = *reload != 0;
    if (w < nw) {
        u64 v = 0;
        if (!rl) {
            const u64 lo = gamma - r + (w << 6);
            const u64 hi = (lo + 64 < gamma) ? lo + 64 : gamma;
            const u32 nb = (u32)(hi - lo);  // 1..64
            const u64 wi = lo >> 6;
            const u32 sh = (u32)(lo & 63);
            v = __ldg(t + wi) >> sh;
            if (sh != 0 && sh + nb > 64) v |= __ldg(t + wi + 1) << (64 - sh);
            if (nb < 64) v &= (1ULL << nb) - 1;
        }
        out[w] = v;
    }
    if (w == 0 && status) *status = rl ? 1 : 0;
}

__global__ void k_canonical_zero(const int *__restrict__ flag, u64 *__restrict__ y, u64 words) {
    pdl_wait();
    if (*flag == 0) return;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (u64)gridDim.x * blockDim.x) y[i] = 0;
}

// Element-wise F_q arithmetic of the transforms, for host-side checking:
// out[4i] = a+b, out[4i+1] = a-b, out[4i+2] = a*b, out[4i+3] = (a mod 2^32)*b
// (canonical); any 64-bit inputs.
__global__ void k_selftest_field(const u64 *__restrict__ a, const u64 *__restrict__ b, u64 *__restrict__ out, u64 n) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        out[4 * i] = gd_canon(gd_add(a[i], b[i]));
        out[4 * i + 1] = gd_canon(gd_sub(a[i], b[i]));
        out[4 * i + 2] = gd_canon(gd_mul(a[i], b[i]));
        out[4 * i + 3] = gd_canon(gd_mul_small((u32)a[i], b[i]));
    }
}

// coltw[r C + c] = omega_N^(c bitrev_R(r)) * theta^((-G c) mod N), canonical.
__global__ void k_fill_coltw(Xform X, u64 *__restrict__ out) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < X.N; i += (u64)gridDim.x * blockDim.x) {
        const u32 r = (u32)(i >> X.logC), c = (u32)(i & (X.C - 1));
        const u64 e = (u64)c * bitrev(r, X.logR);
        const u64 alpha = (0ULL - X.G * (u64)c) & (X.N - 1);
        out[i] = gd_canon(gd_mul(tbl2(X.ipw_lo, X.ipw_hi, e, X.hb), tbl2(X.wt_lo, X.wt_hi, alpha, X.hb)));
    }
}

int launch_fill_coltw(const Xform &X, u64 *coltw, void *stream) {
    k_fill_coltw<<<256, 256, 0, (cudaStream_t)stream>>>(X, coltw);
    return (int)cudaGetLastError();
}

int launch_selftest_field(const u64 *a, const u64 *b, u64 *out, u64 n, void *stream) {
    k_selftest_field<<<64, 256, 0, (cudaStream_t)stream>>>(a, b, out, n);
    return (int)cudaGetLastError();
}

// -------------------------------------------------------------- launchers --

static inline u32 pidx_host(u32 i) { return i + (i >> 4); }


static size_t col_smem(const Xform &X) { return (size_t)pidx_host(X.R * X.tc) * sizeof(u64); }
static size_t row_smem(const Xform &X) { return (size_t)2 * pidx_host(X.C) * sizeof(u64); }

// Instantiations with compile-time geometry for the production shapes (the
// default split of 2^20 .. 2^24 transforms); everything else uses LL = TC = 0.
#define PA_FOR_COL_SHAPES(F) F(0, 0) F(10, 4) F(11, 2)
#define PA_FOR_ROW_SHAPES8(F) F(0) F(10) F(11) F(12)
#define PA_FOR_ROW_SHAPES16(F) F(0) F(13)

int prepare_kernels() {
    // kernel attributes are per device: set them once on each device used
    static std::atomic<unsigned long long> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
    const unsigned long long bit = dev < 64 ? 1ULL << dev : 0;  // devices >= 64: set every time
    if (done_mask.load() & bit) return 0;
    cudaError_t e;
    const int big = 200 * 1024;
#define PA_ATTR_COL(LLV, TCV)                                                                                   \
    if ((e = cudaFuncSetAttribute(k_fwd_col<true, LLV, TCV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
        return e;                                                                                               \
    if ((e = cudaFuncSetAttribute(k_fwd_col<false, LLV, TCV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
        return e;                                                                                               \
    if ((e = cudaFuncSetAttribute(k_inv_col<LLV, TCV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    PA_FOR_COL_SHAPES(PA_ATTR_COL)
#undef PA_ATTR_COL
#define PA_ATTR_ROW(A, LLV)                                                                                          \
    if ((e = cudaFuncSetAttribute(k_row_mac<A, ROW_PAIRS, LLV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))    \
        return e;                                                                                                    \
    if ((e = cudaFuncSetAttribute(k_row_mac<A, ROW_STORE, LLV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))    \
        return e;                                                                                                    \
    if ((e = cudaFuncSetAttribute(k_row_mac<A, ROW_PREPARED, LLV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
        return e;
#define PA_ATTR_ROW8(LLV) PA_ATTR_ROW(8, LLV)
#define PA_ATTR_ROW16(LLV) PA_ATTR_ROW(16, LLV)
    PA_FOR_ROW_SHAPES8(PA_ATTR_ROW8)
    PA_FOR_ROW_SHAPES16(PA_ATTR_ROW16)
#undef PA_ATTR_ROW8
#undef PA_ATTR_ROW16
#undef PA_ATTR_ROW
    done_mask.fetch_or(bit);
    return 0;
}

template <bool PAIR>
static int launch_cols(const char *name, const Xform &X, const Operands &S, int count, u64 *Y, void *stream) {
    if (int e = prepare_kernels()) return e;
    dim3 grid(X.C / X.tc, count);
    const size_t smem = (PAIR ? 2 : 1) * col_smem(X);
    cudaStream_t s = (cudaStream_t)stream;
#define PA_LAUNCH_COL(LLV, TCV)                                                                \
    if ((LLV == 0 && TCV == 0) || (X.logR == (u32)LLV && X.tc == (u32)TCV)) {                  \
        TRACED(name, X.stage, stream, (launch_pdl(k_fwd_col<PAIR, LLV, TCV>, grid, dim3(PA_COL_T), smem, s, X, S, Y))); \
        return (int)cudaGetLastError();                                                        \
    }
    PA_LAUNCH_COL(10, 4)
    PA_LAUNCH_COL(11, 2)
    PA_LAUNCH_COL(0, 0)
#undef PA_LAUNCH_COL
    return (int)cudaErrorInvalidValue;
}

int launch_fwd_col(const Xform &X, const Operands &S, int num_pairs, u64 *Y, void *stream) {
    return launch_cols<true>("fwd_col", X, S, num_pairs, Y, stream);
}

int launch_fwd_col_single(const Xform &X, const Operands &S, int num_operands, u64 *Y, void *stream) {
    return launch_cols<false>("fwd_col1", X, S, num_operands, Y, stream);
}

template <int MODE>
static int launch_rows(const char *name, const Xform &X, const u64 *Y, u64 *Spec, u64 *S, void *stream) {
    if (int e = prepare_kernels()) return e;
    cudaStream_t s = (cudaStream_t)stream;
    if (X.C > 4096) {
        if (X.logC == 13)
            TRACED(name, X.stage, stream, (launch_pdl(k_row_mac<16, MODE, 13>, dim3(X.R), dim3(X.C / 16), row_smem(X), s, X, Y, Spec, S)));
        else
            TRACED(name, X.stage, stream, (launch_pdl(k_row_mac<16, MODE, 0>, dim3(X.R), dim3(X.C / 16), row_smem(X), s, X, Y, Spec, S)));
    } else {
        u32 threads = X.C / 8;
        if (threads < 32) threads = 32;
        if (X.logC == 11)
            TRACED(name, X.stage, stream, (launch_pdl(k_row_mac<8, MODE, 11>, dim3(X.R), dim3(threads), row_smem(X), s, X, Y, Spec, S)));
        else if (X.logC == 12)
            TRACED(name, X.stage, stream, (launch_pdl(k_row_mac<8, MODE, 12>, dim3(X.R), dim3(threads), row_smem(X), s, X, Y, Spec, S)));
        else if (X.logC == 10)
            TRACED(name, X.stage, stream, (launch_pdl(k_row_mac<8, MODE, 10>, dim3(X.R), dim3(threads), row_smem(X), s, X, Y, Spec, S)));
        else
            TRACED(name, X.stage, stream, (launch_pdl(k_row_mac<8, MODE, 0>, dim3(X.R), dim3(threads), row_smem(X), s, X, Y, Spec, S)));
    }
    return (int)cudaGetLastError();
}

int launch_row_mac(const Xform &X, const u64 *Y, u64 *S, void *stream) {
    return launch_rows<ROW_PAIRS>("row_mac", X, Y, nullptr, S, stream);
}

int launch_row_store(const Xform &X, const u64 *Y, u64 *Spec, void *stream) {
    return launch_rows<ROW_STORE>("row_store", X, Y, Spec, nullptr, stream);
}

int launch_row_prepared(const Xform &X, const u64 *Y, const u64 *Spec, u64 *S, void *stream) {
    return launch_rows<ROW_PREPARED>("row_prep", X, Y, const_cast<u64 *>(Spec), S, stream);
}

int launch_inv_col(const Xform &X, const u64 *S, u64 *Z, const u64 *add_src, u64 add_base, u64 add_len,
                   void *stream) {
    if (int e = prepare_kernels()) return e;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid(X.C / X.tc);
#define PA_LAUNCH_INV(LLV, TCV)                                                                          \
    if ((LLV == 0 && TCV == 0) || (X.logR == (u32)LLV && X.tc == (u32)TCV)) {                            \
        TRACED("inv_col", X.stage, stream,                                                               \
               (launch_pdl(k_inv_col<LLV, TCV>, grid, dim3(PA_COL_T), col_smem(X), s, X, S, Z, add_src, add_base, add_len))); \
        return (int)cudaGetLastError();                                                                  \
    }
    PA_LAUNCH_INV(10, 4)
    PA_LAUNCH_INV(11, 2)
    PA_LAUNCH_INV(0, 0)
#undef PA_LAUNCH_INV
    return (int)cudaErrorInvalidValue;
}

// Runs of the one-CTA carry: D digits per run (the top run takes the rest),
// every run >= 64 bits wide so that a carry-in below 2^64 leaves a 1-bit
// carry; a single run when the value is too short for two.
void carry_runs(const CarryDev &cd, u64 ndigits, u64 *D_out, u32 *runs_out) {
    auto start = [&](u64 j) -> u64 {
        if (cd.ub) {
            const u64 s = j * cd.ub;
            return s < cd.G ? s : cd.G;
        }
        return (cd.G * j + cd.N - 1) >> cd.logN;
    };
    // narrowest run of D interior digits: D ub bits, or floor(D G / N) - 1
    u64 D = cd.ub ? (64 + cd.ub - 1) / cd.ub : (65 * cd.N + cd.G - 1) / cd.G + 1;
    D = std::max<u64>(D, (ndigits + 1023) / 1024);
    u64 runs = ndigits ? (ndigits + D - 1) / D : 1;
    while (runs > 1 && start(ndigits) - start((runs - 1) * D) < 64) runs--;
    *D_out = D;
    *runs_out = (u32)std::max<u64>(runs, 1);
}

int launch_carry_chunks(const CarryDev &cd, u64 ndigits, bool wide_chunks, u32 stage, u64 *z, u64 *out_bits,
                        u64 out_words, void *stream, bool zeroed, bool pdl) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!zeroed) {
        cudaError_t e = cudaMemsetAsync(out_bits, 0, out_words * sizeof(u64), s);
        if (e) return e;
    }
    // chunks of PA_CARRY_D digits must span >= 64 bits so that adding the
    // previous chunk's carry-out leaves a 1-bit carry
    const bool parallel = cd.nchunks >= PA_CARRY_T && wide_chunks;
    if (!parallel) {
        u64 D = 0;
        u32 runs = 0;
        carry_runs(cd, ndigits, &D, &runs);
        if (pdl)
            TRACED("carry_one", stage, stream,
                   (launch_pdl(k_carry_one, dim3(1), dim3(1024), 0, s, cd, ndigits, D, runs, (const u64 *)z, out_bits)));
        else
            TRACED("carry_one", stage, stream, (k_carry_one<<<1, 1024, 0, s>>>(cd, ndigits, D, runs, z, out_bits)));
        return (int)cudaGetLastError();
    }
    const u32 nctas = (u32)((cd.nchunks + PA_CARRY_T - 1) / PA_CARRY_T);
    if (pdl) {
        TRACED("carry_a", stage, stream, (launch_pdl(k_carry_a, dim3(nctas), dim3(PA_CARRY_T), 0, s, cd, (const u64 *)z, out_bits)));
        TRACED("carry_b", stage, stream, (launch_pdl(k_carry_b, dim3(1), dim3(1024), 0, s, cd, nctas)));
        TRACED("carry_c", stage, stream, (launch_pdl(k_carry_c, dim3(nctas), dim3(PA_CARRY_T), 0, s, cd, out_bits)));
    } else {
        TRACED("carry_a", stage, stream, (k_carry_a<<<nctas, PA_CARRY_T, 0, s>>>(cd, z, out_bits)));
        TRACED("carry_b", stage, stream, (k_carry_b<<<1, 1024, 0, s>>>(cd, nctas)));
        TRACED("carry_c", stage, stream, (k_carry_c<<<nctas, PA_CARRY_T, 0, s>>>(cd, out_bits)));
    }
    return (int)cudaGetLastError();
}

int launch_carry(const Xform &X, const CarryDev &cd_in, u64 *z, u64 *out_bits, u64 out_words, void *stream) {
    // MH stage: only digits [0, N/2) hold bits below gamma; resolve them linearly
    CarryDev cd = cd_in;
    cd.ub = 0;
    const u64 ndigits = (X.stage == 1 && X.N >= 2) ? X.N / 2 : X.N;
    cd.linear = (X.stage == 1 && X.N >= 2) ? 1 : 0;
    cd.nchunks = ndigits / PA_CARRY_D;
    return launch_carry_chunks(cd, ndigits, (X.G >> X.logN) * PA_CARRY_D >= 64, X.stage, z, out_bits, out_words, stream);
}

int launch_extract(const u64 *t, u64 gamma, u64 r, const int *reload, u64 k, u64 *out, int *status, void *stream,
                   bool pdl) {
    (void)k;
    const u64 nw = (r + 63) >> 6;
    const u32 threads = 256;
    const u64 blocks = (nw + threads - 1) / threads;
    if (pdl)
        TRACED("extract", 1, stream,
               (launch_pdl(k_extract, dim3((unsigned)blocks), dim3(threads), 0, (cudaStream_t)stream, t, gamma, r,
                           reload, out, status)));
    else
        TRACED("extract", 1, stream, (k_extract<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(t, gamma, r, reload, out, status)));
    return (int)cudaGetLastError();
}

int launch_canonical_zero(const int *flag, u64 *y, u64 words, void *stream, bool pdl) {
    if (pdl)
        TRACED("canonical_zero", 0, stream,
               (launch_pdl(k_canonical_zero, dim3(64), dim3(256), 0, (cudaStream_t)stream, flag, y, words)));
    else
        TRACED("canonical_zero", 0, stream, (k_canonical_zero<<<64, 256, 0, (cudaStream_t)stream>>>(flag, y, words)));
    return (int)cudaGetLastError();
}

}  // namespace pa
