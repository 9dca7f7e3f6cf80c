// pa_p3.cu -- the three-prime backend: Eq. 2 and Eq. 4 as exact linear
// convolutions over three 30-bit NTT primes, recombined by the Chinese
// remainder theorem.
//
// Each operand (a gamma-bit integer) is cut into M = T/2 digits of b bits at
// bit offsets t*b; the upper half of every length-T transform is zero, so the
// cyclic convolution of two digit vectors is their linear convolution.  A
// coefficient S_e = sum_i sum_{u+v=e} x_{i,u} a_{i,v} is below
// K M (2^b - 1)^2 < p0 p1 p2, so its three residues determine it exactly
// (Garner's algorithm).  The Mersenne reduction of Eq. 2 then places bit
// offset o at o mod gamma (2^gamma = 1 mod 2^gamma - 1); Eq. 4 keeps the
// offsets below gamma (mod 2^gamma).  The digit vector that results is
// resolved by the carry kernels of pa_kernels.cu (uniform-offset mode).
//
// Arithmetic per prime p < 2^30 (4p < 2^32): values live in [0, 2p);
// twiddles w come with w' = floor(w 2^32 / p) and x w mod p is
// x w - floor(x w' / 2^32) p in [0, 2p) (Shoup); the transform-domain
// product of two variable spectra is a Montgomery product (factor 2^-32,
// removed with the 1/T scaling before the CRT).
//
// Data layout: Y[(j * 2K + o) * T + e] (u32) holds operand o's spectrum for
// prime j, o < K the key slices x_i, o >= K the seed slices a_i (or y, b
// for Eq. 4); S3[j * T + e] the accumulated spectrum and, after the inverse
// column pass, the coefficients' residues.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "../../include/pa_gb300.h"
#include "pa_internal.h"

namespace pa {
namespace p3 {

constexpr u32 kColThreads = 256;

// ------------------------------------------------------------ device math --

__device__ __forceinline__ u32 px(u32 i) { return i + (i >> 3); }  // 1 pad word per 8
__device__ __forceinline__ u32 brev(u32 x, u32 bits) { return bits ? (__brev(x) >> (32 - bits)) : 0u; }
__device__ __forceinline__ u32 red2(u32 x, u32 p2) { return min(x, x - p2); }  // [0, 4p) -> [0, 2p)
__device__ __forceinline__ u32 canon(u32 x, u32 p) { return min(x, x - p); }   // [0, 2p) -> [0, p)
// x w mod p in [0, 2p) for any x < 2^32 (w < p, w' = floor(w 2^32 / p))
__device__ __forceinline__ u32 shoup(u32 x, uint2 w, u32 p) { return x * w.x - __umulhi(x, w.y) * p; }
// a b 2^-32 mod p in (0, 2p) for a, b < 2p: with m = lo(a b) p^-1 mod 2^32 the
// low words of a b and m p agree, so (a b - m p) / 2^32 = hi(a b) - hi(m p).
__device__ __forceinline__ u32 mont(u32 a, u32 b, u32 p, u32 pinv) {
    const u32 lo = a * b, hi = __umulhi(a, b);
    return hi - __umulhi(lo * pinv, p) + p;
}

__device__ __forceinline__ u32 rd32(const u64 *__restrict__ src, u64 pos, u32 nb) {
    const u32 *s32 = reinterpret_cast<const u32 *>(src);
    const u64 wi = pos >> 5;
    const u32 sh = (u32)(pos & 31);
    const u32 lo = __ldg(s32 + wi);
    const u32 hi = (sh + nb > 32) ? __ldg(s32 + wi + 1) : 0u;
    return __funnelshift_r(lo, hi, sh) & (nb >= 32 ? 0xFFFFFFFFu : ((1u << nb) - 1u));
}

// Round rd of a length-2^l transform: the first round takes the leftover
// 1..3 stages, every later round 3 (the final round has stride 1, lo = 0).
__device__ __forceinline__ u32 round_ns(u32 l, u32 rd) { return rd ? 3u : l - 3u * ((l + 2) / 3 - 1); }
__device__ __forceinline__ u32 round_s0(u32 l, u32 rd) { return rd ? round_ns(l, 0) + 3u * (rd - 1) : 0u; }

// Lazy reduction.  Values are kept below B p with a bound B tracked per
// element at compile time (the loops are fully unrolled, so every B folds to
// a constant); 2^H p < 2^32 is the headroom of the prime set (H = 4 for the
// primes below 2^28, 2 for those below 2^30).  A sum is formed unreduced while
// its bound fits the headroom, otherwise its inputs are first brought down by
// conditional subtractions; a difference a - b + B_b p is reduced by its Shoup
// product into [0, 2p).  OUT is the bound the caller needs at the end of the
// round (2: [0, 2p), 4: [0, 4p), 8: [0, 8p), 0: any 32-bit value, e.g. before
// a Shoup product) and IB the bound of the round's inputs.  With headroom 16p
// the radix-8 rounds hand their outputs on below 4p (forward) or 8p
// (inverse), which takes the fewest conditional subtractions over a transform.
__device__ __forceinline__ u32 csub(u32 x, u32 kp) { return min(x, x - kp); }  // x < 2 kp -> x < kp

// One conditional subtraction of floor(B/2) p: x < B p -> x < ceil(B/2) p.
__device__ __forceinline__ void halve(u32 &v, int &B, u32 p) {
    v = csub(v, (u32)(B / 2) * p);
    B -= B / 2;
}

// Bring v below bound `to` (2, 4 or 8, in units of p) from bound B <= 32.
__device__ __forceinline__ void reduce_to(u32 &v, int &B, int to, u32 p) {
#pragma unroll
    for (int it = 0; it < 5; it++)
        if (B > to) halve(v, B, p);
}

// Operands a (bound Ba), b (bound Bb) of a sum must satisfy Ba + Bb <= 2^H:
// reduce the larger bound first.
template <int H>
__device__ __forceinline__ void make_room(u32 &a, int &Ba, u32 &b, int &Bb, u32 p) {
#pragma unroll
    for (int it = 0; it < 8; it++) {
        if (Ba + Bb > (1 << H)) {
            if (Ba >= Bb)
                halve(a, Ba, p);
            else
                halve(b, Bb, p);
        }
    }
}

// Radix-2 DIF stages s0 .. s0+NS-1 of a length-L transform on the elements
// base + m*stride (lo = base mod stride); stage s pairs (i, i + L/2^(s+1))
// with twiddle omega_L^((i mod L/2^(s+1)) 2^s).  HZ: the upper half of the
// group is zero on entry.  In the final round (LAST) the twiddles of the
// pairs with i mod L/2^(s+1) = 0 are 1.  Inputs below 2p.
// rt: the task's round twiddles, stage sg's pair jj at q = 2^NS - 2^(NS-sg) + jj.
// TS: the round table is in shared memory (plain loads) rather than global (read-only path).
template <bool TS>
__device__ __forceinline__ uint2 twl(const uint2 *__restrict__ p) { return TS ? *p : __ldg(p); }

// Shared-memory twiddles of one prime in the column kernel (R = 2^10, uint2
// entries): the forward R table from round 2 on -- round 2 (56 entries),
// round 3 (7), the 4-stage first round (960) and one pad entry that the plan
// stores so that the window is 1024 entries, 512 16-byte copies -- then the
// tile's 64 split inter-pass twiddles B[c][m].
constexpr u32 kColTab = 1024, kColTabStride = kColTab + 64, kColTabR3 = 56, kColTab4 = 63;

// Asynchronous 16-byte global -> shared copies (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const u32 d = (u32)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int NS, bool LAST, bool HZ, bool TS = false, int H = 2, int OUT = 2, int IB = 2>
__device__ __forceinline__ void dif3(u32 (&v)[8], const uint2 *__restrict__ rt, u32 p) {
    int B[8];
#pragma unroll
    for (int m = 0; m < 8; m++) B[m] = IB;
#pragma unroll
    for (int sg = 0; sg < NS; sg++) {
        const int half = 1 << (NS - 1 - sg);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (m & half) continue;
            const int jj = m & (half - 1);
            const bool one = LAST && jj == 0;
            const int q = (1 << NS) - (1 << (NS - sg)) + jj;
            u32 a = v[m], b = v[m + half];
            if (HZ && sg == 0) {
                v[m + half] = one ? a : shoup(a, twl<TS>(rt + q), p);
                B[m + half] = one ? B[m] : 2;
                continue;
            }
            int Ba = B[m], Bb = B[m + half];
            make_room<H>(a, Ba, b, Bb, p);
            v[m] = a + b;
            const u32 d = a - b + (u32)Bb * p;
            B[m] = Ba + Bb;
            v[m + half] = one ? d : shoup(d, twl<TS>(rt + q), p);
            B[m + half] = one ? Ba + Bb : 2;
        }
    }
    if (OUT) {
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) reduce_to(v[m], B[m], OUT, p);
    }
}

// Inverse of dif3 up to a factor 2^NS (DIT, stages reversed, inverse
// twiddles in the same table layout).  HO: the upper outputs of the last
// stage are not needed.  Inputs below IB p.
template <int NS, bool LAST, bool HO, int H = 2, int OUT = 2, int IB = 2>
__device__ __forceinline__ void dit3(u32 (&v)[8], const uint2 *__restrict__ rt, u32 p) {
    int B[8];
#pragma unroll
    for (int m = 0; m < 8; m++) B[m] = IB;
#pragma unroll
    for (int sg = NS - 1; sg >= 0; sg--) {
        const int half = 1 << (NS - 1 - sg);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (m & half) continue;
            const int jj = m & (half - 1);
            const bool one = LAST && jj == 0;
            const int q = (1 << NS) - (1 << (NS - sg)) + jj;
            u32 a = v[m];
            int Ba = B[m];
            u32 t = v[m + half];
            int Bt = B[m + half];
            if (!one) {
                t = shoup(t, __ldg(rt + q), p);
                Bt = 2;
            }
            make_room<H>(a, Ba, t, Bt, p);
            v[m] = a + t;
            if (!(HO && sg == 0)) v[m + half] = a - t + (u32)Bt * p;
            B[m] = B[m + half] = Ba + Bt;
        }
    }
    if (OUT) {
#pragma unroll
        for (int m = 0; m < (1 << NS); m++)
            if (!(HO && m >= (1 << (NS - 1)))) reduce_to(v[m], B[m], OUT, p);
    }
}

// Stages 0..3 of a length-L transform on 16 elements lo + m L/16 whose upper
// 8 are zero on entry (the zero-padded half), twiddles rt[16 - 2^(4-sg) + jj]
// = omega_L^((lo + jj L/16) 2^sg); the round table is in shared memory.
// Inputs below IB p (2 or 4: raw digits of up to log2(4p) bits).
template <int H = 2, int OUT = 2, int IB = 2>
__device__ __forceinline__ void dif16_hz(u32 (&v)[16], const uint2 *__restrict__ rt, u32 p) {
    int B[16];
#pragma unroll
    for (int m = 0; m < 16; m++) B[m] = m < 8 ? IB : 2;
#pragma unroll
    for (int sg = 0; sg < 4; sg++) {
        const int half = 8 >> sg;
#pragma unroll
        for (int m = 0; m < 16; m++) {
            if (m & half) continue;
            const int q = 16 - (16 >> sg) + (m & (half - 1));
            u32 a = v[m];
            if (sg == 0) {
                v[m + half] = shoup(a, rt[q], p);  // (a, 0) -> (a, a w)
                B[m + half] = 2;
                continue;
            }
            u32 b = v[m + half];
            int Ba = B[m], Bb = B[m + half];
            make_room<H>(a, Ba, b, Bb, p);
            v[m] = a + b;
            v[m + half] = shoup(a - b + (u32)Bb * p, rt[q], p);
            B[m] = Ba + Bb;
            B[m + half] = 2;
        }
    }
    if (OUT) {
#pragma unroll
        for (int m = 0; m < 16; m++) reduce_to(v[m], B[m], OUT, p);
    }
}

// Inverse of the 4-stage round (DIT, stages 3..0, inverse twiddles in the same
// layout); HO: the upper 8 outputs are not needed.  Inputs below 2p.
template <bool HO, int H = 2, int OUT = 2>
__device__ __forceinline__ void dit16(u32 (&v)[16], const uint2 *__restrict__ rt, u32 p) {
    int B[16];
#pragma unroll
    for (int m = 0; m < 16; m++) B[m] = 2;
#pragma unroll
    for (int sg = 3; sg >= 0; sg--) {
        const int half = 8 >> sg;
#pragma unroll
        for (int m = 0; m < 16; m++) {
            if (m & half) continue;
            const int q = 16 - (16 >> sg) + (m & (half - 1));
            u32 a = v[m];
            int Ba = B[m];
            u32 t = shoup(v[m + half], __ldg(rt + q), p);
            int Bt = 2;
            make_room<H>(a, Ba, t, Bt, p);
            v[m] = a + t;
            if (!(HO && sg == 0)) v[m + half] = a - t + (u32)Bt * p;
            B[m] = B[m + half] = Ba + Bt;
        }
    }
    if (OUT) {
#pragma unroll
        for (int m = 0; m < 16; m++)
            if (!(HO && m >= 8)) reduce_to(v[m], B[m], OUT, p);
    }
}

// Shared-memory word of element i: one pad word per 8 (px(i + 8k) = px(i) + 9k,
// so elements m * d apart, d a multiple of 8, are px(i) + m * (d + d / 8)).
__device__ __forceinline__ u32 pstep(u32 d) { return d + (d >> 3); }

// Column tiles ([row][8 columns]) use 8 pad words per 64: a warp's 4 rows x 8
// columns are 32 consecutive words of one 64-word block (no conflicts), and
// the final round's 4 groups of 8 rows land in 4 different bank octets.
// Steps of 8 words stay inside a block; steps of 64k words add 72k.
__device__ __forceinline__ u32 pxc(u32 i) { return i + ((i >> 6) << 3); }
__device__ __forceinline__ u32 pstepc(u32 d) { return d >= 64 ? d + (d >> 3) : d; }

#define P3_DISPATCH_NS(ns, F) \
    do {                      \
        if ((ns) == 3)        \
            F(3);             \
        else if ((ns) == 2)   \
            F(2);             \
        else                  \
            F(1);             \
    } while (0)

// ---------------------------------------------------------------- operands --

struct Desc {
    const u64 *src;
    u64 base, len;  // operand = bits [base, base + len) of src
    int force_odd, check_ones, zero;
};

// Algorithm 1 slices: pair i of Eq. 2 is (x_{i+1}, a_{i+1}); the pair of
// Eq. 4 is (y, b) with b forced odd.  Single operands (PAIR false: seed
// preparation and prepared hashing) come in dx: mode 2 = a_{i+1}, 3 = x_{i+1},
// 4 = b, 5 = y.
template <bool PAIR>
__device__ __forceinline__ void descs(const Operands &S, u32 i, Desc &dx, Desc &da) {
    dx.force_odd = da.force_odd = 0;
    dx.check_ones = da.check_ones = 0;
    dx.zero = da.zero = 0;
    if constexpr (!PAIR) {
        da.src = S.seed;
        da.base = 0;
        da.len = 0;
        da.zero = 1;
        dx.src = S.mode == 3 ? S.key : S.mode == 5 ? S.y : S.seed;
        dx.base = S.mode == 4 ? S.k * S.gamma : S.mode == 5 ? 0 : (u64)i * S.gamma;
        dx.len = S.gamma;
        if (S.mode == 3) {
            const u64 rem = S.n - dx.base;
            dx.len = rem < S.gamma ? rem : S.gamma;
            dx.check_ones = 1;
        }
        dx.force_odd = S.mode == 4;
        dx.zero = S.mode == 5 && *S.y_zero != 0;
        return;
    }
    if (S.mode == 0) {
        dx.src = S.key;
        dx.base = (u64)i * S.gamma;
        const u64 rem = S.n - dx.base;
        dx.len = rem < S.gamma ? rem : S.gamma;
        dx.check_ones = 1;
        da.src = S.seed;
        da.base = (u64)i * S.gamma;
        da.len = S.gamma;
    } else if (S.mode == 6) {
        // Toeplitz block (blk, i): key segment i, and the 2 rb - 1 seed bits of
        // the block's diagonals, starting at n + (blk - i) rb in the shifted seed
        dx.src = S.key;
        dx.base = (u64)i * S.rb;
        const u64 rem = S.n - dx.base;
        dx.len = rem < S.rb ? rem : S.rb;
        da.src = S.seed;
        da.base = S.n + (u64)S.blk * S.rb - (u64)i * S.rb;
        const u64 avail = S.seed_bits > da.base ? S.seed_bits - da.base : 0;
        da.len = avail < 2 * S.rb - 1 ? avail : 2 * S.rb - 1;
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

// The digit at bit offset pos of the operand (b bits, fewer at the top),
// reduced into [0, 2p).
__device__ __forceinline__ u32 digit_at(const Geo3 &X, const Desc &d, u64 pos, uint2 red, u32 p, bool &ones) {
    if (d.zero || pos >= d.len) {
        if (d.check_ones && pos < X.G) ones = false;  // zero padding below gamma: not all ones
        return 0;
    }
    const u64 left = d.len - pos;
    const u32 nb = left < X.b ? (u32)left : X.b;
    u32 v = rd32(d.src, d.base + pos, nb);
    if (d.check_ones) ones = ones && (v == (nb >= 32 ? 0xFFFFFFFFu : (1u << nb) - 1u));
    if (d.force_odd && pos == 0) v |= 1u;
    return shoup(v, red, p);
}

// The raw digit at bit offset pos (b bits, fewer at the top; 0 past the operand).
__device__ __forceinline__ u32 digit_raw(const Geo3 &X, const Desc &d, u64 pos, bool &ones) {
    if (d.zero || pos >= d.len) {
        if (d.check_ones && pos < X.G) ones = false;
        return 0;
    }
    const u64 left = d.len - pos;
    const u32 nb = left < X.b ? (u32)left : X.b;
    u32 v = rd32(d.src, d.base + pos, nb);
    if (d.check_ones) ones = ones && (v == (nb >= 32 ? 0xFFFFFFFFu : (1u << nb) - 1u));
    if (d.force_odd && pos == 0) v |= 1u;
    return v;
}

// ------------------------------------------------------------ column pass --

// LL, TC: log2 R and the tile width when fixed at compile time (0: from X).
// SPLIT (the last round of k3_fwd_col_all: stride 1, R = 2^10, 512 threads):
// the inter-pass twiddle of row 8 g + m is A[g][c] -- loaded by the caller a
// round early, one per task (apre) -- times the staged sB[c][m].
template <int NS, bool PAIR, bool FIRST, bool LAST, int LL, int TC, bool TS = false, int H = 2, bool SPLIT = false,
          int RIB = 2, int ROUT = 2>
__device__ __forceinline__ void fwd3_round(const Geo3 &X, u32 j, const Desc &dx, const Desc &da, u32 *__restrict__ smx,
                                           u32 *__restrict__ sma, u32 *__restrict__ Yx, u32 *__restrict__ Ya, u32 c0,
                                           u32 s0, u32 rd, bool &ones, const uint2 *__restrict__ stw = nullptr,
                                           const uint2 *__restrict__ sB = nullptr, uint2 apre0 = uint2{},
                                           uint2 apre1 = uint2{}) {
    const u32 l = LL ? (u32)LL : X.logR, tc = TC ? (u32)TC : X.tc, p = X.p[j];
    const u32 sh = l - s0 - NS, stride = 1u << sh;
    const u32 ntask = ((1u << l) >> NS) * tc;
    const u32 logtc = TC ? (u32)__builtin_ctz(TC) : (u32)(__ffs(tc) - 1);
    const u32 dsm = pstepc(stride * tc);  // tc = 8
    const u64 dY = (u64)stride * X.C;
    const uint2 red = X.red[j];
    // shared-memory tables (TS: R = 2^10) start at round 2 of the forward R table
    const uint2 *tw = TS ? stw + (rd == 2 ? 0u : kColTabR3) : X.twR[j] + X.rofR[rd];
    for (u32 task = threadIdx.x; task < ntask; task += blockDim.x) {
        const u32 c = task & (tc - 1), g = task >> logtc;
        const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
        const u32 a0 = pxc(base * tc + c);
        const u64 e0 = (u64)base * X.C + c0 + c;
        u32 vx[8], va[8];
        uint2 ct[(LAST && !SPLIT) ? 8 : 1];
        if (LAST && SPLIT) {
            ct[0] = task >= blockDim.x ? apre1 : apre0;
        } else if (LAST) {  // inter-pass twiddles first: their L2 latency overlaps the round's arithmetic
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) ct[(LAST && !SPLIT) ? m : 0] = __ldg(X.ctw[j] + e0 + m * dY);
        }
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (FIRST && m >= (1 << (NS - 1))) {  // rows >= R/2: digit slots >= T/2 are zero
                vx[m] = 0;
                va[m] = 0;
            } else if (FIRST) {
                const u64 pos = (e0 + m * dY) * X.b;
                vx[m] = digit_at(X, dx, pos, red, p, ones);
                if (PAIR) va[m] = digit_at(X, da, pos, red, p, ones);
            } else {
                vx[m] = smx[a0 + m * dsm];
                if (PAIR) va[m] = sma[a0 + m * dsm];
            }
        }
        const uint2 *rt = tw + lo * ((1u << NS) - 1);
        // the last round's outputs go straight into Shoup products (any bound)
        dif3<NS, LAST, FIRST, TS, H, LAST ? 0 : ROUT, RIB>(vx, rt, p);
        if (PAIR) dif3<NS, LAST, FIRST, TS, H, LAST ? 0 : ROUT, RIB>(va, rt, p);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (LAST && SPLIT) {
                const u64 e = e0 + m * dY;
                // B[c][0] = 1 (bitrev(0) = 0): row 8 g takes the A factor alone
                const uint2 bm = sB[c * 8 + m];
                Yx[e] = shoup(m == 0 ? vx[m] : shoup(vx[m], bm, p), ct[0], p);
                if (PAIR) Ya[e] = shoup(m == 0 ? va[m] : shoup(va[m], bm, p), ct[0], p);
            } else if (LAST) {
                // position r holds column frequency bitrev(r): times omega_T^(c bitrev(r))
                const u64 e = e0 + m * dY;
                const uint2 t = ct[(LAST && !SPLIT) ? m : 0];
                Yx[e] = shoup(vx[m], t, p);
                if (PAIR) Ya[e] = shoup(va[m], t, p);
            } else {
                smx[a0 + m * dsm] = vx[m];
                if (PAIR) sma[a0 + m * dsm] = va[m];
            }
        }
    }
}

// grid (C / tc, pairs, 3 primes): a tile of tc columns of pair blockIdx.y + pair0.
template <bool PAIR, int LL, int TC, int H>
__global__ void __launch_bounds__(kColThreads) k3_fwd_col(Geo3 X, Operands S, u32 *__restrict__ Y) {
    pdl_wait();
    extern __shared__ u32 sm3[];
    const u32 j = blockIdx.z, tc = TC ? (u32)TC : X.tc, c0 = blockIdx.x * tc, i = blockIdx.y + S.pair0;
    Desc dx, da;
    descs<PAIR>(S, i, dx, da);
    if (j) dx.check_ones = 0;
    u32 *Yx = Y + ((u64)j * 2 * X.K + i) * X.T, *Ya = Y + ((u64)j * 2 * X.K + X.K + i) * X.T;
    u32 *smx = sm3, *sma = sm3 + pxc(X.R * tc);
    bool ones = true;
    const u32 l = LL ? (u32)LL : X.logR, nr = (l + 2) / 3;
#pragma unroll(LL > 0 ? 8 : 1)
    for (u32 rd = 0; rd < nr; rd++) {
        const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
        const bool first = rd == 0, last = rd == nr - 1;
#define P3_FWD(NSV)                                                                                   \
    do {                                                                                              \
        if (first)                                                                                    \
            fwd3_round<NSV, PAIR, true, false, LL, TC, false, H>(X, j, dx, da, smx, sma, Yx, Ya, c0, s0, rd, ones);  \
        else if (last)                                                                                \
            fwd3_round<NSV, PAIR, false, true, LL, TC, false, H>(X, j, dx, da, smx, sma, Yx, Ya, c0, s0, rd, ones);  \
        else                                                                                          \
            fwd3_round<NSV, PAIR, false, false, LL, TC, false, H>(X, j, dx, da, smx, sma, Yx, Ya, c0, s0, rd, ones); \
    } while (0)
        P3_DISPATCH_NS(ns, P3_FWD);
#undef P3_FWD
        __syncthreads();
    }
    pdl_trigger();
    if (dx.check_ones) {
        // Algorithm 1 reload rule: slice i is all ones iff every CTA of the slice saw only ones
        const int all = __syncthreads_and(ones ? 1 : 0);
        if (threadIdx.x == 0 && all) {
            int *cnt = S.reload + 4 + i;
            if (atomicAdd(cnt, 1) + 1 == (int)gridDim.x) atomicExch(S.reload, 1);
        }
    }
}

// Start the copies of prime j's twiddles into the buffer tb (512 threads).
template <int TC>
__device__ __forceinline__ void col_tables_async(const Geo3 &X, u32 j, uint2 *tb, u32 c0) {
    cp_async16(tb + 2 * threadIdx.x, X.twR[j] + X.rofR[2] + 2 * threadIdx.x);
    if (threadIdx.x < 4 * TC) cp_async16(tb + kColTab + 2 * threadIdx.x, X.ctwB[j] + (u64)c0 * 8 + 2 * threadIdx.x);
    cp_async_commit();
}

// All three primes in one CTA (R = 2^10, 8-column tiles, 512 threads): each
// thread reads the 8 nonzero digits of its first-round group once into
// registers; each prime then runs its column transform through the same
// shared tile in three rounds -- stages 0-3 in registers on 16 elements
// (upper half zero), then 4-6 and 7-9 -- with its round twiddles in shared
// memory, copied asynchronously one prime ahead (two buffers).  PAIR: both
// operands of pair i; else the single operand i.
template <int LL, int TC, bool PAIR, int H>
__global__ void __launch_bounds__(512, 2) k3_fwd_col_all(Geo3 X, Operands S, u32 *__restrict__ Y) {
    pdl_wait();
    static_assert(LL == 10 && TC == 8, "one task per thread: R/16 x 8 columns = 512");
    constexpr int RB = H >= 4 ? 4 : 2;  // bound of the rounds' outputs (units of p)
    extern __shared__ u32 sm3[];
    // pairs vary fastest across the grid, so the tile's inter-pass twiddles are
    // reused from L2 by the CTAs of all pairs
    const u32 i = blockIdx.x + S.pair0, c0 = blockIdx.y * TC;
    Desc dx, da;
    descs<PAIR>(S, i, dx, da);
    u32 *smx = sm3, *sma = sm3 + pxc((1u << LL) * TC);
    uint2 *stw = reinterpret_cast<uint2 *>(sm3 + (PAIR ? 2 : 1) * pxc((1u << LL) * TC));  // two twiddle buffers
    col_tables_async<TC>(X, 0, stw, c0);
    bool ones = true;
    const u32 c = threadIdx.x & (TC - 1), lo = threadIdx.x >> 3;  // group lo: rows lo + 64 m
    constexpr u32 D64 = 64;
    u32 rx[8], ra[8];
    {
        const u64 P0 = ((u64)lo * X.C + c0 + c) * X.b, stride = (u64)D64 * X.C * X.b;
#pragma unroll
        for (u32 m = 0; m < 8; m++) {
            rx[m] = digit_raw(X, dx, P0 + m * stride, ones);
            if (PAIR) ra[m] = digit_raw(X, da, P0 + m * stride, ones);
        }
    }
    const u32 a0 = pxc(lo * TC + c);
    constexpr u32 dsm = D64 * TC + ((D64 * TC) >> 3);  // 64 rows = 512 words apart
#pragma unroll 1
    for (u32 j = 0; j < 3; j++) {
        const u32 p = X.p[j];
        const uint2 red = X.red[j];
        // b-bit digits enter unreduced when they lie in [0, 4p) (the first stage only
        // multiplies them; later sums reduce as their bounds require), else through a
        // Shoup product into [0, 2p)
        const bool raw = (1ULL << X.b) <= 4ULL * p;
        u32 *Yx = Y + ((u64)j * 2 * X.K + i) * X.T, *Ya = Y + ((u64)j * 2 * X.K + X.K + i) * X.T;
        uint2 *tb = stw + (j & 1) * kColTabStride;
        // prime j's twiddles have landed, and prime j - 1's rounds are done with
        // the tile and with the other buffer, which now receives prime j + 1's
        cp_async_wait_all();
        __syncthreads();
        const uint2 *sB = tb + kColTab;  // this tile's split inter-pass twiddles B[c][m]
        const uint2 *rt = tb + kColTab4 + lo * 15;
        {
            u32 v[16];
#pragma unroll
            for (u32 m = 0; m < 16; m++) v[m] = m < 8 ? (raw ? rx[m] : shoup(rx[m], red, p)) : 0u;
            if (raw)
                dif16_hz<H, RB, 4>(v, rt, p);
            else
                dif16_hz<H, RB, 2>(v, rt, p);
#pragma unroll
            for (u32 m = 0; m < 16; m++) smx[a0 + m * dsm] = v[m];
        }
        if (PAIR) {
            u32 v[16];
#pragma unroll
            for (u32 m = 0; m < 16; m++) v[m] = m < 8 ? (raw ? ra[m] : shoup(ra[m], red, p)) : 0u;
            if (raw)
                dif16_hz<H, RB, 4>(v, rt, p);
            else
                dif16_hz<H, RB, 2>(v, rt, p);
#pragma unroll
            for (u32 m = 0; m < 16; m++) sma[a0 + m * dsm] = v[m];
        }
        __syncthreads();
        if (j + 1 < 3) col_tables_async<TC>(X, j + 1, stw + ((j + 1) & 1) * kColTabStride, c0);
        // the last round's A twiddles of this thread's two tasks (rows 8 g + m,
        // g = lo and lo + 64), loaded now so that round 2 hides their latency
        const uint2 apre0 = __ldg(X.ctwA[j] + (u64)lo * X.C + c0 + c);
        const uint2 apre1 = __ldg(X.ctwA[j] + (u64)(lo + 64) * X.C + c0 + c);
        // stages 4-6 and 7-9: the standard partition's rounds 2 and 3
        fwd3_round<3, PAIR, false, false, LL, TC, true, H, false, RB, RB>(X, j, dx, da, smx, sma, Yx, Ya, c0, 4, 2, ones,
                                                                          tb);
        __syncthreads();
        fwd3_round<3, PAIR, false, true, LL, TC, true, H, true, RB>(X, j, dx, da, smx, sma, Yx, Ya, c0, 7, 3, ones, tb,
                                                                     sB, apre0, apre1);
    }
    pdl_trigger();
    if (dx.check_ones) {
        // Algorithm 1 reload rule: slice i is all ones iff every CTA of the slice saw only ones
        const int all = __syncthreads_and(ones ? 1 : 0);
        if (threadIdx.x == 0 && all) {
            int *cnt = S.reload + 4 + i;
            if (atomicAdd(cnt, 1) + 1 == (int)gridDim.y) atomicExch(S.reload, 1);
        }
    }
}

// --------------------------------------------------- rows + MAC (Eq. 2) --

// Row rounds: elements base + m*stride with stride >= 8 or (stride = 1 and
// base a multiple of 8), so their padded words are px(base) + m * pstep(stride).
// MODE 0: both rows of pair i, product into acc; 1: row x only, its spectrum
// stored to spec; 2: row x only, times the stored spectrum held in fa.
template <int NS, int ACC, bool LAST, int LL, int MODE, int H, int RIB, int ROUT>
__device__ __forceinline__ void row_fwd3(const Geo3 &X, u32 j, const u32 (&fx)[ACC], const u32 (&fa)[ACC],
                                         u32 *__restrict__ smx, u32 *__restrict__ sma, u32 s0, u32 rd, bool first,
                                         u32 (&acc)[ACC], u32 *__restrict__ spec) {
    constexpr bool TWO = MODE == 0;
    const u32 l = LL ? (u32)LL : X.logC, sh = l - s0 - NS, stride = 1u << sh, ngroups = (1u << l) >> NS;
    const u32 p = X.p[j], pinv = X.pinv[j];
    const u32 dsm = pstep(stride);
    const uint2 *tw = X.twC[j] + X.rofC[rd];
#pragma unroll
    for (int t = 0; t < (ACC >> NS); t++) {
        const u32 g = threadIdx.x + t * blockDim.x;
        if (g < ngroups) {
            const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
            const u32 a0 = px(base);
            u32 vx[8], va[8];
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) {
                vx[m] = first ? fx[t * (1 << NS) + m] : smx[a0 + m * dsm];
                if (TWO) va[m] = first ? fa[t * (1 << NS) + m] : sma[a0 + m * dsm];
            }
            const uint2 *rt = tw + lo * ((1u << NS) - 1);
            // the last round feeds the Montgomery products (inputs below 4p when p < 2^28,
            // whose product then stays below 2^32 p) or the stored spectra ([0, 2p))
            constexpr int OUTL = (MODE == 1 || H < 4) ? 2 : 4;
            dif3<NS, LAST, false, false, H, LAST ? OUTL : ROUT, RIB>(vx, rt, p);
            if (TWO) dif3<NS, LAST, false, false, H, LAST ? OUTL : ROUT, RIB>(va, rt, p);
            if constexpr (LAST && MODE == 1) {  // the last round has stride 1: elements base + m
                if constexpr (NS == 3) {
                    uint4 *d = reinterpret_cast<uint4 *>(spec + base);
                    d[0] = make_uint4(vx[0], vx[1], vx[2], vx[3]);
                    d[1] = make_uint4(vx[4], vx[5], vx[6], vx[7]);
                } else {
#pragma unroll
                    for (int m = 0; m < (1 << NS); m++) spec[base + m] = vx[m];
                }
            } else {
#pragma unroll
                for (int m = 0; m < (1 << NS); m++) {
                    if (LAST) {
                        // Montgomery outputs lie in (0, 2p); with headroom 16p the sum
                        // takes 7 of them before the caller reduces it (mac_reduce)
                        u32 &a = acc[t * (1 << NS) + m];
                        const u32 prod = mont(vx[m], TWO ? va[m] : fa[t * (1 << NS) + m], p, pinv);
                        a = H >= 4 ? a + prod : red2(a + prod, 2 * p);
                    } else {
                        smx[a0 + m * dsm] = vx[m];
                        if (TWO) sma[a0 + m * dsm] = va[m];
                    }
                }
            }
        }
    }
}

// Accumulators of the lazy multiply-accumulate (H = 4): below 16p after at
// most 7 products since the last reduction, brought below 2p.
template <int ACC>
__device__ __forceinline__ void mac_reduce(u32 (&acc)[ACC], u32 p) {
#pragma unroll
    for (int m = 0; m < ACC; m++) acc[m] = csub(csub(csub(acc[m], 8 * p), 4 * p), 2 * p);
}

// The first round's inputs of one row pair (elements g + m C/2^NS of group g).
template <int NS, int ACC, int LL, bool TWO>
__device__ __forceinline__ void row_load3(const Geo3 &X, const u32 *__restrict__ xrow, const u32 *__restrict__ arow,
                                          u32 (&fx)[ACC], u32 (&fa)[ACC]) {
    const u32 l = LL ? (u32)LL : X.logC, stride = 1u << (l - NS), ngroups = (1u << l) >> NS;
#pragma unroll
    for (int t = 0; t < (ACC >> NS); t++) {
        const u32 g = threadIdx.x + t * blockDim.x;
        if (g < ngroups) {
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) {
                fx[t * (1 << NS) + m] = __ldg(xrow + g + m * stride);
                if (TWO) fa[t * (1 << NS) + m] = __ldg(arow + g + m * stride);
            }
        }
    }
}

template <int NS, int ACC, bool LAST, int LL, int H>
__device__ __forceinline__ void row_inv3(const Geo3 &X, u32 j, u32 *__restrict__ sm, u32 *__restrict__ Srow, u32 row,
                                         u32 s0, u32 rd, bool to_global, const u32 (&acc)[ACC]) {
    const u32 l = LL ? (u32)LL : X.logC, sh = l - s0 - NS, stride = 1u << sh, ngroups = (1u << l) >> NS, p = X.p[j];
    const u32 dsm = pstep(stride);
    const uint2 *ictw = X.ictw[j] + ((u64)row << l);
    const uint2 *itw = X.itwC[j] + X.rofC[rd];
#pragma unroll
    for (int t = 0; t < (ACC >> NS); t++) {
        const u32 g = threadIdx.x + t * blockDim.x;
        if (g < ngroups) {
            const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
            const u32 a0 = px(base);
            u32 v[8];
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) v[m] = LAST ? acc[t * (1 << NS) + m] : sm[a0 + m * dsm];
            // the first inverse round takes the accumulators (below 2p), later ones the
            // previous round's outputs (below RBI p)
            constexpr int RBI = H >= 4 ? 8 : 2, IB = LAST ? 2 : RBI;
            if (to_global)  // followed by the Shoup product with the inverse inter-pass twiddle
                dit3<NS, LAST, false, H, 0, IB>(v, itw + lo * ((1u << NS) - 1), p);
            else
                dit3<NS, LAST, false, H, RBI, IB>(v, itw + lo * ((1u << NS) - 1), p);
#pragma unroll
            for (int m = 0; m < (1 << NS); m++) {
                if (to_global) {
                    const u32 idx = base + m * stride;
                    Srow[idx] = shoup(v[m], __ldg(ictw + idx), p);  // omega_T^(-c bitrev(row))
                } else {
                    sm[a0 + m * dsm] = v[m];
                }
            }
        }
    }
}

// A stored row spectrum in the last forward round's order: thread group g
// holds elements g 2^NS + m, m < 2^NS.
template <int NS, int ACC>
__device__ __forceinline__ void row_load_spec(u32 ngroups, const u32 *__restrict__ srow, u32 (&f)[ACC]) {
#pragma unroll
    for (int t = 0; t < (ACC >> NS); t++) {
        const u32 g = threadIdx.x + t * blockDim.x;
        if (g < ngroups) {
            if constexpr (NS == 3) {
                const uint4 *q = reinterpret_cast<const uint4 *>(srow + (g << 3));
                const uint4 u = __ldg(q), w = __ldg(q + 1);
                f[t * 8 + 0] = u.x, f[t * 8 + 1] = u.y, f[t * 8 + 2] = u.z, f[t * 8 + 3] = u.w;
                f[t * 8 + 4] = w.x, f[t * 8 + 5] = w.y, f[t * 8 + 6] = w.z, f[t * 8 + 7] = w.w;
            } else {
#pragma unroll
                for (int m = 0; m < (1 << NS); m++) f[t * (1 << NS) + m] = __ldg(srow + (g << NS) + m);
            }
        }
    }
}

// grid (R, 3 primes); blockDim = C / ACC threads, ACC accumulators each.
// MODE 0: Eq. 2 / Eq. 4 product of the pairs' rows, then the inverse rows;
// 1 (seed preparation): forward rows of the single operands, spectra stored
// to spec ([prime][operand][T], last-round order); 2 (prepared hashing):
// forward rows of the single operands times the stored spectra, then the
// inverse rows.
template <int ACC, int LL, int MODE, int H>
__global__ void __launch_bounds__(1024) k3_row_mac(Geo3 X, const u32 *__restrict__ Y, u32 *__restrict__ S3,
                                                   u32 *__restrict__ spec) {
    pdl_wait();
    extern __shared__ u32 sm3[];
    const u32 j = blockIdx.y, row = blockIdx.x, l = LL ? (u32)LL : X.logC, C = 1u << l;
    u32 *smx = sm3, *sma = sm3 + px(C);
    u32 acc[ACC], fx[ACC], fa[ACC];
    constexpr int RB = H >= 4 ? 4 : 2;  // bound of the forward rounds' outputs (units of p)
#pragma unroll
    for (int m = 0; m < ACC; m++) acc[m] = 0;
    const u32 nr = (l + 2) / 3, ns0 = round_ns(l, 0), nsl = round_ns(l, nr - 1);
    for (u32 i = 0; i < X.K; i++) {
        u32 *srow = MODE ? spec + ((u64)j * X.K + i) * X.T + (u64)row * C : nullptr;
        {  // the first round's inputs, loaded right before use (short register lifetimes)
            const u32 *xr = Y + ((u64)j * 2 * X.K + i) * X.T + (u64)row * C;
            const u32 *ar = MODE ? xr : Y + ((u64)j * 2 * X.K + X.K + i) * X.T + (u64)row * C;
#define P3_LOAD(NSV) row_load3<NSV, ACC, LL, MODE == 0>(X, xr, ar, fx, fa)
            P3_DISPATCH_NS(ns0, P3_LOAD);
#undef P3_LOAD
            if (MODE == 2) {
#define P3_LOADS(NSV) row_load_spec<NSV, ACC>(C >> NSV, srow, fa)
                P3_DISPATCH_NS(nsl, P3_LOADS);
#undef P3_LOADS
            }
        }
#pragma unroll(LL > 0 ? 8 : 1)
        for (u32 rd = 0; rd < nr; rd++) {
            const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
            const bool first = rd == 0, last = rd == nr - 1;
// inputs of the first round (spectra of the column pass) below 2p, of later rounds below RB p
#define P3_ROWF(NSV)                                                                                              \
    do {                                                                                                          \
        if (last && first)                                                                                        \
            row_fwd3<NSV, ACC, true, LL, MODE, H, 2, RB>(X, j, fx, fa, smx, sma, s0, rd, first, acc, srow);       \
        else if (last)                                                                                            \
            row_fwd3<NSV, ACC, true, LL, MODE, H, RB, RB>(X, j, fx, fa, smx, sma, s0, rd, first, acc, srow);      \
        else if (first)                                                                                           \
            row_fwd3<NSV, ACC, false, LL, MODE, H, 2, RB>(X, j, fx, fa, smx, sma, s0, rd, first, acc, srow);      \
        else                                                                                                      \
            row_fwd3<NSV, ACC, false, LL, MODE, H, RB, RB>(X, j, fx, fa, smx, sma, s0, rd, first, acc, srow);     \
    } while (0)
            P3_DISPATCH_NS(ns, P3_ROWF);
#undef P3_ROWF
            __syncthreads();
        }
        if (H >= 4 && MODE != 1 && (i % 7 == 6 || i + 1 == X.K)) mac_reduce(acc, X.p[j]);
    }
    if (MODE == 1) {
        pdl_trigger();
        return;
    }
    u32 *Srow = S3 + (u64)j * X.T + (u64)row * C;
#pragma unroll(LL > 0 ? 8 : 1)
    for (int rd = (int)nr - 1; rd >= 0; rd--) {
        const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
        const bool from_acc = rd == (int)nr - 1, to_global = rd == 0;
#define P3_ROWI(NSV)                                                          \
    do {                                                                      \
        if (from_acc)                                                         \
            row_inv3<NSV, ACC, true, LL, H>(X, j, smx, Srow, row, s0, rd, to_global, acc);  \
        else                                                                  \
            row_inv3<NSV, ACC, false, LL, H>(X, j, smx, Srow, row, s0, rd, to_global, acc); \
    } while (0)
        P3_DISPATCH_NS(ns, P3_ROWI);
#undef P3_ROWI
        __syncthreads();
    }
    pdl_trigger();
}

// -------------------------------------------------------- inverse columns --

template <int NS, bool FIRSTR, bool TOGLOBAL, bool HO, int LL, int TC, int H>
__device__ __forceinline__ void inv3_round(const Geo3 &X, u32 j, u32 *__restrict__ S3, u32 *__restrict__ sm, u32 c0,
                                           u32 s0, u32 rd) {
    const u32 l = LL ? (u32)LL : X.logR, tc = TC ? (u32)TC : X.tc, p = X.p[j];
    const u32 sh = l - s0 - NS, stride = 1u << sh;
    const u32 ntask = ((1u << l) >> NS) * tc;
    const u32 logtc = TC ? (u32)__builtin_ctz(TC) : (u32)(__ffs(tc) - 1);
    const u32 dsm = pstepc(stride * tc);
    const u64 dY = (u64)stride * X.C;
    const uint2 *itw = X.itwR[j] + X.rofR[rd];
    u32 *Sj = S3 + (u64)j * X.T;
    for (u32 task = threadIdx.x; task < ntask; task += blockDim.x) {
        const u32 c = task & (tc - 1), g = task >> logtc;
        const u32 lo = g & (stride - 1), base = ((g >> sh) << (l - s0)) + lo;
        const u32 a0 = pxc(base * tc + c);
        const u64 e0 = (u64)base * X.C + c0 + c;
        u32 v[8];
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) v[m] = FIRSTR ? Sj[e0 + m * dY] : sm[a0 + m * dsm];
        // the residues written to S3 only feed Shoup products (the CRT): any bound
        dit3<NS, FIRSTR, HO, H, TOGLOBAL ? 0 : 2>(v, itw + lo * ((1u << NS) - 1), p);
#pragma unroll
        for (int m = 0; m < (1 << NS); m++) {
            if (TOGLOBAL) {
                if (HO && m >= (1 << (NS - 1))) continue;  // rows >= R/2: coefficients >= T/2, unused
                Sj[e0 + m * dY] = v[m];
            } else {
                sm[a0 + m * dsm] = v[m];
            }
        }
    }
}

// grid (C / tc, 3 primes).  In place on S3: every CTA reads its own columns
// completely (first round) before it writes them (last round).
template <int LL, int TC, int H>
__global__ void __launch_bounds__(kColThreads) k3_inv_col(Geo3 X, u32 *__restrict__ S3, u64 *__restrict__ zero_out,
                                                          u64 zero_words) {
    pdl_wait();
    {  // the output bits of the fused carry (k3_resolve_a ORs into them)
        const u64 nthr = (u64)gridDim.x * gridDim.y * blockDim.x;
        for (u64 i = ((u64)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; i < zero_words; i += nthr)
            zero_out[i] = 0;
    }
    extern __shared__ u32 sm3[];
    const u32 j = blockIdx.y, tc = TC ? (u32)TC : X.tc, c0 = blockIdx.x * tc;
    const u32 l = LL ? (u32)LL : X.logR, nr = (l + 2) / 3;
    const bool ho = X.stage == 1;  // Eq. 4: only t mod 2^gamma, i.e. coefficients < T/2
    // R = 2^10 with the 4-stage table: stages 3..0 in one register round at the end
    constexpr bool M4 = LL == 10 && TC == 8;
    const int rlast = (M4 && X.rof4Ri) ? 2 : 0;
#pragma unroll(LL > 0 ? 8 : 1)
    for (int rd = (int)nr - 1; rd >= rlast; rd--) {
        const u32 s0 = round_s0(l, rd), ns = round_ns(l, rd);
        const bool first = rd == (int)nr - 1, last = rd == 0;
#define P3_INV(NSV)                                                       \
    do {                                                                  \
        if (first)                                                        \
            inv3_round<NSV, true, false, false, LL, TC, H>(X, j, S3, sm3, c0, s0, (u32)rd);   \
        else if (last && ho)                                              \
            inv3_round<NSV, false, true, true, LL, TC, H>(X, j, S3, sm3, c0, s0, (u32)rd);    \
        else if (last)                                                    \
            inv3_round<NSV, false, true, false, LL, TC, H>(X, j, S3, sm3, c0, s0, (u32)rd);   \
        else                                                              \
            inv3_round<NSV, false, false, false, LL, TC, H>(X, j, S3, sm3, c0, s0, (u32)rd);  \
    } while (0)
        P3_DISPATCH_NS(ns, P3_INV);
#undef P3_INV
        __syncthreads();
    }
    if constexpr (M4) {
        if (rlast == 2) {
            // stages 3..0: 16 rows lo + 64 m of one column per task, written to S3
            const u32 p = X.p[j];
            const uint2 *itw = X.itwR[j] + X.rof4Ri;
            u32 *Sj = S3 + (u64)j * X.T;
            for (u32 task = threadIdx.x; task < 64 * TC; task += blockDim.x) {
                const u32 c = task & (TC - 1), lo = task >> 3;
                const u32 a0 = pxc(lo * TC + c);
                const u64 e0 = (u64)lo * X.C + c0 + c, dY = (u64)64 * X.C;
                u32 v[16];
#pragma unroll
                for (u32 m = 0; m < 16; m++) v[m] = sm3[a0 + m * 576];  // 64 rows apart: pstepc(512)
                if (ho) {
                    dit16<true, H, 0>(v, itw + lo * 15, p);
#pragma unroll
                    for (u32 m = 0; m < 8; m++) Sj[e0 + m * dY] = v[m];
                } else {
                    dit16<false, H, 0>(v, itw + lo * 15, p);
#pragma unroll
                    for (u32 m = 0; m < 16; m++) Sj[e0 + m * dY] = v[m];
                }
            }
        }
    }
    pdl_trigger();
}

// ------------------------------------------------------ CRT and Mersenne fold --

// Coefficient e from its three residues (scaled by 2^32 / T): Garner's mixed
// radix x1 + p0 x2 + p0 p1 x3.
__device__ __forceinline__ unsigned __int128 crt_combine(const Geo3 &X, u32 res0, u32 res1, u32 res2) {
    const u32 p0 = X.p[0], p1 = X.p[1], p2 = X.p[2];
    const u32 r0 = canon(shoup(res0, X.scale[0], p0), p0);
    const u32 r1 = canon(shoup(res1, X.scale[1], p1), p1);
    const u32 r2 = canon(shoup(res2, X.scale[2], p2), p2);
    const u32 x1 = r0;
    const u32 u1 = canon(shoup(x1, X.red[1], p1), p1);
    const u32 x2 = canon(shoup(r1 - u1 + p1, X.c12, p1), p1);
    const u32 u2 = canon(shoup(x1, X.red[2], p2), p2);
    const u32 w2 = canon(shoup(x2, X.p0m2, p2), p2);
    const u32 s2 = canon(u2 + w2, p2);
    const u32 x3 = canon(shoup(r2 - s2 + p2, X.c3, p2), p2);
    return (unsigned __int128)x1 + (unsigned __int128)((u64)p0 * x2) + (unsigned __int128)X.p01 * x3;
}

__device__ __forceinline__ unsigned __int128 crt_value(const Geo3 &X, const u32 *__restrict__ S3, u64 e) {
    return crt_combine(X, __ldg(S3 + e), __ldg(S3 + X.T + e), __ldg(S3 + 2 * X.T + e));
}

// Digit t (bit offset t b) of the value to resolve.  Coefficient e's value V_e
// sits at bit offset e b; its b-bit pieces (V_e, V_e >> b, V_e >> 2b) land on
// positions e, e+1, e+2.  Eq. 2 (RING): position P's offset P b is taken mod
// gamma; position t + nd (nd = ceil(gamma / b)) lands on digit t shifted by
// D1 = nd b - gamma, position t + n2 (n2 = ceil(2 gamma / b)) by
// D2 = n2 b - 2 gamma, as long as t b + D < gamma (the top digit is short:
// larger offsets belong to a lower digit of the next wrap).  Eq. 4: position t
// only, plus digit t of c (bits [c_base, c_base + gamma) of c_src).  A CTA of
// 256 digits computes each coefficient it needs once (258 per wrap), shares
// the pieces through shared memory, and zeroes the carry output first.
template <bool RING>
__global__ void __launch_bounds__(256) k3_digits(Geo3 X, const u32 *__restrict__ S3, u64 *__restrict__ z, u64 npad,
                                                 const u64 *__restrict__ c_src, u64 c_base, u64 *__restrict__ zero_out,
                                                 u64 zero_words) {
    pdl_wait();
    __shared__ u64 pc[3][258];
    const u64 t0 = (u64)blockIdx.x * 256, t = t0 + threadIdx.x;
    if (t < zero_words) zero_out[t] = 0;  // the carry kernels OR their bits into it
    const u64 b = X.b, G = X.G, mask = (1ULL << b) - 1;
    const u64 ncoef = RING ? 2 * X.M - 1 : X.M;
    const u64 nd = X.nd, n2 = (2 * G + b - 1) / b;
    u64 acc = 0;
#pragma unroll 1
    for (u32 w = 0; w < (RING ? 3u : 1u); w++) {
        const u64 off = w == 0 ? 0 : (w == 1 ? nd : n2);
        const u64 D = w == 0 ? 0 : (w == 1 ? nd * b - G : n2 * b - 2 * G);
        // the block's first digit has the smallest offset: if it cannot take wrap w, none can
        if (w > 0 && (t0 * b + D >= G || t0 + off > 2 * X.M)) break;
        const u64 P0 = t0 + off;  // position of this block's first digit
        for (u32 i = threadIdx.x; i < 258; i += 256) {
            const u64 e = P0 + i - 2;  // wraps below 0 when P0 < 2: skipped by the range check
            u64 v0 = 0, v1 = 0, v2 = 0;
            if (P0 + i >= 2 && e < ncoef) {
                const unsigned __int128 V = crt_value(X, S3, e);
                v0 = (u64)V & mask;
                v1 = (u64)(V >> b) & mask;
                v2 = (u64)(V >> (2 * b));
            }
            pc[0][i] = v0;
            pc[1][i] = v1;
            pc[2][i] = v2;
        }
        __syncthreads();
        if (t < nd && (w == 0 || (t * b + D < G && t + off <= 2 * X.M))) {
            const u32 i = threadIdx.x + 2;
            acc += (pc[0][i] + pc[1][i - 1] + pc[2][i - 2]) << D;
        }
        __syncthreads();
    }
    if (!RING && c_src && t < nd) {
        const u64 pos = t * b;
        const u32 nb = (u32)min(b, G - pos);
        acc += rd32(c_src, c_base + pos, nb);
    }
    if (t < npad) z[t] = t < nd ? acc : 0;
    pdl_trigger();
}

// ------------------------------------- fused digit gather + carry (large) --
//
// The digits of k3_digits and the chunk carries of the carry kernels in one
// pass, for vectors whose chunks of PA_CARRY_D digits span >= 64 bits: thread
// t of CTA q owns chunk q (NT - 1) - 1 + t (thread 0 the last chunk of the previous
// CTA -- around the ring for CTA 0 -- whose carry-out it provides).  A thread
// computes the CRT values of its chunk's 8 positions once per wrap and takes
// the pieces its first two digits need from the previous lane (shuffles), the
// previous warp (shared memory) or, for thread 0, two extra CRT values.  The
// digits never go to memory: the chunk's carry-out H (zero carry-in), its bits
// with carry-in H of the previous chunk (OR-ed into y, which the inverse
// column pass zeroed), and its generate / propagate state are derived in
// registers; the CTA's state feeds k3_resolve_c.
// NT threads per CTA (256, or 64 for short vectors so that they still spread
// over the SMs): NT - 1 chunks written per CTA (thread 0 only provides a
// carry-out).
constexpr u32 kResolveMinChunks = 63;  // the smallest CTA's chunks: sizes the per-CTA state arrays

__device__ __forceinline__ bool digit_takes_wrap(const Geo3 &X, u64 t, u32 w, u64 off, u64 D) {
    return t < X.nd && (w == 0 || (t * X.b + D < X.G && t + off <= 2 * X.M));
}

// b-bit pieces of coefficient e (0 outside [0, ncoef)): v0, v1 < 2^b <= 2^30.
__device__ __forceinline__ void crt_pieces(const Geo3 &X, const u32 *__restrict__ S3, long long e, u64 ncoef, u32 &v0,
                                           u32 &v1, u64 &v2) {
    v0 = v1 = 0;
    v2 = 0;
    if (e < 0 || (u64)e >= ncoef) return;
    const unsigned __int128 V = crt_value(X, S3, (u64)e);
    const u64 mask = (1ULL << X.b) - 1;
    v0 = (u32)((u64)V & mask);
    v1 = (u32)((u64)(V >> X.b) & mask);
    v2 = (u64)(V >> (2 * X.b));
}

template <bool RING, int NT>
__global__ void __launch_bounds__(NT) k3_resolve_a(Geo3 X, const u32 *__restrict__ S3, CarryDev cd,
                                                   const u64 *__restrict__ c_src, u64 c_base, u64 *__restrict__ y) {
    pdl_wait();
    constexpr int NW = NT / 32;
    __shared__ u64 Hs[NT];
    __shared__ u64 xw[NW][3];  // per warp: pieces v1(7), v2(6), v2(7) of its last lane
    __shared__ unsigned wg[NW], wp[NW];
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long cq = (long long)blockIdx.x * (NT - 1) - 1 + tid;
    // chunk whose digits this thread forms (thread 0 of CTA 0: the top chunk around the ring)
    const bool exists = cq >= 0 ? (u64)cq < cd.nchunks : RING;
    const u64 ch = cq >= 0 ? (u64)cq : cd.nchunks - 1;
    const bool real = tid > 0 && cq >= 0 && (u64)cq < cd.nchunks;  // chunks this CTA writes
    const u64 t0 = ch * PA_CARRY_D;
    const u64 b = X.b, G = X.G;
    const u64 ncoef = RING ? 2 * X.M - 1 : X.M;
    const u64 nd = X.nd, n2 = (2 * G + b - 1) / b;
    u64 z[PA_CARRY_D];
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) z[d] = 0;
    // threads whose previous thread holds a chunk that is not the one below:
    // thread 0, and at the ring's wrap the thread of chunk 0
    const bool own_prev = tid == 0 || cq == 0;
#pragma unroll 1
    for (u32 w = 0; w < (RING ? 3u : 1u); w++) {
        const u64 off = w == 0 ? 0 : (w == 1 ? nd : n2);
        const u64 D = w == 0 ? 0 : (w == 1 ? nd * b - G : n2 * b - 2 * G);
        // positions t0 + j + off, j = 0..7; digit t0 + j needs pieces of j, j - 1, j - 2.
        // All residues of the wrap are loaded before any CRT (memory-level parallelism).
        u32 q0[PA_CARRY_D + 2], q1[PA_CARRY_D + 2], q2[PA_CARRY_D + 2];  // [0..7]: j, [8], [9]: j = -1, -2
        bool need[PA_CARRY_D];
#pragma unroll
        for (u32 j = 0; j < PA_CARRY_D; j++) need[j] = exists && digit_takes_wrap(X, t0 + j, w, off, D);
        // a wrap none of the CTA's digits takes is skipped (validity falls with the digit index)
        if (!__syncthreads_or(need[0] ? 1 : 0)) continue;
#pragma unroll
        for (u32 j = 0; j < PA_CARRY_D + 2; j++) {
            const long long e = j < PA_CARRY_D ? (long long)(t0 + off + j) : (long long)(t0 + off) - (long long)(j - 7);
            const bool ld = (j < PA_CARRY_D ? need[j] : (own_prev && need[0])) && e >= 0 && (u64)e < ncoef;
            q0[j] = ld ? __ldg(S3 + e) : 0u;
            q1[j] = ld ? __ldg(S3 + X.T + e) : 0u;
            q2[j] = ld ? __ldg(S3 + 2 * X.T + e) : 0u;
        }
        auto pieces = [&](u32 j, u32 &c0, u32 &c1, u64 &c2) {
            if (!(j < PA_CARRY_D ? need[j] : (own_prev && need[0]))) {  // no digit of this thread takes them
                c0 = c1 = 0;
                c2 = 0;
                return;
            }
            const unsigned __int128 V = crt_combine(X, q0[j], q1[j], q2[j]);
            const u64 mask = (1ULL << b) - 1;
            c0 = (u32)((u64)V & mask);
            c1 = (u32)((u64)(V >> b) & mask);
            c2 = (u64)(V >> (2 * b));
        };
        // pieces the next lane needs (j = 6, 7) first; a residue triple of zeros gives zero pieces
        u32 v0_6, v1_6, v0_7, v1_7;
        u64 v2_6, v2_7;
        pieces(6, v0_6, v1_6, v2_6);
        pieces(7, v0_7, v1_7, v2_7);
        // pieces of positions j = -1, -2 from the previous lane / warp / own CRT
        u32 p1m1 = __shfl_up_sync(0xFFFFFFFFu, v1_7, 1);
        u64 p2m1 = __shfl_up_sync(0xFFFFFFFFu, v2_7, 1), p2m2 = __shfl_up_sync(0xFFFFFFFFu, v2_6, 1);
        if (lane == 31) {
            xw[warp][0] = v1_7;
            xw[warp][1] = v2_7;
            xw[warp][2] = v2_6;
        }
        __syncthreads();
        if (lane == 0 && warp > 0) {
            p1m1 = (u32)xw[warp - 1][0];
            p2m1 = xw[warp - 1][1];
            p2m2 = xw[warp - 1][2];
        }
        if (own_prev) {
            u32 a0, a1;
            u64 a2;
            pieces(8, a0, a1, a2);
            p1m1 = a1;
            p2m1 = a2;
            pieces(9, a0, a1, a2);
            p2m2 = a2;
        }
        u32 w1 = p1m1;               // v1 of position j - 1
        u64 w2a = p2m1, w2b = p2m2;  // v2 of positions j - 1, j - 2
#pragma unroll
        for (u32 j = 0; j < PA_CARRY_D; j++) {
            u32 c0, c1;
            u64 c2;
            if (j == 6) {
                c0 = v0_6, c1 = v1_6, c2 = v2_6;
            } else if (j == 7) {
                c0 = v0_7, c1 = v1_7, c2 = v2_7;
            } else {
                pieces(j, c0, c1, c2);
            }
            if (need[j]) z[j] += ((u64)c0 + w1 + w2b) << D;
            w1 = c1;
            w2b = w2a;
            w2a = c2;
        }
        __syncthreads();
    }
    if (!RING && c_src && exists) {
#pragma unroll
        for (u32 j = 0; j < PA_CARRY_D; j++) {
            const u64 t = t0 + j;
            if (t < nd) z[j] += rd32(c_src, c_base + t * b, (u32)min(b, G - t * b));
        }
    }
    // chunk carry-out with zero carry-in
    u32 bd[PA_CARRY_D];
    u64 s = min(t0 * b, G);
    const u64 s_begin = s;
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) {
        const u64 s1 = min((t0 + d + 1) * b, G);
        bd[d] = (u32)(s1 - s);
        s = s1;
    }
    unsigned __int128 acc = 0;
#pragma unroll
    for (u32 d = 0; d < PA_CARRY_D; d++) {
        acc += z[d];
        acc >>= bd[d];
    }
    const u64 Ht = exists ? (u64)acc : 0;
    Hs[tid] = Ht;
    if (blockIdx.x == 0 && tid == 0) *cd.allones = 1;  // cleared by k3_resolve_c unless every chunk is all ones
    __syncthreads();
    bool g = false, p = true;
    if (real) {
        const u64 Hin = Hs[tid - 1];
        acc = Hin;
        bool ones = true;
        u64 wi = s_begin >> 6, wv = 0;
        u32 bo = (u32)(s_begin & 63);
#pragma unroll
        for (u32 d = 0; d < PA_CARRY_D; d++) {
            acc += z[d];
            const u64 mask = (1ULL << bd[d]) - 1;
            const u64 bits = (u64)acc & mask;
            ones = ones && (bits == mask);
            acc >>= bd[d];
            wv |= bits << bo;
            const u32 nb = bo + bd[d];
            if (nb >= 64) {
                atomicOr(y + wi, wv);
                wi++;
                wv = (nb > 64) ? (bits >> (64 - bo)) : 0;
                bo = nb - 64;
            } else {
                bo = nb;
            }
        }
        if (bo) atomicOr(y + wi, wv);
        g = (u64)acc != Ht;  // acc == H_t + (carry out of adding H_{t-1})
        p = !g && ones;
        cd.state[cq] = (unsigned char)((g ? 1 : 0) | (p ? 2 : 0));
    }
    pdl_trigger();
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, g), pm = __ballot_sync(0xFFFFFFFFu, p);
    if (lane == 0) {
        wg[warp] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wp[warp] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    if (tid == 0) {
        unsigned Gc = 0, Pc = 1;
        for (u32 q = 0; q < NW; q++) {
            Gc = wg[q] | (wp[q] & Gc);
            Pc = wp[q] & Pc;
        }
        cd.cta_state[blockIdx.x] = (unsigned char)(Gc | (Pc << 1));
    }
}

// Generate / propagate of the states [lo, hi) composed in order, by the CTA
// (NT threads): (G, P) with G = carry out given no carry in, P = a carry in
// passes through.  Every thread gets the result.
template <int NT>
__device__ __forceinline__ void fold_states(const unsigned char *__restrict__ st, u32 lo, u32 hi, unsigned &Gout,
                                            unsigned &Pout, unsigned *wG, unsigned *wP) {
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 n = hi > lo ? hi - lo : 0, per = (n + NT - 1) / NT;
    const u32 b0 = lo + min(tid * per, n), b1 = lo + min(tid * per + per, n);
    unsigned G = 0, P = 1;
    for (u32 q = b0; q < b1; q++) {
        const unsigned v = st[q];
        G = (v & 1) | (((v >> 1) & 1) & G);
        P = ((v >> 1) & 1) & P;
    }
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, G), pm = __ballot_sync(0xFFFFFFFFu, P);
    __syncthreads();  // wG / wP may still be read from a previous call
    if (lane == 0) {
        wG[warp] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wP[warp] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    G = 0;
    P = 1;
    for (u32 q = 0; q < NT / 32; q++) {
        G = wG[q] | (wP[q] & G);
        P = wP[q] & P;
    }
    Gout = G;
    Pout = P;
}

// Carries between chunks: the CTA's carry-in from the states of the CTAs below
// it (and, around the ring, the carry out of the top with none in -- the
// end-around carry of the Mersenne fold), then per chunk from the chunk states,
// and the chunks receiving a carry increment their bit range.
template <bool RING, int NT>
__global__ void __launch_bounds__(NT) k3_resolve_c(CarryDev cd, u32 nctas, u64 *__restrict__ y) {
    pdl_wait();
    constexpr int NW = NT / 32;
    __shared__ unsigned wG[NW], wP[NW], wg[NW], wp[NW];
    const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned Gpre, Ppre, Gall = 0, Pall = 1;
    fold_states<NT>(cd.cta_state, 0, blockIdx.x, Gpre, Ppre, wG, wP);
    if (RING) fold_states<NT>(cd.cta_state, 0, nctas, Gall, Pall, wG, wP);
    const unsigned ewrap = RING ? Gall : 0u;
    const unsigned cin = Gpre | (Ppre & ewrap);
    const long long cq = (long long)blockIdx.x * (NT - 1) - 1 + tid;
    const bool real = tid > 0 && cq >= 0 && (u64)cq < cd.nchunks;
    const unsigned st = real ? cd.state[cq] : 2u;
    const unsigned gm = __ballot_sync(0xFFFFFFFFu, st & 1), pm = __ballot_sync(0xFFFFFFFFu, (st >> 1) & 1);
    if (lane == 0) {
        wg[warp] = (unsigned)((((u64)(gm | pm)) + gm) >> 32);
        wp[warp] = (pm == 0xFFFFFFFFu);
    }
    __syncthreads();
    unsigned cw = cin;
    for (u32 q = 0; q < warp; q++) cw = wg[q] | (wp[q] & cw);
    const u64 a = gm | pm, sum = a + gm + cw;
    const bool e = ((sum ^ a ^ gm) >> lane) & 1;
    pdl_trigger();
    bool fin_ones = true;
    if (real) {
        const u64 j0 = (u64)cq * PA_CARRY_D;
        const u64 s_lo = min(j0 * cd.ub, cd.G), s_hi = min((j0 + PA_CARRY_D) * cd.ub, cd.G);
        bool flipping = e;
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
    }
    const int all = __syncthreads_and(fin_ones ? 1 : 0);
    if (tid == 0 && !all) *cd.allones = 0;
}

// ----------------------------------------------------- Toeplitz parity --

// Output block blk of the Toeplitz product: bit i' is the parity of
// coefficient rb - 1 + i' of sum_J w_J * x_J (its exact value from the CRT;
// all primes are odd).  Thread per bit, two ballots per output word.
__global__ void __launch_bounds__(256) k3_toeplitz_bits(Geo3 X, const u32 *__restrict__ S3, u64 rb, u64 bit0, u64 r,
                                                        u32 *__restrict__ out32) {
    pdl_wait();
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;  // bit within the block
    bool bit = false;
    if (i < rb && bit0 + i < r) bit = ((u64)crt_value(X, S3, rb - 1 + i) & 1) != 0;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, bit);
    if ((threadIdx.x & 31) == 0 && i < rb && bit0 + i < r) out32[(bit0 + i) >> 5] = m;
    pdl_trigger();
}

// ------------------------------------------------------------------ tables --

// ctw[r C + c] = omega_T^(dir * c bitrev_R(r)) with its Shoup companion; the
// power comes from two host tables, lo[e mod 2^h] * hi[e >> h].
__global__ void k3_fill_ctw(u32 logR, u32 logC, u32 h, const u32 *__restrict__ lo, const u32 *__restrict__ hi, u32 p,
                            uint2 *__restrict__ out) {
    const u64 T = 1ULL << (logR + logC);
    for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; idx < T; idx += (u64)gridDim.x * blockDim.x) {
        const u32 r = (u32)(idx >> logC), c = (u32)(idx & ((1u << logC) - 1));
        const u64 e = ((u64)c * brev(r, logR)) & (T - 1);
        const u32 w = (u32)(((u64)__ldg(lo + (e & ((1ULL << h) - 1))) * __ldg(hi + (e >> h))) % p);
        out[idx] = make_uint2(w, (u32)(((u64)w << 32) / p));
    }
}

// The split inter-pass twiddles of R = 2^10 plans: out[r C + c] =
// omega_T^(c bitrev_7(r)) for r < 128 (A), or out[c 8 + m] =
// omega_T^(128 c bitrev_3(m)) (B), with Shoup companions.
__global__ void k3_fill_split(u32 logC, u32 logT, u32 h, bool b_table, const u32 *__restrict__ lo,
                              const u32 *__restrict__ hi, u32 p, uint2 *__restrict__ out) {
    const u64 T = 1ULL << logT, C = 1ULL << logC, n = (b_table ? 8 : 128) * C;
    for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (u64)gridDim.x * blockDim.x) {
        u64 e;
        if (b_table)
            e = (128 * (idx >> 3) * brev((u32)(idx & 7), 3)) & (T - 1);
        else
            e = ((idx & (C - 1)) * brev((u32)(idx >> logC), 7)) & (T - 1);
        const u32 w = (u32)(((u64)__ldg(lo + (e & ((1ULL << h) - 1))) * __ldg(hi + (e >> h))) % p);
        out[idx] = make_uint2(w, (u32)(((u64)w << 32) / p));
    }
}

}  // namespace p3

// ---------------------------------------------------------------- launchers --

using namespace p3;

static size_t col_smem3(const Geo3 &X, bool pair) {
    return (size_t)(pair ? 2 : 1) * (X.R * X.tc + ((X.R * X.tc >> 6) << 3) + 8) * sizeof(u32);
}
static size_t row_smem3(const Geo3 &X) { return (size_t)2 * (X.C + (X.C >> 3) + 8) * sizeof(u32); }

// Instantiated shapes.  Transforms up to 2^22 use primes below 2^28
// (headroom H = 4), longer ones primes below 2^30 (H = 2); with R = 2^10 for
// T >= 2^20 the row length fixes H: rows of 2^10, 2^11 (and every shorter
// transform) H = 4, rows of 2^12 H = 4 or (operands beyond the smaller
// primes' bound) 2, rows of 2^13 and 2^14 H = 2.
template <int MODE>
static cudaError_t p3_row_attrs(int big) {
    cudaError_t e;
#define P3_ATTR(f) \
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    P3_ATTR((k3_row_mac<8, 0, MODE, 4>))
    P3_ATTR((k3_row_mac<8, 10, MODE, 4>))
    P3_ATTR((k3_row_mac<8, 11, MODE, 4>))
    P3_ATTR((k3_row_mac<8, 12, MODE, 4>))
    P3_ATTR((k3_row_mac<8, 12, MODE, 2>))
    P3_ATTR((k3_row_mac<8, 13, MODE, 2>))
    P3_ATTR((k3_row_mac<16, 14, MODE, 2>))
#undef P3_ATTR
    return cudaSuccess;
}

int p3_prepare_kernels() {
    // kernel attributes are per device: set them once on each device used
    static std::atomic<unsigned long long> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
    const unsigned long long bit = dev < 64 ? 1ULL << dev : 0;  // devices >= 64: set every time
    if (done_mask.load() & bit) return 0;
    const int big = 200 * 1024;
    cudaError_t e;
#define P3_ATTR(f) \
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    P3_ATTR((k3_fwd_col<true, 0, 0, 4>))
    P3_ATTR((k3_fwd_col<false, 0, 0, 4>))
    P3_ATTR((k3_fwd_col_all<10, 8, true, 4>))
    P3_ATTR((k3_fwd_col_all<10, 8, false, 4>))
    P3_ATTR((k3_fwd_col_all<10, 8, true, 2>))
    P3_ATTR((k3_fwd_col_all<10, 8, false, 2>))
    P3_ATTR((k3_inv_col<0, 0, 4>))
    P3_ATTR((k3_inv_col<10, 8, 4>))
    P3_ATTR((k3_inv_col<10, 8, 2>))
#undef P3_ATTR
    if ((e = p3_row_attrs<0>(big)) || (e = p3_row_attrs<1>(big)) || (e = p3_row_attrs<2>(big))) return e;
    done_mask.fetch_or(bit);
    return 0;
}

// Compile-time geometry for the production shapes (R = 2^10, 8-column tiles;
// rows of 2^10 .. 2^14), runtime geometry otherwise.  pair: both operands of
// each pair (Eq. 2 / Eq. 4), else the single operands of S.mode.
template <int H>
static void p3_fwd_all(const Geo3 &X, const Operands &S, int pairs, u32 *Y, void *stream, bool pair, size_t smem) {
    cudaStream_t s = (cudaStream_t)stream;
    if (pair)
        TRACED("p3_fwd_col", X.stage, stream,
               (launch_pdl(k3_fwd_col_all<10, 8, true, H>, dim3(pairs, X.C / X.tc), dim3(512), smem, s, X, S, Y)));
    else
        TRACED("p3_fwd_col", X.stage, stream,
               (launch_pdl(k3_fwd_col_all<10, 8, false, H>, dim3(pairs, X.C / X.tc), dim3(512), smem, s, X, S, Y)));
}

int p3_launch_fwd_col(const Geo3 &X, const Operands &S, int pairs, u32 *Y, void *stream, bool pair) {
    if (int e = p3_prepare_kernels()) return e;
    const dim3 grid(X.C / X.tc, pairs, 3);
    const size_t smem = col_smem3(X, pair);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem_all = smem + 2 * kColTabStride * sizeof(uint2);
    if (X.logR == 10 && X.tc == 8 && X.rof4R) {
        if (X.head == 4)
            p3_fwd_all<4>(X, S, pairs, Y, stream, pair, smem_all);
        else
            p3_fwd_all<2>(X, S, pairs, Y, stream, pair, smem_all);
    } else {
        if (X.head != 4) return (int)cudaErrorInvalidValue;  // short transforms use the primes below 2^28
        if (pair)
            TRACED("p3_fwd_col", X.stage, stream,
                   (launch_pdl(k3_fwd_col<true, 0, 0, 4>, grid, dim3(kColThreads), smem, s, X, S, Y)));
        else
            TRACED("p3_fwd_col", X.stage, stream,
                   (launch_pdl(k3_fwd_col<false, 0, 0, 4>, grid, dim3(kColThreads), smem, s, X, S, Y)));
    }
    return (int)cudaGetLastError();
}

template <int MODE>
static int p3_row_launch(const Geo3 &X, const u32 *Y, u32 *S3, u32 *spec, cudaStream_t s, void *stream) {
    const dim3 grid(X.R, 3);
    const size_t smem = row_smem3(X);
    const char *name = MODE == 1 ? "p3_row_store" : "p3_row_mac";
#define P3_ROW(A, L, H)                                                                                     \
    do {                                                                                                    \
        if (X.head != (u32)(H)) return (int)cudaErrorInvalidValue;                                          \
        TRACED(name, X.stage, stream,                                                                       \
               (launch_pdl(k3_row_mac<A, L, MODE, H>, grid, dim3(X.C / A), smem, s, X, Y, S3, spec)));      \
    } while (0)
    switch (X.logC) {
    case 10: P3_ROW(8, 10, 4); break;
    case 11: P3_ROW(8, 11, 4); break;
    case 12:
        if (X.head == 4)
            P3_ROW(8, 12, 4);
        else
            P3_ROW(8, 12, 2);
        break;
    case 13: P3_ROW(8, 13, 2); break;
    case 14: P3_ROW(16, 14, 2); break;
    default:
        if (X.C > 8192) return (int)cudaErrorInvalidValue;
        P3_ROW(8, 0, 4);
    }
#undef P3_ROW
    return 0;
}

// mode 0: pairs (spec unused); 1: store the single operands' spectra to
// spec; 2: single operands times the spectra stored in spec.
int p3_launch_row_mac(const Geo3 &X, const u32 *Y, u32 *S3, void *stream, int mode, u32 *spec) {
    if (int e = p3_prepare_kernels()) return e;
    cudaStream_t s = (cudaStream_t)stream;
    int e = 0;
    if (mode == 0)
        e = p3_row_launch<0>(X, Y, S3, spec, s, stream);
    else if (mode == 1)
        e = p3_row_launch<1>(X, Y, S3, spec, s, stream);
    else
        e = p3_row_launch<2>(X, Y, S3, spec, s, stream);
    return e ? e : (int)cudaGetLastError();
}

int p3_launch_inv_col(const Geo3 &X, u32 *S3, u64 *zero_out, u64 zero_words, void *stream) {
    if (int e = p3_prepare_kernels()) return e;
    const dim3 grid(X.C / X.tc, 3);
    const size_t smem = col_smem3(X, false);
    cudaStream_t s = (cudaStream_t)stream;
    if (X.logR == 10 && X.tc == 8) {
        if (X.head == 4)
            TRACED("p3_inv_col", X.stage, stream,
                   (launch_pdl(k3_inv_col<10, 8, 4>, grid, dim3(kColThreads), smem, s, X, S3, zero_out, zero_words)));
        else
            TRACED("p3_inv_col", X.stage, stream,
                   (launch_pdl(k3_inv_col<10, 8, 2>, grid, dim3(kColThreads), smem, s, X, S3, zero_out, zero_words)));
    } else {
        if (X.head != 4) return (int)cudaErrorInvalidValue;
        TRACED("p3_inv_col", X.stage, stream,
               (launch_pdl(k3_inv_col<0, 0, 4>, grid, dim3(kColThreads), smem, s, X, S3, zero_out, zero_words)));
    }
    return (int)cudaGetLastError();
}

// Fused digit gather and carry of a stage whose chunks are wide (the parallel
// carry): output bits y zeroed beforehand (by the inverse column pass).
template <int NT>
static void p3_resolve_nt(const Geo3 &X, const u32 *S3, const CarryDev &cd, const u64 *c_src, u64 c_base, u64 *y,
                          void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const u32 nctas = (u32)((cd.nchunks + NT - 2) / (NT - 1));
    if (X.stage == 0) {
        TRACED("p3_resolve_a", 0, stream,
               (launch_pdl(k3_resolve_a<true, NT>, dim3(nctas), dim3(NT), 0, s, X, S3, cd, c_src, c_base, y)));
        TRACED("p3_resolve_c", 0, stream,
               (launch_pdl(k3_resolve_c<true, NT>, dim3(nctas), dim3(NT), 0, s, cd, nctas, y)));
    } else {
        TRACED("p3_resolve_a", 1, stream,
               (launch_pdl(k3_resolve_a<false, NT>, dim3(nctas), dim3(NT), 0, s, X, S3, cd, c_src, c_base, y)));
        TRACED("p3_resolve_c", 1, stream,
               (launch_pdl(k3_resolve_c<false, NT>, dim3(nctas), dim3(NT), 0, s, cd, nctas, y)));
    }
}

static int p3_launch_resolve(const Geo3 &X, const u32 *S3, const CarryDev &cd, const u64 *c_src, u64 c_base, u64 *y,
                             void *stream) {
    // 256-thread CTAs while they number at least 64; 64-thread CTAs below
    if (cd.nchunks >= 64 * 255)
        p3_resolve_nt<256>(X, S3, cd, c_src, c_base, y, stream);
    else
        p3_resolve_nt<64>(X, S3, cd, c_src, c_base, y, stream);
    return (int)cudaGetLastError();
}

int p3_launch_digits(const Geo3 &X, const u32 *S3, u64 *z, u64 npad, const u64 *c_src, u64 c_base, u64 *zero_out,
                     u64 zero_words, void *stream) {
    const u32 threads = 256;
    const u64 blocks = (std::max(npad, zero_words) + threads - 1) / threads;
    cudaStream_t s = (cudaStream_t)stream;
    if (X.stage == 0)
        TRACED("p3_digits", X.stage, stream,
               (launch_pdl(k3_digits<true>, dim3((unsigned)blocks), dim3(threads), 0, s, X, S3, z, npad, c_src, c_base,
                           zero_out, zero_words)));
    else
        TRACED("p3_digits", X.stage, stream,
               (launch_pdl(k3_digits<false>, dim3((unsigned)blocks), dim3(threads), 0, s, X, S3, z, npad, c_src, c_base,
                           zero_out, zero_words)));
    return (int)cudaGetLastError();
}

int p3_launch_fill_ctw(u32 logR, u32 logC, u32 h, const u32 *lo, const u32 *hi, u32 p, uint2 *out, void *stream) {
    k3_fill_ctw<<<152 * 8, 256, 0, (cudaStream_t)stream>>>(logR, logC, h, lo, hi, p, out);
    return (int)cudaGetLastError();
}

static int p3_launch_fill_split(u32 logC, u32 logT, u32 h, bool b_table, const u32 *lo, const u32 *hi, u32 p,
                                uint2 *out, void *stream) {
    k3_fill_split<<<152 * 2, 256, 0, (cudaStream_t)stream>>>(logC, logT, h, b_table, lo, hi, p, out);
    return (int)cudaGetLastError();
}

// ----------------------------------------------------------------- host plan --

namespace {

struct PrimeSet {
    u32 p[3];
    u32 maxlog;  // 2^maxlog divides every p - 1
    u32 head;    // 2^head p < 2^32: the lazy-reduction headroom of the butterflies
};
// Transforms up to 2^21: the three largest primes below 2^28 with 2^21 | p - 1
// (product 2^83.6; values may grow to 16p between reductions); 2^22: the
// three largest below 2^28 with 2^22 | p - 1 (product 2^82.4, headroom 16p as
// well).  2^23: the three largest below 2^30 with 2^23 | p - 1 (below 2^28
// there is only one); 2^24: the three below 2^30 with 2^24 | p - 1 (the only
// ones); both with headroom 4p.
const PrimeSet kSetA4 = {{257949697u, 249561089u, 230686721u}, 21, 4};
const PrimeSet kSetA4b = {{230686721u, 167772161u, 163577857u}, 22, 4};
const PrimeSet kSetA = {{998244353u, 754974721u, 469762049u}, 23, 2};
const PrimeSet kSetB = {{754974721u, 469762049u, 167772161u}, 24, 2};

const PrimeSet &prime_set(u32 logT) {
    return logT <= kSetA4.maxlog ? kSetA4 : logT <= kSetA4b.maxlog ? kSetA4b : logT <= kSetA.maxlog ? kSetA : kSetB;
}

u32 powmod(u64 b, u64 e, u32 p) {
    u64 r = 1;
    b %= p;
    while (e) {
        if (e & 1) r = r * b % p;
        b = b * b % p;
        e >>= 1;
    }
    return (u32)r;
}
u32 invmod(u64 a, u32 p) { return powmod(a % p, p - 2, p); }

u32 primitive_root(u32 p) {
    std::vector<u32> f;
    u32 m = p - 1;
    for (u32 d = 2; (u64)d * d <= m; d++)
        if (m % d == 0) {
            f.push_back(d);
            while (m % d == 0) m /= d;
        }
    if (m > 1) f.push_back(m);
    for (u32 g = 2;; g++) {
        bool ok = true;
        for (u32 q : f) ok = ok && powmod(g, (p - 1) / q, p) != 1;
        if (ok) return g;
    }
}

uint2 shoup_pair(u32 w, u32 p) { return make_uint2(w, (u32)(((u64)w << 32) / p)); }

u32 inv2_32(u32 p) {  // p^-1 mod 2^32 (p odd), Newton: each step doubles the correct bits
    u32 x = p;
    for (int i = 0; i < 5; i++) x *= 2u - p * x;
    return x;
}

struct Choice {
    u32 logT = 0, b = 0;
    const PrimeSet *ps = nullptr;
};

// Smallest transform (2^8 .. 2^24) and digit size for operands of G bits and
// K products: K M (2^b - 1)^2 < p0 p1 p2 with M b >= G; for Eq. 2 (ring) the
// top carry chunk must span >= 64 bits whenever the parallel carry runs.
bool choose(uint64_t G, uint64_t K, bool ring, Choice *out) {
    for (u32 l = 8; l <= 24; l++) {
        // at 2^22 the primes below 2^30 (a larger product) serve the operands
        // whose bound the primes below 2^28 cannot meet, before a longer transform
        const PrimeSet *cand[2] = {&prime_set(l), l == kSetA4b.maxlog ? &kSetA : nullptr};
        for (const PrimeSet *pc : cand) {
            if (!pc) continue;
            const PrimeSet &ps = *pc;
            const unsigned __int128 P = (unsigned __int128)ps.p[0] * ps.p[1] * ps.p[2];
            const u64 M = 1ULL << (l - 1);
            const u64 bmin = std::max<u64>(1, (G + M - 1) / M);
            for (u64 b = bmin; b <= 30; b++) {
                const unsigned __int128 m = ((unsigned __int128)1 << b) - 1;
                if ((unsigned __int128)K * M * m * m >= P) break;
                const u64 nd = (G + b - 1) / b;
                const u64 nch = (nd + PA_CARRY_D - 1) / PA_CARRY_D;
                const bool parallel = nch >= PA_CARRY_T && b * PA_CARRY_D >= 64;
                if (ring && parallel && G - (nch - 1) * PA_CARRY_D * b < 64) continue;
                out->logT = l;
                out->b = (u32)b;
                out->ps = &ps;
                return true;
            }
        }
    }
    return false;
}

void geometry(Geo3 &X, const Choice &ch, uint64_t G, uint64_t K, u32 stage) {
    const u32 l = ch.logT;
    X.head = ch.ps->head;
    X.logT = l;
    X.T = 1ULL << l;
    X.M = X.T / 2;
    X.b = ch.b;
    X.G = G;
    X.nd = (G + ch.b - 1) / ch.b;
    X.K = (u32)K;
    X.stage = stage;
    X.logR = std::min<u32>(l / 2, 10);
    X.logC = l - X.logR;
    X.R = 1u << X.logR;
    X.C = 1u << X.logC;
    // tile width 8: 32-byte row segments, and the padded addressing of pxc()
    X.tc = 8;
}

// Round twiddle table of a length-2^l transform with root w (see Geo3).
std::vector<uint2> round_table(u32 w, u32 l, u32 p, u32 *rof) {
    std::vector<u32> pw(1u << l);
    u64 a = 1;
    for (size_t e = 0; e < pw.size(); e++, a = a * w % p) pw[e] = (u32)a;
    std::vector<uint2> t;
    const u32 nr = (l + 2) / 3, ns0 = l - 3 * (nr - 1);
    u32 s0 = 0;
    for (u32 rd = 0; rd < nr; rd++) {
        const u32 ns = rd ? 3 : ns0, stride = 1u << (l - s0 - ns);
        rof[rd] = (u32)t.size();
        for (u32 lo = 0; lo < stride; lo++)
            for (u32 sg = 0; sg < ns; sg++)
                for (u32 jj = 0; jj < (1u << (ns - 1 - sg)); jj++)
                    t.push_back(shoup_pair(pw[((lo + jj * stride) << (s0 + sg)) & ((1u << l) - 1)], p));
        s0 += ns;
    }
    return t;
}

uint64_t table_bytes(const Geo3 &X) { return 3ULL * (4 * X.R + 4 * X.C + 2 * X.T + 136 * X.C) * sizeof(uint2); }

}  // namespace

struct P3Plan {
    uint64_t n = 0, r = 0, k = 0;
    uint32_t gamma = 0;
    Geo3 mmh{}, mh{};
    DevAlloc mem;  // every device buffer and table of the plan
    uint64_t ws_bytes = 0;
    u32 *Y = nullptr, *S3 = nullptr;
    u64 *ybuf = nullptr, *tbuf = nullptr, *H = nullptr;
    unsigned char *cstate = nullptr, *cta_state = nullptr, *cta_cin = nullptr;
    int *flags = nullptr;
    size_t flags_bytes = 0;
    // seed reuse: spectra of a_1..a_k ([prime][i][T]) and b ([prime][T]), seed copy
    u32 *spec_a = nullptr, *spec_b = nullptr;
    u64 *seed_copy = nullptr;
    bool prepared = false;
    // Toeplitz hashing: output blocks and key segments of rb bits, the seed
    // shifted up by rb zero bits (pseed)
    bool toep = false;
    uint64_t rb = 0, nblk = 0;
    u64 *pseed = nullptr;
    // Eq. 4's seed operand b is transformed on `side` while the Eq. 2 stage runs
    // (fork / join events); its column pass writes Yb (3 x 2 T_mh words, the column
    // layout of a stage with one pair), its row pass the spectrum bspec (3 T_mh)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    u32 *Yb = nullptr, *bspec = nullptr;
    ~P3Plan() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        mem.release();
    }
    void *alloc(size_t bytes, int *err) {
        void *p = mem.take(bytes, err);
        if (p) ws_bytes += bytes;
        return p;
    }
};

namespace {

// Twiddle tables and constants of one stage; tables are shared with `other`
// when both stages use the same transform shape.
int build_tables(P3Plan *pl, Geo3 &X, const PrimeSet &ps, const Geo3 *other) {
    for (int j = 0; j < 3; j++) {
        const u32 p = ps.p[j];
        X.p[j] = p;
        X.pinv[j] = inv2_32(p);
        X.red[j] = make_uint2(1u, (u32)((1ULL << 32) / p));
        X.scale[j] = shoup_pair((u32)((u64)powmod(2, 32, p) * invmod(X.T, p) % p), p);
    }
    const u32 p0 = ps.p[0], p1 = ps.p[1], p2 = ps.p[2];
    X.p01 = (u64)p0 * p1;
    X.c12 = shoup_pair(invmod(p0, p1), p1);
    X.p0m2 = shoup_pair(p0 % p2, p2);
    X.c3 = shoup_pair(invmod((u64)p0 * p1 % p2, p2), p2);
    if (other && other->T == X.T && other->logR == X.logR && other->p[0] == X.p[0] && other->twR[0]) {
        for (int j = 0; j < 3; j++) {
            X.twR[j] = other->twR[j];
            X.itwR[j] = other->itwR[j];
            X.twC[j] = other->twC[j];
            X.itwC[j] = other->itwC[j];
            X.ctw[j] = other->ctw[j];
            X.ictw[j] = other->ictw[j];
            X.ctwA[j] = other->ctwA[j];
            X.ctwB[j] = other->ctwB[j];
        }
        for (int rd = 0; rd < 6; rd++) {
            X.rofR[rd] = other->rofR[rd];
            X.rofC[rd] = other->rofC[rd];
        }
        X.rof4R = other->rof4R;
        X.rof4Ri = other->rof4Ri;
        return PA_OK;
    }
    int err = PA_OK;
    const u32 l = X.logT, h = (l + 1) / 2;
    std::vector<u32> lo(1u << h), hi(1u << (l - h));
    u32 *dlo = (u32 *)pl->alloc(lo.size() * 4, &err), *dhi = (u32 *)pl->alloc(hi.size() * 4, &err);
    for (int j = 0; j < 3 && !err; j++) {
        const u32 p = ps.p[j], g = primitive_root(p);
        const u32 wT = powmod(g, (p - 1) >> l, p);
        for (int dir = 0; dir < 2 && !err; dir++) {
            const u32 w = dir ? invmod(wT, p) : wT;
            const u32 wR = powmod(w, X.C, p), wC = powmod(w, X.R, p);
            std::vector<uint2> tR = round_table(wR, X.logR, p, X.rofR), tC = round_table(wC, X.logC, p, X.rofC);
            if (dir == 1 && X.logR == 10) {
                // inverse of the 4-stage round (stages 0-3 of the inverse column pass)
                X.rof4Ri = (u32)tR.size();
                std::vector<u32> pw(X.R);
                u64 a4 = 1;
                for (u32 e = 0; e < X.R; e++, a4 = a4 * wR % p) pw[e] = (u32)a4;
                for (u32 lo = 0; lo < 64; lo++)
                    for (u32 sg = 0; sg < 4; sg++)
                        for (u32 jj = 0; jj < (8u >> sg); jj++) tR.push_back(shoup_pair(pw[((lo + jj * 64) << sg) % X.R], p));
            }
            if (dir == 0 && X.logR == 10) {
                // 4-stage first round of the column kernel: per lo < 64, stage sg's twiddles
                // omega_R^((lo + jj 64) 2^sg), jj < 2^(3 - sg)
                X.rof4R = (u32)tR.size();
                std::vector<u32> pw(X.R);
                u64 a4 = 1;
                for (u32 e = 0; e < X.R; e++, a4 = a4 * wR % p) pw[e] = (u32)a4;
                for (u32 lo = 0; lo < 64; lo++)
                    for (u32 sg = 0; sg < 4; sg++)
                        for (u32 jj = 0; jj < (8u >> sg); jj++) tR.push_back(shoup_pair(pw[((lo + jj * 64) << sg) % X.R], p));
                // the column kernel copies entries [rofR[2], rofR[2] + kColTab) in 16-byte pieces
                while (tR.size() < (size_t)X.rofR[2] + kColTab) tR.push_back(make_uint2(0u, 0u));
                if (tR.size() != (size_t)X.rofR[2] + kColTab || X.rofR[3] - X.rofR[2] != kColTabR3 ||
                    X.rof4R - X.rofR[2] != kColTab4 || (X.rofR[2] & 1))
                    err = PA_ERR_INVALID;
            }
            u64 a = 1;
            uint2 *dR = (uint2 *)pl->alloc(tR.size() * sizeof(uint2), &err);
            uint2 *dC = (uint2 *)pl->alloc(tC.size() * sizeof(uint2), &err);
            uint2 *dT = (uint2 *)pl->alloc(X.T * sizeof(uint2), &err);
            if (err) break;
            pl->mem.upload(dR, tR.data(), tR.size() * sizeof(uint2), &err);
            pl->mem.upload(dC, tC.data(), tC.size() * sizeof(uint2), &err);
            if (err) break;
            a = 1;
            for (size_t e = 0; e < lo.size(); e++, a = a * w % p) lo[e] = (u32)a;
            const u32 wh = powmod(w, 1ULL << h, p);
            a = 1;
            for (size_t e = 0; e < hi.size(); e++, a = a * wh % p) hi[e] = (u32)a;
            // on the plan's private stream: building a plan waits for nothing else on the device;
            // the stream orders the reuse of dlo / dhi by the next table
            pl->mem.upload(dlo, lo.data(), lo.size() * 4, &err);
            pl->mem.upload(dhi, hi.data(), hi.size() * 4, &err);
            if (!err && p3_launch_fill_ctw(X.logR, X.logC, h, dlo, dhi, p, dT, pl->mem.stream)) err = PA_ERR_CUDA;
            if (!err && dir == 0 && X.logR == 10) {
                uint2 *dA = (uint2 *)pl->alloc(128ULL * X.C * sizeof(uint2), &err);
                uint2 *dB = (uint2 *)pl->alloc(8ULL * X.C * sizeof(uint2), &err);
                if (!err && (p3_launch_fill_split(X.logC, X.logT, h, false, dlo, dhi, p, dA, pl->mem.stream) ||
                             p3_launch_fill_split(X.logC, X.logT, h, true, dlo, dhi, p, dB, pl->mem.stream)))
                    err = PA_ERR_CUDA;
                X.ctwA[j] = dA;
                X.ctwB[j] = dB;
            }
            if (err) break;
            (dir ? X.itwR : X.twR)[j] = dR;
            (dir ? X.itwC : X.twC)[j] = dC;
            (dir ? X.ictw : X.ctw)[j] = dT;
        }
    }
    return err;
}

}  // namespace

int p3_feasible(uint32_t gamma, uint64_t k, uint32_t *logT_mmh, uint32_t *logT_mh) {
    Choice c1, c2;
    if (!choose(gamma, k, true, &c1) || !choose(gamma, 1, false, &c2)) return PA_ERR_UNSUPPORTED;
    if (logT_mmh) *logT_mmh = c1.logT;
    if (logT_mh) *logT_mh = c2.logT;
    return PA_OK;
}

static void ws_parts(const Geo3 &A, const Geo3 &B, uint64_t k, uint64_t *total_no_tables) {
    const uint64_t Tm = std::max(A.T, B.T);
    const uint64_t nch = std::max((A.nd + 7) / 8, (B.nd + 7) / 8) + 1;
    uint64_t s = 0;
    s += 3 * std::max<uint64_t>(2 * k * A.T, 2 * B.T) * 4;  // Y (also the digit vector)
    s += 3 * Tm * 4;                                       // S3
    s += 2 * ((A.G + 63) / 64 + 2) * 8;                    // ybuf, tbuf
    s += nch * 9 + 2 * (nch / kResolveMinChunks + 2);      // carry state
    s += (4 + k) * sizeof(int);
    s += (3 * 2 + 3) * B.T * 4;  // Yb, bspec
    *total_no_tables = s;
}

uint64_t p3_plan_bytes(uint32_t gamma, uint64_t k) {
    Choice c1, c2;
    if (!choose(gamma, k, true, &c1) || !choose(gamma, 1, false, &c2)) return 0;
    Geo3 A{}, B{};
    geometry(A, c1, gamma, k, 0);
    geometry(B, c2, gamma, 1, 1);
    uint64_t s;
    ws_parts(A, B, k, &s);
    const bool shared = A.T == B.T && A.logR == B.logR && c1.ps == c2.ps;
    return s + table_bytes(A) + (shared ? 0 : table_bytes(B)) + 2 * (1ULL << ((std::max(A.logT, B.logT) + 1) / 2)) * 4;
}

int p3_plan_create(uint64_t n, uint64_t r, uint32_t gamma, uint64_t k, bool stream_ordered, P3Plan **out) {
    *out = nullptr;
    Choice c1, c2;
    if (!choose(gamma, k, true, &c1) || !choose(gamma, 1, false, &c2)) return PA_ERR_UNSUPPORTED;
    if (p3_prepare_kernels()) return PA_ERR_CUDA;
    P3Plan *pl = new (std::nothrow) P3Plan();
    if (!pl) return PA_ERR_NOMEM;
    if (pl->mem.init(stream_ordered)) {
        delete pl;
        return PA_ERR_CUDA;
    }
    pl->n = n;
    pl->r = r;
    pl->gamma = gamma;
    pl->k = k;
    geometry(pl->mmh, c1, gamma, k, 0);
    geometry(pl->mh, c2, gamma, 1, 1);
    int err = build_tables(pl, pl->mmh, *c1.ps, nullptr);
    if (!err) err = build_tables(pl, pl->mh, *c2.ps, &pl->mmh);
    const Geo3 &A = pl->mmh, &B = pl->mh;
    const uint64_t Tm = std::max(A.T, B.T);
    const uint64_t nch = std::max((A.nd + 7) / 8, (B.nd + 7) / 8) + 1;
    pl->Y = (u32 *)pl->alloc(3 * std::max<uint64_t>(2 * k * A.T, 2 * B.T) * 4, &err);
    pl->S3 = (u32 *)pl->alloc(3 * Tm * 4, &err);
    pl->ybuf = (u64 *)pl->alloc(((gamma + 63) / 64 + 2) * 8, &err);
    pl->tbuf = (u64 *)pl->alloc(((gamma + 63) / 64 + 2) * 8, &err);
    pl->H = (u64 *)pl->alloc(nch * 8, &err);
    pl->cstate = (unsigned char *)pl->alloc(nch, &err);
    pl->cta_state = (unsigned char *)pl->alloc(nch / kResolveMinChunks + 2, &err);
    pl->cta_cin = (unsigned char *)pl->alloc(nch / kResolveMinChunks + 2, &err);
    pl->flags_bytes = (4 + k) * sizeof(int);
    pl->flags = (int *)pl->alloc(pl->flags_bytes, &err);
    // the column pass lays operand i of prime j at (2 K j + i) T, K = 1 for Eq. 4
    pl->Yb = (u32 *)pl->alloc(3 * 2 * B.T * 4, &err);
    pl->bspec = (u32 *)pl->alloc(3 * B.T * 4, &err);
    if (!err && (cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking) ||
                 cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) ||
                 cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming)))
        err = PA_ERR_CUDA;
    if (!err) err = pl->mem.sync();  // the tables are filled
    if (err) {
        delete pl;
        return err;
    }
    pl->ws_bytes = pl->mem.bytes;  // workspace and tables
    *out = pl;
    return PA_OK;
}

void p3_plan_destroy(P3Plan *pl) { delete pl; }

void p3_plan_query(const P3Plan *pl, uint64_t *len_mmh, uint64_t *len_mh, uint64_t *ws_bytes) {
    if (len_mmh) *len_mmh = pl->mmh.T;
    if (len_mh) *len_mh = pl->mh.T;
    if (ws_bytes) *ws_bytes = pl->ws_bytes;
}

const Geo3 *p3_stage(const P3Plan *pl, int stage) { return stage ? &pl->mh : &pl->mmh; }

// The fused digit gather + carry runs where the parallel carry would (enough
// chunks, each spanning >= 64 bits); smaller vectors take the digit kernel and
// the one-CTA carry.
static bool p3_fused_carry(const Geo3 &X, const CarryDev &cd) {
    return cd.nchunks >= PA_CARRY_T && X.b * PA_CARRY_D >= 64;
}

static CarryDev p3_carry_dev(P3Plan *pl, const Geo3 &X, bool ring, int *allones) {
    CarryDev cd;
    cd.N = 1;
    cd.G = X.G;
    cd.logN = 0;
    cd.ub = X.b;
    cd.linear = ring ? 0 : 1;
    cd.nchunks = (X.nd + PA_CARRY_D - 1) / PA_CARRY_D;
    cd.H = pl->H;
    cd.state = pl->cstate;
    cd.cta_state = pl->cta_state;
    cd.cta_cin = pl->cta_cin;
    cd.allones = allones;
    return cd;
}

// Eq. 2: y = sum_i a_i x_i mod 2^gamma - 1 into y (gamma bits).  prep: the
// spectra of a_i come from the plan (seed reuse), only the x_i are transformed.
static int mmh_impl(P3Plan *pl, const u64 *key, const u64 *seed, u64 *y, bool canonical, void *stream, bool prep) {
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
    ops.mode = prep ? 3 : 0;
    const Geo3 &X = pl->mmh;
    if ((e = p3_launch_fwd_col(X, ops, (int)pl->k, pl->Y, stream, !prep))) return e;
    if ((e = p3_launch_row_mac(X, pl->Y, pl->S3, stream, prep ? 2 : 0, prep ? pl->spec_a : nullptr))) return e;
    const CarryDev cd = p3_carry_dev(pl, X, true, pl->flags + 1);
    const u64 npad = cd.nchunks * PA_CARRY_D;
    const u64 ywords = (pl->gamma + 63) / 64;
    if (p3_fused_carry(X, cd)) {
        if ((e = p3_launch_inv_col(X, pl->S3, y, ywords, stream))) return e;
        if ((e = p3_launch_resolve(X, pl->S3, cd, nullptr, 0, y, stream))) return e;
    } else {
        u64 *z = (u64 *)pl->Y;
        if ((e = p3_launch_inv_col(X, pl->S3, nullptr, 0, stream))) return e;
        if ((e = p3_launch_digits(X, pl->S3, z, npad, nullptr, 0, y, ywords, stream))) return e;
        if ((e = launch_carry_chunks(cd, npad, X.b * PA_CARRY_D >= 64, 0, z, y, ywords, stream, true, true))) return e;
    }
    if (canonical && (e = launch_canonical_zero(pl->flags + 1, y, ywords, stream, true))) return e;
    return 0;
}

// Eq. 4: out = ((b y + c) mod 2^gamma) >> (gamma - r), y from the plan's
// buffer.  prep: the spectrum of b comes from the plan, only y is transformed.
// Eq. 4: z from y and the seed.  spec: b's spectrum (seed reuse, or computed
// beside the Eq. 2 stage); null: b is transformed here with y.
static int mh_impl(P3Plan *pl, const u64 *seed, u64 *out, int *status, void *stream, const u32 *spec) {
    const bool prep = spec != nullptr;
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
    ops.mode = prep ? 5 : 1;
    const Geo3 &X = pl->mh;
    if ((e = p3_launch_fwd_col(X, ops, 1, pl->Y, stream, !prep))) return e;
    if ((e = p3_launch_row_mac(X, pl->Y, pl->S3, stream, prep ? 2 : 0, const_cast<u32 *>(spec)))) return e;
    const CarryDev cd = p3_carry_dev(pl, X, false, pl->flags + 2);
    const u64 npad = cd.nchunks * PA_CARRY_D;
    const u64 twords = (pl->gamma + 63) / 64;
    const u64 c_base = (pl->k + 1) * (u64)pl->gamma;
    if (p3_fused_carry(X, cd)) {
        if ((e = p3_launch_inv_col(X, pl->S3, pl->tbuf, twords, stream))) return e;
        if ((e = p3_launch_resolve(X, pl->S3, cd, seed, c_base, pl->tbuf, stream))) return e;
    } else {
        u64 *z = (u64 *)pl->Y;
        if ((e = p3_launch_inv_col(X, pl->S3, nullptr, 0, stream))) return e;
        if ((e = p3_launch_digits(X, pl->S3, z, npad, seed, c_base, pl->tbuf, twords, stream))) return e;
        if ((e = launch_carry_chunks(cd, npad, X.b * PA_CARRY_D >= 64, 1, z, pl->tbuf, twords, stream, true, true)))
            return e;
    }
    if ((e = launch_extract(pl->tbuf, pl->gamma, pl->r, pl->flags, pl->k, out, status, stream, true))) return e;
    return 0;
}

int p3_enqueue_mmh(P3Plan *pl, const u64 *key, const u64 *seed, u64 *y, bool canonical, void *stream) {
    return mmh_impl(pl, key, seed, y, canonical, stream, false);
}

// A whole block (Algorithm 1).  b's column and row transforms (Eq. 4) do not
// depend on y: for Eq. 4 transforms of 2^20 and 2^21 (whose single-pair
// column pass fills less than a wave) they run on the plan's side stream,
// forked from `stream` at the start and joined before Eq. 4, filling SMs the
// Eq. 2 kernels leave idle; Eq. 4 then transforms y alone and multiplies by
// the stored spectrum of b.  Shorter blocks (latency-bound) and longer ones
// (an Eq. 4 column pass of several waves, rows of 2^12 or more) keep the pair
// (y, b) in Eq. 4: measured faster there.
int p3_enqueue_hash(P3Plan *pl, const u64 *key, const u64 *seed, u64 *out, int *status, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int e;
    if (pl->mh.T < (1ULL << 20) || pl->mh.T > (1ULL << 21)) {
        if ((e = mmh_impl(pl, key, seed, pl->ybuf, false, stream, false))) return e;
        return mh_impl(pl, seed, out, status, stream, nullptr);
    }
    if ((e = cudaEventRecord(pl->ev_fork, s)) || (e = cudaStreamWaitEvent(pl->side, pl->ev_fork, 0))) return e;
    Geo3 Xb = pl->mh;
    Xb.stage = 2;  // traced as mh_b.*
    Operands ops;
    ops.pair0 = 0;
    ops.key = nullptr;
    ops.seed = seed;
    ops.y = nullptr;
    ops.y_zero = nullptr;
    ops.reload = pl->flags;
    ops.n = pl->n;
    ops.gamma = pl->gamma;
    ops.k = pl->k;
    ops.mode = 4;  // b
    if ((e = p3_launch_fwd_col(Xb, ops, 1, pl->Yb, pl->side, false))) return e;
    if ((e = p3_launch_row_mac(Xb, pl->Yb, nullptr, pl->side, 1, pl->bspec))) return e;
    if ((e = cudaEventRecord(pl->ev_join, pl->side))) return e;
    if ((e = mmh_impl(pl, key, seed, pl->ybuf, false, stream, false))) return e;
    if ((e = cudaStreamWaitEvent(s, pl->ev_join, 0))) return e;
    return mh_impl(pl, seed, out, status, stream, pl->bspec);
}

// Seed reuse: forward transforms (columns, then rows) of a_1..a_k and of b,
// their spectra kept in the plan with a copy of the seed (c is read from it).
int p3_seed_prepare(P3Plan *pl, const u64 *seed, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t sw = ((pl->k + 2) * pl->gamma + 63) / 64;
    if (!pl->spec_a || !pl->spec_b || !pl->seed_copy) {  // first call, or a retry after a failed allocation
        int err = PA_OK;
        if (!pl->spec_a) pl->spec_a = (u32 *)pl->alloc(3 * pl->k * pl->mmh.T * 4, &err);
        if (!pl->spec_b) pl->spec_b = (u32 *)pl->alloc(3 * pl->mh.T * 4, &err);
        if (!pl->seed_copy) pl->seed_copy = (u64 *)pl->alloc(sw * 8, &err);
        if (err) return err;
    }
    pl->prepared = false;
    int e;
    if ((e = cudaMemcpyAsync(pl->seed_copy, seed, sw * 8, cudaMemcpyDeviceToDevice, s))) return e;
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
    if ((e = p3_launch_fwd_col(pl->mmh, ops, (int)pl->k, pl->Y, stream, false))) return e;
    if ((e = p3_launch_row_mac(pl->mmh, pl->Y, pl->S3, stream, 1, pl->spec_a))) return e;
    ops.mode = 4;  // b
    if ((e = p3_launch_fwd_col(pl->mh, ops, 1, pl->Y, stream, false))) return e;
    if ((e = p3_launch_row_mac(pl->mh, pl->Y, pl->S3, stream, 1, pl->spec_b))) return e;
    pl->prepared = true;
    return 0;
}

int p3_hash_prepared(P3Plan *pl, const u64 *key, u64 *out, int *status, void *stream) {
    int e = mmh_impl(pl, key, pl->seed_copy, pl->ybuf, false, stream, true);
    if (!e) e = mh_impl(pl, pl->seed_copy, out, status, stream, pl->spec_b);
    return e;
}

bool p3_prepared(const P3Plan *pl) { return pl->prepared; }

// ------------------------------------------------------ Toeplitz hashing --
// The comparison scheme of Sec. 1 / Table 1 (Toeplitz hashing with the key
// split into segments): z = T x over GF(2), T[i][j] = s[i - j + n - 1].  With
// segments x_J of rb bits and output blocks z_I of rb bits, block (I, J) of T
// is Toeplitz, so z_I = sum_J w_IJ * x_J taken at positions rb - 1 .. 2 rb - 2
// and mod 2, w_IJ the 2 rb - 1 seed bits starting at n - rb + (I - J) rb (bits
// before 0 read as 0).  Each term is an exact integer convolution of 1-bit
// digits on the transforms of length 4 rb (both operands in the lower half),
// accumulated in the transform domain like the k products of Eq. 2; the
// coefficients (at most n) come back through the CRT and their parities are
// the output bits.
int p3_toeplitz_create(uint64_t n, uint64_t r, uint32_t rb_log, P3Plan **out) {
    *out = nullptr;
    if (rb_log < 6 || rb_log > 22) return PA_ERR_UNSUPPORTED;
    const uint64_t rb = 1ULL << rb_log, K = (n + rb - 1) / rb, nblk = (r + rb - 1) / rb;
    if (K > 65535) return PA_ERR_UNSUPPORTED;  // segments index the column grid
    if (p3_prepare_kernels()) return PA_ERR_CUDA;
    Choice ch;
    ch.logT = rb_log + 2;
    ch.b = 1;
    ch.ps = &prime_set(ch.logT);
    // coefficients are at most n (< every prime): exact
    P3Plan *pl = new (std::nothrow) P3Plan();
    if (!pl) return PA_ERR_NOMEM;
    if (pl->mem.init(false)) {
        delete pl;
        return PA_ERR_CUDA;
    }
    pl->n = n;
    pl->r = r;
    pl->k = K;
    pl->toep = true;
    pl->rb = rb;
    pl->nblk = nblk;
    geometry(pl->mmh, ch, 2 * rb, K, 0);
    int err = build_tables(pl, pl->mmh, *ch.ps, nullptr);
    const Geo3 &A = pl->mmh;
    pl->Y = (u32 *)pl->alloc(3 * 2 * K * A.T * 4, &err);
    pl->S3 = (u32 *)pl->alloc(3 * A.T * 4, &err);
    pl->pseed = (u64 *)pl->alloc(((n + r - 1 + rb + 63) / 64 + 1) * 8, &err);
    pl->flags_bytes = (4 + K) * sizeof(int);
    pl->flags = (int *)pl->alloc(pl->flags_bytes, &err);
    if (!err) err = pl->mem.sync();
    if (err) {
        delete pl;
        return err;
    }
    pl->ws_bytes = pl->mem.bytes;
    *out = pl;
    return PA_OK;
}

int p3_toeplitz_hash(P3Plan *pl, const u64 *key, const u64 *seed, u64 *out, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t n = pl->n, r = pl->r, rb = pl->rb;
    const uint64_t sw = (n + r - 1 + 63) / 64;
    int e;
    if ((e = cudaMemsetAsync(out, 0, ((r + 63) / 64) * 8, s))) return e;
    if ((e = cudaMemsetAsync(pl->pseed, 0, (rb / 64) * 8, s))) return e;
    if ((e = cudaMemcpyAsync(pl->pseed + rb / 64, seed, sw * 8, cudaMemcpyDeviceToDevice, s))) return e;
    if ((e = cudaMemsetAsync(pl->flags, 0, pl->flags_bytes, s))) return e;
    Operands ops;
    ops.pair0 = 0;
    ops.key = key;
    ops.seed = pl->pseed;
    ops.y = nullptr;
    ops.y_zero = nullptr;
    ops.reload = pl->flags;
    ops.n = n;
    ops.gamma = 2 * rb;
    ops.k = pl->k;
    ops.mode = 6;
    ops.rb = rb;
    ops.seed_bits = n + r - 1 + rb;
    const Geo3 &X = pl->mmh;
    for (uint64_t I = 0; I < pl->nblk; I++) {
        ops.blk = (u32)I;
        if ((e = p3_launch_fwd_col(X, ops, (int)pl->k, pl->Y, stream, true))) return e;
        if ((e = p3_launch_row_mac(X, pl->Y, pl->S3, stream))) return e;
        if ((e = p3_launch_inv_col(X, pl->S3, nullptr, 0, stream))) return e;
        const uint64_t nbits = std::min<uint64_t>(rb, r - I * rb);
        const unsigned blocks = (unsigned)((nbits + 255) / 256);
        TRACED("p3_toeplitz_bits", 0, stream,
               (launch_pdl(k3_toeplitz_bits, dim3(blocks), dim3(256), 0, s, X, (const u32 *)pl->S3, rb, I * rb, r,
                           reinterpret_cast<u32 *>(out))));
        if ((e = (int)cudaGetLastError())) return e;
    }
    return 0;
}

void p3_toeplitz_query(const P3Plan *pl, uint64_t *rb, uint64_t *segments, uint64_t *blocks) {
    if (rb) *rb = pl->rb;
    if (segments) *segments = pl->k;
    if (blocks) *blocks = pl->nblk;
}

int *p3_flags(P3Plan *pl) { return pl->flags; }
size_t p3_flags_bytes(const P3Plan *pl) { return pl->flags_bytes; }

}  // namespace pa
