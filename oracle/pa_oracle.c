/*
 * pa_oracle.c -- reference oracle for the MMH-MH privacy-amplification hash
 * of "An efficient hybrid hash based privacy amplification algorithm for QKD"
 * (arXiv 2105.13678).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * table or header with the CUDA library; the two are checked against each
 * other bit for bit.
 *
 * The oracle evaluates the paper's definitions directly, single-threaded, on
 * exact integers stored as little-endian arrays of 64-bit limbs:
 *
 *   step 0 (Sec. 4, Table 3): p = M_gamma = 2^gamma - 1 with gamma a Mersenne
 *       prime exponent, n = k * gamma.  Reading used here: gamma is the
 *       smallest known Mersenne exponent >= r + margin, k = ceil(n / gamma),
 *       the last segment is zero-padded at its high end.
 *   Algorithm 1, splitting: x = <x_1..x_k>, a = <a_1..a_k>, gamma-bit slices.
 *   Algorithm 1, reload rule: if some x_i = 2^gamma - 1 the key is reloaded;
 *       the oracle returns ORA_RELOAD and a zero output.
 *   Eq. 2 / Algorithm 1 (MMH): y = sum_i a_i * x_i mod p, the products
 *       taken as exact integers, one reduction mod p at the end.  The
 *       reduction uses the Mersenne identity of Sec. 3.1
 *       (x mod M_gamma == floor(x / 2^gamma) + x mod 2^gamma, applied until
 *       the value is below 2^gamma, then 2^gamma - 1 -> 0).
 *   Eq. 4 / Algorithm 1 (MH): z = ((b * y + c) mod 2^alpha) / 2^(alpha-beta)
 *       with alpha = gamma, beta = r, b forced odd (gcd(b, 2) = 1).
 *
 * Seed layout (reading of Algorithm 1's random numbers): (k + 2) * gamma bits;
 * a_i = bits [(i-1)gamma, i*gamma) reduced mod p, b = bits [k*gamma,
 * (k+1)gamma) with bit 0 set, c = bits [(k+1)gamma, (k+2)gamma).
 * Bit order everywhere: bit t of a string lives in word t/64 at position t%64.
 *
 * Large products use the schoolbook method (Knuth, TAOCP vol. 2, 4.3.1,
 * Algorithm M) below a limb threshold and textbook Karatsuba
 * (TAOCP 4.3.3) above it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORA_OK 0
#define ORA_RELOAD 1
#define ORA_ERR_INVALID (-1)
#define ORA_ERR_NOMEM (-2)

/* Exponents of the known Mersenne primes (the public list cited in Sec. 3.1). */
static const uint32_t ORA_MERSENNE[] = {
    2u,        3u,        5u,        7u,        13u,       17u,       19u,
    31u,       61u,       89u,       107u,      127u,      521u,      607u,
    1279u,     2203u,     2281u,     3217u,     4253u,     4423u,     9689u,
    9941u,     11213u,    19937u,    21701u,    23209u,    44497u,    86243u,
    110503u,   132049u,   216091u,   756839u,   859433u,   1257787u,  1398269u,
    2976221u,  3021377u,  6972593u,  13466917u, 20996011u, 24036583u, 25964951u,
    30402457u, 32582657u, 37156667u, 42643801u, 43112609u, 57885161u, 74207281u,
    77232917u, 82589933u, 136279841u};
#define ORA_N_MERSENNE (sizeof(ORA_MERSENNE) / sizeof(ORA_MERSENNE[0]))

int ora_mersenne_count(void) { return (int)ORA_N_MERSENNE; }
uint32_t ora_mersenne_at(int i) { return ORA_MERSENNE[i]; }

/* Step 0 (Sec. 4, Table 3): gamma = smallest exponent >= r + margin (or the
 * caller's exponent when gamma_override != 0), k = ceil(n / gamma). */
int ora_plan(uint64_t n, uint64_t r, uint32_t margin, uint32_t gamma_override,
             uint32_t *gamma_out, uint64_t *k_out) {
    if (n == 0 || r == 0 || !gamma_out || !k_out) return ORA_ERR_INVALID;
    uint32_t g = 0;
    if (gamma_override) {
        for (size_t i = 0; i < ORA_N_MERSENNE; i++)
            if (ORA_MERSENNE[i] == gamma_override) g = gamma_override;
        if (g == 0 || (uint64_t)g <= r) return ORA_ERR_INVALID;
    } else {
        uint64_t need = r + (uint64_t)margin;
        if (need <= r) need = r + 1; /* gamma > beta strictly (Algorithm 1 output) */
        for (size_t i = 0; i < ORA_N_MERSENNE; i++)
            if ((uint64_t)ORA_MERSENNE[i] >= need) { g = ORA_MERSENNE[i]; break; }
        if (g == 0) return ORA_ERR_INVALID;
    }
    *gamma_out = g;
    *k_out = (n + g - 1) / g;
    return ORA_OK;
}

/* ---------------------------------------------------------------- bits -- */

static size_t words_for(uint64_t bits) { return (size_t)((bits + 63) / 64); }

/* dst[0..dst_words) = the integer made of src bits [off, off+len); bits at or
 * beyond src_bits count as zero. */
static void bits_extract(uint64_t *dst, size_t dst_words, const uint64_t *src,
                         uint64_t src_bits, uint64_t off, uint64_t len) {
    memset(dst, 0, dst_words * sizeof(uint64_t));
    for (uint64_t t = 0; t < len; t += 64) {
        uint64_t pos = off + t;
        uint64_t v = 0;
        if (pos < src_bits) {
            uint64_t wi = pos >> 6;
            unsigned sh = (unsigned)(pos & 63);
            v = src[wi] >> sh;
            if (sh != 0 && (wi + 1) * 64 < src_bits) v |= src[wi + 1] << (64 - sh);
            uint64_t avail = src_bits - pos;
            if (avail < 64) v &= (1ULL << avail) - 1;
        }
        uint64_t take = len - t;
        if (take < 64) v &= (1ULL << take) - 1;
        dst[t >> 6] = v;
    }
}

/* ------------------------------------------------------------- bignums -- */

static size_t bn_len(const uint64_t *a, size_t n) {
    while (n > 0 && a[n - 1] == 0) n--;
    return n;
}

static uint64_t bn_bitlen(const uint64_t *a, size_t n) {
    n = bn_len(a, n);
    if (n == 0) return 0;
    return (uint64_t)(n - 1) * 64 + (64 - (uint64_t)__builtin_clzll(a[n - 1]));
}

/* x[0..nx) += y[0..ny), ny <= nx; returns the carry out of x. */
static uint64_t bn_add_into(uint64_t *x, size_t nx, const uint64_t *y, size_t ny) {
    uint64_t carry = 0;
    size_t i = 0;
    for (; i < ny; i++) {
        u128 s = (u128)x[i] + y[i] + carry;
        x[i] = (uint64_t)s;
        carry = (uint64_t)(s >> 64);
    }
    for (; carry && i < nx; i++) {
        x[i] += 1;
        carry = (x[i] == 0);
    }
    return carry;
}

/* x[0..nx) -= y[0..ny), requires x >= y. */
static void bn_sub_into(uint64_t *x, size_t nx, const uint64_t *y, size_t ny) {
    uint64_t borrow = 0;
    size_t i = 0;
    for (; i < ny; i++) {
        uint64_t yi = y[i];
        uint64_t d = x[i] - yi - borrow;
        borrow = (x[i] < yi) || (x[i] - yi < borrow);
        x[i] = d;
    }
    for (; borrow && i < nx; i++) {
        borrow = (x[i] == 0);
        x[i] -= 1;
    }
}

/* Schoolbook product, Knuth 4.3.1 Algorithm M: w[0..m+n) = u[0..m) * v[0..n). */
static void mul_school(uint64_t *w, const uint64_t *u, size_t m, const uint64_t *v, size_t n) {
    memset(w, 0, (m + n) * sizeof(uint64_t));
    for (size_t j = 0; j < n; j++) {
        uint64_t k = 0;
        for (size_t i = 0; i < m; i++) {
            u128 t = (u128)u[i] * v[j] + w[i + j] + k;
            w[i + j] = (uint64_t)t;
            k = (uint64_t)(t >> 64);
        }
        w[j + m] = k;
    }
}

static size_t g_kara_threshold = 32;

/* Karatsuba (Knuth 4.3.3): r[0..2n) = a[0..n) * b[0..n).  Splitting
 * a = a1*B^lo + a0, b = b1*B^lo + b0 (B = 2^64, lo = floor(n/2)):
 *   a*b = z2*B^(2lo) + z1*B^lo + z0, z0 = a0 b0, z2 = a1 b1,
 *   z1 = (a0 + a1)(b0 + b1) - z0 - z2.
 * ws must hold kara_ws(n) limbs. */
static size_t kara_ws(size_t n) {
    if (n < g_kara_threshold) return 0;
    size_t hi = n - n / 2;
    return 4 * hi + 4 + kara_ws(hi + 1);
}

static void mul_kara(uint64_t *r, const uint64_t *a, const uint64_t *b, size_t n, uint64_t *ws) {
    if (n < g_kara_threshold) {
        mul_school(r, a, n, b, n);
        return;
    }
    size_t lo = n / 2, hi = n - lo;
    uint64_t *sa = ws, *sb = ws + (hi + 1), *z1 = ws + 2 * (hi + 1), *rest = ws + 4 * (hi + 1);

    mul_kara(r, a, b, lo, rest);                       /* z0 -> r[0, 2lo)       */
    mul_kara(r + 2 * lo, a + lo, b + lo, hi, rest);    /* z2 -> r[2lo, 2n)      */

    memset(sa, 0, (hi + 1) * sizeof(uint64_t));        /* sa = a0 + a1          */
    memcpy(sa, a + lo, hi * sizeof(uint64_t));
    bn_add_into(sa, hi + 1, a, lo);
    memset(sb, 0, (hi + 1) * sizeof(uint64_t));        /* sb = b0 + b1          */
    memcpy(sb, b + lo, hi * sizeof(uint64_t));
    bn_add_into(sb, hi + 1, b, lo);

    mul_kara(z1, sa, sb, hi + 1, rest);                /* z1 = sa * sb          */
    bn_sub_into(z1, 2 * (hi + 1), r, 2 * lo);          /* z1 -= z0              */
    bn_sub_into(z1, 2 * (hi + 1), r + 2 * lo, 2 * hi); /* z1 -= z2              */
    bn_add_into(r + lo, 2 * n - lo, z1, bn_len(z1, 2 * (hi + 1)));
}

/* r[0..na+nb) = a * b.  method 0: schoolbook only, 1: Karatsuba above the
 * threshold (operands zero-padded to a common length). */
static int bn_mul(uint64_t *r, const uint64_t *a, size_t na, const uint64_t *b, size_t nb, int method) {
    if (na == 0 || nb == 0) {
        memset(r, 0, (na + nb) * sizeof(uint64_t));
        return ORA_OK;
    }
    if (method == 0) {
        mul_school(r, a, na, b, nb);
        return ORA_OK;
    }
    size_t n = na > nb ? na : nb;
    uint64_t *pa = calloc(n, sizeof(uint64_t)), *pb = calloc(n, sizeof(uint64_t));
    uint64_t *pr = calloc(2 * n, sizeof(uint64_t));
    size_t wsn = kara_ws(n) + 1;
    uint64_t *ws = calloc(wsn, sizeof(uint64_t));
    if (!pa || !pb || !pr || !ws) {
        free(pa); free(pb); free(pr); free(ws);
        return ORA_ERR_NOMEM;
    }
    memcpy(pa, a, na * sizeof(uint64_t));
    memcpy(pb, b, nb * sizeof(uint64_t));
    mul_kara(pr, pa, pb, n, ws);
    memcpy(r, pr, (na + nb) * sizeof(uint64_t));
    free(pa); free(pb); free(pr); free(ws);
    return ORA_OK;
}

/* In place: s[0..ns) <- s mod (2^gamma - 1), canonical in [0, 2^gamma - 1).
 * Sec. 3.1: x mod M_gamma == floor(x / 2^gamma) + x mod 2^gamma (a congruence;
 * applied until the value is below 2^gamma, then M_gamma itself maps to 0). */
static int bn_mod_mersenne(uint64_t *s, size_t ns, uint32_t gamma) {
    size_t gw = words_for(gamma);
    uint64_t *lo = calloc(ns + 1, sizeof(uint64_t)), *hi = calloc(ns + 1, sizeof(uint64_t));
    if (!lo || !hi) { free(lo); free(hi); return ORA_ERR_NOMEM; }
    while (bn_bitlen(s, ns) > gamma) {
        uint64_t bits = (uint64_t)ns * 64;
        bits_extract(lo, ns, s, bits, 0, gamma);
        bits_extract(hi, ns, s, bits, gamma, bits - gamma);
        bn_add_into(lo, ns, hi, ns);
        memcpy(s, lo, ns * sizeof(uint64_t));
    }
    /* s < 2^gamma now; s == 2^gamma - 1 (all ones) is p itself == 0 */
    int all_ones = 1;
    for (uint64_t t = 0; t < gamma && all_ones; t++)
        all_ones = (int)((s[t >> 6] >> (t & 63)) & 1);
    if (all_ones) memset(s, 0, ns * sizeof(uint64_t));
    (void)gw;
    free(lo); free(hi);
    return ORA_OK;
}

/* ------------------------------------------------------------ MMH, MH -- */

/* Algorithm 1, MMH part (Eq. 2): y = sum_{i=1..k} a_i x_i mod p.  key has n bits, seed
 * has (k+2)*gamma bits.  Writes y (ceil(gamma/64) words).  Returns ORA_RELOAD
 * if some x_i == 2^gamma - 1 (Algorithm 1 reload rule), y then unspecified. */
static int mmh(const uint64_t *key, uint64_t n, const uint64_t *seed, uint32_t gamma, uint64_t k,
               uint64_t *y) {
    size_t gw = words_for(gamma);
    size_t sw = 2 * gw + 2; /* room for sum of k products (< k * 2^(2 gamma)) */
    uint64_t seed_bits = (k + 2) * (uint64_t)gamma;
    uint64_t *x = calloc(gw, 8), *a = calloc(gw, 8), *prod = calloc(2 * gw, 8);
    uint64_t *s = calloc(sw + 2, 8);
    int rc = ORA_OK;
    if (!x || !a || !prod || !s) { rc = ORA_ERR_NOMEM; goto out; }
    /* k can exceed 2^64/2^(2gamma) only for absurd sizes; widen s for the carries */
    for (uint64_t i = 0; i < k; i++) {
        bits_extract(x, gw, key, n, i * (uint64_t)gamma, gamma);
        int all_ones = 1;
        for (uint64_t t = 0; t < gamma && all_ones; t++)
            all_ones = (int)((x[t >> 6] >> (t & 63)) & 1);
        if (all_ones) { rc = ORA_RELOAD; goto out; }
        bits_extract(a, gw, seed, seed_bits, i * (uint64_t)gamma, gamma);
        /* a_i in Z_p: the all-ones slice is p == 0 */
        bn_mod_mersenne(a, gw, gamma);
        rc = bn_mul(prod, a, gw, x, gw, 1);
        if (rc != ORA_OK) goto out;
        if (bn_add_into(s, sw + 2, prod, 2 * gw)) { rc = ORA_ERR_INVALID; goto out; }
    }
    rc = bn_mod_mersenne(s, sw + 2, gamma);
    if (rc != ORA_OK) goto out;
    memcpy(y, s, gw * sizeof(uint64_t));
out:
    free(x); free(a); free(prod); free(s);
    return rc;
}

/* Eq. 4 (Algorithm 1, MH part) with alpha = gamma, beta = r:
 * out = ((b * y + c) mod 2^gamma) >> (gamma - r), r bits, high bits zero. */
static int mh(const uint64_t *y, const uint64_t *seed, uint32_t gamma, uint64_t k, uint64_t r,
              uint64_t *out) {
    size_t gw = words_for(gamma);
    uint64_t seed_bits = (k + 2) * (uint64_t)gamma;
    uint64_t *b = calloc(gw, 8), *c = calloc(gw, 8), *t = calloc(2 * gw + 1, 8);
    int rc = ORA_OK;
    if (!b || !c || !t) { rc = ORA_ERR_NOMEM; goto out; }
    bits_extract(b, gw, seed, seed_bits, k * (uint64_t)gamma, gamma);
    b[0] |= 1; /* gcd(b, 2) = 1 */
    bits_extract(c, gw, seed, seed_bits, (k + 1) * (uint64_t)gamma, gamma);
    rc = bn_mul(t, b, gw, y, gw, 1);
    if (rc != ORA_OK) goto out;
    bn_add_into(t, 2 * gw + 1, c, gw);
    /* bits [gamma - r, gamma) of t; bits >= gamma are dropped (mod 2^gamma) */
    bits_extract(out, words_for(r), t, gamma, gamma - r, r);
out:
    free(b); free(c); free(t);
    return rc;
}

/* Full Algorithm 1.  key: ceil(n/64) words (bits >= n ignored); seed:
 * ceil((k+2)gamma/64) words; out: ceil(r/64) words; y_out (optional):
 * ceil(gamma/64) words receiving the MMH value y.  Returns ORA_OK,
 * ORA_RELOAD (out zero-filled) or a negative error. */
int ora_pa_hash(const uint64_t *key, uint64_t n, const uint64_t *seed, uint64_t r,
                uint32_t gamma, uint64_t k, uint64_t *out, uint64_t *y_out) {
    if (!key || !seed || !out || n == 0 || r == 0 || gamma < 2 || (uint64_t)gamma <= r || k == 0 ||
        k * (uint64_t)gamma < n)
        return ORA_ERR_INVALID;
    size_t gw = words_for(gamma);
    uint64_t *y = calloc(gw, 8);
    if (!y) return ORA_ERR_NOMEM;
    memset(out, 0, words_for(r) * sizeof(uint64_t));
    int rc = mmh(key, n, seed, gamma, k, y);
    if (rc == ORA_OK) rc = mh(y, seed, gamma, k, r, out);
    if (rc != ORA_OK) memset(out, 0, words_for(r) * sizeof(uint64_t));
    if (y_out) memcpy(y_out, y, gw * sizeof(uint64_t));
    free(y);
    return rc;
}

/* Stand-alone pieces, exported for the oracle's own pin tests. */
int ora_mul(const uint64_t *a, size_t na, const uint64_t *b, size_t nb, uint64_t *r, int method) {
    return bn_mul(r, a, na, b, nb, method);
}

int ora_mod_mersenne(uint64_t *s, size_t ns, uint32_t gamma) { return bn_mod_mersenne(s, ns, gamma); }

int ora_mmh(const uint64_t *key, uint64_t n, const uint64_t *seed, uint32_t gamma, uint64_t k,
            uint64_t *y) {
    return mmh(key, n, seed, gamma, k, y);
}

int ora_mh(const uint64_t *y, const uint64_t *seed, uint32_t gamma, uint64_t k, uint64_t r,
           uint64_t *out) {
    memset(out, 0, words_for(r) * sizeof(uint64_t));
    return mh(y, seed, gamma, k, r, out);
}

void ora_set_karatsuba_threshold(size_t limbs) { g_kara_threshold = limbs < 4 ? 4 : limbs; }

/* ----------------------------------------------------- Toeplitz hashing -- */
/* The comparison scheme of Sec. 1 / Table 1: Toeplitz-hashing privacy
 * amplification, z = T x over GF(2) with T the r x n Toeplitz matrix whose
 * entries are constant along diagonals, T[i][j] = s[i - j + n - 1], drawn
 * from a seed s of n + r - 1 bits (s[0] is T[0][n - 1], s[n + r - 2] is
 * T[r - 1][0]).  Reading used: that diagonal convention (the paper fixes
 * none; any fixed one gives the same family); key, seed and output bit order
 * as everywhere (bit t of a string is bit t % 64 of word t / 64).  Plain
 * double loop: z_i = XOR_j T[i][j] x_j. */
static int bit_at(const uint64_t *w, uint64_t t) { return (int)((w[t >> 6] >> (t & 63)) & 1u); }

int ora_toeplitz(const uint64_t *key, uint64_t n, const uint64_t *seed, uint64_t r, uint64_t *out) {
    if (!key || !seed || !out || n == 0 || r == 0) return ORA_ERR_INVALID;
    memset(out, 0, words_for(r) * sizeof(uint64_t));
    for (uint64_t i = 0; i < r; i++) {
        int acc = 0;
        for (uint64_t j = 0; j < n; j++) acc ^= bit_at(key, j) & bit_at(seed, i - j + n - 1);
        if (acc) out[i >> 6] |= 1ULL << (i & 63);
    }
    return ORA_OK;
}

/* Selected output bits of the same product: out_bits[q] = z_(idx[q]). */
int ora_toeplitz_bits(const uint64_t *key, uint64_t n, const uint64_t *seed, uint64_t r, const uint64_t *idx,
                      uint64_t count, uint8_t *out_bits) {
    if (!key || !seed || !idx || !out_bits || n == 0 || r == 0) return ORA_ERR_INVALID;
    for (uint64_t q = 0; q < count; q++) {
        const uint64_t i = idx[q];
        if (i >= r) return ORA_ERR_INVALID;
        int acc = 0;
        for (uint64_t j = 0; j < n; j++) acc ^= bit_at(key, j) & bit_at(seed, i - j + n - 1);
        out_bits[q] = (uint8_t)acc;
    }
    return ORA_OK;
}
