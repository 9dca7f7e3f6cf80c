// gl_device.cuh -- device arithmetic in F_q, q = 2^64 - 2^32 + 1, on 32-bit
// limbs with PTX carry chains.
//
// Representation: any 64-bit value x stands for x mod q ("lazy": values in
// [q, 2^64) are allowed everywhere inside the transforms).  Reductions use
// 2^64 = 2^32 - 1 (mod q) and 2^96 = -1 (mod q).  The carry chains keep the
// integer ALU pipe short and put the multiply-adds on the FMA pipe.
#pragma once
#include <stdint.h>

namespace pa {

typedef unsigned long long u64;
typedef unsigned int u32;

__device__ __forceinline__ u32 lo32(u64 x) { return (u32)x; }
__device__ __forceinline__ u32 hi32(u64 x) { return (u32)(x >> 32); }
__device__ __forceinline__ u64 mk64(u32 lo, u32 hi) { return ((u64)hi << 32) | lo; }

// a + b (mod q), a, b < 2^64.  A carry out of bit 64 adds 2^32 - 1; that add
// can itself carry only once more.
__device__ __forceinline__ u64 gd_add(u64 a, u64 b) {
    u32 s0, s1;
    asm("{\n\t"
        ".reg .u32 c;\n\t"
        "add.cc.u32 %0, %2, %4;\n\t"
        "addc.cc.u32 %1, %3, %5;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "mad.lo.cc.u32 %0, c, 0xFFFFFFFF, %0;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "mad.lo.cc.u32 %0, c, 0xFFFFFFFF, %0;\n\t"
        "addc.u32 %1, %1, 0;\n\t"
        "}"
        : "=&r"(s0), "=&r"(s1)
        : "r"(lo32(a)), "r"(hi32(a)), "r"(lo32(b)), "r"(hi32(b)));
    return mk64(s0, s1);
}

// a - b (mod q), a, b < 2^64.  A borrow subtracts 2^32 - 1 (the borrow mask
// 0xFFFFFFFF is that constant); that subtraction can borrow only once more.
__device__ __forceinline__ u64 gd_sub(u64 a, u64 b) {
    u32 d0, d1;
    asm("{\n\t"
        ".reg .u32 m;\n\t"
        "sub.cc.u32 %0, %2, %4;\n\t"
        "subc.cc.u32 %1, %3, %5;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, m;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, m;\n\t"
        "subc.u32 %1, %1, 0;\n\t"
        "}"
        : "=&r"(d0), "=&r"(d1)
        : "r"(lo32(a)), "r"(hi32(a)), "r"(lo32(b)), "r"(hi32(b)));
    return mk64(d0, d1);
}

// a * b (mod q), a, b < 2^64, result < 2^64.  The 128-bit product
// p3:p2:p1:p0 (32-bit limbs) is p1:p0 + p2 (2^32 - 1) - p3 (mod q):
//   t = p1:p0 - p3        (a borrow subtracts 2^32 - 1; no second borrow)
//   r = t + p2 (2^32 - 1) (a carry adds 2^32 - 1; no second carry)
__device__ __forceinline__ u64 gd_mul(u64 a, u64 b) {
    u32 r0, r1;
    asm("{\n\t"
        ".reg .u32 p0, p1, p2, p3, m;\n\t"
        "mul.lo.u32 p0, %2, %4;\n\t"
        "mul.hi.u32 p1, %2, %4;\n\t"
        "mad.lo.cc.u32 p1, %2, %5, p1;\n\t"
        "madc.hi.u32 p2, %2, %5, 0;\n\t"
        "mad.lo.cc.u32 p1, %3, %4, p1;\n\t"
        "madc.hi.cc.u32 p2, %3, %4, p2;\n\t"
        "addc.u32 p3, 0, 0;\n\t"
        "mad.lo.cc.u32 p2, %3, %5, p2;\n\t"
        "madc.hi.u32 p3, %3, %5, p3;\n\t"
        "sub.cc.u32 %0, p0, p3;\n\t"
        "subc.cc.u32 %1, p1, 0;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, m;\n\t"
        "subc.u32 %1, %1, 0;\n\t"
        "mad.lo.cc.u32 %0, p2, 0xFFFFFFFF, %0;\n\t"
        "madc.hi.cc.u32 %1, p2, 0xFFFFFFFF, %1;\n\t"
        "addc.u32 m, 0, 0;\n\t"
        "mad.lo.cc.u32 %0, m, 0xFFFFFFFF, %0;\n\t"
        "addc.u32 %1, %1, 0;\n\t"
        "}"
        : "=&r"(r0), "=&r"(r1)
        : "r"(lo32(a)), "r"(hi32(a)), "r"(lo32(b)), "r"(hi32(b)));
    return mk64(r0, r1);
}

// d * w (mod q) for a digit d < 2^32 and any w < 2^64: the 96-bit product
// p2:p1:p0 is p1:p0 + p2 (2^32 - 1) (mod q); one carry adds 2^32 - 1.
__device__ __forceinline__ u64 gd_mul_small(u32 d, u64 w) {
    u32 r0, r1;
    asm("{\n\t"
        ".reg .u32 p0, p1, p2, t1, m;\n\t"
        "mul.lo.u32 p0, %2, %3;\n\t"
        "mul.hi.u32 t1, %2, %3;\n\t"
        "mad.lo.cc.u32 p1, %2, %4, t1;\n\t"
        "madc.hi.u32 p2, %2, %4, 0;\n\t"
        "mad.lo.cc.u32 %0, p2, 0xFFFFFFFF, p0;\n\t"
        "madc.hi.cc.u32 %1, p2, 0xFFFFFFFF, p1;\n\t"
        "addc.u32 m, 0, 0;\n\t"
        "mad.lo.cc.u32 %0, m, 0xFFFFFFFF, %0;\n\t"
        "addc.u32 %1, %1, 0;\n\t"
        "}"
        : "=&r"(r0), "=&r"(r1)
        : "r"(d), "r"(lo32(w)), "r"(hi32(w)));
    return mk64(r0, r1);
}

// Canonical representative in [0, q).
__device__ __forceinline__ u64 gd_canon(u64 x) { return x >= 0xFFFFFFFF00000001ULL ? x - 0xFFFFFFFF00000001ULL : x; }

}  // namespace pa
