// pa_tc_probe.cu -- the tensor-core limb-convolution alternative to the
// number-theoretic transforms, measured rather than assumed.
//
// An exact product of two integers cut into 8-bit limbs is a convolution of
// limb vectors.  With 32-limb blocks A_p, B_q (A = sum_p A_p 2^(256 p)), the
// block products are a matrix product: the 64 x 32 Toeplitz matrix of B_q
// (T[i][j] = B_q[i - j]) times a 32 x P matrix whose columns are the A_p;
// every entry is below 32 * 255^2 < 2^24, exact in int32.  An n-limb product
// thus costs 64 * 32 * (n / 32)^2 = 2 n^2 int8 multiply-adds.  GB300 (sm_103a)
// has no int8 kind of tcgen05.mma (ptxas rejects .kind::i8 for sm_103a), so
// the only int8 tensor path is the warp-level mma.sync; this file holds one
// exact tile of the block product and a throughput loop for that instruction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pa_gb300.h"

namespace {

// D (16 x 8, s32) += A (16 x 32, u8, row-major) * B (32 x 8, u8, column-major).
__device__ __forceinline__ void mma_u8(int (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp per tile: out[t] (64 x 8, row-major int32) = Toeplitz(bq[t]) (64 x 32)
// times a[t] (32 x 8, column c = limbs a[t][c * 32 .. c * 32 + 31]).
// Fragment layout of m16n8k32 (8-bit): lane = 4 g + q; A bytes (row g or g + 8,
// columns 4 q + 0..3 and 16 + 4 q + 0..3); B bytes (rows 4 q + 0..3 and
// 16 + 4 q + 0..3, column g); D (rows g, g + 8; columns 2 q, 2 q + 1).
__global__ void k_limbconv_tile(const uint8_t *__restrict__ bq, const uint8_t *__restrict__ a, int32_t *__restrict__ out,
                                int ntiles) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= ntiles) return;
    const uint8_t *B = bq + (size_t)warp * 32, *Am = a + (size_t)warp * 256;
    const int g = lane >> 2, q = lane & 3;
    unsigned bf[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        unsigned w = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) w |= (unsigned)Am[g * 32 + 16 * h + 4 * q + i] << (8 * i);
        bf[h] = w;
    }
#pragma unroll
    for (int mt = 0; mt < 4; mt++) {
        unsigned af[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int row = 16 * mt + g + ((r & 1) ? 8 : 0), col0 = ((r & 2) ? 16 : 0) + 4 * q;
            unsigned w = 0;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int s = row - (col0 + i);
                w |= (unsigned)((s >= 0 && s < 32) ? B[s] : 0) << (8 * i);
            }
            af[r] = w;
        }
        int d[4] = {0, 0, 0, 0};
        mma_u8(d, af, bf);
        int32_t *o = out + (size_t)warp * 512 + (16 * mt) * 8;
        o[g * 8 + 2 * q] = d[0];
        o[g * 8 + 2 * q + 1] = d[1];
        o[(g + 8) * 8 + 2 * q] = d[2];
        o[(g + 8) * 8 + 2 * q + 1] = d[3];
    }
}

// Throughput: every warp issues `iters` rounds of 8 independent m16n8k32 int8
// products on register operands; the accumulators are folded into `sink`.
__global__ void __launch_bounds__(256) k_mma_rate(uint64_t iters, int *sink) {
    unsigned af[4], bf[2];
#pragma unroll
    for (int r = 0; r < 4; r++) af[r] = 0x01010101u * (threadIdx.x + r);
    bf[0] = 0x02020202u;
    bf[1] = 0x03030303u;
    int d[8][4];
#pragma unroll
    for (int u = 0; u < 8; u++)
#pragma unroll
        for (int r = 0; r < 4; r++) d[u][r] = 0;
    for (uint64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) mma_u8(d[u], af, bf);
    }
    int s = 0;
#pragma unroll
    for (int u = 0; u < 8; u++) s += d[u][0] + d[u][1] + d[u][2] + d[u][3];
    if (s == 0x7FFFFFFF) *sink = s;  // keeps the loop; never true for these operands
}

}  // namespace

extern "C" {

int pa_tc_limbconv_tile(const uint8_t *bq, const uint8_t *a, int32_t *out, int ntiles, void *stream) {
    if (!bq || !a || !out || ntiles <= 0) return PA_ERR_INVALID;
    const int threads = 128, blocks = (ntiles * 32 + threads - 1) / threads;
    k_limbconv_tile<<<blocks, threads, 0, (cudaStream_t)stream>>>(bq, a, out, ntiles);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

int pa_tc_int8_rate(uint64_t iters, uint32_t ctas_per_sm, double *tops, double *ms) {
    if (!tops || !ms || iters == 0 || ctas_per_sm == 0) return PA_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) return PA_ERR_CUDA;
    int *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PA_OK;
    if (cudaMalloc(&sink, sizeof(int)) || cudaEventCreate(&e0) || cudaEventCreate(&e1)) rc = PA_ERR_CUDA;
    const unsigned blocks = (unsigned)sms * ctas_per_sm;
    if (!rc) {
        k_mma_rate<<<blocks, 256>>>(iters / 10 + 1, sink);  // warm-up
        cudaEventRecord(e0);
        k_mma_rate<<<blocks, 256>>>(iters, sink);
        cudaEventRecord(e1);
        float t = 0.f;
        if (cudaEventSynchronize(e1) || cudaEventElapsedTime(&t, e0, e1)) rc = PA_ERR_CUDA;
        const double ops = 2.0 * 16 * 8 * 32 * 8 * (double)iters * blocks * (256 / 32);
        *ms = t;
        *tops = ops / (t * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return rc;
}

}  // extern "C"
