// rates_probe.cu -- throughput of the arithmetic units that an FP64 panel
// update could use on this GPU: SIMT FP64 fused multiply-add, the FP64
// tensor-core instruction mma.sync.m8n8k4.f64, the INT8 tensor-core
// instruction mma.sync.m16n8k32.s8 (the building block of integer-slice
// emulation of FP64 products), and, as yardsticks, SIMT FP32 and the BF16
// instruction mma.sync.m16n8k16.bf16.  Each kernel runs independent
// dependency chains per thread (enough instruction-level parallelism to fill
// the pipe) on every SM; the host times it with CUDA events.  Test
// infrastructure only (built by the test that uses it).
#include <cuda_runtime.h>
#include <cstdint>

namespace {

constexpr int kChains = 8;

__global__ void k_dfma(double* out, int iters, double a) {
    double x[kChains];
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, 1e-7);
    double s = 0;
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 123.456) out[0] = s;
}

__global__ void k_ffma(float* out, int iters, float a) {
    float x[kChains];
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, 1e-7f);
    float s = 0;
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 123.456f) out[0] = s;
}

// D(8x8) += A(8x4) B(4x8), FP64: per warp 2*8*8*4 = 512 flops
__global__ void k_dmma(double* out, int iters) {
    double a = 1.0 + threadIdx.x * 1e-6, b = 1.0 - threadIdx.x * 1e-6;
    double d[kChains][2];
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 0.0;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
    double s = 0;
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
    if (s == 123.456) out[0] = s;
}

// D(16x8) += A(16x32) B(32x8), s8 -> s32: per warp 2*16*8*32 = 8192 ops
__global__ void k_imma(int* out, int iters) {
    uint32_t a0 = 0x01010101u + threadIdx.x, a1 = a0 ^ 0x02020202u, a2 = a0 + 3, a3 = a1 + 5;
    uint32_t b0 = 0x01020304u ^ threadIdx.x, b1 = b0 + 7;
    int d[kChains][4];
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                         "{%0,%1,%2,%3};"
                         : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    int s = 0;
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == 123456) out[0] = s;
}

// D(16x8) += A(16x16) B(16x8), bf16 -> f32: per warp 2*16*8*16 = 4096 flops
__global__ void k_hmma(float* out, int iters) {
    uint32_t a0 = 0x3f803f80u, a1 = 0x3f813f81u, a2 = 0x3f823f82u, a3 = 0x3f833f83u;
    uint32_t b0 = 0x3f7f3f7fu, b1 = 0x3f7e3f7eu;
    float d[kChains][4];
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0.f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                         "{%8,%9}, {%0,%1,%2,%3};"
                         : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    float s = 0;
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == 123.456f) out[0] = s;
}

}  // namespace

// kind: 0 DFMA, 1 FFMA, 2 DMMA, 3 IMMA, 4 HMMA(bf16).  Returns the rate in
// tera-operations per second (a multiply-add counts as two), timed with CUDA
// events over `reps` launches after one warm-up launch; <0 on a CUDA error.
extern "C" double rates_probe(int kind, int reps) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) return -1;
    const int threads = 256, blocks = sms * 4, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double per_iter = 0;  // operations per launch-iteration per thread
    auto launch = [&]() {
        switch (kind) {
            case 0: k_dfma<<<blocks, threads>>>((double*)buf, iters, 0.999999); per_iter = 2.0 * kChains; break;
            case 1: k_ffma<<<blocks, threads>>>((float*)buf, iters, 0.999999f); per_iter = 2.0 * kChains; break;
            case 2: k_dmma<<<blocks, threads>>>((double*)buf, iters); per_iter = 512.0 / 32 * kChains; break;
            case 3: k_imma<<<blocks, threads>>>((int*)buf, iters); per_iter = 8192.0 / 32 * kChains; break;
            default: k_hmma<<<blocks, threads>>>((float*)buf, iters); per_iter = 4096.0 / 32 * kChains; break;
        }
    };
    launch();
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) return -2;
    const double ops = per_iter * iters * (double)threads * blocks * reps;
    return ops / (ms * 1e-3) / 1e12;
}
