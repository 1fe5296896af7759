// Throughput of the scan's arithmetic on one SM sub-partition: how many cycles 16 independent
// operations of each kind take per warp when two warps share a scheduler (the occupancy of the
// scan kernels), and the same for one Gray step's mix of the scan (adds, 3-input mins over the
// columns, the running minimum).  It measures the roofline the scan is bound by: which
// operations share a pipe and what one operation costs.  Not part of the library.
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

namespace {
constexpr int kN = 16;  // independent chains per thread (the scan's columns per thread)

__device__ __forceinline__ float fadd(float a, float b) { float d; asm("add.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); return d; }
__device__ __forceinline__ float fmin2(float a, float b) { float d; asm("min.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); return d; }
__device__ __forceinline__ float fmin3(float a, float b, float c) { float d; asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c)); return d; }
__device__ __forceinline__ int iadd(int a, int b) { int d; asm("add.s32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
__device__ __forceinline__ void fadd2(float &x, float &y, float a, float b)
{
    asm("{\n\t.reg .b64 p, q;\n\tmov.b64 p, {%0, %1};\n\tmov.b64 q, {%2, %3};\n\tadd.rn.f32x2 p, p, q;\n\tmov.b64 {%0, %1}, p;\n\t}"
                 : "+f"(x), "+f"(y) : "f"(a), "f"(b));
}

// MODE: 0 FADD, 1 FMNMX (2 inputs), 2 FMNMX3, 3 FADD2 (pairs), 4 IADD (eight pairs of chains that
// feed each other: integer adds of one chain would fold), 5 IMNMX3 (__vimin3_s32),
// 6 VIMNMX3 on u16x2, 7 the FP32-lane step (16 adds, one pair in four as FADD2, 3-input min
// tree, running minimum), 8 the int32 step (16 IADD, __vimin3_s32 tree), 9 the packed step (16
// 32-bit adds, __vimin3_u16x2 tree, lane combine).
template <int MODE>
__global__ void __launch_bounds__(128, 2) probe(float *out, int iters, float s)
{
    float v[kN], c[kN], e[kN];
    int iv[kN], ic[kN];
    unsigned uv[kN];
    for (int i = 0; i < kN; ++i) {
        v[i] = threadIdx.x * 1e-3f + i;
        c[i] = -i * s;
        e[i] = i * s;
        iv[i] = threadIdx.x + i;
        ic[i] = i - 7;
        uv[i] = 0x40004000u + i;
    }
    float red = 1e30f;
    int ired = 1 << 30;
    for (int it = 0; it < iters; ++it) {
        if constexpr (MODE == 0) {
#pragma unroll
            for (int i = 0; i < kN; ++i) v[i] = fadd(v[i], c[i]);
        } else if constexpr (MODE == 1) {
#pragma unroll
            for (int i = 0; i < kN; ++i) v[i] = fmin2(v[i], c[i]);
        } else if constexpr (MODE == 2) {
#pragma unroll
            for (int i = 0; i < kN; ++i) v[i] = fmin3(v[i], c[i], e[i]);
        } else if constexpr (MODE == 3) {
#pragma unroll
            for (int i = 0; i < kN; i += 2) fadd2(v[i], v[i + 1], c[i], c[i + 1]);
        } else if constexpr (MODE == 4) {
            // pairs of chains feed each other, so no run of adds folds into one
#pragma unroll
            for (int i = 0; i < kN / 2; ++i) {
                iv[i] = iadd(iv[i], iv[i + kN / 2]);
                iv[i + kN / 2] = iadd(iv[i + kN / 2], iv[i]);
            }
        } else if constexpr (MODE == 5) {
#pragma unroll
            for (int i = 0; i < kN; ++i) iv[i] = __vimin3_s32(iv[i], ic[i], it);
        } else if constexpr (MODE == 6) {
#pragma unroll
            for (int i = 0; i < kN; ++i) uv[i] = __vimin3_u16x2(uv[i], (unsigned)ic[i], (unsigned)it);
        } else if constexpr (MODE == 7) {
#pragma unroll
            for (int i = 0; i < kN; i += 2) {
                if (i % 8 == 0) {
                    fadd2(v[i], v[i + 1], c[i], c[i + 1]);
                } else {
                    v[i] = fadd(v[i], c[i]);
                    v[i + 1] = fadd(v[i + 1], c[i + 1]);
                }
            }
            float m[6];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = fmin3(v[3 * q], v[3 * q + 1], v[3 * q + 2]);
            m[5] = v[15];
            red = fmin2(red, fadd(fmin2(fmin3(m[0], m[1], m[2]), fmin3(m[3], m[4], m[5])), s));
        } else if constexpr (MODE == 8) {
#pragma unroll
            for (int i = 0; i < kN; ++i) iv[i] = iadd(iv[i], ic[i]);
            int m[6];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = __vimin3_s32(iv[3 * q], iv[3 * q + 1], iv[3 * q + 2]);
            m[5] = iv[15];
            ired = min(ired, iadd(min(__vimin3_s32(m[0], m[1], m[2]), __vimin3_s32(m[3], m[4], m[5])), it));
        } else {
#pragma unroll
            for (int i = 0; i < kN; ++i) uv[i] = (unsigned)iadd((int)uv[i], ic[i]);
            unsigned m[6];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = __vimin3_u16x2(uv[3 * q], uv[3 * q + 1], uv[3 * q + 2]);
            m[5] = uv[15];
            const unsigned w = __vminu2(__vimin3_u16x2(m[0], m[1], m[2]), __vimin3_u16x2(m[3], m[4], m[5]));
            ired = min(ired, iadd((int)min(w & 0xffffu, w >> 16), it));
        }
    }
    float acc = red + (float)ired;
    for (int i = 0; i < kN; ++i)
        acc += v[i] + e[i] + (float)iv[i] + (float)uv[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int MODE>
float time_mode(int blocks, float *out, int iters)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
        cudaEventRecord(a);
        probe<MODE><<<blocks, 128>>>(out, iters, 1e-7f);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}
}  // namespace

int main(int argc, char **argv)
{
    const double clock_hz = argc > 1 ? std::atof(argv[1]) * 1e6 : 2.07e9;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) {
        std::printf("no CUDA device\n");
        return 1;
    }
    const int blocks = 2 * sms;  // two blocks of four warps per SM: two warps per scheduler
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * 128) != cudaSuccess) {
        std::printf("allocation failed\n");
        return 1;
    }
    const int iters = 1 << 15;
    const char *names[] = {"FADD", "FMNMX (2 inputs)", "FMNMX3 (3 inputs)", "FADD2 (16 elements = 8 pairs)", "IADD",
                           "IMNMX3 (__vimin3_s32)", "VIMNMX3 u16x2", "FP32-lane Gray step", "int32 Gray step",
                           "packed 16-bit Gray step"};
    float ms[10];
    ms[0] = time_mode<0>(blocks, out, iters);
    ms[1] = time_mode<1>(blocks, out, iters);
    ms[2] = time_mode<2>(blocks, out, iters);
    ms[3] = time_mode<3>(blocks, out, iters);
    ms[4] = time_mode<4>(blocks, out, iters);
    ms[5] = time_mode<5>(blocks, out, iters);
    ms[6] = time_mode<6>(blocks, out, iters);
    ms[7] = time_mode<7>(blocks, out, iters);
    ms[8] = time_mode<8>(blocks, out, iters);
    ms[9] = time_mode<9>(blocks, out, iters);
    const cudaError_t err = cudaDeviceSynchronize();
    // warp-iterations each scheduler executes: blocks x 4 warps x iters / (SMs x 4 schedulers)
    const double per_smsp = (double)blocks * 4 * iters / (sms * 4.0);
    std::printf("SMs %d, clock %.0f MHz, 2 warps per scheduler, 16 independent operations per warp-iteration\n", sms,
                clock_hz / 1e6);
    for (int m = 0; m < 10; ++m)
        std::printf("%-32s %8.3f ms  %6.2f cycles per warp-iteration per scheduler\n", names[m], ms[m],
                    ms[m] * 1e-3 * clock_hz / per_smsp);
    std::printf("status %s\n", cudaGetErrorString(err));
    cudaFree(out);
    return err == cudaSuccess ? 0 : 1;
}
