// Peak-rate probes: the denominators of the roofline fractions the benchmark
// reports for kernels bound by FP32 or FP64 arithmetic or by the TF32 tensor
// pipe.  Each probe runs a dense stream of the one operation on every SM,
// with enough independent work per thread (or back-to-back MMAs) to keep the
// pipe full, and returns operations per second measured with CUDA events.
//   FP32 / FP64: 8 independent FMA chains per thread, 1024 threads, 4 blocks
//                per SM; 2 flops per FMA.
//   TF32:        one CTA per SM issues back-to-back tcgen05.mma kind::tf32
//                (M = 128, N = 256, K = 8, operands in shared memory,
//                accumulator in tensor memory); 2 M N K flops per MMA.
// The paper has no counterpart (it reports no hardware rates).
#include <cstdint>

#include "../../include/rks.h"
#include "common.cuh"
#include "kernels.h"

template <typename T>
__global__ void __launch_bounds__(1024) fma_probe_kernel(T *out, int iters, T x, T y) {
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int k = 0; k < 8; k++) a[k] = a[k] * x + y;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
    if (s == (T)12345.678) out[0] = s;  // keeps the chains live; never true for these inputs
}

#define PROBE_N 256
#define PROBE_K 8
#define PROBE_SPIN 4000000

__device__ __forceinline__ uint32_t probe_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(128, 1) tf32_probe_kernel(int iters, int *err) {
    __shared__ __align__(1024) float A[128 * PROBE_K];
    __shared__ __align__(1024) float B[PROBE_N * PROBE_K];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const int t = threadIdx.x;
    for (int i = t; i < 128 * PROBE_K; i += blockDim.x) A[i] = 1e-3f * (float)(i % 7);
    for (int i = t; i < PROBE_N * PROBE_K; i += blockDim.x) B[i] = 1e-3f * (float)(i % 5);
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(probe_smem(&slot)),
                     "r"(PROBE_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(probe_smem(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = slot;
    if (t == 0) {
        // K-major, no swizzle: cores of 8 rows x 16 B; the two K cores 128 B
        // apart, 8-row groups 256 B apart
        auto desc = [](uint32_t a) -> uint64_t {
            return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
                   ((uint64_t)1 << 46);
        };
        const uint64_t da = desc(probe_smem(A)), db = desc(probe_smem(B));
        const uint32_t id = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PROBE_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        for (int it = 0; it < iters; it++) {
            const uint32_t acc = it > 0;
            asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tm),
                         "l"(da), "l"(db), "r"(id), "r"(acc)
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         probe_smem(&bar))
                     : "memory");
    }
    uint32_t done = 0;
    for (int it = 0; it < PROBE_SPIN && !done; it++)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(probe_smem(&bar)), "r"(0u)
                     : "memory");
    if (!done) atomicOr(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (t < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(PROBE_N) : "memory");
}

int probe_rate(int kind, cudaStream_t s, double *ops_per_s) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    void *out = nullptr;
    int *err = nullptr;
    CUDA_OK(cudaMalloc(&out, 64));
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(out);
        return rks_cuda_fail(e, "probe", __FILE__, __LINE__);
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaMemsetAsync(err, 0, sizeof(int), s);
    double ops = 0.0;
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {  // first launch is the warm-up
        cudaEventRecord(a, s);
        if (kind == RKS_PROBE_FP32_FMA) {
            const int iters = 2048;
            fma_probe_kernel<float><<<4 * nsm, 1024, 0, s>>>((float *)out, iters, 0.999f, 1e-4f);
            ops = 2.0 * 16 * 8 * (double)iters * 1024 * 4 * nsm;
        } else if (kind == RKS_PROBE_FP64_FMA) {
            const int iters = 128;
            fma_probe_kernel<double><<<4 * nsm, 1024, 0, s>>>((double *)out, iters, 0.999, 1e-4);
            ops = 2.0 * 16 * 8 * (double)iters * 1024 * 4 * nsm;
        } else {
            const int iters = 20000;
            tf32_probe_kernel<<<nsm, 128, 0, s>>>(iters, err);
            ops = 2.0 * 128 * PROBE_N * PROBE_K * (double)iters * nsm;
        }
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    cudaFree(err);
    if (e != cudaSuccess) return rks_cuda_fail(e, "probe", __FILE__, __LINE__);
    if (herr) return RKS_EDEVICE;
    *ops_per_s = ops / (best * 1e-3);
    return RKS_OK;
}
