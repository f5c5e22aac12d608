// mma_rate.cu -- the measured rate of dense tcgen05.mma of kind::f16 (fp16 x fp16 operands
// from shared memory, fp32 accumulator in tensor memory) on this GPU: the tensor peak that
// the tensor-core pointwise form is measured against.  GB300 (sm_103a) has no integer tensor
// MMA (ptxas rejects .kind::i8 for that target), so the 16-bit floating-point kinds are the
// only exact tensor path for modular limb products.
//
// One CTA per SM; one thread issues `iters` MMAs of 128 x N x 16 into one accumulator, commits
// them to an mbarrier, and the block waits (bounded: a wait that runs out sets the status and
// the block returns after a second bounded wait for the commit).  Operands are zeros: the
// rate does not depend on the values.  The host times the launch with CUDA events.
#include <cuda_runtime.h>

#include "common.cuh"
#include "pmat.h"

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no-swizzle shared-memory matrix descriptor: 8-row x 16-byte core matrices, LBO
// between the two K-adjacent ones of a 16-element K step, SBO between 8-row groups
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int polls)
{
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; it++)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(bar), "r"(parity));
    return done != 0;
}

__global__ void __launch_bounds__(128) k_mma_rate(int N, int iters, int *status)
{
    __shared__ __align__(1024) unsigned char op[4096 + 8192];   // A 128 x 16, B N x 16 (fp16)
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x;
    for (int x = tid; x < (int)sizeof(op) / 16; x += 128) ((uint4 *)op)[x] = make_uint4(0, 0, 0, 0);
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tbase;
    // D f32, A f16, B f16, both K-major; N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
    const uint64_t ad = desc(smem_addr(op), 128, 256), bd = desc(smem_addr(op + 4096), 128, 256);
    if (tid == 0) {
        for (int i = 0; i < iters; i++)
            asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(i));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_addr(&bar)));
    }
    bool ok = mbar_wait(smem_addr(&bar), 0, 1 << 26);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        if (tid == 0) atomicExch(status, PM_ETIMEOUT);
        mbar_wait(smem_addr(&bar), 0, 1 << 26);   // the commit, before the memory is freed
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace

extern "C" int pm_mma_rate(int device, int n_cols, int iters, double *tflops)
{
    if (!tflops || n_cols < 16 || n_cols > 256 || (n_cols & 15) || iters < 1 || iters > (1 << 20)) return PM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return PM_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PM_ECUDA;
    int *status = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = PM_OK;
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess || cudaMemset(status, 0, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess)
        rc = PM_ECUDA;
    float best = 0;
    for (int rep = 0; rc == PM_OK && rep < 4; rep++) {     // the first launch warms up
        cudaEventRecord(a, st);
        k_mma_rate<<<sms, 128, 0, st>>>(n_cols, iters, status);
        cudaEventRecord(b, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = PM_ECUDA; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && (best == 0 || ms < best)) best = ms;
    }
    int hs = 0;
    if (rc == PM_OK && cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = PM_ECUDA;
    if (rc == PM_OK && hs) rc = hs;
    if (rc == PM_OK) *tflops = 2.0 * 128 * n_cols * 16 * (double)iters * sms / (best * 1e-3) / 1e12;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (status) cudaFree(status);
    return rc;
}
