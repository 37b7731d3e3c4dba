// Tensor-pipe peak probe (hz_tensor_peak): the rate at which one GB300 executes dense tcgen05
// MMAs of a given kind and shape when nothing else limits them.  The substitution kernels'
// roofline is stated against this measured rate.
//
// One block per SM; warp 0 allocates tensor memory, lane 0 issues `iters` MMAs (M = 128, N as
// requested, K = one instruction's worth: 8 for tf32, 16 for bf16) from operands that stay
// resident in shared memory, alternating between two accumulators, then commits them to an
// mbarrier and waits (bounded) until they have completed.  No global memory is touched on the
// way, so the rate is the tensor pipe's.  Operand values are small normal numbers (the rate does
// not depend on them).
#include <algorithm>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"

namespace hz {
namespace {

constexpr int PK_LBO = 128;   // bytes between the two core matrices along K
constexpr int PK_SBO = 256;   // bytes between 8-row groups (K = 32 bytes per row)

__device__ inline uint32_t pk_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t pk_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(PK_LBO >> 4) << 16;
    d |= (uint64_t)(PK_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version; no swizzle
    return d;
}

// A from tensor memory (address of the first of K columns holding the 128 x K operand, lane = row)
__device__ inline void pk_mma_tmem_a(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc));
}

template <int KIND>
__device__ inline void pk_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (KIND == 0) {
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                     :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                     :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

// KIND 0: tf32 x tf32 -> f32; 1: bf16 x bf16 -> f32; 2: tf32 with the A operand in tensor memory.
// Dynamic shared memory of the probe: operands and barrier use the first 12 KB; the rest only
// keeps a second block off the SM, so that every SM runs exactly one issuing block.
constexpr int PK_SMEM = 120 * 1024;

template <int KIND>
__global__ void __launch_bounds__(128, 1) k_tensor_peak(long long iters, int N, int* flag) {
    extern __shared__ __align__(1024) unsigned char pk_smem[];
    unsigned char* a_s = pk_smem;              // 128 rows x 32 bytes
    unsigned char* b_s = pk_smem + 4096;       // up to 256 rows x 32 bytes
    uint64_t& bar = *(uint64_t*)(pk_smem + 12288);
    uint32_t& tptr = *(uint32_t*)(pk_smem + 12296);
    const int t = threadIdx.x, w = t >> 5;
    // operands: 1/64 in every element (tf32: 0x3C800000; bf16 pairs: 0x3C80)
    const uint32_t v = KIND == 0 ? 0x3C800000u : 0x3C803C80u;
    for (int i = t; i < 128 * 8; i += blockDim.x) ((uint32_t*)a_s)[i] = v;
    for (int i = t; i < 256 * 8; i += blockDim.x) ((uint32_t*)b_s)[i] = v;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(pk_smem_u32(&tptr)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(pk_smem_u32(&bar)), "r"(1));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tptr;
    // KIND 2: the A operand (128 lanes x 8 columns of 1/64) sits in tensor memory after the two
    // accumulators (columns 256 + 8k .. for N <= 128; one accumulator of N = 256 ends at 256)
    const uint32_t a_col = 384u;
    if (KIND == 2) {
        const uint32_t taddr = tmem + ((uint32_t)(32 * w) << 16) + a_col;
        const uint32_t v1 = 0x3C800000u;
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                     :: "r"(taddr), "r"(v1), "r"(v1), "r"(v1), "r"(v1), "r"(v1), "r"(v1), "r"(v1), "r"(v1) : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    bool ok = true;
    if (t == 0) {
        const uint32_t fmt = KIND == 1 ? 1u : 2u;   // operand format: tf32 = 2 (kind::tf32), bf16 = 1 (kind::f16)
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24);
        const uint64_t ad = pk_desc(pk_smem_u32(a_s)), bd = pk_desc(pk_smem_u32(b_s));
        const uint32_t accw = N <= 128 ? 128u : 0u;   // second accumulator (N <= 128 only)
        for (long long i = 0; i < iters; ++i) {
            const uint32_t acc = (uint32_t)(i & 1) * accw;
            if (KIND == 2) pk_mma_tmem_a(tmem + acc, tmem + a_col, bd, idesc, i >= 2 ? 1u : 0u);
            else pk_mma<KIND>(tmem + acc, ad, bd, idesc, i >= 2 ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(pk_smem_u32(&bar)));
        // bounded wait for every issued MMA (polls and 10 s of wall time)
        unsigned long long t0 = 0;
        ok = false;
        for (long long it = 0; it < (1LL << 34); ++it) {
            uint32_t done;
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                         : "=r"(done) : "r"(pk_smem_u32(&bar)), "r"(0u) : "memory");
            if (done) { ok = true; break; }
            if ((it & 1023) == 1023) {
                unsigned long long now;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                if (t0 == 0) t0 = now;
                else if (now - t0 > 10000000000ull) break;
            }
        }
        if (!ok) atomicExch(flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

}  // namespace
}  // namespace hz

extern "C" hz_status hz_tensor_peak(int32_t kind, int32_t n, double seconds, double* tflops, double* ms) {
    using namespace hz;
    if ((kind < 0 || kind > 2) || (n != 64 && n != 128 && n != 256) || !(seconds > 0.0) || seconds > 30.0 ||
        !tflops)
        return HZ_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HZ_ERR_CUDA;
    }
    const int K = kind == 1 ? 16 : 8;
    const double flops_per_mma = 2.0 * 128.0 * n * K;
    int* flag = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hz_status st = HZ_OK;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return HZ_ERR_OOM;
    }
    cudaMemset(flag, 0, sizeof(int));
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (cudaFuncSetAttribute(k_tensor_peak<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, PK_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_tensor_peak<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, PK_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_tensor_peak<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PK_SMEM) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(flag);
        return HZ_ERR_CUDA;
    }
    auto run = [&](long long iters) -> float {
        cudaEventRecord(e0);
        if (kind == 0) k_tensor_peak<0><<<sms, 128, PK_SMEM>>>(iters, n, flag);
        else if (kind == 1) k_tensor_peak<1><<<sms, 128, PK_SMEM>>>(iters, n, flag);
        else k_tensor_peak<2><<<sms, 128, PK_SMEM>>>(iters, n, flag);
        g_launch_count.fetch_add(1, std::memory_order_relaxed);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        return t;
    };
    // calibrate the count on a short run, then one run of about `seconds`
    long long iters = 1 << 16;
    float t = run(iters);
    for (int k = 0; k < 4 && t < 50.f; ++k) {
        iters *= 8;
        t = run(iters);
    }
    iters = std::max<long long>(iters, (long long)((double)iters * seconds * 1e3 / std::max(t, 1e-3f)));
    t = run(iters);
    int hflag = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = HZ_ERR_CUDA;
    else if (hflag)
        st = HZ_ERR_TIMEOUT;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(flag);
    if (st != HZ_OK) return st;
    *tflops = flops_per_mma * (double)iters * sms / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return HZ_OK;
}
