// tcgen05 building blocks shared by the tensor-core kernels (substitution and factorization):
// operand layout constants, shared-memory and instruction descriptors, TF32 splitting,
// cp.async copies, bounded mbarrier waits, tensor-memory loads and the complex split-TF32 MMA
// sequence of one pipeline stage.
//
// Operands are K-major core matrices without swizzle: a [rows x KC] operand of 4-byte elements
// stores 8-row x 16-byte core matrices, LBO bytes apart along K and SBO bytes apart along rows.
#pragma once

#include <cstdint>

#include "hz_internal.cuh"

namespace hz {
namespace tcc {

constexpr int KC = 16;                 // complex reduction indices per stage
constexpr int LBO = 128;               // bytes between core matrices along K
constexpr int SBO = (KC / 4) * 128;    // bytes between 8-row groups (K = 16 tf32 per row)
constexpr int MR = 128;                // complex output rows per work item (4 tiles)
constexpr int TROW = KC * 8 + 16;      // padded raw row (transposed tiles): 144 bytes
constexpr long long WAIT_LIMIT = 1LL << 26;            // polls of one mbarrier wait at most ...
constexpr unsigned long long WAIT_NS = 2000000000ull;  // ... and at most 2 s of wall time
constexpr int NLOAD = 128, NCONV = 256;                // loader and converter threads

__device__ __forceinline__ long long tri_idx(int rt, int ct) { return (long long)rt * (rt + 1) / 2 + ct; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(LBO >> 4) << 16;
    d |= (uint64_t)(SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; base offset 0; no swizzle
    return d;
}

// byte offset of (row, k) in a [rows x KC] K-major core-matrix operand (4-byte elements)
__device__ __forceinline__ int coff(int row, int k) { return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4; }

__device__ __forceinline__ float tf32_hi(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// 16-byte asynchronous global->shared copy; src_bytes = 0 zero-fills without reading
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of the given parity: gives up (false) after max_polls polls (the
// pipeline waits take the launch's limit; waits that drain a block's own MMAs keep WAIT_LIMIT),
// WAIT_NS of wall time, or as soon as another role of the block has raised *abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          long long max_polls = WAIT_LIMIT) {
    unsigned long long t0 = 0;
    for (long long it = 0; it < max_polls; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if ((it & 255) == 255) {
            if (*abort) return false;
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > WAIT_NS) break;
        }
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" :: "r"(smem_u32(b)) : "memory");
}
// arrive on b once all of this thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(b)));
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes (real and imaginary part)
__device__ __forceinline__ void tmem_ld16(uint32_t ar, uint32_t ai, uint32_t (&vr)[16], uint32_t (&vi)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]), "=r"(vr[7]),
                   "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]), "=r"(vr[12]), "=r"(vr[13]), "=r"(vr[14]), "=r"(vr[15])
                 : "r"(ar));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]), "=r"(vi[7]),
                   "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]), "=r"(vi[13]), "=r"(vi[14]), "=r"(vi[15])
                 : "r"(ai));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// MMA part of a stage (one thread): 2 x (4 or 12) MMAs of 8 complex reduction indices.  The
// converted operands of a stage sit at `base`: Ar_hi, Ar_lo, Ai_hi, Ai_lo (MR x KC each), then
// Xr_hi, Xr_lo, Xi_hi, Xi_lo (NT x KC each); the product is Y[MR x NT] = A X^T.
template <int NT, int SPLIT>
__device__ __forceinline__ void mma_stage(uint32_t base, uint32_t tm_r, uint32_t tm_i, bool first_stage) {
    constexpr int A_MAT = MR * KC * 4, X_MAT = NT * KC * 4;   // one real operand matrix of A / of X
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(MR >> 4) << 24);
    const uint32_t idesc_neg = idesc | (1u << 13);
#pragma unroll
    for (int ks = 0; ks < KC / 8; ++ks) {
        const uint32_t ko = ks * 2 * LBO;
        const uint64_t arh = smem_desc(base + 0 * A_MAT + ko), arl = smem_desc(base + 1 * A_MAT + ko);
        const uint64_t aih = smem_desc(base + 2 * A_MAT + ko), ail = smem_desc(base + 3 * A_MAT + ko);
        const uint32_t xb = base + 4 * A_MAT + ko;
        const uint64_t xrh = smem_desc(xb), xrl = smem_desc(xb + X_MAT);
        const uint64_t xih = smem_desc(xb + 2 * X_MAT), xil = smem_desc(xb + 3 * X_MAT);
        const uint32_t first = (first_stage && ks == 0) ? 0u : 1u;
        mma_tf32(tm_r, arh, xrh, idesc, first);      // Yr = Ar Xr - Ai Xi
        mma_tf32(tm_r, aih, xih, idesc_neg, 1u);
        mma_tf32(tm_i, aih, xrh, idesc, first);      // Yi = Ai Xr + Ar Xi
        mma_tf32(tm_i, arh, xih, idesc, 1u);
        if (SPLIT == 3) {                             // hi x lo and lo x hi terms
            mma_tf32(tm_r, arh, xrl, idesc, 1u);
            mma_tf32(tm_r, arl, xrh, idesc, 1u);
            mma_tf32(tm_r, aih, xil, idesc_neg, 1u);
            mma_tf32(tm_r, ail, xih, idesc_neg, 1u);
            mma_tf32(tm_i, aih, xrl, idesc, 1u);
            mma_tf32(tm_i, ail, xrh, idesc, 1u);
            mma_tf32(tm_i, arh, xil, idesc, 1u);
            mma_tf32(tm_i, arl, xih, idesc, 1u);
        }
    }
}


}  // namespace tcc
}  // namespace hz
