// Tensor-core (tcgen05) variant of the substitution products for complex64 factors.
//
// A block computes 128 complex output rows (four factor tile rows) x NT right-hand-side
// columns of one of the four node products of the substitution (see solve.cu), for the
// nodes whose products are large enough to fill it; smaller nodes of the same tree level run
// on the CUDA-core kernel in the same phase.
//
// The complex product Y = A X is four real products with two accumulators in tensor memory:
//     Yr = Ar Xr - Ai Xi,    Yi = Ai Xr + Ar Xi,
// (the minus sign through the instruction descriptor's negate-A bit).  Each real product runs
// in TF32 with a three-term split of both operands (a = a_hi + a_lo, x = x_hi + x_lo;
// a x ~ a_hi x_hi + a_hi x_lo + a_lo x_hi) and FP32 accumulation, which keeps every product at
// FP32-level accuracy (about 2^-21 relative): 12 MMAs (M = 128, N = NT, K = 8) per 8 complex
// reduction indices.  SPLIT = 1 keeps only a_hi x_hi (plain TF32, about 2^-11 relative; 4 MMAs);
// it is an option (HZ_PRECOND_SPLIT=1) for the local solves inside the preconditioner, whose
// accuracy changes how fast GMRES converges but not the solution it converges to.
//
// Warp-specialized pipeline (416 threads, 16 complex reduction indices per stage, two-deep
// rings of raw and converted buffers, every hand-off an mbarrier):
//   4 loader warps    : cp.async 16-byte copies of the factor tiles and vector rows into a raw
//                       buffer (masked rows / absent tiles zero-filled by the copy), completion
//                       signalled with cp.async.mbarrier.arrive;
//   8 converter warps : raw -> split hi/lo TF32 operands in the K-major core-matrix layout
//                       (no swizzle), 16-byte stores;
//   1 MMA warp        : one thread issues the 24 MMAs of a stage and commits them to the
//                       mbarrier that releases the converted buffer.
// The epilogue (converter warps) stages both accumulators from tensor memory (tcgen05.ld;
// lane = complex row) through shared memory and writes whole rows with 16-byte accesses: a
// task that covers the full reduction of its rows stores them, split reductions and the
// shared update rows of FB accumulate with vector atomics.  Every mbarrier wait is bounded and
// the outcome block-uniform; on timeout the block records an error flag, waits once more
// (bounded) for its own MMAs, frees its tensor memory and exits.
#include <algorithm>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"
#include "hz_solve.cuh"

namespace hz {

namespace {

enum { FA = 0, FB = 1, BA = 2, BB = 3 };

constexpr int KC = 16;                 // complex reduction indices per stage
constexpr int LBO = 128;               // bytes between core matrices along K
constexpr int SBO = (KC / 4) * 128;    // bytes between 8-row groups (K = 16 tf32 per row)
constexpr int MR = 128;                // complex output rows per block (4 tiles)
constexpr int TROW = KC * 8 + 16;      // padded raw row (transposed tiles): 144 bytes
constexpr long long WAIT_LIMIT = 1LL << 26;

__device__ inline long long tri_idx(int rt, int ct) { return (long long)rt * (rt + 1) / 2 + ct; }

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(LBO >> 4) << 16;
    d |= (uint64_t)(SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; base offset 0; no swizzle
    return d;
}

// byte offset of (row, k) in a [rows x KC] K-major core-matrix operand (4-byte elements)
__device__ inline int coff(int row, int k) { return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4; }

__device__ inline float tf32_hi(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// 16-byte asynchronous global->shared copy; src_bytes = 0 zero-fills without reading
__device__ inline void cp16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ inline void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

template <int NT> struct Layout {
    static constexpr int A_MAT = MR * KC * 4;            // one real operand matrix (8 KB)
    static constexpr int X_MAT = NT * KC * 4;
    static constexpr int CONV = 4 * A_MAT + 4 * X_MAT;   // Ar_h Ar_l Ai_h Ai_l  Xr_h Xr_l Xi_h Xi_l
    static constexpr int RAW_A = 4 * 32 * TROW;          // large enough for both raw tile layouts
    static constexpr int RAW_X = KC * NT * 8;
    static constexpr int RAW = RAW_A + RAW_X;
    static constexpr int TOTAL = 2 * CONV + 2 * RAW + 128;
};

// thread roles (warp-specialized): 4 loader warps, 8 converter warps, 1 MMA warp
constexpr int NLOAD = 128, NCONVT = 256, NTHREADS = NLOAD + NCONVT + 32;

__device__ inline void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count));
}
__device__ inline void mbar_arrive(uint64_t* b) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" :: "r"(smem_u32(b)) : "memory");
}
// arrive on b once all of this thread's earlier cp.async copies have landed
__device__ inline void cp_async_arrive(uint64_t* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(smem_u32(b)) : "memory");
}

template <int NT, int MODE, int SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1) k_subst_tc(const Task* __restrict__ tasks, const JobDev<float2>* __restrict__ jobs,
                                                          int ldc, int nchunks, int KS, int* flag) {
    using LY = Layout<NT>;
    constexpr bool TR = (MODE == BA || MODE == BB);  // factor tiles used transposed
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* conv = smem;
    unsigned char* raw = smem + 2 * LY::CONV;
    uint64_t* bars = (uint64_t*)(raw + 2 * LY::RAW);
    uint64_t* raw_full = bars + 0;    // [2] loaders' copies landed (count NLOAD)
    uint64_t* raw_empty = bars + 2;   // [2] converters done reading (count NCONVT)
    uint64_t* conv_full = bars + 4;   // [2] converted operands written (count NCONVT)
    uint64_t* conv_empty = bars + 6;  // [2] MMAs of the buffer done (tcgen05.commit)
    uint32_t* tptr = (uint32_t*)(bars + 8);

    const int chunk = blockIdx.x % nchunks;
    const Task tk = tasks[blockIdx.x / nchunks];
    const JobDev<float2> jb = jobs[tk.job];
    const NodeDev nd = jb.nodes[tk.node];
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const int col0 = chunk * NT;
    const int o0 = tk.tile;  // first of the four output tiles
    const int nout_t = (MODE == FB) ? nd.upd_t : nd.own_t;
    const int kbeg = tk.pad_;
    const int kend = min((MODE == FA) ? min(o0 + 4, nd.own_t) : ((MODE == BA) ? nd.upd_t : nd.own_t), kbeg + KS);
    const int nst = max(0, kend - kbeg) * 2;
    const float2* vec = (MODE == FA || MODE == BB) ? jb.acc : jb.x;
    const int* upd = jb.upd_idx + nd.upd_off;
    const int nrows_k = (MODE == BA) ? nd.nupd : nd.nown;   // valid vector rows
    const int mma_warp = (NLOAD + NCONVT) / 32;

    if (w == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tptr)), "r"(2 * NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(raw_full + b, NLOAD);
            mbar_init(raw_empty + b, NCONVT);
            mbar_init(conv_full + b, NCONVT);
            mbar_init(conv_empty + b, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tptr;
    const uint32_t tm_r = tmem, tm_i = tmem + NT;  // accumulators: real part cols [0, NT), imag [NT, 2NT)
    bool ok = true;

    if (t < NLOAD) {
        // ------------------------------------------------------------ loaders
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s & 1;
            if (s >= 2) ok = mbar_wait(smem_u32(raw_empty + slot), (uint32_t)(((s >> 1) - 1) & 1));
            if (!ok) break;
            unsigned char* rb = raw + slot * LY::RAW;
            const int kt = kbeg + (s >> 1), hk = s & 1;
#pragma unroll
            for (int i = 0; i < 8; ++i) {     // factor tiles: 1024 chunks of 16 bytes
                const int c = t + NLOAD * i;
                const int oi = c >> 8, q = c & 255;
                const int o = o0 + oi;
                bool exists = o < nout_t;
                if (MODE == FA) exists = exists && kt <= o;
                if (MODE == BB) exists = exists && kt >= o;
                long long toff = 0;
                if (exists) {
                    if (MODE == FA) toff = nd.linv_off + tri_idx(o, kt);
                    else if (MODE == FB) toff = nd.l21_off + (long long)o * nd.own_t + kt;
                    else if (MODE == BA) toff = nd.l21_off + (long long)kt * nd.own_t + o;
                    else toff = nd.linv_off + tri_idx(kt, o);
                }
                const float2* tl = jb.fac + toff * TILE2;
                uint32_t dst;
                const float2* src;
                if (!TR) {
                    dst = smem_u32(rb + oi * 4096 + q * 16);
                    src = tl + hk * KC * 32 + q * 2;
                } else {
                    const int r = q >> 3, j = q & 7;
                    dst = smem_u32(rb + oi * 32 * TROW + r * TROW + j * 16);
                    src = tl + 32 * r + hk * KC + j * 2;
                }
                cp16(dst, exists ? (const void*)src : (const void*)jb.fac, exists ? 16 : 0);
            }
            for (int c = t; c < KC * NT / 2; c += NLOAD) {  // vector rows: KC x NT, raw [k][n]
                const int k = c / (NT / 2), j = c % (NT / 2);
                const int rr = kt * TILE + hk * KC + k;
                const bool v = rr < nrows_k;
                long long row = 0;
                if (v) row = (MODE == BA) ? (long long)upd[rr] : (long long)(nd.own0 + rr);
                cp16(smem_u32(rb + LY::RAW_A + k * NT * 8 + j * 16), vec + row * ldc + col0 + 2 * j, v ? 16 : 0);
            }
            cp_async_arrive(raw_full + slot);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (t < NLOAD + NCONVT) {
        // ------------------------------------------------------------ converters
        const int ct = t - NLOAD;
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s & 1;
            ok = mbar_wait(smem_u32(raw_full + slot), (uint32_t)((s >> 1) & 1));
            if (ok && s >= 2) ok = mbar_wait(smem_u32(conv_empty + slot), (uint32_t)(((s >> 1) - 1) & 1));
            if (!ok) break;
            unsigned char* rb = raw + slot * LY::RAW;
            unsigned char* cv = conv + slot * LY::CONV;
#pragma unroll
            for (int i = 0; i < 2; ++i) {     // factor operand: 128 rows x 16 k, (row, 4 consecutive k)
                const int id = ct + NCONVT * i;
                const int row = id & 127, kq = id >> 7;
                const int oi = row >> 5, r = row & 31;
                float re[4], im[4];
                if (!TR) {
                    const float2* src = (const float2*)(rb + oi * 4096);
#pragma unroll
                    for (int j = 0; j < 4; ++j) { float2 a = src[(4 * kq + j) * 32 + r]; re[j] = a.x; im[j] = a.y; }
                } else {
                    const float4* src = (const float4*)(rb + oi * 32 * TROW + r * TROW + kq * 32);
                    float4 a0 = src[0], a1 = src[1];
                    re[0] = a0.x; im[0] = a0.y; re[1] = a0.z; im[1] = a0.w;
                    re[2] = a1.x; im[2] = a1.y; re[3] = a1.z; im[3] = a1.w;
                }
                float4 rh, ih;
                rh.x = tf32_hi(re[0]); rh.y = tf32_hi(re[1]); rh.z = tf32_hi(re[2]); rh.w = tf32_hi(re[3]);
                ih.x = tf32_hi(im[0]); ih.y = tf32_hi(im[1]); ih.z = tf32_hi(im[2]); ih.w = tf32_hi(im[3]);
                const int off = coff(row, 4 * kq);
                *(float4*)(cv + 0 * LY::A_MAT + off) = rh;
                *(float4*)(cv + 2 * LY::A_MAT + off) = ih;
                if (SPLIT == 3) {
                    *(float4*)(cv + 1 * LY::A_MAT + off) = make_float4(re[0] - rh.x, re[1] - rh.y, re[2] - rh.z, re[3] - rh.w);
                    *(float4*)(cv + 3 * LY::A_MAT + off) = make_float4(im[0] - ih.x, im[1] - ih.y, im[2] - ih.z, im[3] - ih.w);
                }
            }
            for (int id = ct; id < NT * 4; id += NCONVT) {   // vector operand: NT rows x 16 k
                const int n = id % NT, kq = id / NT;
                const float2* src = (const float2*)(rb + LY::RAW_A);
                float re[4], im[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) { float2 a = src[(4 * kq + j) * NT + n]; re[j] = a.x; im[j] = a.y; }
                float4 rh, ih;
                rh.x = tf32_hi(re[0]); rh.y = tf32_hi(re[1]); rh.z = tf32_hi(re[2]); rh.w = tf32_hi(re[3]);
                ih.x = tf32_hi(im[0]); ih.y = tf32_hi(im[1]); ih.z = tf32_hi(im[2]); ih.w = tf32_hi(im[3]);
                const int off = 4 * LY::A_MAT + coff(n, 4 * kq);
                *(float4*)(cv + off + 0 * LY::X_MAT) = rh;
                *(float4*)(cv + off + 2 * LY::X_MAT) = ih;
                if (SPLIT == 3) {
                    *(float4*)(cv + off + 1 * LY::X_MAT) = make_float4(re[0] - rh.x, re[1] - rh.y, re[2] - rh.z, re[3] - rh.w);
                    *(float4*)(cv + off + 3 * LY::X_MAT) = make_float4(im[0] - ih.x, im[1] - ih.y, im[2] - ih.z, im[3] - ih.w);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(raw_empty + slot);
            mbar_arrive(conv_full + slot);
        }
    } else if (l == 0) {
        // ------------------------------------------------------------ MMA issuer
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(MR >> 4) << 24);
        const uint32_t idesc_neg = idesc | (1u << 13);
        for (int s = 0; s < nst && ok; ++s) {
            const int cb = s & 1;
            ok = mbar_wait(smem_u32(conv_full + cb), (uint32_t)((s >> 1) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(conv + cb * LY::CONV);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t ko = ks * 2 * LBO;
                const uint64_t arh = smem_desc(base + 0 * LY::A_MAT + ko), arl = smem_desc(base + 1 * LY::A_MAT + ko);
                const uint64_t aih = smem_desc(base + 2 * LY::A_MAT + ko), ail = smem_desc(base + 3 * LY::A_MAT + ko);
                const uint32_t xb = base + 4 * LY::A_MAT + ko;
                const uint64_t xrh = smem_desc(xb), xrl = smem_desc(xb + LY::X_MAT);
                const uint64_t xih = smem_desc(xb + 2 * LY::X_MAT), xil = smem_desc(xb + 3 * LY::X_MAT);
                const uint32_t first = (s == 0 && ks == 0) ? 0u : 1u;
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
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(conv_empty + cb)));
        }
    }

    // every role arrives here (their waits are bounded); make the outcome block-uniform
    ok = __syncthreads_and(ok) != 0;
    bool done = true;
    if (nst > 0) {
        const bool got = mbar_wait(smem_u32(conv_empty + ((nst - 1) & 1)), (uint32_t)(((nst - 1) >> 1) & 1));
        done = __syncthreads_and(got) != 0;
    }
    if (!ok || !done) {
        if (t == 0) atomicExch(flag, 1);
        ok = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue (converter warps), in two passes so that global memory sees whole rows:
    //  (1) tensor memory -> shared staging tile [128 rows][NT + 2] (warp w reads lanes
    //      32 (w % 4) .. +31 = output tile o0 + w % 4, column half by the converter-warp index);
    //  (2) each converter warp writes 16 staged rows, lane = pair of columns (16-byte accesses).
    //  A task that covers the whole reduction of its outputs is their only writer and stores;
    //  split reductions (and FB, whose update rows are shared between nodes) accumulate.
    if (ok && t >= NLOAD && t < NLOAD + NCONVT) {
        constexpr int SP = NT + 2;           // staging pitch (complex): 16-byte rows, odd in 16-byte units
        float2* stg = (float2*)smem;         // operand and raw buffers are free once the MMAs are done
        const int cw = (t - NLOAD) >> 5;     // converter warp 0..7
        {
            const int q4 = w & 3;
            const int rl = 32 * q4 + l;
            const int cbeg = (cw >> 2) * (NT / 2);
            for (int c0 = cbeg; c0 < cbeg + NT / 2; c0 += 16) {
                uint32_t vr[16], vi[16];
                if (nst > 0) {
                    const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                 : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]), "=r"(vr[7]),
                                   "=r"(vr[8]), "=r"(vr[9]), "=r"(vr[10]), "=r"(vr[11]), "=r"(vr[12]), "=r"(vr[13]), "=r"(vr[14]), "=r"(vr[15])
                                 : "r"(tm_r + lane_off + (uint32_t)c0));
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                                 : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]), "=r"(vi[7]),
                                   "=r"(vi[8]), "=r"(vi[9]), "=r"(vi[10]), "=r"(vi[11]), "=r"(vi[12]), "=r"(vi[13]), "=r"(vi[14]), "=r"(vi[15])
                                 : "r"(tm_i + lane_off + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) { vr[j] = 0u; vi[j] = 0u; }
                }
#pragma unroll
                for (int j = 0; j < 16; j += 2)
                    *(float4*)&stg[rl * SP + c0 + j] = make_float4(__uint_as_float(vr[j]), __uint_as_float(vi[j]),
                                                                   __uint_as_float(vr[j + 1]), __uint_as_float(vi[j + 1]));
            }
        }
        asm volatile("bar.sync 1, %0;" :: "n"(NCONVT) : "memory");   // converter warps only

        const int kfull0 = (MODE == BB) ? o0 : 0;
        const int kfull1 = (MODE == FA) ? min(o0 + 4, nd.own_t) : ((MODE == BA) ? nd.upd_t : nd.own_t);
        const bool unique = kbeg == kfull0 && kend == kfull1 && MODE != FB;
        const int nrows_out = (MODE == FB) ? nd.nupd : nd.nown;
        constexpr int RB = 4, NV = NT / 64;  // rows per batch; 16-byte column pairs per lane and row
        for (int i0 = 0; i0 < 16; i0 += RB) {
            long long base[RB];
            bool vrow[RB];
            float2 di[RB];
            float4 z[RB][NV];
            // all loads of the batch first (row indices, D^{-1}, z), then the writes
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int rl2 = cw * 16 + i0 + r;
                const int row = o0 * TILE + rl2;
                vrow[r] = (o0 + (rl2 >> 5)) < nout_t && row < nrows_out;
                base[r] = 0;
                if (vrow[r]) base[r] = ((MODE == FB) ? (long long)upd[row] : (long long)(nd.own0 + row)) * ldc + col0;
                if (MODE == BA && kbeg == 0 && vrow[r]) {
                    di[r] = jb.dinv[nd.own0 + row];
#pragma unroll
                    for (int v = 0; v < NV; ++v) z[r][v] = *(const float4*)(jb.x + base[r] + 2 * l + 64 * v);
                }
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (!vrow[r]) continue;
                const int rl2 = cw * 16 + i0 + r;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int c = 2 * l + 64 * v;
                    float4 y = *(const float4*)&stg[rl2 * SP + c];
                    if (MODE == FB) {
                        atomicAdd((float4*)(jb.acc + base[r] + c), make_float4(-y.x, -y.y, -y.z, -y.w));
                    } else if (MODE == FA || MODE == BB) {
                        if (unique) *(float4*)(jb.x + base[r] + c) = y;
                        else atomicAdd((float4*)(jb.x + base[r] + c), y);
                    } else {  // BA: acc = Dinv z - partial; the first split clears z
                        if (kbeg == 0) {
                            const float2 d = di[r];
                            const float4 q = z[r][v];
                            y.x -= d.x * q.x - d.y * q.y; y.y -= d.x * q.y + d.y * q.x;
                            y.z -= d.x * q.z - d.y * q.w; y.w -= d.x * q.w + d.y * q.z;
                            *(float4*)(jb.x + base[r] + c) = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        const float4 ny = make_float4(-y.x, -y.y, -y.z, -y.w);
                        if (unique) *(float4*)(jb.acc + base[r] + c) = ny;
                        else atomicAdd((float4*)(jb.acc + base[r] + c), ny);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * NT));
}

template <int NT, int MODE, int SPLIT>
void launch_one(const Task* tasks, long long n, const JobDev<float2>* jobs, int ldc, int KS, int* flag, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        HZ_CUDA(cudaFuncSetAttribute(k_subst_tc<NT, MODE, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Layout<NT>::TOTAL));
        attr = true;
    }
    const int nchunks = ldc / NT;
    k_subst_tc<NT, MODE, SPLIT><<<(unsigned)(n * nchunks), NTHREADS, Layout<NT>::TOTAL, st>>>(tasks, jobs, ldc, nchunks,
                                                                                               KS, flag);
    HZ_CHECK_LAUNCH();
}

template <int NT, int SPLIT>
void launch_mode(const Batch& b, int h, int mode, int ldc, int* flag, cudaStream_t st) {
    const long long off = b.pair_off[mode][h], n = b.pair_cnt[mode][h];
    if (n == 0) return;
    const Task* tasks = b.d_tasks + off;
    const JobDev<float2>* jobs = (const JobDev<float2>*)b.d_jobs;
    switch (mode) {
        case FA: launch_one<NT, FA, SPLIT>(tasks, n, jobs, ldc, b.KS_tc, flag, st); break;
        case FB: launch_one<NT, FB, SPLIT>(tasks, n, jobs, ldc, b.KS_tc, flag, st); break;
        case BA: launch_one<NT, BA, SPLIT>(tasks, n, jobs, ldc, b.KS_tc, flag, st); break;
        default: launch_one<NT, BB, SPLIT>(tasks, n, jobs, ldc, b.KS_tc, flag, st); break;
    }
}

}  // namespace

int tc_columns(int ldc) {
    if (ldc % 128 == 0) return 128;
    if (ldc % 64 == 0) return 64;
    return 0;
}

void launch_level_tc(const Batch& b, int h, int mode, int ldc, int* flag, cudaStream_t st) {
    const bool wide = tc_columns(ldc) == 128;
    if (b.split == 1) {
        if (wide) launch_mode<128, 1>(b, h, mode, ldc, flag, st);
        else launch_mode<64, 1>(b, h, mode, ldc, flag, st);
    } else {
        if (wide) launch_mode<128, 3>(b, h, mode, ldc, flag, st);
        else launch_mode<64, 3>(b, h, mode, ldc, flag, st);
    }
}

}  // namespace hz
