// Tensor-core (tcgen05) variant of the substitution products for complex64 factors.
//
// A work item computes 128 complex output rows (four factor tile rows) x NT right-hand-side
// columns of one of the four node products of the substitution (see solve.cu), for the nodes
// whose products are large enough to fill it; smaller nodes of the same tree level run on the
// CUDA-core kernel in the same phase.
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
// Warp-specialized pipeline (16 complex reduction indices per stage, two-deep rings of raw and
// converted buffers, every hand-off an mbarrier):
//   4 loader warps    : cp.async 16-byte copies of the factor tiles and vector rows into a raw
//                       buffer (masked rows / absent tiles zero-filled by the copy), completion
//                       signalled with cp.async.mbarrier.arrive;
//   8 converter warps : raw -> split hi/lo TF32 operands in the K-major core-matrix layout
//                       (no swizzle), 16-byte stores;
//   1 MMA warp        : one thread issues the MMAs of a stage and commits them to the mbarrier
//                       that releases the converted buffer.
// Two kernels share these stages:
//   k_subst_tc  (one block per work item, 416 threads): after the last MMA the converter warps
//               stage the accumulators through shared memory and write whole rows;
//   k_subst_tcp (persistent, one block per SM, 544 threads): the block walks the launch's work
//               items with stride gridDim.x; the rings run on across items, the accumulators
//               alternate between two TMEM buffers, and 4 epilogue warps drain item i while the
//               MMA warp accumulates item i+1, so block start-up, pipeline fill and epilogue are
//               paid once per SM instead of once per item.
// Output rule of both: an item that covers the full reduction of its rows stores them; split
// reductions and the shared update rows of FB accumulate with vector atomics.  Every mbarrier
// wait is bounded (polls and wall time); a wait that gives up raises an abort flag in shared
// memory that ends the block's other waits; the block then records an error flag, waits
// (bounded) for its own MMAs, frees its tensor memory and exits.
#include <algorithm>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"
#include "hz_solve.cuh"
#include "tc_common.cuh"

namespace hz {

namespace {

using namespace tcc;

enum { FA = 0, FB = 1, BA = 2, BB = 3 };

// Sizes of one ring stage for NT columns.
template <int NT> struct Ring {
    static constexpr int A_MAT = MR * KC * 4;            // one real operand matrix (8 KB)
    static constexpr int X_MAT = NT * KC * 4;
    static constexpr int CONV = 4 * A_MAT + 4 * X_MAT;   // Ar_h Ar_l Ai_h Ai_l  Xr_h Xr_l Xi_h Xi_l
    static constexpr int RAW_A = 4 * 32 * TROW;          // large enough for both raw tile layouts
    static constexpr int RAW_X = KC * NT * 8;
    static constexpr int RAW = RAW_A + RAW_X;
    static constexpr int BYTES = 2 * (CONV + RAW);       // two-deep rings
};

// One work item: 128 output rows (tiles o0 .. o0+3) x NT columns of one node product, reduction
// tiles [kbeg, kend).
struct Item {
    JobDev<float2> jb;
    NodeDev nd;
    int col0, o0, nout_t, nrows_out, nrows_k, kbeg, kend, nst;
    bool unique;
};

template <int NT, int MODE>
__device__ inline Item decode(const Task* tasks, const JobDev<float2>* jobs, long long item, int nchunks, int KS) {
    Item it;
    const Task tk = tasks[item / nchunks];
    it.jb = jobs[tk.job];
    it.nd = it.jb.nodes[tk.node];
    const NodeDev& nd = it.nd;
    it.col0 = (int)(item % nchunks) * NT;
    it.o0 = tk.tile;
    it.nout_t = (MODE == FB) ? nd.upd_t : nd.own_t;
    it.nrows_out = (MODE == FB) ? nd.nupd : nd.nown;
    it.nrows_k = (MODE == BA) ? nd.nupd : nd.nown;
    it.kbeg = tk.pad_;
    const int kfull0 = (MODE == BB) ? it.o0 : 0;
    const int kfull1 = (MODE == FA) ? min(it.o0 + 4, nd.own_t) : ((MODE == BA) ? nd.upd_t : nd.own_t);
    it.kend = min(kfull1, it.kbeg + KS);
    it.nst = max(0, it.kend - it.kbeg) * 2;
    it.unique = it.kbeg == kfull0 && it.kend == kfull1 && MODE != FB;
    return it;
}

// Vector rows a loader thread copies in stage s of an item (-1: beyond the node, zero-filled).
// They are looked up one stage ahead, so that BA's gather through the update index list is not
// on the copy's critical path.
template <int NT> struct Vrows { int r[KC * NT / 2 / NLOAD]; };

template <int NT, int MODE>
__device__ inline Vrows<NT> stage_rows(const Item& it, int s, int t) {
    Vrows<NT> v;
    const int kt = it.kbeg + (s >> 1), hk = s & 1;
    const int* upd = it.jb.upd_idx + it.nd.upd_off;
#pragma unroll
    for (int i = 0; i < KC * NT / 2 / NLOAD; ++i) {
        const int k = (t + NLOAD * i) / (NT / 2);
        const int rr = kt * TILE + hk * KC + k;
        v.r[i] = -1;
        if (rr < it.nrows_k) v.r[i] = (MODE == BA) ? upd[rr] : it.nd.own0 + rr;
    }
    return v;
}

// Loader part of stage s of an item: the four factor tiles' 16-column halves and 16 vector rows.
template <int NT, int MODE>
__device__ inline void load_stage(unsigned char* rb, const Item& it, int s, int ldc, int t, const Vrows<NT>& vr) {
    using RG = Ring<NT>;
    constexpr bool TR = (MODE == BA || MODE == BB);  // factor tiles used transposed
    const NodeDev& nd = it.nd;
    const int kt = it.kbeg + (s >> 1), hk = s & 1;
    for (int c = t; c < 1024; c += NLOAD) {     // factor tiles: 1024 chunks of 16 bytes
        const int oi = c >> 8, q = c & 255;
        const int o = it.o0 + oi;
        bool exists = o < it.nout_t;
        if (MODE == FA) exists = exists && kt <= o;
        if (MODE == BB) exists = exists && kt >= o;
        long long toff = 0;
        if (exists) {
            if (MODE == FA) toff = nd.linv_off + tri_idx(o, kt);
            else if (MODE == FB) toff = nd.l21_off + (long long)o * nd.own_t + kt;
            else if (MODE == BA) toff = nd.l21_off + (long long)kt * nd.own_t + o;
            else toff = nd.linv_off + tri_idx(kt, o);
        }
        const float2* tl = it.jb.fac + toff * TILE2;
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
        cp16(dst, exists ? (const void*)src : (const void*)it.jb.fac, exists ? 16 : 0);
    }
    const float2* vec = (MODE == FA || MODE == BB) ? it.jb.acc : it.jb.x;
#pragma unroll
    for (int i = 0; i < KC * NT / 2 / NLOAD; ++i) {  // vector rows: KC x NT, raw [k][n]
        const int c = t + NLOAD * i;
        const int k = c / (NT / 2), j = c % (NT / 2);
        const bool v = vr.r[i] >= 0;
        const long long row = v ? vr.r[i] : 0;
        cp16(smem_u32(rb + RG::RAW_A + k * NT * 8 + j * 16), vec + row * ldc + it.col0 + 2 * j, v ? 16 : 0);
    }
}

// Converter part of a stage: raw -> hi (and lo) TF32 operands.
template <int NT, int MODE, int SPLIT>
__device__ inline void convert_stage(const unsigned char* rb, unsigned char* cv, int ct) {
    using RG = Ring<NT>;
    constexpr bool TR = (MODE == BA || MODE == BB);
    for (int id = ct; id < MR * 4; id += NCONV) {   // factor operand: 128 rows x 16 k, (row, 4 consecutive k)
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
        *(float4*)(cv + 0 * RG::A_MAT + off) = rh;
        *(float4*)(cv + 2 * RG::A_MAT + off) = ih;
        if (SPLIT == 3) {
            *(float4*)(cv + 1 * RG::A_MAT + off) = make_float4(re[0] - rh.x, re[1] - rh.y, re[2] - rh.z, re[3] - rh.w);
            *(float4*)(cv + 3 * RG::A_MAT + off) = make_float4(im[0] - ih.x, im[1] - ih.y, im[2] - ih.z, im[3] - ih.w);
        }
    }
    for (int id = ct; id < NT * 4; id += NCONV) {   // vector operand: NT rows x 16 k
        const int n = id % NT, kq = id / NT;
        const float2* src = (const float2*)(rb + RG::RAW_A);
        float re[4], im[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) { float2 a = src[(4 * kq + j) * NT + n]; re[j] = a.x; im[j] = a.y; }
        float4 rh, ih;
        rh.x = tf32_hi(re[0]); rh.y = tf32_hi(re[1]); rh.z = tf32_hi(re[2]); rh.w = tf32_hi(re[3]);
        ih.x = tf32_hi(im[0]); ih.y = tf32_hi(im[1]); ih.z = tf32_hi(im[2]); ih.w = tf32_hi(im[3]);
        const int off = 4 * RG::A_MAT + coff(n, 4 * kq);
        *(float4*)(cv + off + 0 * RG::X_MAT) = rh;
        *(float4*)(cv + off + 2 * RG::X_MAT) = ih;
        if (SPLIT == 3) {
            *(float4*)(cv + off + 1 * RG::X_MAT) = make_float4(re[0] - rh.x, re[1] - rh.y, re[2] - rh.z, re[3] - rh.w);
            *(float4*)(cv + off + 3 * RG::X_MAT) = make_float4(im[0] - ih.x, im[1] - ih.y, im[2] - ih.z, im[3] - ih.w);
        }
    }
}

// Writes one 16-byte column pair y of an output row (global offset base + c) by the output rule.
template <int MODE>
__device__ inline void write_pair(const Item& it, long long base, int c, float4 y, float2 d, float4 z) {
    float4* dx = (float4*)(it.jb.x + base + c);
    float4* da = (float4*)(it.jb.acc + base + c);
    if (MODE == FB) {
        atomicAdd(da, make_float4(-y.x, -y.y, -y.z, -y.w));
    } else if (MODE == FA || MODE == BB) {
        if (it.unique) *dx = y;
        else atomicAdd(dx, y);
    } else {  // BA: acc = Dinv z - partial; the first split clears z
        if (it.kbeg == 0) {
            y.x -= d.x * z.x - d.y * z.y; y.y -= d.x * z.y + d.y * z.x;
            y.z -= d.x * z.z - d.y * z.w; y.w -= d.x * z.w + d.y * z.z;
            *dx = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float4 ny = make_float4(-y.x, -y.y, -y.z, -y.w);
        if (it.unique) *da = ny;
        else atomicAdd(da, ny);
    }
}

// global offset (row x ldc + chunk column) of local output row r of an item, -1 if absent
template <int MODE>
__device__ inline long long row_base(const Item& it, int r, int ldc) {
    const int row = it.o0 * TILE + r;
    if ((it.o0 + (r >> 5)) >= it.nout_t || row >= it.nrows_out) return -1;
    const int* upd = it.jb.upd_idx + it.nd.upd_off;
    return ((MODE == FB) ? (long long)upd[row] : (long long)(it.nd.own0 + row)) * ldc + it.col0;
}

// ------------------------------------------------------------------------------------------
// k_subst_tc: one block per work item
// ------------------------------------------------------------------------------------------
template <int NT> struct OneLayout {
    using RG = Ring<NT>;
    static constexpr int NTHREADS = NLOAD + NCONV + 32;
    static constexpr int HALF = NT / 2;                  // output columns staged per epilogue pass
    static constexpr int SP = HALF + 2;                  // staging pitch (complex): 16-byte rows, odd in 16 B
    static_assert(MR * SP * 8 <= RG::BYTES, "staging tile must fit in the ring buffers");
    static constexpr int ROWS_OFF = RG::BYTES;           // long long rowbase[128], float2 dinv[128]
    static constexpr int BAR_OFF = ROWS_OFF + MR * 8 + MR * 8;
    static constexpr int TOTAL = BAR_OFF + 8 * 8 + 16;
};

template <int NT, int MODE, int SPLIT>
__global__ void __launch_bounds__(OneLayout<NT>::NTHREADS, 1)
k_subst_tc(const Task* __restrict__ tasks, const JobDev<float2>* __restrict__ jobs, int ldc, int nchunks, int KS,
           int* flag, long long polls) {
    using RG = Ring<NT>;
    using LY = OneLayout<NT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* conv = smem;                  // [2][CONV]
    unsigned char* raw = smem + 2 * RG::CONV;    // [2][RAW]
    long long* rowbase = (long long*)(smem + LY::ROWS_OFF);
    float2* dinv_s = (float2*)(smem + LY::ROWS_OFF + MR * 8);
    uint64_t* bars = (uint64_t*)(smem + LY::BAR_OFF);
    uint64_t* raw_full = bars;        // [2] loaders' copies landed (count NLOAD)
    uint64_t* raw_empty = bars + 2;   // [2] converters done reading (count NCONV)
    uint64_t* conv_full = bars + 4;   // [2] converted operands written (count NCONV)
    uint64_t* conv_empty = bars + 6;  // [2] MMAs of the buffer done (tcgen05.commit)
    uint32_t* tptr = (uint32_t*)(bars + 8);
    volatile int* abort = (volatile int*)(bars + 8) + 1;
    volatile int* committed = (volatile int*)(bars + 8) + 2;   // stages whose MMAs were committed

    const Item it = decode<NT, MODE>(tasks, jobs, blockIdx.x, nchunks, KS);
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const int nst = it.nst;
    const int mma_warp = (NLOAD + NCONV) / 32;

    if (w == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tptr)), "r"(2 * NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(raw_full + b, NLOAD);
            mbar_init(raw_empty + b, NCONV);
            mbar_init(conv_full + b, NCONV);
            mbar_init(conv_empty + b, 1);
        }
        *abort = 0;
        *committed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tptr;
    const uint32_t tm_r = tmem, tm_i = tmem + NT;  // accumulators: real part cols [0, NT), imag [NT, 2NT)
    bool ok = true;

    if (t < NLOAD) {
        Vrows<NT> rows = stage_rows<NT, MODE>(it, 0, t);
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s & 1, use = s >> 1;
            const Vrows<NT> next = stage_rows<NT, MODE>(it, s + 1, t);   // looked up ahead
            if (s >= 2) ok = mbar_wait(smem_u32(raw_empty + slot), (uint32_t)((use - 1) & 1), abort, polls);
            if (!ok) break;
            load_stage<NT, MODE>(raw + slot * RG::RAW, it, s, ldc, t, rows);
            cp_async_arrive(raw_full + slot);
            rows = next;
        }
        // row descriptors of the epilogue, fetched while the pipeline drains
        for (int r = t; r < MR; r += NLOAD) {
            const long long base = row_base<MODE>(it, r, ldc);
            rowbase[r] = base;
            if (MODE == BA) dinv_s[r] = base >= 0 ? it.jb.dinv[it.nd.own0 + it.o0 * TILE + r] : make_float2(0.f, 0.f);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (t < NLOAD + NCONV) {
        const int ct = t - NLOAD;
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s & 1, use = s >> 1;
            ok = mbar_wait(smem_u32(raw_full + slot), (uint32_t)(use & 1), abort, polls);
            if (ok && s >= 2) ok = mbar_wait(smem_u32(conv_empty + slot), (uint32_t)((use - 1) & 1), abort, polls);
            if (!ok) break;
            convert_stage<NT, MODE, SPLIT>(raw + slot * RG::RAW, conv + slot * RG::CONV, ct);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(raw_empty + slot);
            mbar_arrive(conv_full + slot);
        }
    } else if (l == 0) {
        for (int s = 0; s < nst && ok; ++s) {
            const int cb = s & 1, use = s >> 1;
            ok = mbar_wait(smem_u32(conv_full + cb), (uint32_t)(use & 1), abort, polls);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mma_stage<NT, SPLIT>(smem_u32(conv + cb * RG::CONV), tm_r, tm_i, s == 0);
            mma_commit(conv_empty + cb);
            *committed = s + 1;
        }
    }

    // every role arrives here (their waits are bounded); make the outcome block-uniform
    ok = __syncthreads_and(ok) != 0;
    bool done = true;
    const int ncommit = *committed;
    if (ncommit > 0) {   // the last committed stage's MMAs, waited for even after an abort
        const int sl = ncommit - 1;
        int no_abort = 0;
        const bool got = mbar_wait(smem_u32(conv_empty + (sl & 1)), (uint32_t)((sl >> 1) & 1), &no_abort);
        done = __syncthreads_and(got) != 0;
    }
    if (!ok || !done) {
        if (t == 0) atomicExch(flag, 1);
        ok = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue (converter warps), per column half of the tile:
    //  (1) tensor memory -> shared staging tile [128 rows][HALF + 2]; warp w may read TMEM lanes
    //      32 (w % 4) .. +31 (output tile o0 + w % 4); the two warps of a lane quarter split the columns;
    //  (2) each converter warp writes 16 staged rows, lane = pair of columns (16-byte accesses),
    //      all loads of a batch of rows (BA's z) before its writes.
    if (ok && t >= NLOAD && t < NLOAD + NCONV) {
        constexpr int HALF = LY::HALF, SP = LY::SP;
        constexpr int CPW = HALF / 2;            // columns per warp per pass
        constexpr int RPW = MR / (NCONV / 32);   // staged rows written per warp
        constexpr int NP = HALF / 2;             // 16-byte column pairs per row and pass
        constexpr int RB = 8;                    // rows per load batch
        static_assert(CPW % 16 == 0 && RPW % RB == 0, "epilogue tiling");
        float2* stg = (float2*)smem;             // operand and raw buffers are free after the MMAs
        const int cw = (t - NLOAD) >> 5;
        const int q4 = w & 3, sub = cw >> 2;
        const int rl = 32 * q4 + l;
        for (int pass = 0; pass < 2; ++pass) {
            const int cbeg = pass * HALF + sub * CPW;
            for (int c0 = cbeg; c0 < cbeg + CPW; c0 += 16) {
                uint32_t vr[16], vi[16];
                if (nst > 0) {
                    const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
                    tmem_ld16(tm_r + lane_off + (uint32_t)c0, tm_i + lane_off + (uint32_t)c0, vr, vi);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) { vr[j] = 0u; vi[j] = 0u; }
                }
                const int cl = c0 - pass * HALF;
#pragma unroll
                for (int j = 0; j < 16; j += 2)
                    *(float4*)&stg[rl * SP + cl + j] = make_float4(__uint_as_float(vr[j]), __uint_as_float(vi[j]),
                                                                   __uint_as_float(vr[j + 1]), __uint_as_float(vi[j + 1]));
            }
            asm volatile("bar.sync 1, %0;" :: "n"(NCONV) : "memory");   // converter warps only
            const bool lane_on = l < NP;
            const int c = pass * HALF + 2 * l;
            for (int i0 = 0; i0 < RPW; i0 += RB) {
                float4 z[RB];
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    z[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                    const long long base = rowbase[cw * RPW + i0 + r];
                    if (MODE == BA && it.kbeg == 0 && lane_on && base >= 0) z[r] = *(const float4*)(it.jb.x + base + c);
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int rl2 = cw * RPW + i0 + r;
                    const long long base = rowbase[rl2];
                    if (!lane_on || base < 0) continue;
                    const float2 d = (MODE == BA) ? dinv_s[rl2] : make_float2(0.f, 0.f);
                    write_pair<MODE>(it, base, c, *(const float4*)&stg[rl2 * SP + 2 * l], d, z[r]);
                }
            }
            asm volatile("bar.sync 1, %0;" :: "n"(NCONV) : "memory");   // staging reused by the next pass
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * NT));
}

// ------------------------------------------------------------------------------------------
// k_subst_tcp: persistent, one block per SM
// ------------------------------------------------------------------------------------------
template <int NT> struct PLayout {
    using RG = Ring<NT>;
    static constexpr int NEPI = 128;                       // epilogue threads (4 warps)
    static constexpr int NTHREADS = NLOAD + NCONV + 32 + NEPI;
    static constexpr int EP = 18;                          // staging pitch (complex) of a 32 x 16 chunk
    static constexpr int STG_OFF = RG::BYTES;              // 4 warps x 32 rows x EP complex
    static constexpr int BAR_OFF = STG_OFF + 4 * 32 * EP * 8;
    static constexpr int TOTAL = BAR_OFF + 12 * 8 + 16;
    static constexpr int TMEM_COLS = 4 * NT;               // two accumulator buffers (re, im) x NT
};

template <int NT, int MODE, int SPLIT>
__global__ void __launch_bounds__(PLayout<NT>::NTHREADS, 1)
k_subst_tcp(const Task* __restrict__ tasks, const JobDev<float2>* __restrict__ jobs, int ldc, int nchunks, int KS,
            long long nitems, int* flag, long long polls) {
    using RG = Ring<NT>;
    using LY = PLayout<NT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* conv = smem;                  // [2][CONV]
    unsigned char* raw = smem + 2 * RG::CONV;    // [2][RAW]
    uint64_t* bars = (uint64_t*)(smem + LY::BAR_OFF);
    uint64_t* raw_full = bars;         // [2] loaders' copies landed (count NLOAD)
    uint64_t* raw_empty = bars + 2;    // [2] converters done reading (count NCONV)
    uint64_t* conv_full = bars + 4;    // [2] converted operands written (count NCONV)
    uint64_t* conv_empty = bars + 6;   // [2] MMAs of the buffer done (tcgen05.commit)
    uint64_t* acc_full = bars + 8;     // [2] all MMAs of an item's accumulator done (tcgen05.commit)
    uint64_t* acc_empty = bars + 10;   // [2] epilogue done reading the accumulator (count NEPI)
    uint32_t* tptr = (uint32_t*)(bars + 12);
    volatile int* abort = (volatile int*)(bars + 12) + 1;

    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const int mma_warp = (NLOAD + NCONV) / 32;
    const int epi_warp0 = (NLOAD + NCONV + 32) / 32;

    if (w == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tptr)),
                     "r"(LY::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(raw_full + b, NLOAD);
            mbar_init(raw_empty + b, NCONV);
            mbar_init(conv_full + b, NCONV);
            mbar_init(conv_empty + b, 1);
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, LY::NEPI);
        }
        *abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tptr;
    bool ok = true;
    bool mma_drained = true;

    if (t < NLOAD) {
        // ------------------------------------------------------------ loaders
        // the next item is decoded, and the next stage's vector rows looked up, while the
        // current stage's copies are issued
        long long gs = 0;  // stage counter across this block's items
        long long item = blockIdx.x;
        Item cur;
        Vrows<NT> rows;
        if (item < nitems) {
            cur = decode<NT, MODE>(tasks, jobs, item, nchunks, KS);
            rows = stage_rows<NT, MODE>(cur, 0, t);
        }
        for (; item < nitems && ok; item += gridDim.x) {
            const long long nxt_item = item + gridDim.x;
            Item nxt = cur;
            if (nxt_item < nitems) nxt = decode<NT, MODE>(tasks, jobs, nxt_item, nchunks, KS);
            for (int s = 0; s < cur.nst && ok; ++s, ++gs) {
                const int slot = (int)(gs & 1);
                const long long use = gs >> 1;
                Vrows<NT> next_rows;
                if (s + 1 < cur.nst) next_rows = stage_rows<NT, MODE>(cur, s + 1, t);
                else if (nxt_item < nitems) next_rows = stage_rows<NT, MODE>(nxt, 0, t);
                if (gs >= 2) ok = mbar_wait(smem_u32(raw_empty + slot), (uint32_t)((use - 1) & 1), abort, polls);
                if (!ok) break;
                load_stage<NT, MODE>(raw + slot * RG::RAW, cur, s, ldc, t, rows);
                cp_async_arrive(raw_full + slot);
                rows = next_rows;
            }
            cur = nxt;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (t < NLOAD + NCONV) {
        // ------------------------------------------------------------ converters
        const int ct = t - NLOAD;
        long long gs = 0;
        int nst_next = blockIdx.x < nitems ? decode<NT, MODE>(tasks, jobs, blockIdx.x, nchunks, KS).nst : 0;
        for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int nst = nst_next;   // decoded one item ahead
            if (item + gridDim.x < nitems) nst_next = decode<NT, MODE>(tasks, jobs, item + gridDim.x, nchunks, KS).nst;
            for (int s = 0; s < nst && ok; ++s, ++gs) {
                const int slot = (int)(gs & 1);
                const long long use = gs >> 1;
                ok = mbar_wait(smem_u32(raw_full + slot), (uint32_t)(use & 1), abort, polls);
                if (ok && gs >= 2) ok = mbar_wait(smem_u32(conv_empty + slot), (uint32_t)((use - 1) & 1), abort, polls);
                if (!ok) break;
                convert_stage<NT, MODE, SPLIT>(raw + slot * RG::RAW, conv + slot * RG::CONV, ct);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(raw_empty + slot);
                mbar_arrive(conv_full + slot);
            }
        }
    } else if (w == mma_warp) {
        // ------------------------------------------------------------ MMA issuer (lane 0)
        if (l == 0) {
            long long gs = 0;
            int nit = 0;  // items of this block so far
            int nst_next = blockIdx.x < nitems ? decode<NT, MODE>(tasks, jobs, blockIdx.x, nchunks, KS).nst : 0;
            for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++nit) {
                const int nst = nst_next;   // decoded one item ahead
                if (item + gridDim.x < nitems) nst_next = decode<NT, MODE>(tasks, jobs, item + gridDim.x, nchunks, KS).nst;
                const int b = nit & 1;
                if (nit >= 2) ok = mbar_wait(smem_u32(acc_empty + b), (uint32_t)(((nit >> 1) - 1) & 1), abort, polls);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tm_r = tmem + (uint32_t)(b * 2 * NT), tm_i = tm_r + NT;
                for (int s = 0; s < nst && ok; ++s, ++gs) {
                    const int cb = (int)(gs & 1);
                    ok = mbar_wait(smem_u32(conv_full + cb), (uint32_t)((gs >> 1) & 1), abort, polls);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    mma_stage<NT, SPLIT>(smem_u32(conv + cb * RG::CONV), tm_r, tm_i, s == 0);
                    mma_commit(conv_empty + cb);
                }
                mma_commit(acc_full + b);   // arrives when every MMA issued so far has completed
            }
            // before the tensor memory is freed every issued MMA must have completed: the last
            // item begun (nit - 1; an interrupted one was committed too) is waited for, even
            // after an abort
            if (nit > 0) {
                int no_abort = 0;
                mma_drained = mbar_wait(smem_u32(acc_full + ((nit - 1) & 1)), (uint32_t)(((nit - 1) >> 1) & 1), &no_abort);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue warps
        // warp w reads TMEM lanes 32 (w % 4) .. +31 = output rows of tile o0 + w % 4 (lane = row);
        // per 16-column chunk: stage 32 x 16 in this warp's shared slice, then write 4 rows per
        // instruction (8 lanes x 16 bytes per row)
        const int q4 = w & 3;
        float2* stg = (float2*)(smem + LY::STG_OFF) + (size_t)(w - epi_warp0) * 32 * LY::EP;
        const int r4 = l >> 3, p = l & 7;   // write phase: row within a group of 4, column pair
        int nit = 0;
        for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++nit) {
            const Item it = decode<NT, MODE>(tasks, jobs, item, nchunks, KS);
            const int b = nit & 1;
            // this lane's row descriptor, shuffled to the writing lanes below
            const long long my_base = row_base<MODE>(it, 32 * q4 + l, ldc);
            float2 my_d = make_float2(0.f, 0.f);
            if (MODE == BA && my_base >= 0) my_d = it.jb.dinv[it.nd.own0 + it.o0 * TILE + 32 * q4 + l];
            ok = mbar_wait(smem_u32(acc_full + b), (uint32_t)((nit >> 1) & 1), abort, polls);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
            const uint32_t tm_r = tmem + (uint32_t)(b * 2 * NT) + lane_off, tm_i = tm_r + NT;
            for (int c0 = 0; c0 < NT; c0 += 16) {
                uint32_t vr[16], vi[16];
                if (it.nst > 0) {
                    tmem_ld16(tm_r + (uint32_t)c0, tm_i + (uint32_t)c0, vr, vi);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) { vr[j] = 0u; vi[j] = 0u; }
                }
#pragma unroll
                for (int j = 0; j < 16; j += 2)
                    *(float4*)&stg[l * LY::EP + j] = make_float4(__uint_as_float(vr[j]), __uint_as_float(vi[j]),
                                                                 __uint_as_float(vr[j + 1]), __uint_as_float(vi[j + 1]));
                __syncwarp();
                const int c = c0 + 2 * p;
                long long base[8];
                float4 z[8];
#pragma unroll
                for (int g = 0; g < 8; ++g) {   // all loads of the chunk before its writes
                    base[g] = __shfl_sync(0xffffffffu, my_base, 4 * g + r4);
                    z[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (MODE == BA && it.kbeg == 0 && base[g] >= 0) z[g] = *(const float4*)(it.jb.x + base[g] + c);
                }
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const int rr = 4 * g + r4;
                    float2 d;
                    d.x = __shfl_sync(0xffffffffu, my_d.x, rr);
                    d.y = __shfl_sync(0xffffffffu, my_d.y, rr);
                    if (base[g] < 0) continue;
                    write_pair<MODE>(it, base[g], c, *(const float4*)&stg[rr * LY::EP + 2 * p], d, z[g]);
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(acc_empty + b);
        }
    }

    ok = __syncthreads_and(ok && mma_drained) != 0;
    if (!ok && t == 0) atomicExch(flag, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(LY::TMEM_COLS));
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        HZ_CUDA(cudaGetDevice(&dev));
        HZ_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    }
    return n;
}

template <int NT, int MODE, int SPLIT>
void launch_one(const Batch& b, const Task* tasks, long long n, const JobDev<float2>* jobs, int ldc, int* flag,
                cudaStream_t st) {
    const int nchunks = (b.job_cols > 0 ? b.job_cols : ldc) / NT;
    const long long nitems = n * nchunks;
    if (b.tc_cfg == 1) {
        static bool attr = false;
        if (!attr) {
            HZ_CUDA(cudaFuncSetAttribute(k_subst_tcp<NT, MODE, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         PLayout<NT>::TOTAL));
            attr = true;
        }
        const long long grid = std::min<long long>(nitems, sm_count());
        k_subst_tcp<NT, MODE, SPLIT><<<(unsigned)grid, PLayout<NT>::NTHREADS, PLayout<NT>::TOTAL, st>>>(
            tasks, jobs, ldc, nchunks, b.KS_tc, nitems, flag, b.wait_polls);
    } else {
        static bool attr = false;
        if (!attr) {
            HZ_CUDA(cudaFuncSetAttribute(k_subst_tc<NT, MODE, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OneLayout<NT>::TOTAL));
            attr = true;
        }
        k_subst_tc<NT, MODE, SPLIT><<<(unsigned)nitems, OneLayout<NT>::NTHREADS, OneLayout<NT>::TOTAL, st>>>(
            tasks, jobs, ldc, nchunks, b.KS_tc, flag, b.wait_polls);
    }
    HZ_CHECK_LAUNCH();
}

template <int NT, int SPLIT>
void launch_mode(const Batch& b, int h, int mode, int ldc, int* flag, cudaStream_t st) {
    const long long off = b.pair_off[mode][h], n = b.pair_cnt[mode][h];
    if (n == 0) return;
    const Task* tasks = b.d_tasks + off;
    const JobDev<float2>* jobs = (const JobDev<float2>*)b.d_jobs;
    switch (mode) {
        case FA: launch_one<NT, FA, SPLIT>(b, tasks, n, jobs, ldc, flag, st); break;
        case FB: launch_one<NT, FB, SPLIT>(b, tasks, n, jobs, ldc, flag, st); break;
        case BA: launch_one<NT, BA, SPLIT>(b, tasks, n, jobs, ldc, flag, st); break;
        default: launch_one<NT, BB, SPLIT>(b, tasks, n, jobs, ldc, flag, st); break;
    }
}

}  // namespace

int tc_columns(int ldc) {
    if (ldc % 128 == 0) return 128;
    if (ldc % 64 == 0) return 64;
    return 0;
}

void launch_level_tc(const Batch& b, int h, int mode, int ldc, int* flag, cudaStream_t st) {
    const bool wide = tc_columns(b.job_cols > 0 ? b.job_cols : ldc) == 128;
    if (b.split == 1) {
        if (wide) launch_mode<128, 1>(b, h, mode, ldc, flag, st);
        else launch_mode<64, 1>(b, h, mode, ldc, flag, st);
    } else {
        if (wide) launch_mode<128, 3>(b, h, mode, ldc, flag, st);
        else launch_mode<64, 3>(b, h, mode, ldc, flag, st);
    }
}

}  // namespace hz
