// Tensor-core (tcgen05, split-TF32) products of the multifrontal factorization (Algorithm 1,
// "Local Solves: Parallel Multi-frontal Methods" section) for complex64 fronts.
//
// A front F = [F11 F21^T; F21 F22] (own unknowns first, column-major, lower triangle) is
// factored in three steps once its pivot block F11 = L11 D L11^T has been factored and L11
// inverted (the CUDA-core kernels of factor.cu, FP64 pivot blocks):
//   L21  = F21 L11^{-T} D^{-1}          (GEMM_L21: A = F21 from the front, B = L11^{-1} packed
//                                        tiles; the output goes straight into the packed L21
//                                        tiles of the factor storage, scaled by D^{-1} per column)
//   F22 -= L21 D L21^T                  (GEMM_SCHUR: A = L21, B = L21 scaled by D(k) per
//                                        reduction index; lower 128 x 128 output tiles only)
// so the Schur update reads F22 once (K = the number of own unknowns) instead of once per
// 32-column panel.  Both are complex products C = sum_k A(i,k) B(j,k) (no conjugation): four
// real products, each with a three-term TF32 split of both operands (hi*hi + hi*lo + lo*hi)
// and FP32 accumulation in tensor memory, i.e. FP32-level accuracy, as in the substitution
// kernels (tc_common.cuh).
//
// One block per 128 x 128 output tile (416 threads): 4 loader warps (cp.async into a two-deep
// raw ring: 16-byte copies of packed tiles, 8-byte copies of front columns, zero-filled beyond
// the front), 8 converter warps (hi/lo split into K-major core matrices, the D(k) scaling of the
// Schur product's B operand), one MMA warp (one thread issues, tcgen05.commit releases the
// buffer); the converter warps then read the accumulators (lane = output row) and write each
// output column's 32 rows per warp instruction.  Every wait is bounded; a block that gives up
// raises the error flag, waits (bounded) for its own MMAs, frees its tensor memory and exits.
#include <algorithm>
#include <vector>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"
#include "tc_common.cuh"

namespace hz {

namespace {

using namespace tcc;

enum { GEMM_L21 = 0, GEMM_SCHUR = 1 };

constexpr int GN = 128;                         // output columns per item (N of the MMA)
constexpr int G_AMAT = MR * KC * 4;             // one converted real operand matrix (8 KB)
constexpr int G_CONV = 4 * G_AMAT + 4 * G_AMAT; // A (re/im x hi/lo) and B (re/im x hi/lo)
constexpr int G_RAW_A = 4 * KC * 32 * 8;        // 128 rows x 16 k complex, [tile][k][row]
constexpr int G_RAW = 2 * G_RAW_A + KC * 8;     // A, B and the 16 D(k) of the stage
constexpr int G_BAR_OFF = 2 * G_CONV + 2 * G_RAW;
constexpr int G_SMEM = G_BAR_OFF + 8 * 8 + 16;
constexpr int G_THREADS = NLOAD + NCONV + 32;

__device__ __forceinline__ void cp8(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// 16-byte chunks of the four packed 32x32 tiles (rows rt0 .. rt0+3, column tile kt, half hk)
// of one operand into raw [tile][k][row] layout; `tile_off(rt)` < 0 means absent (zero-filled).
template <class TileOff>
__device__ __forceinline__ void load_packed(unsigned char* dst0, const float2* fac, int rt0, int hk, int t,
                                            TileOff tile_off) {
    for (int c = t; c < 1024; c += NLOAD) {
        const int oi = c >> 8, q = c & 255;
        const long long toff = tile_off(rt0 + oi);
        const float2* src = fac + (toff >= 0 ? toff : 0) * TILE2 + hk * KC * 32 + q * 2;
        cp16(smem_u32(dst0 + oi * 4096 + q * 16), toff >= 0 ? (const void*)src : (const void*)fac, toff >= 0 ? 16 : 0);
    }
}

// raw [tile][k][row] (128 rows x 16 k complex) -> split operand matrices at cv + {0,1,2,3} * G_AMAT
// (re_hi, re_lo, im_hi, im_lo), optionally multiplied by d[k] first
template <bool SCALE>
__device__ __forceinline__ void convert_operand(const unsigned char* rb, const float2* d, unsigned char* cv, int ct) {
    for (int id = ct; id < MR * 4; id += NCONV) {
        const int row = id & 127, kq = id >> 7;
        const float2* src = (const float2*)(rb + (row >> 5) * 4096);
        float re[4], im[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 a = src[(4 * kq + j) * 32 + (row & 31)];
            if (SCALE) {
                const float2 s = d[4 * kq + j];
                a = make_float2(a.x * s.x - a.y * s.y, a.x * s.y + a.y * s.x);
            }
            re[j] = a.x;
            im[j] = a.y;
        }
        float4 rh, ih;
        rh.x = tf32_hi(re[0]); rh.y = tf32_hi(re[1]); rh.z = tf32_hi(re[2]); rh.w = tf32_hi(re[3]);
        ih.x = tf32_hi(im[0]); ih.y = tf32_hi(im[1]); ih.z = tf32_hi(im[2]); ih.w = tf32_hi(im[3]);
        const int off = coff(row, 4 * kq);
        *(float4*)(cv + 0 * G_AMAT + off) = rh;
        *(float4*)(cv + 1 * G_AMAT + off) = make_float4(re[0] - rh.x, re[1] - rh.y, re[2] - rh.z, re[3] - rh.w);
        *(float4*)(cv + 2 * G_AMAT + off) = ih;
        *(float4*)(cv + 3 * G_AMAT + off) = make_float4(im[0] - ih.x, im[1] - ih.y, im[2] - ih.z, im[3] - ih.w);
    }
}

template <int MODE>
__global__ void __launch_bounds__(G_THREADS, 1)
k_front_gemm(const GemmItem* __restrict__ items, const FrontGemmDesc* __restrict__ fronts, int* flag, long long polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* conv = smem;                  // [2][G_CONV]
    unsigned char* raw = smem + 2 * G_CONV;      // [2][G_RAW]
    uint64_t* bars = (uint64_t*)(smem + G_BAR_OFF);
    uint64_t* raw_full = bars;        // [2] loaders' copies landed (count NLOAD)
    uint64_t* raw_empty = bars + 2;   // [2] converters done reading (count NCONV)
    uint64_t* conv_full = bars + 4;   // [2] converted operands written (count NCONV)
    uint64_t* conv_empty = bars + 6;  // [2] MMAs of the buffer done (tcgen05.commit)
    uint32_t* tptr = (uint32_t*)(bars + 8);
    volatile int* abort = (volatile int*)(bars + 8) + 1;
    volatile int* committed = (volatile int*)(bars + 8) + 2;   // stages whose MMAs were committed

    const GemmItem it = items[blockIdx.x];
    const FrontGemmDesc f = fronts[it.front];
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const int nst = it.nst;
    const int mma_warp = (NLOAD + NCONV) / 32;

    if (w == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tptr)), "r"(2 * GN));
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
    const uint32_t tm_r = tmem, tm_i = tmem + GN;
    bool ok = true;

    if (t < NLOAD) {
        // ------------------------------------------------------------ loaders
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s & 1, use = s >> 1;
            if (s >= 2) ok = mbar_wait(smem_u32(raw_empty + slot), (uint32_t)((use - 1) & 1), abort, polls);
            if (!ok) break;
            unsigned char* rb = raw + slot * G_RAW;
            const int kt = s >> 1, hk = s & 1;
            if (MODE == GEMM_L21) {
                // A: F21 rows i0 .. i0+127, columns kt*32 + hk*16 .. +15 (8-byte copies)
#pragma unroll 4
                for (int q = 0; q < 16; ++q) {
                    const int e = t + NLOAD * q;
                    const int r = e & 127, k = e >> 7;
                    const int row = it.ti * MR + r, col = kt * TILE + hk * KC + k;
                    const bool in = row < f.nupd && col < f.nown;
                    const float2* src = f.F + (long long)(f.nown + row) + (long long)col * f.m;
                    cp8(smem_u32(rb + (r >> 5) * 4096 + (k * 32 + (r & 31)) * 8), in ? (const void*)src : (const void*)f.F,
                        in ? 8 : 0);
                }
                // B: L11^{-1} tile rows of the output columns j0 .. j0+127 (lower triangle)
                load_packed(rb + G_RAW_A, f.fac, it.tj * 4, hk, t, [&](int rt) -> long long {
                    return (rt < f.own_t && kt <= rt) ? f.linv_off + tri_idx(rt, kt) : -1;
                });
            } else {
                load_packed(rb, f.fac, it.ti * 4, hk, t, [&](int rt) -> long long {
                    return rt < f.upd_t ? f.l21_off + (long long)rt * f.own_t + kt : -1;
                });
                load_packed(rb + G_RAW_A, f.fac, it.tj * 4, hk, t, [&](int rt) -> long long {
                    return rt < f.upd_t ? f.l21_off + (long long)rt * f.own_t + kt : -1;
                });
                if (t < KC) {   // D(k) from the front's diagonal
                    const int col = kt * TILE + hk * KC + t;
                    const bool in = col < f.nown;
                    cp8(smem_u32(rb + 2 * G_RAW_A + t * 8), in ? (const void*)(f.F + (long long)col * (f.m + 1)) : (const void*)f.F,
                        in ? 8 : 0);
                }
            }
            cp_async_arrive(raw_full + slot);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (t < NLOAD + NCONV) {
        // ------------------------------------------------------------ converters
        const int ct = t - NLOAD;
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s & 1, use = s >> 1;
            ok = mbar_wait(smem_u32(raw_full + slot), (uint32_t)(use & 1), abort, polls);
            if (ok && s >= 2) ok = mbar_wait(smem_u32(conv_empty + slot), (uint32_t)((use - 1) & 1), abort, polls);
            if (!ok) break;
            const unsigned char* rb = raw + slot * G_RAW;
            unsigned char* cv = conv + slot * G_CONV;
            convert_operand<false>(rb, nullptr, cv, ct);
            if (MODE == GEMM_SCHUR) convert_operand<true>(rb + G_RAW_A, (const float2*)(rb + 2 * G_RAW_A), cv + 4 * G_AMAT, ct);
            else convert_operand<false>(rb + G_RAW_A, nullptr, cv + 4 * G_AMAT, ct);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(raw_empty + slot);
            mbar_arrive(conv_full + slot);
        }
    } else if (l == 0) {
        // ------------------------------------------------------------ MMA issuer
        for (int s = 0; s < nst && ok; ++s) {
            const int cb = s & 1, use = s >> 1;
            ok = mbar_wait(smem_u32(conv_full + cb), (uint32_t)(use & 1), abort, polls);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mma_stage<GN, 3>(smem_u32(conv + cb * G_CONV), tm_r, tm_i, s == 0);
            mma_commit(conv_empty + cb);
            *committed = s + 1;
        }
    }

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

    // ---- epilogue (converter warps): warp w reads TMEM lanes 32 (w % 4) .. +31 (output rows,
    // lane = row); the two warps of a lane quarter split the 128 columns
    if (ok && nst > 0 && t >= NLOAD && t < NLOAD + NCONV) {
        const int q4 = w & 3, sub = ((t - NLOAD) >> 5) >> 2;
        const int lr = 32 * q4 + l;                  // output row within the item
        const int i = it.ti * MR + lr;
        const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
        for (int c0 = sub * (GN / 2); c0 < (sub + 1) * (GN / 2); c0 += 16) {
            uint32_t vr[16], vi[16];
            tmem_ld16(tm_r + lane_off + (uint32_t)c0, tm_i + lane_off + (uint32_t)c0, vr, vi);
            if (MODE == GEMM_L21) {
                const int rt = i >> 5;
                if (rt < f.upd_t) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int j = it.tj * GN + c0 + jj;
                        const int ctile = j >> 5;
                        if (ctile >= f.own_t) continue;
                        const float2 d = j < f.nown ? f.dinv[f.own0 + j] : make_float2(0.f, 0.f);
                        const float a = __uint_as_float(vr[jj]), b = __uint_as_float(vi[jj]);
                        f.fac[(f.l21_off + (long long)rt * f.own_t + ctile) * TILE2 + (i & 31) + (j & 31) * TILE] =
                            make_float2(a * d.x - b * d.y, a * d.y + b * d.x);
                    }
                }
            } else if (i < f.nupd) {
                float2* col0 = f.F + (long long)(f.nown + i) + (long long)f.nown * f.m;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = it.tj * GN + c0 + jj;
                    if (j > i) continue;
                    float2* p = col0 + (long long)j * f.m;
                    float2 v = *p;
                    v.x -= __uint_as_float(vr[jj]);
                    v.y -= __uint_as_float(vi[jj]);
                    *p = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * GN));
}

}  // namespace

bool front_gemm_eligible(int nown, int nupd, int min_upd) { return nupd >= min_upd && nown >= TILE; }

// Work items of the two products for the given fronts (longest reductions first).
void front_gemm_items(const std::vector<FrontGemmDesc>& fr, std::vector<GemmItem>& l21, std::vector<GemmItem>& schur) {
    l21.clear();
    schur.clear();
    for (int q = 0; q < (int)fr.size(); ++q) {
        const FrontGemmDesc& f = fr[q];
        const int T = cdiv(f.nupd, MR), J = cdiv(f.nown, GN);
        for (int ti = 0; ti < T; ++ti) {
            for (int tj = 0; tj < J; ++tj) {
                const int kend = std::min((tj + 1) * (GN / TILE), f.own_t);
                l21.push_back({q, ti, tj, 2 * kend});
            }
            for (int tj = 0; tj <= ti; ++tj) schur.push_back({q, ti, tj, 2 * f.own_t});
        }
    }
    auto longer = [](const GemmItem& a, const GemmItem& b) { return a.nst > b.nst; };
    std::stable_sort(l21.begin(), l21.end(), longer);
    std::stable_sort(schur.begin(), schur.end(), longer);
}

void launch_front_gemm(int mode, const GemmItem* d_items, long long n, const FrontGemmDesc* d_fronts, int* flag,
                       long long polls, cudaStream_t st) {
    if (n <= 0) return;
    static bool attr[2] = {false, false};
    if (!attr[mode]) {
        if (mode == GEMM_L21)
            HZ_CUDA(cudaFuncSetAttribute(k_front_gemm<GEMM_L21>, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM));
        else
            HZ_CUDA(cudaFuncSetAttribute(k_front_gemm<GEMM_SCHUR>, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM));
        attr[mode] = true;
    }
    for (long long b0 = 0; b0 < n; b0 += 65535LL * 16) {
        const unsigned grid = (unsigned)std::min<long long>(n - b0, 65535LL * 16);
        if (mode == GEMM_L21)
            k_front_gemm<GEMM_L21><<<grid, G_THREADS, G_SMEM, st>>>(d_items + b0, d_fronts, flag, polls);
        else
            k_front_gemm<GEMM_SCHUR><<<grid, G_THREADS, G_SMEM, st>>>(d_items + b0, d_fronts, flag, polls);
        HZ_CHECK_LAUNCH();
    }
}

}  // namespace hz
