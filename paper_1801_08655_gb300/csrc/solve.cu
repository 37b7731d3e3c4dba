// Multi-RHS forward/backward substitution through the packed multifrontal factors.
//
// This is the local solve w = (H^l)^{-1} g that every step of the online phase calls
// (Algorithm 2 local and inner solves; Algorithms 4-9 in the sweeps and the blocks of the
// polarized matrix).  With the diagonal blocks of the fronts stored inverted, each tree
// node costs four dense products on a block of columns:
//   forward  (leaves -> root):  z = Linv * acc[own];         acc[upd] -= L21 * z   (scatter)
//   backward (root -> leaves):  v = Dinv z - L21^T x[upd];   x[own]   = Linv^T * v
// Nodes of equal height are independent; a launch covers one phase of one height for all
// layers of a batch.  Every block computes a TILE-row slab of one product for a chunk of
// CC right-hand-side columns over a range of at most KS reduction tiles (split-K keeps the
// top of the tree, where a level has few nodes with long reductions, spread over the whole
// GPU).  Outputs are zeroed beforehand; a task covering the whole reduction of its rows stores
// them, split reductions and FB's update rows (shared between the nodes of a level) accumulate
// with atomics.  The factor tile stream is the HBM traffic that bounds the kernel at small
// column counts.  Complex64 blocks of >= 64 columns can instead run on the tensor-core kernels
// of subst_tc.cu; the autotuner decides per batch signature.
#include <algorithm>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"
#include "hz_solve.cuh"

namespace hz {

namespace {

enum { FA = 0, FB = 1, BA = 2, BB = 3 };

__device__ inline long long tri_idx(int rt, int ct) { return (long long)rt * (rt + 1) / 2 + ct; }

template <class C> __device__ inline void atomic_sub(C* p, C v);
template <> __device__ inline void atomic_sub<float2>(float2* p, float2 v) {
    atomicAdd(p, make_float2(-v.x, -v.y));
}
template <> __device__ inline void atomic_sub<double2>(double2* p, double2 v) {
    atomicAdd(&p->x, -v.x);
    atomicAdd(&p->y, -v.y);
}
template <class C> __device__ inline void atomic_add(C* p, C v) { atomic_sub(p, cneg(v)); }

// Writes the TILE x CC output block of one task, staged in shared memory (Ys, row pitch YP),
// to the solve vectors: consecutive threads take consecutive columns of a row, and every thread
// issues all of its loads (row indices, D^{-1}, z) before any of its writes.  A task covering
// the whole reduction of its rows is their only writer and stores; split reductions and FB
// (update rows are shared between the nodes of a level) accumulate atomically.  Outputs are
// zeroed beforehand (x before the forward pass and, for BB, by BA; acc before the backward).
template <class C, int CC, int MODE>
__device__ inline void write_out(const C* Ys, int YP, const JobDev<C>& jb, const NodeDev& nd, const int* upd,
                                 int tile, int col0, int ldc, int kt0, bool unique) {
    constexpr int EPT = (TILE * CC + 255) / 256;   // elements per thread
    constexpr int EB = EPT < 4 ? EPT : 4;          // elements per load batch
    const int nrows = (MODE == FB) ? nd.nupd : nd.nown;
#pragma unroll
    for (int i0 = 0; i0 < EPT; i0 += EB) {
        long long dst[EB];
        C y[EB], z[EB], di[EB];
        bool v[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) {
            const int e = threadIdx.x + 256 * (i0 + i);
            const int r = e / CC, c = e % CC;
            const int row = tile * TILE + r;
            v[i] = e < TILE * CC && row < nrows;
            dst[i] = 0;
            y[i] = czero<C>();
            z[i] = czero<C>();
            di[i] = czero<C>();
            if (v[i]) {
                dst[i] = ((MODE == FB) ? (long long)upd[row] : (long long)(nd.own0 + row)) * ldc + col0 + c;
                y[i] = Ys[r * YP + c];
                if (MODE == BA && kt0 == 0) {
                    di[i] = jb.dinv[nd.own0 + row];
                    z[i] = jb.x[dst[i]];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < EB; ++i) {
            if (!v[i]) continue;
            if (MODE == FB) {
                atomic_sub(jb.acc + dst[i], y[i]);
            } else if (MODE == FA || MODE == BB) {
                if (unique) jb.x[dst[i]] = y[i];
                else atomic_add(jb.x + dst[i], y[i]);
            } else {  // BA: acc = Dinv z - L21^T x_upd; the task with the first reduction tile clears z
                C val = y[i];
                if (kt0 == 0) {
                    val = csub(val, cmul(di[i], z[i]));
                    jb.x[dst[i]] = czero<C>();
                }
                if (unique) jb.acc[dst[i]] = cneg(val);
                else atomic_sub(jb.acc + dst[i], val);
            }
        }
    }
}

template <class C, int CC, int MODE>
__global__ void __launch_bounds__(256) k_subst(const Task* __restrict__ tasks,
                                               const JobDev<C>* __restrict__ jobs, int ldc, int nchunks,
                                               int KS) {
    constexpr int WC = CC >= 8 ? 8 : CC;  // warps along the columns
    constexpr int WK = 8 / WC;            // warps along the reduction dimension
    constexpr int NCT = CC / WC;          // columns per thread
    constexpr int KPW = TILE / WK;        // reduction indices per warp per tile
    __shared__ C Ms[TILE][TILE + 1];      // Ms[col][row] of the stored (column-major) tile
    __shared__ C Xs[TILE][CC];            // Xs[k][c]
    __shared__ C Red[WK > 1 ? WK : 1][WK > 1 ? TILE * CC : 1];

    const int chunk = blockIdx.x % nchunks;
    const Task tk = tasks[blockIdx.x / nchunks];
    const JobDev<C> jb = jobs[tk.job];
    const NodeDev nd = jb.nodes[tk.node];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int wc = warp % WC, wk = warp / WC;
    const int col0 = chunk * CC;

    // reduction range of this task: [tk.pad_ (first tile), +KS) within the product's range
    int kend;
    if (MODE == FA) kend = tk.tile + 1;
    else if (MODE == FB) kend = nd.own_t;
    else if (MODE == BA) kend = nd.upd_t;
    else kend = nd.own_t;
    const int kt0 = tk.pad_;
    const int kt1 = min(kend, kt0 + KS);

    const C* vec = (MODE == FA || MODE == BB) ? jb.acc : jb.x;
    const int* upd = jb.upd_idx + nd.upd_off;

    C acc[NCT];
#pragma unroll
    for (int u = 0; u < NCT; ++u) acc[u] = czero<C>();

    // register-staged prefetch: the next tile's loads are in flight while this tile is used
    constexpr int XPT = (TILE * CC + 255) / 256;   // vector elements per thread per tile
    auto mat_ptr = [&](int kt) -> const C* {
        if (MODE == FA) return jb.fac + (nd.linv_off + tri_idx(tk.tile, kt)) * TILE2;
        if (MODE == FB) return jb.fac + (nd.l21_off + (long long)tk.tile * nd.own_t + kt) * TILE2;
        if (MODE == BA) return jb.fac + (nd.l21_off + (long long)kt * nd.own_t + tk.tile) * TILE2;
        return jb.fac + (nd.linv_off + tri_idx(kt, tk.tile)) * TILE2;
    };
    C pm[TILE2 / 256], px[XPT];
    auto fetch = [&](int kt) {
        const C* mt = mat_ptr(kt);
#pragma unroll
        for (int i = 0; i < TILE2 / 256; ++i) pm[i] = mt[t + i * 256];
#pragma unroll
        for (int i = 0; i < XPT; ++i) {
            const int e = t + i * 256;
            C v = czero<C>();
            if (e < TILE * CC) {
                const int k = e / CC, c = e % CC;
                const int r = kt * TILE + k;
                if (MODE == BA) {
                    if (r < nd.nupd) v = vec[(long long)upd[r] * ldc + col0 + c];
                } else {
                    if (r < nd.nown) v = vec[(long long)(nd.own0 + r) * ldc + col0 + c];
                }
            }
            px[i] = v;
        }
    };
    if (kt0 < kt1) fetch(kt0);
    for (int kt = kt0; kt < kt1; ++kt) {
#pragma unroll
        for (int i = 0; i < TILE2 / 256; ++i) {
            const int e = t + i * 256;
            Ms[e / TILE][e % TILE] = pm[i];
        }
#pragma unroll
        for (int i = 0; i < XPT; ++i) {
            const int e = t + i * 256;
            if (e < TILE * CC) Xs[e / CC][e % CC] = px[i];
        }
        __syncthreads();
        if (kt + 1 < kt1) fetch(kt + 1);
#pragma unroll 4
        for (int kk = 0; kk < KPW; ++kk) {
            const int k = wk * KPW + kk;
            const C a = (MODE == FA || MODE == FB) ? Ms[k][lane] : Ms[lane][k];
#pragma unroll
            for (int u = 0; u < NCT; ++u) cfma(acc[u], a, Xs[k][wc * NCT + u]);
        }
        __syncthreads();
    }

    // stage the TILE x CC outputs in Ms (free after the loop), then write them row-wise
    if (WK > 1) {
#pragma unroll
        for (int u = 0; u < NCT; ++u) Red[wk][lane * CC + wc * NCT + u] = acc[u];
        __syncthreads();
        if (wk == 0) {
#pragma unroll
            for (int u = 0; u < NCT; ++u) {
                C s = czero<C>();
                for (int q = 0; q < WK; ++q) s = cadd(s, Red[q][lane * CC + wc * NCT + u]);
                acc[u] = s;
            }
        }
    }
    if (wk == 0) {
#pragma unroll
        for (int u = 0; u < NCT; ++u) Ms[lane][wc * NCT + u] = acc[u];
    }
    __syncthreads();
    const bool unique = kt0 == ((MODE == BB) ? tk.tile : 0) && kt1 == kend;
    write_out<C, CC, MODE>(&Ms[0][0], TILE + 1, jb, nd, upd, tk.tile, col0, ldc, kt0, unique);
}

// 64-column variant for complex64: each thread owns a 2-row x 4-column register tile, fed by
// three 16-byte shared loads per 8 complex MACs.  The factor tile is kept as [k][row] in shared
// memory (rows padded to 34 complex, so every row pair is one aligned 16-byte load), transposed
// on the way in for the transposed phases.
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_subst64(const Task* __restrict__ tasks,
                                                    const JobDev<float2>* __restrict__ jobs, int ldc, int nchunks,
                                                    int KS) {
    constexpr int CC = 64;
    constexpr int MS = 34;                       // padded row length (complex) of the [k][row] tile
    constexpr int XP = CC + 2;                   // padded row length of the vector / output tile
    __shared__ __align__(16) float2 Ms[TILE][MS];
    __shared__ __align__(16) float2 Xs[TILE][XP];

    const int chunk = blockIdx.x % nchunks;
    const Task tk = tasks[blockIdx.x / nchunks];
    const JobDev<float2> jb = jobs[tk.job];
    const NodeDev nd = jb.nodes[tk.node];
    const int t = threadIdx.x;
    const int rp = t & 15, cq = t >> 4;          // rows 2rp, 2rp+1; columns 4cq .. 4cq+3
    const int col0 = chunk * CC;

    int kend;
    if (MODE == FA) kend = tk.tile + 1;
    else if (MODE == FB) kend = nd.own_t;
    else if (MODE == BA) kend = nd.upd_t;
    else kend = nd.own_t;
    const int kt0 = tk.pad_;
    const int kt1 = min(kend, kt0 + KS);
    const float2* vec = (MODE == FA || MODE == BB) ? jb.acc : jb.x;
    const int* upd = jb.upd_idx + nd.upd_off;

    float2 acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    auto mat_ptr = [&](int kt) -> const float2* {
        if (MODE == FA) return jb.fac + (nd.linv_off + tri_idx(tk.tile, kt)) * TILE2;
        if (MODE == FB) return jb.fac + (nd.l21_off + (long long)tk.tile * nd.own_t + kt) * TILE2;
        if (MODE == BA) return jb.fac + (nd.l21_off + (long long)kt * nd.own_t + tk.tile) * TILE2;
        return jb.fac + (nd.linv_off + tri_idx(kt, tk.tile)) * TILE2;
    };
    float2 pm[4], px[8];
    auto fetch = [&](int kt) {
        const float2* mt = mat_ptr(kt);
#pragma unroll
        for (int i = 0; i < 4; ++i) pm[i] = mt[t + i * 256];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = t + i * 256;
            const int k = e >> 6, c = e & 63;
            const int r = kt * TILE + k;
            float2 v = make_float2(0.f, 0.f);
            if (MODE == BA) {
                if (r < nd.nupd) v = vec[(long long)upd[r] * ldc + col0 + c];
            } else {
                if (r < nd.nown) v = vec[(long long)(nd.own0 + r) * ldc + col0 + c];
            }
            px[i] = v;
        }
    };
    if (kt0 < kt1) fetch(kt0);
    for (int kt = kt0; kt < kt1; ++kt) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = t + i * 256;           // stored element (row e % 32, column e / 32)
            if (MODE == FA || MODE == FB) Ms[e >> 5][e & 31] = pm[i];   // A(row, k) = stored(row, k)
            else Ms[e & 31][e >> 5] = pm[i];                              // A(row, k) = stored(k, row)
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = t + i * 256;
            Xs[e >> 6][e & 63] = px[i];
        }
        __syncthreads();
        if (kt + 1 < kt1) fetch(kt + 1);
#pragma unroll 8
        for (int k = 0; k < TILE; ++k) {
            const float4 a2 = *(const float4*)&Ms[k][2 * rp];
            const float4 x01 = *(const float4*)&Xs[k][4 * cq];
            const float4 x23 = *(const float4*)&Xs[k][4 * cq + 2];
            const float2 a0 = make_float2(a2.x, a2.y), a1 = make_float2(a2.z, a2.w);
            const float2 xs[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w),
                                  make_float2(x23.x, x23.y), make_float2(x23.z, x23.w)};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cfma(acc[0][j], a0, xs[j]);
                cfma(acc[1][j], a1, xs[j]);
            }
        }
        __syncthreads();
    }

    // stage the 32 x 64 outputs in Xs (free after the loop), then write them row-wise
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        *(float4*)&Xs[2 * rp + i][4 * cq] = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
        *(float4*)&Xs[2 * rp + i][4 * cq + 2] = make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y);
    }
    __syncthreads();
    const bool unique = kt0 == ((MODE == BB) ? tk.tile : 0) && kt1 == kend;
    write_out<float2, CC, MODE>(&Xs[0][0], XP, jb, nd, upd, tk.tile, col0, ldc, kt0, unique);
}

template <class C, int CC>
void launch_level(const Batch& b, int h, int mode, int ldc, cudaStream_t st) {
    const int nchunks = (b.job_cols > 0 ? b.job_cols : ldc) / CC;
    const long long off = b.off[mode][h], n = b.cnt[mode][h];
    if (n == 0) return;
    const Task* tasks = b.d_tasks + off;
    const JobDev<C>* jobs = (const JobDev<C>*)b.d_jobs;
    dim3 grid((unsigned)(n * nchunks));
    if constexpr (CC == 64 && sizeof(C) == 8) {
        const JobDev<float2>* j64 = (const JobDev<float2>*)b.d_jobs;
        switch (mode) {
            case FA: k_subst64<FA><<<grid, 256, 0, st>>>(tasks, j64, ldc, nchunks, b.KS); break;
            case FB: k_subst64<FB><<<grid, 256, 0, st>>>(tasks, j64, ldc, nchunks, b.KS); break;
            case BA: k_subst64<BA><<<grid, 256, 0, st>>>(tasks, j64, ldc, nchunks, b.KS); break;
            default: k_subst64<BB><<<grid, 256, 0, st>>>(tasks, j64, ldc, nchunks, b.KS); break;
        }
    } else {
        switch (mode) {
            case FA: k_subst<C, CC, FA><<<grid, 256, 0, st>>>(tasks, jobs, ldc, nchunks, b.KS); break;
            case FB: k_subst<C, CC, FB><<<grid, 256, 0, st>>>(tasks, jobs, ldc, nchunks, b.KS); break;
            case BA: k_subst<C, CC, BA><<<grid, 256, 0, st>>>(tasks, jobs, ldc, nchunks, b.KS); break;
            default: k_subst<C, CC, BB><<<grid, 256, 0, st>>>(tasks, jobs, ldc, nchunks, b.KS); break;
        }
    }
    HZ_CHECK_LAUNCH();
}

template <class C>
void zero_vectors(const Batch& b, bool x_vec, int ldc, cudaStream_t st) {
    for (size_t j = 0; j < b.vec_ptrs.size(); ++j) {
        void* p = x_vec ? b.vec_ptrs[j].second : b.vec_ptrs[j].first;
        HZ_CUDA(cudaMemsetAsync(p, 0, (size_t)b.vec_rows[j] * ldc * sizeof(C), st));
    }
}

// Records a CUDA event pair around one launch in profiling detail mode.
struct LaunchTimer {
    std::vector<ProfRec>* out;
    cudaStream_t st;
    ProfRec r{};
    LaunchTimer(std::vector<ProfRec>* o, cudaStream_t s, int kind, double bytes, double flops, int mode, int level,
                long long tasks)
        : out(o), st(s) {
        if (!out) return;
        r.kind = kind;
        r.mode = mode;
        r.level = level;
        r.tasks = tasks;
        r.bytes = bytes;
        r.flops = flops;
        HZ_CUDA(cudaEventCreate(&r.e0));
        HZ_CUDA(cudaEventCreate(&r.e1));
        HZ_CUDA(cudaEventRecord(r.e0, st));
    }
    void done() {
        if (!out) return;
        HZ_CUDA(cudaEventRecord(r.e1, st));
        out->push_back(r);
    }
};

template <class C, int CC>
void run_batch(const Batch& b, int ldc, int ncols, bool tc, int* flag, cudaStream_t st, std::vector<ProfRec>* pl) {
    auto level = [&](int h, int mode) {
        if (b.cnt[mode][h] > 0) {
            LaunchTimer lt(pl, st, 0, b.lvl_bytes[0][mode][h], b.lvl_flops[0][mode][h] * ncols, mode, h, b.cnt[mode][h]);
            launch_level<C, CC>(b, h, mode, ldc, st);
            lt.done();
        }
        if (tc && b.pair_cnt[mode][h] > 0) {
            LaunchTimer lt(pl, st, 1, b.lvl_bytes[1][mode][h], b.lvl_flops[1][mode][h] * ncols, mode, h,
                           b.pair_cnt[mode][h]);
            launch_level_tc(b, h, mode, ldc, flag, st);
            lt.done();
        }
    };
    zero_vectors<C>(b, true, ldc, st);
    for (int h = 0; h < b.H; ++h)
        for (int mode : {FA, FB}) level(h, mode);
    zero_vectors<C>(b, false, ldc, st);
    for (int h = b.H - 1; h >= 0; --h)
        for (int mode : {BA, BB}) level(h, mode);
}

}  // namespace

int chunk_cols(bool is_double, int ncols) {
    const int cmax = is_double ? 32 : 64;
    int c = 1;
    while (c < ncols && c < cmax) c *= 2;
    return c;
}

int padded_ldc(bool is_double, int ncols) {
    const int cc = chunk_cols(is_double, ncols);
    return (ncols + cc - 1) / cc * cc;
}

template <class C>
void substitute(Ctx& ctx, const Batch& b, int ncols, cudaStream_t st) {
    const bool dbl = sizeof(C) == 16;
    const int ldc = padded_ldc(dbl, ncols);
    const int cc = (b.CC > 0 && ldc % b.CC == 0) ? b.CC : chunk_cols(dbl, ncols);
    ProfRec rec{};
    if (ctx.prof) {
        HZ_CUDA(cudaEventCreate(&rec.e0));
        HZ_CUDA(cudaEventCreate(&rec.e1));
        HZ_CUDA(cudaEventRecord(rec.e0, st));
    }
    const bool tc = b.tc;
    int* flag = ctx.d_flag + 1;
    std::vector<ProfRec>* pl = (ctx.prof && ctx.prof_detail) ? &ctx.prof_launch : nullptr;
    switch (cc) {
        case 1: run_batch<C, 1>(b, ldc, ncols, tc, flag, st, pl); break;
        case 2: run_batch<C, 2>(b, ldc, ncols, tc, flag, st, pl); break;
        case 4: run_batch<C, 4>(b, ldc, ncols, tc, flag, st, pl); break;
        case 8: run_batch<C, 8>(b, ldc, ncols, tc, flag, st, pl); break;
        case 16: run_batch<C, 16>(b, ldc, ncols, tc, flag, st, pl); break;
        case 32: run_batch<C, 32>(b, ldc, ncols, tc, flag, st, pl); break;
        default:
            if constexpr (sizeof(C) == 8) run_batch<C, 64>(b, ldc, ncols, tc, flag, st, pl);
            else throw Error{HZ_ERR_ARG, "chunk width"};
    }
    if (ctx.prof) {
        HZ_CUDA(cudaEventRecord(rec.e1, st));
        rec.bytes = b.alg_bytes;
        rec.flops = b.flops_per_col * ncols;
        ctx.prof_recs.push_back(rec);
    }
}

// Tensor-core eligibility of one node product: at least min_tiles output tiles and a reduction
// over at least two tiles (of any length when min_tiles <= 2, the autotuner's candidate that
// puts almost every product on the tensor cores).
static bool tc_node(int mode, const Node& nd, int min_tiles) {
    const int out_t = mode == 1 ? nd.upd_t : nd.own_t;
    const int red_t = mode == 2 ? nd.upd_t : nd.own_t;
    return out_t >= min_tiles && red_t >= (min_tiles <= 2 ? 1 : 2);
}

static std::string tune_key(const Ctx& ctx, const std::vector<int>& layers, int ldc, int split, int sparse) {
    std::vector<int> shapes;
    for (int l : layers) shapes.push_back(ctx.layers[l].shape);
    std::sort(shapes.begin(), shapes.end());
    std::string key = "n" + std::to_string(ldc) + (split == 1 ? "s1" : "") + (sparse ? "p" + std::to_string(sparse) : "") + ":";
    for (int s : shapes) key += std::to_string(s) + ",";
    return key;
}

template <class C>
Batch& get_batch(Ctx& ctx, const std::vector<int>& layers, int ncols, int split, int sparse) {
    const bool dbl = sizeof(C) == 16;
    const int ldc = padded_ldc(dbl, ncols);
    const bool tc_ok = !dbl && tc_columns(ldc) > 0;
    auto it = ctx.tuned.find(tune_key(ctx, layers, ldc, split, sparse));
    if (it != ctx.tuned.end()) {
        const auto& ch = it->second;
        return get_batch_cfg<C>(ctx, layers, ncols, ch.KS, ch.CC, tc_ok && ch.tc, ch.KS_tc, ch.min_t, split, ch.tc_cfg,
                                sparse);
    }
    // default: split the reductions when the batch alone cannot fill the GPU
    const int nchunks = ldc / chunk_cols(dbl, ncols);
    const int KS = ((long long)layers.size() * nchunks >= 64) ? (1 << 30) : 8;
    const bool tc = tc_ok && ctx.tc_mode == 1;
    const int nchunks_tc = tc ? ldc / tc_columns(ldc) : 1;
    const int KS_tc = ((long long)layers.size() * nchunks_tc >= 32) ? (1 << 30) : ctx.tc_ks;
    return get_batch_cfg<C>(ctx, layers, ncols, KS, 0, tc, KS_tc, ctx.tc_min_tiles, split, ctx.tc_cfg, sparse);
}

template <class C>
void ensure_tuned(Ctx& ctx, const std::vector<int>& layers, int ncols, int split, int sparse) {
    const bool dbl = sizeof(C) == 16;
    const int ldc = padded_ldc(dbl, ncols);
    const bool tc_ok = !dbl && tc_columns(ldc) > 0;
    const std::string key = tune_key(ctx, layers, ldc, split, sparse);
    if (!ctx.autotune || ctx.tuned.count(key)) return;
    const int cc0 = chunk_cols(dbl, ncols);
    std::vector<Ctx::TuneChoice> cands;
    const bool try_tc = tc_ok && ctx.tc_mode >= 1;
    if (ctx.tc_mode != 1 || !tc_ok) {
        // CUDA-core candidates (fewer when the tensor-core kernel competes for these columns)
        std::vector<int> ccs{cc0};
        if (!try_tc && cc0 >= 16 && ldc % (cc0 / 2) == 0) ccs.push_back(cc0 / 2);
        for (int cc : ccs)
            for (int ks : {4, 8, 16, 1 << 30})
                if (!try_tc || ks == 8 || ks == (1 << 30)) cands.push_back({ks, cc, 0, 1 << 30, 0, 0});
    }
    if (try_tc)
        for (int cfg : {1, 0})   // persistent / one block per work item
            for (int mt : {2, 4, ctx.tc_min_tiles})
                for (int kstc : {16, 1 << 30}) cands.push_back({8, cc0, 1, kstc, mt, cfg});
    cudaEvent_t e0, e1;
    HZ_CUDA(cudaEventCreate(&e0));
    HZ_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Ctx::TuneChoice choice = cands.front();
    const bool prof = ctx.prof;
    ctx.prof = false;
    std::string log = key + " ->";
    for (const auto& cd : cands) {
        Batch& b = get_batch_cfg<C>(ctx, layers, ncols, cd.KS, cd.CC, cd.tc != 0, cd.KS_tc, cd.min_t, split, cd.tc_cfg,
                                    sparse);
        for (size_t j = 0; j < b.vec_ptrs.size(); ++j)
            HZ_CUDA(cudaMemsetAsync(b.vec_ptrs[j].first, 0, (size_t)b.vec_rows[j] * ldc * sizeof(C), ctx.stream));
        substitute<C>(ctx, b, ncols, ctx.stream);  // warm-up
        HZ_CUDA(cudaEventRecord(e0, ctx.stream));
        substitute<C>(ctx, b, ncols, ctx.stream);
        HZ_CUDA(cudaEventRecord(e1, ctx.stream));
        HZ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        HZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const int ks_shown = cd.tc ? cd.KS_tc : cd.KS;
        log += std::string(cd.tc ? " (TC, KS " : " (KS ") + std::to_string(ks_shown > 1000 ? 0 : ks_shown) +
               ", CC " + std::to_string(cd.CC) +
               (cd.tc ? ", min " + std::to_string(cd.min_t) + ", cfg " + std::to_string(cd.tc_cfg) : std::string()) + ") " +
               std::to_string(ms) + " ms;";
        if (ms < best) { best = ms; choice = cd; }
    }
    ctx.prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx.tuned[key] = choice;
    ctx.tune_log.push_back(log);
}

template <class C>
Batch& get_batch_cfg(Ctx& ctx, const std::vector<int>& layers, int ncols, int KS, int CC, bool tc, int KS_tc,
                     int min_t, int split, int tc_cfg, int sparse) {
    const bool dbl = sizeof(C) == 16;
    const int ldc = padded_ldc(dbl, ncols);
    std::string key = "KS" + std::to_string(KS) + "C" + std::to_string(CC) + "n" + std::to_string(ldc) +
                      (tc ? "tc" + std::to_string(KS_tc) + "m" + std::to_string(min_t) + "s" + std::to_string(split) +
                                "c" + std::to_string(tc_cfg)
                          : "") + "p" + std::to_string(sparse) + ":";
    for (int l : layers) key += std::to_string(l) + ",";
    auto it = ctx.batches.find(key);
    if (it != ctx.batches.end()) return it->second;
    Batch b;
    b.layers = layers;
    b.KS = KS;
    b.CC = CC;
    b.tc = tc;
    b.KS_tc = KS_tc;
    b.min_t = min_t;
    b.split = split;
    b.tc_cfg = tc_cfg;
    b.sparse = sparse;
    b.wait_polls = ctx.tc_wait_polls;
    // per-block sparsity: job j * nblk + q is block q (columns [q * job_cols, (q + 1) * job_cols))
    // of layer j; the caller has checked that the blocks tile the columns in whole chunks
    const int nblk = block_count(sparse);
    if (nblk > 1 && (ncols % nblk != 0 || (ncols / nblk) % 64 != 0 || ldc != ncols))
        throw Error{HZ_ERR_ARG, "per-block sparsity needs column blocks of a multiple of 64"};
    b.job_cols = nblk > 1 ? ncols / nblk : 0;
    int H = 0;
    for (int l : layers) H = std::max(H, (int)ctx.shapes[ctx.layers[l].shape].levels.size());
    b.H = H;
    std::vector<std::vector<Task>> lists[4], quads[4];
    for (auto& v : lists) v.assign(H, {});
    for (auto& v : quads) v.assign(H, {});
    for (int k = 0; k < 2; ++k)
        for (int mode = 0; mode < 4; ++mode) {
            b.lvl_bytes[k][mode].assign(H, 0.0);
            b.lvl_flops[k][mode].assign(H, 0.0);
        }
    auto add_tasks = [&](std::vector<Task>& out, int j, int nid, int tile, int k0, int k1, int ks) {
        if (k1 <= k0) { out.push_back(Task{j, nid, tile, k0}); return; }
        for (int k = k0; k < k1; k += ks) out.push_back(Task{j, nid, tile, k});
    };
    for (int j = 0; j < (int)layers.size(); ++j) {
        const Layer& ly = ctx.layers[layers[j]];
        const Shape& sh = ctx.shapes[ly.shape];
        // local z planes that carry the interface sources (forward) and read-outs (backward) of
        // this layer: the plane pair next to its top interface and/or the pair next to its bottom
        // interface, as the batch's sparsity code selects (SP_*, forward in bits 0-1, backward in
        // bits 2-3).  A node whose subtree box misses every forward plane has a zero forward
        // result; one that misses every backward plane has no read-out below it.
        auto plane_set = [&](int code) {
            std::vector<int> pl;
            const bool top = layers[j] > 0, bot = layers[j] < ctx.L - 1;
            if (top && (code == SP_BOTH || code == SP_TOP)) { pl.push_back(ly.lo - 1 - ly.zlo); pl.push_back(ly.lo - ly.zlo); }
            if (bot && (code == SP_BOTH || code == SP_BOT)) { pl.push_back(ly.hi - ly.zlo); pl.push_back(ly.hi + 1 - ly.zlo); }
            return pl;
        };
        int fcode[4], bcode[4];
        std::vector<int> fplanes[4], bplanes[4];
        for (int q = 0; q < nblk; ++q) {
            const int code = block_code(sparse, q);
            fcode[q] = code & 3;
            bcode[q] = (code >> 2) & 3;
            fplanes[q] = plane_set(fcode[q]);
            bplanes[q] = plane_set(bcode[q]);
        }
        for (int h = 0; h < (int)sh.levels.size(); ++h)
            for (int nid : sh.levels[h]) {
                const Node& nd = sh.nodes[nid];
                auto touches = [&](const std::vector<int>& pl) {
                    for (int z : pl)
                        if (z >= nd.box[4] && z < nd.box[5]) return true;
                    return false;
                };
                for (int mode = 0; mode < 4; ++mode) {
                    const bool fwd = mode == FA || mode == FB;
                    const int out_t = mode == 1 ? nd.upd_t : nd.own_t;
                    const bool on_tc = tc && tc_node(mode, nd, b.min_t);
                    int nact = 0;
                    for (int q = 0; q < nblk; ++q) {
                        const bool on = fwd ? (fcode[q] == SP_ALL || touches(fplanes[q]))
                                            : (bcode[q] == SP_ALL || touches(bplanes[q]));
                        if (!on) continue;
                        ++nact;
                        const int jq = j * nblk + q;
                        if (on_tc) {
                            for (int t = 0; t < out_t; t += 4) {
                                if (mode == 0) add_tasks(quads[0][h], jq, nid, t, 0, std::min(t + 4, nd.own_t), b.KS_tc);
                                if (mode == 1) add_tasks(quads[1][h], jq, nid, t, 0, nd.own_t, b.KS_tc);
                                if (mode == 2) add_tasks(quads[2][h], jq, nid, t, 0, nd.upd_t, b.KS_tc);
                                if (mode == 3) add_tasks(quads[3][h], jq, nid, t, t, nd.own_t, b.KS_tc);
                            }
                        } else {
                            for (int t = 0; t < out_t; ++t) {
                                if (mode == 0) add_tasks(lists[0][h], jq, nid, t, 0, t + 1, KS);      // FA: Linv row tile t
                                if (mode == 1) add_tasks(lists[1][h], jq, nid, t, 0, nd.own_t, KS);   // FB: L21 row tile t
                                if (mode == 2) add_tasks(lists[2][h], jq, nid, t, 0, nd.upd_t, KS);   // BA (>= 1 task)
                                if (mode == 3) add_tasks(lists[3][h], jq, nid, t, t, nd.own_t, KS);   // BB
                            }
                        }
                    }
                    if (nact == 0) continue;
                    // stored factor entries this product reads (triangular L^{-1} or L21): once
                    // algorithmically, however many column blocks use them
                    const double ent = (mode == FA || mode == BB) ? (double)nd.nown * (nd.nown + 1) / 2.0
                                                                  : (double)nd.nown * nd.nupd;
                    b.lvl_bytes[on_tc][mode][h] += ent * sizeof(C);
                    b.lvl_flops[on_tc][mode][h] += 8.0 * ent * nact / nblk;
                }
            }
    }
    // tensor-core work items longest reduction first: the persistent kernel deals them out
    // round-robin, and either kernel then ends a launch on short items
    for (int mode = 0; mode < 4; ++mode)
        for (int h = 0; h < H; ++h) {
            auto red_len = [&](const Task& tk) {
                const Node& nd = ctx.shapes[ctx.layers[layers[tk.job / nblk]].shape].nodes[tk.node];
                const int kend = mode == 0 ? std::min(tk.tile + 4, nd.own_t) : (mode == 2 ? nd.upd_t : nd.own_t);
                return std::min(kend, tk.pad_ + std::min(b.KS_tc, 1 << 28)) - tk.pad_;
            };
            std::stable_sort(quads[mode][h].begin(), quads[mode][h].end(),
                             [&](const Task& x, const Task& y) { return red_len(x) > red_len(y); });
        }
    std::vector<Task> all;
    for (int mode = 0; mode < 4; ++mode) {
        b.pair_off[mode].assign(H, 0);
        b.pair_cnt[mode].assign(H, 0);
        for (int h = 0; h < H; ++h) {
            b.pair_off[mode][h] = (long long)all.size();
            b.pair_cnt[mode][h] = (long long)quads[mode][h].size();
            all.insert(all.end(), quads[mode][h].begin(), quads[mode][h].end());
        }
    }
    for (int mode = 0; mode < 4; ++mode) {
        b.off[mode].assign(H, 0);
        b.cnt[mode].assign(H, 0);
        for (int h = 0; h < H; ++h) {
            b.off[mode][h] = (long long)all.size();
            b.cnt[mode][h] = (long long)lists[mode][h].size();
            all.insert(all.end(), lists[mode][h].begin(), lists[mode][h].end());
        }
    }
    HZ_CUDA(cudaMalloc(&b.d_tasks, std::max<size_t>(1, all.size()) * sizeof(Task)));
    HZ_CUDA(cudaMemcpyAsync(b.d_tasks, all.data(), all.size() * sizeof(Task), cudaMemcpyHostToDevice, ctx.stream));
    HZ_CUDA(cudaStreamSynchronize(ctx.stream));
    std::vector<JobDev<C>> jobs;
    for (int l : layers) {
        const Layer& ly = ctx.layers[l];
        const Shape& sh = ctx.shapes[ly.shape];
        for (int q = 0; q < nblk; ++q) {
            JobDev<C> jd;
            jd.fac = (const C*)ly.d_fac;
            jd.dinv = (const C*)ly.d_dinv;
            jd.nodes = sh.d_nodes;
            jd.upd_idx = sh.d_upd_idx;
            jd.acc = (C*)ctx.slot_acc[l] + (long long)q * b.job_cols;
            jd.x = (C*)ctx.slot_x[l] + (long long)q * b.job_cols;
            jobs.push_back(jd);
        }
        b.vec_ptrs.push_back({ctx.slot_acc[l], ctx.slot_x[l]});
        b.vec_rows.push_back(sh.N);
    }
    // algorithmic work of the products this batch runs (each stored factor entry of an active
    // product read once, 8 real flops per entry and column)
    for (int k = 0; k < 2; ++k)
        for (int mode = 0; mode < 4; ++mode)
            for (int h = 0; h < H; ++h) {
                b.alg_bytes += b.lvl_bytes[k][mode][h];
                b.flops_per_col += b.lvl_flops[k][mode][h];
            }
    HZ_CUDA(cudaMalloc(&b.d_jobs, jobs.size() * sizeof(JobDev<C>)));
    HZ_CUDA(cudaMemcpyAsync(b.d_jobs, jobs.data(), jobs.size() * sizeof(JobDev<C>), cudaMemcpyHostToDevice,
                            ctx.stream));
    HZ_CUDA(cudaStreamSynchronize(ctx.stream));
    return ctx.batches.emplace(key, b).first->second;
}

void free_batches(Ctx& ctx) {
    for (auto& kv : ctx.batches) {
        cudaFree(kv.second.d_tasks);
        cudaFree(kv.second.d_jobs);
    }
    ctx.batches.clear();
}

template void substitute<float2>(Ctx&, const Batch&, int, cudaStream_t);
template void substitute<double2>(Ctx&, const Batch&, int, cudaStream_t);
template Batch& get_batch<float2>(Ctx&, const std::vector<int>&, int, int, int);
template Batch& get_batch<double2>(Ctx&, const std::vector<int>&, int, int, int);
template Batch& get_batch_cfg<float2>(Ctx&, const std::vector<int>&, int, int, int, bool, int, int, int, int, int);
template Batch& get_batch_cfg<double2>(Ctx&, const std::vector<int>&, int, int, int, bool, int, int, int, int, int);
template void ensure_tuned<float2>(Ctx&, const std::vector<int>&, int, int, int);
template void ensure_tuned<double2>(Ctx&, const std::vector<int>&, int, int, int);

}  // namespace hz
