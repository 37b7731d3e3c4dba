// Numeric multifrontal factorization of the local operators (Algorithm 1).
//
// Per layer and per tree node, a dense front F (own + update unknowns, column-major,
// lower triangle) is assembled from the original 7-point entries of the local operator
// H^l (Eq. 8 with the PML stretching of Eqs. 3-5) and the children's Schur complements
// (extend-add), then partially factored F11 = L11 D L11^T (unpivoted complex-symmetric
// LDL^T, right-looking in panels of TILE columns, pivot blocks in FP64), L21 = F21 L11^{-T} D^{-1},
// Schur complement F22 - L21 D L21^T for the parent.  L11 is then inverted explicitly
// (selective inversion, the alternative the paper cites for parallel triangular solves in
// its Local Solves section) so that every substitution step becomes a dense
// matrix-times-block product; L^{-1} and L21 are packed into TILE x TILE tiles.
//
// Fronts of all nodes at the same tree height, across a group of layers, are processed by
// the same launches.
#include <algorithm>
#include <cmath>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"

namespace hz {

namespace {

template <class C> struct FrontDesc {
    C* F;                 // dense front (m x m, column-major)
    C* fac;               // layer's packed factor tiles
    C* dinv;              // layer's D^{-1} (elimination indexed)
    const AsmEntry* ent;  // this node's assembly entries
    long long linv_off, l21_off;
    int m, nown, nupd, own0, nasm, layer;
    int lim;              // rows/columns the panel steps update: m, or nown when the L21 and Schur
                          // products run on the tensor cores afterwards (factor_tc.cu)
    int tc;               // 1: L21 and the Schur update come from the tensor-core products
};

template <class C> struct ExtDesc {
    C* P;                 // parent front
    const C* F;           // child front
    const int* emap;      // child update index -> parent front position
    int mp, mc, ownc, nupdc;
};

__device__ inline long long tri_index(int rt, int ct) { return (long long)rt * (rt + 1) / 2 + ct; }

// Stencil coefficient of the local operator for the column unknown `cell` and direction d
// (0 = diagonal, 1..6 = x-, x+, y-, y+, z-, z+), in FP64: symmetric form of the stretched
// 7-point operator (s_a at half nodes for the derivative along a, at nodes otherwise), times b at
// the half node for a variable density (div(b grad u), b = 1/rho).
__device__ double2 stencil_coef(const LayerCoef& lc, int cell, int d) {
    int x = cell % lc.nx;
    int y = (cell / lc.nx) % lc.ny;
    int z = cell / (lc.nx * lc.ny);
    double2 sx = lc.sx_n[x], sy = lc.sy_n[y], sz = lc.sz_n[z];
    double2 syz = cmul(sy, sz), sxz = cmul(sx, sz), sxy = cmul(sx, sy);
    double2 c[7];
    c[1] = cscale(cmul(syz, lc.isx_h[x]), lc.inv_h2);
    c[2] = cscale(cmul(syz, lc.isx_h[x + 1]), lc.inv_h2);
    c[3] = cscale(cmul(sxz, lc.isy_h[y]), lc.inv_h2);
    c[4] = cscale(cmul(sxz, lc.isy_h[y + 1]), lc.inv_h2);
    c[5] = cscale(cmul(sxy, lc.isz_h[z]), lc.inv_h2);
    c[6] = cscale(cmul(sxy, lc.isz_h[z + 1]), lc.inv_h2);
    if (lc.b) {   // variable density: b at the half nodes
        const long long P = (long long)lc.nx * lc.ny;
        c[1] = cscale(c[1], bhalf(lc.b, cell, x, lc.nx, 1, -1));
        c[2] = cscale(c[2], bhalf(lc.b, cell, x, lc.nx, 1, +1));
        c[3] = cscale(c[3], bhalf(lc.b, cell, y, lc.ny, lc.nx, -1));
        c[4] = cscale(c[4], bhalf(lc.b, cell, y, lc.ny, lc.nx, +1));
        c[5] = cscale(c[5], bhalf(lc.b, cell, z, lc.nzl, P, -1));
        c[6] = cscale(c[6], bhalf(lc.b, cell, z, lc.nzl, P, +1));
    }
    if (d > 0) return c[d];
    double2 dg = cscale(cmul(sxy, sz), lc.omega2 * lc.m[cell]);
    for (int k = 1; k <= 6; ++k) dg = csub(dg, c[k]);
    return dg;
}

template <class C>
__global__ void k_assemble(const FrontDesc<C>* fd, const LayerCoef* coefs) {
    const FrontDesc<C>& f = fd[blockIdx.y];
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= f.nasm) return;
    AsmEntry a = f.ent[e];
    double2 v = stencil_coef(coefs[f.layer], a.cell, a.dir);
    f.F[a.foff] = from_d<C>(v);
}

template <class C>
__global__ void k_extend_add(const ExtDesc<C>* ed) {
    const ExtDesc<C>& e = ed[blockIdx.y];
    long long n = (long long)e.nupdc * e.nupdc;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        int a = (int)(q % e.nupdc), b = (int)(q / e.nupdc);
        if (a < b) continue;
        C v = e.F[(long long)(e.ownc + a) + (long long)(e.ownc + b) * e.mc];
        long long dst = (long long)e.emap[a] + (long long)e.emap[b] * e.mp;
        e.P[dst] = cadd(e.P[dst], v);
    }
}

// Diagonal block of panel k0: unpivoted LDL^T in FP64 in shared memory, D and D^{-1}
// stored, and the inverse of the unit lower block written as the packed diagonal tile.
template <class C>
__global__ void k_diag(const FrontDesc<C>* fd, int k0, int* flag) {
    const FrontDesc<C>& f = fd[blockIdx.x];
    if (k0 >= f.nown) return;
    const int nb = min(TILE, f.nown - k0);
    __shared__ double2 a[TILE][TILE + 1];
    __shared__ double2 xinv[TILE][TILE + 1];
    __shared__ double2 dinv_s[TILE];
    const int t = threadIdx.x;
    for (int q = t; q < TILE * TILE; q += blockDim.x) {
        int i = q % TILE, j = q / TILE;
        double2 v = make_double2(0.0, 0.0);
        if (i < nb && j < nb && i >= j) v = to_d(f.F[(long long)(k0 + i) + (long long)(k0 + j) * f.m]);
        a[i][j] = v;
    }
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        double2 d = a[k][k];
        double dd = d.x * d.x + d.y * d.y;
        if (t == 0) {
            if (!(dd > 1e-280) || !isfinite(dd)) atomicExch(flag, 1);
            dinv_s[k] = (dd > 0.0) ? crecip(d) : make_double2(0.0, 0.0);
        }
        __syncthreads();
        double2 di = dinv_s[k];
        int cnt = nb - k - 1;
        for (int q = t; q < cnt * cnt; q += blockDim.x) {
            int i = k + 1 + q % cnt, j = k + 1 + q / cnt;
            if (i >= j) a[i][j] = csub(a[i][j], cmul(cmul(a[i][k], di), a[j][k]));
        }
        __syncthreads();
        for (int i = k + 1 + t; i < nb; i += blockDim.x) a[i][k] = cmul(a[i][k], di);
        __syncthreads();
    }
    // inverse of the unit lower triangular block, one column per thread
    if (t < TILE) {
        int j = t;
        for (int i = 0; i < TILE; ++i) xinv[i][j] = make_double2(0.0, 0.0);
        if (j < nb) {
            xinv[j][j] = make_double2(1.0, 0.0);
            for (int i = j + 1; i < nb; ++i) {
                double2 s = make_double2(0.0, 0.0);
                for (int k = j; k < i; ++k) s = cadd(s, cmul(a[i][k], xinv[k][j]));
                xinv[i][j] = cneg(s);
            }
        }
    }
    __syncthreads();
    // write back: strict lower L, D on the diagonal, D^{-1}, packed inverse tile
    for (int q = t; q < nb * nb; q += blockDim.x) {
        int i = q % nb, j = q / nb;
        if (i >= j) f.F[(long long)(k0 + i) + (long long)(k0 + j) * f.m] = from_d<C>(a[i][j]);
    }
    for (int k = t; k < nb; k += blockDim.x) f.dinv[f.own0 + k0 + k] = from_d<C>(dinv_s[k]);
    const int kt = k0 / TILE;
    C* tile = f.fac + (f.linv_off + tri_index(kt, kt)) * TILE2;
    for (int q = t; q < TILE2; q += blockDim.x) {
        int i = q % TILE, j = q / TILE;
        tile[q] = from_d<C>(xinv[i][j]);
    }
}

// Panel rows below the diagonal block: L[i, panel] = F[i, panel] * Linv_kk^T * D^{-1}.
template <class C>
__global__ void k_panel(const FrontDesc<C>* fd, int k0) {
    using R = typename real_of<C>::type;
    const FrontDesc<C>& f = fd[blockIdx.y];
    if (k0 >= f.nown) return;
    const int nb = min(TILE, f.nown - k0);
    const int r0 = k0 + nb + blockIdx.x * TILE;
    if (r0 >= f.lim) return;
    __shared__ C A[TILE][TILE + 1];   // A[k][r]
    __shared__ C X[TILE][TILE + 1];   // X[k][c] = Linv_kk[c][k]
    __shared__ C Di[TILE];
    const int t = threadIdx.x;
    const int kt = k0 / TILE;
    const C* tile = f.fac + (f.linv_off + tri_index(kt, kt)) * TILE2;
    for (int q = t; q < TILE2; q += blockDim.x) {
        int r = q % TILE, k = q / TILE;
        C v = czero<C>();
        if (r0 + r < f.lim && k < nb) v = f.F[(long long)(r0 + r) + (long long)(k0 + k) * f.m];
        A[k][r] = v;
        // tile is column-major: element (row=c, col=k) at c + k*TILE
        int c = q % TILE, kk = q / TILE;
        X[kk][c] = tile[q];
    }
    if (t < TILE) Di[t] = (t < nb) ? f.dinv[f.own0 + k0 + t] : czero<C>();
    __syncthreads();
    const int r = t % TILE;
    const int cg = t / TILE;   // 8 groups of 4 columns
    C acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = czero<C>();
    for (int k = 0; k < nb; ++k) {
        C av = A[k][r];
#pragma unroll
        for (int u = 0; u < 4; ++u) cfma(acc[u], av, X[k][cg * 4 + u]);
    }
    if (r0 + r < f.lim) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int c = cg * 4 + u;
            if (c < nb) f.F[(long long)(r0 + r) + (long long)(k0 + c) * f.m] = cmul(acc[u], Di[c]);
        }
    }
    (void)sizeof(R);
}

// Trailing update of the lower triangle: F[i, j] -= sum_k L[i,k] D[k] L[j,k] for
// k0+nb <= j <= i < lim, one TILE x TILE output tile per block.
template <class C>
__global__ void k_update(const FrontDesc<C>* fd, int k0) {
    const FrontDesc<C>& f = fd[blockIdx.y];
    if (k0 >= f.nown) return;
    const int nb = min(TILE, f.nown - k0);
    const int s = k0 + nb;
    const int T = cdiv_dev(f.lim - s, TILE);
    const long long q = blockIdx.x;
    if (T <= 0 || q >= (long long)T * (T + 1) / 2) return;
    int ti = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((long long)(ti + 1) * (ti + 2) / 2 <= q) ++ti;
    while ((long long)ti * (ti + 1) / 2 > q) --ti;
    const int tj = (int)(q - (long long)ti * (ti + 1) / 2);
    const int i0 = s + ti * TILE, j0 = s + tj * TILE;
    __shared__ C Li[TILE][TILE + 1];  // Li[k][r]
    __shared__ C Lj[TILE][TILE + 1];  // Lj[k][c] * D[k]
    const int t = threadIdx.x;
    for (int e = t; e < TILE2; e += blockDim.x) {
        int r = e % TILE, k = e / TILE;
        C vi = czero<C>(), vj = czero<C>();
        if (k < nb) {
            long long col = (long long)(k0 + k) * f.m;
            if (i0 + r < f.lim) vi = f.F[(i0 + r) + col];
            if (j0 + r < f.lim) vj = cmul(f.F[(j0 + r) + col], f.F[(long long)(k0 + k) + col]);
        }
        Li[k][r] = vi;
        Lj[k][r] = vj;
    }
    __syncthreads();
    const int r = t % TILE;
    const int cg = t / TILE;
    C acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = czero<C>();
    for (int k = 0; k < nb; ++k) {
        C av = Li[k][r];
#pragma unroll
        for (int u = 0; u < 4; ++u) cfma(acc[u], av, Lj[k][cg * 4 + u]);
    }
    if (i0 + r < f.lim) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int c = j0 + cg * 4 + u;
            if (c < f.lim && c <= i0 + r) {
                long long idx = (long long)(i0 + r) + (long long)c * f.m;
                f.F[idx] = csub(f.F[idx], acc[u]);
            }
        }
    }
}

// Selective inversion, block row i: X_ij = -Linv_ii * sum_{k=j}^{i-1} L_ik X_kj, j < i.
template <class C>
__global__ void k_inverse_row(const FrontDesc<C>* fd, int i) {
    const FrontDesc<C>& f = fd[blockIdx.y];
    const int own_t = cdiv_dev(f.nown, TILE);
    const int j = blockIdx.x;
    if (i >= own_t || j >= i) return;
    __shared__ C A[TILE][TILE + 1];   // A[k][r]: L_ik (row r, col k)  /  later Linv_ii
    __shared__ C B[TILE][TILE + 1];   // B[k][c]: X_kj (row k, col c)  /  later acc
    const int t = threadIdx.x;
    const int r = t % TILE, cg = t / TILE;
    C acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = czero<C>();
    for (int k = j; k < i; ++k) {
        const C* xt = f.fac + (f.linv_off + tri_index(k, j)) * TILE2;
        for (int e = t; e < TILE2; e += blockDim.x) {
            int rr = e % TILE, kk = e / TILE;
            int row = i * TILE + rr, col = k * TILE + kk;
            C v = czero<C>();
            if (row < f.nown && col < f.nown) v = f.F[(long long)row + (long long)col * f.m];
            A[kk][rr] = v;
            B[e % TILE][e / TILE] = xt[e];   // xt column-major: (row=e%T, col=e/T)
        }
        __syncthreads();
        for (int kk = 0; kk < TILE; ++kk) {
            C av = A[kk][r];
#pragma unroll
            for (int u = 0; u < 4; ++u) cfma(acc[u], av, B[kk][cg * 4 + u]);
        }
        __syncthreads();
    }
    // out = -Linv_ii * acc
    const C* dt = f.fac + (f.linv_off + tri_index(i, i)) * TILE2;
    for (int e = t; e < TILE2; e += blockDim.x) A[e / TILE][e % TILE] = dt[e];  // A[k][r] = Linv_ii(r, k)
#pragma unroll
    for (int u = 0; u < 4; ++u) B[r][cg * 4 + u] = acc[u];
    __syncthreads();
    C out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = czero<C>();
    for (int kk = 0; kk < TILE; ++kk) {
        C av = A[kk][r];
#pragma unroll
        for (int u = 0; u < 4; ++u) cfma(out[u], av, B[kk][cg * 4 + u]);
    }
    C* ot = f.fac + (f.linv_off + tri_index(i, j)) * TILE2;
#pragma unroll
    for (int u = 0; u < 4; ++u) ot[r + (cg * 4 + u) * TILE] = cneg(out[u]);
}

// Copy L21 (rows nown..m-1, columns 0..nown-1 of the front) into packed tiles.
template <class C>
__global__ void k_pack_l21(const FrontDesc<C>* fd) {
    const FrontDesc<C>& f = fd[blockIdx.y];
    if (f.tc) return;   // written by the tensor-core L21 product
    const int own_t = cdiv_dev(f.nown, TILE), upd_t = cdiv_dev(f.nupd, TILE);
    const int q = blockIdx.x;
    if (q >= own_t * upd_t) return;
    const int rt = q / own_t, ct = q % own_t;
    C* ot = f.fac + (f.l21_off + (long long)q) * TILE2;
    for (int e = threadIdx.x; e < TILE2; e += blockDim.x) {
        int r = e % TILE, c = e / TILE;
        int row = rt * TILE + r, col = ct * TILE + c;
        C v = czero<C>();
        if (row < f.nupd && col < f.nown) v = f.F[(long long)(f.nown + row) + (long long)col * f.m];
        ot[e] = v;
    }
}

}  // namespace

// Kernel kinds of the factorization, for the optional per-kind timing (HZ_FACTOR_PROFILE=1).
enum { FK_ASSEMBLE, FK_EXTEND, FK_DIAG, FK_PANEL, FK_UPDATE, FK_INVERSE, FK_GEMM_L21, FK_GEMM_SCHUR, FK_PACK, FK_N };
const char* const kFactorKindNames[FK_N] = {"k_assemble", "k_extend_add", "k_diag", "k_panel", "k_update",
                                            "k_inverse_row", "k_front_gemm L21", "k_front_gemm Schur", "k_pack_l21"};

template <class C>
void factor_layers(Ctx& ctx) {
    cudaStream_t st = ctx.stream;
    // per-kind launch timing: an event pair around every launch, read after the factorization
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> fprof;
    cudaEvent_t fp_e0 = nullptr;
#define FP_BEGIN()                                                            \
    do {                                                                      \
        if (ctx.factor_prof) {                                                \
            HZ_CUDA(cudaEventCreate(&fp_e0));                                 \
            HZ_CUDA(cudaEventRecord(fp_e0, st));                              \
        }                                                                     \
    } while (0)
#define FP_END(kind)                                                          \
    do {                                                                      \
        if (ctx.factor_prof) {                                                \
            cudaEvent_t e1_;                                                  \
            HZ_CUDA(cudaEventCreate(&e1_));                                   \
            HZ_CUDA(cudaEventRecord(e1_, st));                                \
            fprof.push_back({(kind), {fp_e0, e1_}});                          \
        }                                                                     \
    } while (0)
    const int L = (int)ctx.layers.size();
    // front arena: as many layers per group as the budget allows
    long long max_front = 0;
    for (auto& sh : ctx.shapes) max_front = std::max(max_front, sh.front_total);
    size_t free_b = 0, total_b = 0;
    HZ_CUDA(cudaMemGetInfo(&free_b, &total_b));
    long long per_layer = max_front * (long long)sizeof(C);
    long long budget = (long long)(free_b * 0.6);
    int G = (int)std::max(1LL, std::min<long long>(L, budget / std::max(1LL, per_layer)));
    // fronts of one level across the group index gridDim.y (<= 65535)
    size_t max_level = 1;
    for (auto& sh : ctx.shapes)
        for (auto& lv : sh.levels) max_level = std::max(max_level, lv.size());
    G = std::max(1, std::min(G, (int)(65535 / max_level)));
    if (max_level > 65535) throw Error{HZ_ERR_ARG, "too many fronts in one tree level"};
    if (per_layer > (long long)(free_b * 0.9))
        throw Error{HZ_ERR_OOM, "front workspace of one layer exceeds free device memory"};
    C* arena = nullptr;
    if (cudaMalloc(&arena, (size_t)per_layer * G) != cudaSuccess) {
        cudaGetLastError();
        throw Error{HZ_ERR_OOM, "cannot allocate the front workspace"};
    }
    ctx.workspace_bytes = std::max<long long>(ctx.workspace_bytes, per_layer * G);
    FrontDesc<C>* d_fd = nullptr;
    ExtDesc<C>* d_ed = nullptr;
    size_t fd_cap = 0, ed_cap = 0;
    void* d_gd = nullptr;
    void* d_gi = nullptr;
    size_t gd_cap = 0, gi_cap = 0;
    // the L21 and Schur products of large complex64 fronts run on the tensor cores
    const bool use_tc = sizeof(C) == 8 && ctx.factor_tc_min_upd > 0;
    try {
        for (int g0 = 0; g0 < L; g0 += G) {
            const int g1 = std::min(L, g0 + G);
            HZ_CUDA(cudaMemsetAsync(arena, 0, (size_t)per_layer * (g1 - g0), st));
            int Hmax = 0;
            for (int l = g0; l < g1; ++l)
                Hmax = std::max(Hmax, (int)ctx.shapes[ctx.layers[l].shape].levels.size());
            for (int h = 0; h < Hmax; ++h) {
                std::vector<FrontDesc<C>> fds;
                std::vector<FrontGemmDesc> gds;
                std::vector<ExtDesc<C>> eds[2];
                int max_nasm = 0, max_own = 0, max_rt = 0, max_tri = 0, max_pack = 0, max_ext = 0;
                for (int l = g0; l < g1; ++l) {
                    Layer& ly = ctx.layers[l];
                    Shape& sh = ctx.shapes[ly.shape];
                    if (h >= (int)sh.levels.size()) continue;
                    C* base = arena + (long long)(l - g0) * max_front;
                    for (int nid : sh.levels[h]) {
                        const Node& nd = sh.nodes[nid];
                        FrontDesc<C> f;
                        f.F = base + nd.front_off;
                        f.fac = (C*)ly.d_fac;
                        f.dinv = (C*)ly.d_dinv;
                        f.linv_off = nd.linv_off;
                        f.l21_off = nd.l21_off;
                        f.ent = sh.d_asm + nd.asm_off;
                        f.m = nd.m; f.nown = nd.nown; f.nupd = nd.nupd; f.own0 = nd.own0;
                        f.nasm = nd.nasm; f.layer = l;
                        f.tc = (use_tc && front_gemm_eligible(nd.nown, nd.nupd, ctx.factor_tc_min_upd)) ? 1 : 0;
                        f.lim = f.tc ? nd.nown : nd.m;
                        fds.push_back(f);
                        if (f.tc) {
                            FrontGemmDesc g;
                            g.F = (float2*)f.F;
                            g.fac = (float2*)f.fac;
                            g.dinv = (const float2*)f.dinv;
                            g.linv_off = nd.linv_off;
                            g.l21_off = nd.l21_off;
                            g.m = nd.m; g.nown = nd.nown; g.nupd = nd.nupd; g.own0 = nd.own0;
                            g.own_t = nd.own_t; g.upd_t = nd.upd_t;
                            gds.push_back(g);
                        }
                        max_nasm = std::max(max_nasm, nd.nasm);
                        max_own = std::max(max_own, nd.nown);
                        int rows = f.lim - std::min(nd.nown, TILE);
                        max_rt = std::max(max_rt, cdiv(std::max(rows, 0), TILE));
                        int T = cdiv(std::max(rows, 0), TILE);
                        max_tri = std::max(max_tri, T * (T + 1) / 2);
                        if (!f.tc) max_pack = std::max(max_pack, nd.own_t * nd.upd_t);
                        for (int k = 0; k < nd.nchild; ++k) {
                            const Node& ch = sh.nodes[nd.child[k]];
                            ExtDesc<C> e;
                            e.P = f.F;
                            e.F = base + ch.front_off;
                            e.emap = sh.d_emap + ch.emap_off;
                            e.mp = nd.m; e.mc = ch.m; e.ownc = ch.nown; e.nupdc = ch.nupd;
                            eds[k].push_back(e);
                            max_ext = std::max(max_ext, ch.nupd);
                        }
                    }
                }
                if (fds.empty()) continue;
                const int nf = (int)fds.size();
                if (fds.size() > fd_cap) {
                    if (d_fd) cudaFree(d_fd);
                    fd_cap = fds.size() * 2;
                    HZ_CUDA(cudaMalloc(&d_fd, fd_cap * sizeof(FrontDesc<C>)));
                }
                HZ_CUDA(cudaMemcpyAsync(d_fd, fds.data(), fds.size() * sizeof(FrontDesc<C>),
                                        cudaMemcpyHostToDevice, st));
                // 1. original entries
                if (max_nasm > 0) {
                    FP_BEGIN();
                    k_assemble<C><<<dim3(cdiv(max_nasm, 256), nf), 256, 0, st>>>(d_fd, ctx.d_coefs);
                    HZ_CHECK_LAUNCH();
                    FP_END(FK_ASSEMBLE);
                }
                // 2. extend-add, one child slot at a time (siblings overlap in the parent)
                {
                    size_t n0 = eds[0].size(), n1 = eds[1].size();
                    if (n0 + n1 > ed_cap) {
                        if (d_ed) cudaFree(d_ed);
                        ed_cap = (n0 + n1) * 2;
                        HZ_CUDA(cudaMalloc(&d_ed, ed_cap * sizeof(ExtDesc<C>)));
                    }
                    std::vector<ExtDesc<C>> all(eds[0]);
                    all.insert(all.end(), eds[1].begin(), eds[1].end());
                    if (!all.empty())
                        HZ_CUDA(cudaMemcpyAsync(d_ed, all.data(), all.size() * sizeof(ExtDesc<C>),
                                                cudaMemcpyHostToDevice, st));
                    long long work = (long long)max_ext * max_ext;
                    int gx = (int)std::min<long long>(4096, std::max<long long>(1, (work + 255) / 256));
                    if (n0) {
                        FP_BEGIN();
                        k_extend_add<C><<<dim3(gx, (unsigned)n0), 256, 0, st>>>(d_ed);
                        HZ_CHECK_LAUNCH();
                        FP_END(FK_EXTEND);
                    }
                    if (n1) {
                        FP_BEGIN();
                        k_extend_add<C><<<dim3(gx, (unsigned)n1), 256, 0, st>>>(d_ed + n0);
                        HZ_CHECK_LAUNCH();
                        FP_END(FK_EXTEND);
                    }
                }
                // 3. blocked partial LDL^T
                for (int k0 = 0; k0 < max_own; k0 += TILE) {
                    FP_BEGIN();
                    k_diag<C><<<nf, 256, 0, st>>>(d_fd, k0, ctx.d_flag);
                    HZ_CHECK_LAUNCH();
                    FP_END(FK_DIAG);
                    if (max_rt > 0) {
                        FP_BEGIN();
                        k_panel<C><<<dim3(max_rt, nf), 256, 0, st>>>(d_fd, k0);
                        HZ_CHECK_LAUNCH();
                        FP_END(FK_PANEL);
                    }
                    if (max_tri > 0) {
                        FP_BEGIN();
                        k_update<C><<<dim3(max_tri, nf), 256, 0, st>>>(d_fd, k0);
                        HZ_CHECK_LAUNCH();
                        FP_END(FK_UPDATE);
                    }
                }
                // 4. selective inversion of L11
                const int max_own_t = cdiv(max_own, TILE);
                for (int i = 1; i < max_own_t; ++i) {
                    FP_BEGIN();
                    k_inverse_row<C><<<dim3(i, nf), 256, 0, st>>>(d_fd, i);
                    HZ_CHECK_LAUNCH();
                    FP_END(FK_INVERSE);
                }
                // 5. tensor-core fronts: L21 = F21 L11^{-T} D^{-1} into the packed tiles, then the
                //    Schur complement F22 -= L21 D L21^T
                if (!gds.empty()) {
                    std::vector<GemmItem> it_l21, it_schur;
                    front_gemm_items(gds, it_l21, it_schur);
                    const size_t need_g = gds.size() * sizeof(FrontGemmDesc);
                    const size_t need_i = (it_l21.size() + it_schur.size()) * sizeof(GemmItem);
                    if (need_g > gd_cap) {
                        if (d_gd) cudaFree(d_gd);
                        gd_cap = need_g * 2;
                        HZ_CUDA(cudaMalloc(&d_gd, gd_cap));
                    }
                    if (need_i > gi_cap) {
                        if (d_gi) cudaFree(d_gi);
                        gi_cap = need_i * 2;
                        HZ_CUDA(cudaMalloc(&d_gi, gi_cap));
                    }
                    HZ_CUDA(cudaMemcpyAsync(d_gd, gds.data(), need_g, cudaMemcpyHostToDevice, st));
                    GemmItem* d_items = (GemmItem*)d_gi;
                    HZ_CUDA(cudaMemcpyAsync(d_items, it_l21.data(), it_l21.size() * sizeof(GemmItem),
                                            cudaMemcpyHostToDevice, st));
                    HZ_CUDA(cudaMemcpyAsync(d_items + it_l21.size(), it_schur.data(), it_schur.size() * sizeof(GemmItem),
                                            cudaMemcpyHostToDevice, st));
                    FP_BEGIN();
                    launch_front_gemm(0, d_items, (long long)it_l21.size(), (const FrontGemmDesc*)d_gd, ctx.d_flag + 1,
                                      ctx.tc_wait_polls, st);
                    FP_END(FK_GEMM_L21);
                    FP_BEGIN();
                    launch_front_gemm(1, d_items + it_l21.size(), (long long)it_schur.size(), (const FrontGemmDesc*)d_gd,
                                      ctx.d_flag + 1, ctx.tc_wait_polls, st);
                    FP_END(FK_GEMM_SCHUR);
                }
                // 6. pack L21 (fronts factored by the panel steps alone)
                if (max_pack > 0) {
                    FP_BEGIN();
                    k_pack_l21<C><<<dim3(max_pack, nf), 256, 0, st>>>(d_fd);
                    HZ_CHECK_LAUNCH();
                    FP_END(FK_PACK);
                }
                HZ_CUDA(cudaStreamSynchronize(st));
            }
        }
    } catch (...) {
        cudaFree(arena);
        if (d_fd) cudaFree(d_fd);
        if (d_ed) cudaFree(d_ed);
        if (d_gd) cudaFree(d_gd);
        if (d_gi) cudaFree(d_gi);
        throw;
    }
    HZ_CUDA(cudaStreamSynchronize(st));
    cudaFree(arena);
    if (d_fd) cudaFree(d_fd);
    if (d_ed) cudaFree(d_ed);
    if (d_gd) cudaFree(d_gd);
    if (d_gi) cudaFree(d_gi);
    if (ctx.factor_prof) {
        double ms[FK_N] = {};
        long long n[FK_N] = {};
        for (auto& r : fprof) {
            float t = 0.f;
            cudaEventElapsedTime(&t, r.second.first, r.second.second);
            ms[r.first] += t;
            n[r.first] += 1;
            cudaEventDestroy(r.second.first);
            cudaEventDestroy(r.second.second);
        }
        ctx.factor_text = "kernel launch_groups ms\n";
        for (int k = 0; k < FK_N; ++k)
            ctx.factor_text += std::string(kFactorKindNames[k]) + " " + std::to_string(n[k]) + " " + std::to_string(ms[k]) + "\n";
    }
#undef FP_BEGIN
#undef FP_END
}

template void factor_layers<float2>(Ctx&);
template void factor_layers<double2>(Ctx&);

}  // namespace hz
