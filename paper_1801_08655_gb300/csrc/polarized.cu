// Online phase of the method of polarized traces on the GPU.
//
// Indices are 0-based: layers l = 0..L-1, interfaces j = 0..K-1 (K = L-1); interface j
// carries the plane pair (P_j, Q_j) = (last owned plane of layer j, first owned plane of
// layer j+1).  A polarized trace vector per right-hand side is stored as
// [2 (down, up)][K][2 (P, Q)][ny][nx] in complex128, right-hand sides outermost.
//
// Interface sources (the Dirac deltas of the Formulation section, weights taken from the
// assembled matrix so that the discrete Green's representation formula is exact):
//   S_top(t_{l-1}) on layer l:  plane Q_{l-1} += -c t(P_{l-1});  pad plane P_{l-1} += +c t(Q_{l-1})
//   S_bot(t_l)     on layer l:  plane P_l     += -c t(Q_l);      pad plane Q_l     += +c t(P_l)
// with c = s_x s_y / h^2 the z-coupling across a physical half plane.
// Read-outs: "bottom" of layer l = planes (P_l, Q_l), "top" of layer l = (P_{l-1}, Q_{l-1}).
//
// Blocks of the polarized matrix (appendix, Algorithms 6-9) and the preconditioner of
// Eq. 16 (Algorithms 4-6) are built from one batched local solve per layer with the
// four source blocks stacked as columns (M_pol), or one layer at a time (sweeps).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"
#include "hz_solve.cuh"

namespace hz {

namespace {

template <class C> __device__ inline void atomic_addc(C* p, double2 v);
template <> __device__ inline void atomic_addc<float2>(float2* p, double2 v) {
    atomicAdd(p, make_float2((float)v.x, (float)v.y));
}
template <> __device__ inline void atomic_addc<double2>(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

template <class C> struct Inject {
    C* acc;
    const int* pos;
    const double2* src;      // trace pair base for r = 0; plane P at +0, Q at +plane
    long long rstride;       // between right-hand sides in src
    int ldc, col0;
    int zl_m, off_m;         // local plane receiving -c * src[off_m + cell]
    int zl_p, off_p;         // local plane receiving +c * src[off_p + cell]
    const double* b;         // layer's local b = 1/rho, or nullptr (constant density)
};

// Trace vectors keep cells contiguous per right-hand side; the slot vectors keep right-hand sides
// contiguous per row.  The three kernels below move a tile of 32 cells x 32 right-hand sides
// through shared memory so that both sides are read and written along their contiguous index
// (tile[a][b] with a pitch of 33 16-byte elements: conflict-free along either index).
constexpr int IO_T = 32;

template <class C>
__global__ void __launch_bounds__(256) k_inject(const Inject<C>* inj, const double2* sx, const double2* sy,
                                                double inv_h2, int nx, int ny, int R) {
    __shared__ double2 tm[IO_T][IO_T + 1], tp[IO_T][IO_T + 1];   // [r][cell]
    const Inject<C> q = inj[blockIdx.z];
    const int P = nx * ny;
    const int cell0 = blockIdx.x * IO_T, r0 = blockIdx.y * IO_T;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // trace planes, read along cells
    for (int rr = w; rr < IO_T; rr += 8) {
        const int r = r0 + rr, cell = cell0 + lane;
        double2 vm = make_double2(0.0, 0.0), vp = vm;
        if (r < R && cell < P) {
            const double2* src = q.src + (long long)r * q.rstride;
            vm = src[q.off_m + cell];
            vp = src[q.off_p + cell];
        }
        tm[rr][lane] = vm;
        tp[rr][lane] = vp;
    }
    __syncthreads();
    // slot rows, written along the right-hand sides
    const int r = r0 + lane;
    for (int cc = w; cc < IO_T; cc += 8) {
        const int cell = cell0 + cc;
        if (cell >= P) break;
        if (r >= R) continue;
        const int x = cell % nx, y = cell / nx;
        // c = A[(Q,y,x),(P,y,x)]: the z-coupling across the physical half plane between the pair's
        // planes (zl_m and zl_p are the two of them), times b at that half plane
        double2 c = cscale(cmul(sx[x], sy[y]), inv_h2);
        if (q.b) c = cscale(c, 0.5 * (q.b[(long long)q.zl_m * P + cell] + q.b[(long long)q.zl_p * P + cell]));
        atomic_addc(q.acc + (long long)q.pos[q.zl_m * P + cell] * q.ldc + q.col0 + r, cneg(cmul(c, tm[lane][cc])));
        atomic_addc(q.acc + (long long)q.pos[q.zl_p * P + cell] * q.ldc + q.col0 + r, cmul(c, tp[lane][cc]));
    }
}

template <class C> struct Extract {
    const C* x;
    const int* pos;
    double2* dst;            // destination plane for r = 0
    long long rstride;
    int ldc, zl, nblk;
    int cols[4];
    double sign;
};

template <class C>
__global__ void __launch_bounds__(256) k_extract(const Extract<C>* ex, int P, int R) {
    __shared__ double2 t[IO_T][IO_T + 1];   // [cell][r]
    const Extract<C> q = ex[blockIdx.z];
    const int cell0 = blockIdx.x * IO_T, r0 = blockIdx.y * IO_T;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // slot rows, read along the right-hand sides (the column blocks summed)
    for (int cc = w; cc < IO_T; cc += 8) {
        const int cell = cell0 + cc, r = r0 + lane;
        double2 v = make_double2(0.0, 0.0);
        if (cell < P && r < R) {
            const C* xr = q.x + (long long)q.pos[q.zl * P + cell] * q.ldc + r;
            for (int b = 0; b < q.nblk; ++b) v = cadd(v, to_d(xr[q.cols[b]]));
        }
        t[cc][lane] = v;
    }
    __syncthreads();
    // trace plane, updated along cells
    const int cell = cell0 + lane;
    for (int rr = w; rr < IO_T; rr += 8) {
        const int r = r0 + rr;
        if (r >= R) break;
        if (cell >= P) continue;
        double2* d = q.dst + (long long)r * q.rstride + cell;
        *d = cadd(*d, cscale(t[lane][rr], q.sign));
    }
}

template <class C> struct VolIO {
    C* vec;                  // acc (sources) or x (read-out)
    const int* pos;
    int ldc, col0, lo, hi, zlo;
};

// acc[pos(cell)][col0 + r] = S * g[r][z][cell] over the layer's owned planes; blockIdx.y is
// (plane offset) x nrt + (right-hand-side tile).
template <class C>
__global__ void __launch_bounds__(256) k_volume_source(const VolIO<C>* io, const double2* g,
                                                       const double2* const* gslot, int R, int nrt, long long N3,
                                                       int nx, int ny, const double2* sx, const double2* sy,
                                                       const double2* sz, int scale) {
    __shared__ double2 t[IO_T][IO_T + 1];   // [r][cell]
    if (gslot) g = *gslot;   // recorded plans read the caller's volume through the handle's slot
    const VolIO<C> q = io[blockIdx.z];
    const int P = nx * ny;
    const int z = q.lo + (int)blockIdx.y / nrt;
    if (z > q.hi) return;   // uniform over the block
    const int cell0 = blockIdx.x * IO_T, r0 = ((int)blockIdx.y % nrt) * IO_T;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int rr = w; rr < IO_T; rr += 8) {   // volume, read along cells
        const int r = r0 + rr, cell = cell0 + lane;
        t[rr][lane] = (r < R && cell < P) ? g[(long long)r * N3 + (long long)z * P + cell] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int r = r0 + lane;
    for (int cc = w; cc < IO_T; cc += 8) {   // slot rows, written along the right-hand sides
        const int cell = cell0 + cc;
        if (cell >= P) break;
        if (r >= R) continue;
        double2 S = make_double2(1.0, 0.0);
        if (scale) S = cmul(cmul(sx[cell % nx], sy[cell / nx]), sz[z]);
        q.vec[(long long)q.pos[(z - q.zlo) * P + cell] * q.ldc + q.col0 + r] = from_d<C>(cmul(S, t[lane][cc]));
    }
}

// u[r][z][cell] (+)= x[pos(cell)][col0 + r] over the owned planes.
template <class C>
__global__ void k_volume_out(const VolIO<C>* io, double2* u, double2* const* uslot, int R, long long N3, int P,
                             int accumulate) {
    if (uslot) u = *uslot;
    const VolIO<C> q = io[blockIdx.z];
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = q.lo + blockIdx.y;
    if (cell >= P || z > q.hi) return;
    const C* src = q.vec + (long long)q.pos[(z - q.zlo) * P + cell] * q.ldc + q.col0;
    double2* dst = u + (long long)z * P + cell;
    for (int r = 0; r < R; ++r) {
        double2 v = to_d(src[r]);
        if (accumulate) v = cadd(v, dst[(long long)r * N3]);
        dst[(long long)r * N3] = v;
    }
}

// Natural-order local vectors <-> elimination-order slot (stage entry point).
template <class C>
__global__ void k_gather_local(C* acc, const int* pos, int ldc, const double2* g, long long Nl, int ncols) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (i >= Nl) return;
    acc[(long long)pos[i] * ldc + c] = from_d<C>(g[(long long)c * Nl + i]);
}
template <class C>
__global__ void k_scatter_local(const C* x, const int* pos, int ldc, double2* w, long long Nl, int ncols) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (i >= Nl) return;
    w[(long long)c * Nl + i] = to_d(x[(long long)pos[i] * ldc + c]);
}

// y = a * x (+ b * z restricted to one plane of each pair) over trace pairs.
// Pair j of a vector with pair stride 2P: planes [2P j, 2P j + 2P).
__global__ void k_pairs_axpy(double2* y, long long ystride, const double2* x, long long xstride, double a,
                             const double2* z, long long zstride, double b, int zplane, int npairs, int P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    long long n = (long long)npairs * 2 * P;
    if (i >= n) return;
    double2 v = cscale(x[(long long)r * xstride + i], a);
    if (z != nullptr) {
        int pl = (int)((i / P) % 2);
        if (pl == zplane) v = cadd(v, cscale(z[(long long)r * zstride + i], b));
    }
    y[(long long)r * ystride + i] = v;
}


// ------------------------------------------------------------------------------------------
// explicit trace-to-trace Green's blocks: the local Green's function between a layer's interface
// plane pairs (the blocks Algorithms 4-9 apply matrix-free by local solves), stored densely
// ------------------------------------------------------------------------------------------
// One term of a block product: E (2P x 2P, column-major, complex type C) applied to the trace
// pair x0 (+ x1 when given), each pair [r * xstride + k], k < 2P.
template <class C> struct TBTerm {
    const C* E;
    const double2* x0;
    const double2* x1;
};
// y[r * ystride + m] += sign * sum over the terms of (E (x0 + x1))[m], m < 2P, r < R.
template <class C> struct TBJob {
    TBTerm<C> t[2];
    double2* y;
    int nterm;
    double sign;
};

constexpr int TB_ROWS = 256;   // output rows (read-out entries) per block, one per thread
constexpr int TB_KC = 64;      // source entries staged per step

// Complex128 blocks (complex64 ones go through k_trace_block2 below).
// Each thread owns one read-out entry m and NC right-hand-side columns; the block streams the
// columns of E (one unit source trace's read-outs are contiguous, so a warp reads 32 consecutive
// entries of a column per step) against the source values of TB_KC entries x NC columns staged in
// shared memory.  blockIdx: x row tile, y (column group, K slice), z job.  With more than one K
// slice the partial sums are added with FP64 atomics, otherwise each output is read, added to
// and written by its one thread.
template <class C, int NC>
__global__ void __launch_bounds__(TB_ROWS) k_trace_block(const TBJob<C>* jobs, int n2, int R, long long xs,
                                                         long long ys, int kslice, int ncg) {
    __shared__ C xsm[TB_KC][NC];
    const TBJob<C>& jb = jobs[blockIdx.z];
    const int m = blockIdx.x * TB_ROWS + threadIdx.x;
    const int cg = blockIdx.y % ncg, ks = blockIdx.y / ncg;
    const int c0 = cg * NC;
    const int kb = ks * kslice, ke = min(n2, kb + kslice);
    C acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = czero<C>();
    const int nterm = jb.nterm;
    for (int t = 0; t < nterm; ++t) {
        const C* E = jb.t[t].E;
        const double2* x0 = jb.t[t].x0;
        const double2* x1 = jb.t[t].x1;
        for (int kc = kb; kc < ke; kc += TB_KC) {
            __syncthreads();
            for (int i = threadIdx.x; i < TB_KC * NC; i += TB_ROWS) {
                const int kk = i % TB_KC, c = i / TB_KC;
                const int k = kc + kk, r = c0 + c;
                double2 v = make_double2(0.0, 0.0);
                if (k < ke && r < R) {
                    v = x0[(long long)r * xs + k];
                    if (x1) v = cadd(v, x1[(long long)r * xs + k]);
                }
                xsm[kk][c] = from_d<C>(v);
            }
            __syncthreads();
            const int kn = min(TB_KC, ke - kc);
            if (m < n2) {
                const C* Ep = E + (long long)kc * n2 + m;
                for (int kk = 0; kk < kn; kk += 8) {
                    C e[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) e[u] = (kk + u < kn) ? __ldcs(Ep + (long long)(kk + u) * n2) : czero<C>();
#pragma unroll
                    for (int u = 0; u < 8; ++u)
#pragma unroll
                        for (int c = 0; c < NC; ++c) cfma(acc[c], e[u], xsm[kk + u][c]);
                }
            }
        }
    }
    if (m >= n2) return;
    const bool atomic = gridDim.y > (unsigned)ncg;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int r = c0 + c;
        if (r >= R) break;
        const double2 v = cscale(to_d(acc[c]), jb.sign);
        double2* yp = jb.y + (long long)r * ys + m;
        if (atomic) {
            atomicAdd(&yp->x, v.x);
            atomicAdd(&yp->y, v.y);
        } else {
            *yp = cadd(*yp, v);
        }
    }
}

// Complex64 blocks: each thread owns two adjacent read-out rows (one 16-byte load per source
// entry) and streams its own rows of E through a private ring of TB2_ST stages x TB2_KG source
// entries in shared memory with cp.async, so that TB2_ST - 1 stages of loads are in flight while
// it multiplies the stage that has landed (no block barrier is needed for E: a thread reads only
// what it copied itself).  The source values are staged per TB_KC entries as in k_trace_block.
constexpr int TB2_THREADS = 256;
constexpr int TB2_ROWS = 2 * TB2_THREADS;
constexpr int TB2_KG = 8;
constexpr int TB2_ST = 4;
constexpr size_t tb2_smem(int nc) { return (size_t)TB2_ST * TB2_KG * TB2_THREADS * 16 + (size_t)TB_KC * nc * 8; }

__device__ inline void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int NC>
__global__ void __launch_bounds__(TB2_THREADS, 1) k_trace_block2(const TBJob<float2>* jobs, int n2, int R, long long xs,
                                                                 long long ys, int kslice, int ncg) {
    extern __shared__ __align__(16) unsigned char tb2_smem_raw[];
    float4* ring = reinterpret_cast<float4*>(tb2_smem_raw);   // [TB2_ST][TB2_KG][TB2_THREADS]
    float2(*xsm)[NC] = reinterpret_cast<float2(*)[NC]>(tb2_smem_raw + (size_t)TB2_ST * TB2_KG * TB2_THREADS * 16);
    const TBJob<float2>& jb = jobs[blockIdx.z];
    const int tid = threadIdx.x;
    const int m = blockIdx.x * TB2_ROWS + 2 * tid;   // rows m and m + 1 (n2 is even)
    const bool row_ok = m < n2;
    const int cg = blockIdx.y % ncg, ks = blockIdx.y / ncg;
    const int c0 = cg * NC;
    const int kb = ks * kslice, ke = min(n2, kb + kslice);
    const int G = (ke - kb + TB2_KG - 1) / TB2_KG;   // pipeline stages of this slice (uniform over the block)
    float2 a0[NC], a1[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { a0[c] = czero<float2>(); a1[c] = czero<float2>(); }
    const int nterm = jb.nterm;
    for (int t = 0; t < nterm; ++t) {
        const float2* E = jb.t[t].E;
        const double2* x0 = jb.t[t].x0;
        const double2* x1 = jb.t[t].x1;
        auto issue = [&](int g) {   // one commit group per stage
            const int sl = g % TB2_ST;
#pragma unroll
            for (int u = 0; u < TB2_KG; ++u) {
                const int k = kb + g * TB2_KG + u;
                float4* dst = ring + (sl * TB2_KG + u) * TB2_THREADS + tid;
                if (row_ok && k < ke) cp_async16(dst, E + (long long)k * n2 + m);
                else *dst = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            cp_async_commit();
        };
#pragma unroll
        for (int g = 0; g < TB2_ST - 1; ++g) {
            if (g < G) issue(g);
            else cp_async_commit();
        }
        for (int g = 0; g < G; ++g) {
            const int kk0 = (g * TB2_KG) % TB_KC;
            if (kk0 == 0) {   // next TB_KC source entries of x (all threads reach this together)
                __syncthreads();
                const int kc = kb + g * TB2_KG;
                for (int i = tid; i < TB_KC * NC; i += TB2_THREADS) {
                    const int kk = i % TB_KC, c = i / TB_KC;
                    const int k = kc + kk, r = c0 + c;
                    double2 v = make_double2(0.0, 0.0);
                    if (k < ke && r < R) {
                        v = x0[(long long)r * xs + k];
                        if (x1) v = cadd(v, x1[(long long)r * xs + k]);
                    }
                    xsm[kk][c] = to_f(v);
                }
                __syncthreads();
            }
            if (g + TB2_ST - 1 < G) issue(g + TB2_ST - 1);
            else cp_async_commit();
            cp_async_wait<TB2_ST - 1>();   // this thread's copies of stage g have landed
            const int sl = g % TB2_ST;
#pragma unroll
            for (int u = 0; u < TB2_KG; ++u) {
                const float4 e = ring[(sl * TB2_KG + u) * TB2_THREADS + tid];
                const float2 e0 = make_float2(e.x, e.y), e1 = make_float2(e.z, e.w);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float2 xv = xsm[kk0 + u][c];
                    cfma(a0[c], e0, xv);
                    cfma(a1[c], e1, xv);
                }
            }
        }
        cp_async_wait<0>();   // the ring is reused by the next term
    }
    if (!row_ok) return;
    const bool atomic = gridDim.y > (unsigned)ncg;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int r = c0 + c;
        if (r >= R) break;
        double2* yp = jb.y + (long long)r * ys + m;
        const double2 v0 = cscale(to_d(a0[c]), jb.sign), v1 = cscale(to_d(a1[c]), jb.sign);
        if (atomic) {
            atomicAdd(&yp[0].x, v0.x);
            atomicAdd(&yp[0].y, v0.y);
            atomicAdd(&yp[1].x, v1.x);
            atomicAdd(&yp[1].y, v1.y);
        } else {
            yp[0] = cadd(yp[0], v0);
            yp[1] = cadd(yp[1], v1);
        }
    }
}

// U[r][k] = (k == k0 + r), r < ncols, k < n2: unit source traces k0 .. k0 + ncols - 1 (pairs
// flattened as (plane, cell)); columns past the last trace stay zero.
__global__ void k_unit_traces(double2* U, int n2, int ncols, int k0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)ncols * n2) return;
    const int r = (int)(i / n2), k = (int)(i % n2);
    U[i] = make_double2(k == k0 + r ? 1.0 : 0.0, 0.0);
}

// E_b[(k0 + r) * n2 + m] = T[b][r][m] for the chunk's columns r < ncols with k0 + r < n2.
template <class C>
__global__ void k_store_blocks(C* base, const long long* off, const double2* T, int n2, int ncols, int k0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= (long long)ncols * n2) return;
    const int r = (int)(i / n2), m = (int)(i % n2);
    if (k0 + r >= n2) return;
    base[off[b] + (long long)(k0 + r) * n2 + m] = from_d<C>(T[(long long)b * ncols * n2 + i]);
}

// ------------------------------------------------------------------------------------------
// FP64 volume residual r = g - A u, g = S f (scale) or f, with per-column norms
// ------------------------------------------------------------------------------------------
template <int RB>
__global__ void __launch_bounds__(256) k_residual(const double2* f, const double2* u, double2* rout, double* norms,
                                                  int scale, int R, int nx, int ny, int nz, const double2* sxn,
                                                  const double2* isxh, const double2* syn, const double2* isyh,
                                                  const double2* szn, const double2* iszh, const double* m,
                                                  const double* b, double omega2, double inv_h2) {
    // one cell and RB columns per thread: the cell's stencil coefficients (FP64, as in the
    // assembly) are formed once and applied to RB columns, so that the FP64 pipe (the bound of
    // this kernel on a GPU whose FP64 rate is a small fraction of its FP32 rate) spends its
    // work on the products with u
    const long long N3 = (long long)nx * ny * nz;
    const int r0 = blockIdx.y * RB;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rr[RB], gg[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) { rr[j] = 0.0; gg[j] = 0.0; }
    if (i < N3) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        const double2 sx = sxn[x], sy = syn[y], sz = szn[z];
        const double2 syz = cmul(sy, sz), sxz = cmul(sx, sz), sxy = cmul(sx, sy);
        double2 c1 = cscale(cmul(syz, isxh[x]), inv_h2), c2 = cscale(cmul(syz, isxh[x + 1]), inv_h2);
        double2 c3 = cscale(cmul(sxz, isyh[y]), inv_h2), c4 = cscale(cmul(sxz, isyh[y + 1]), inv_h2);
        double2 c5 = cscale(cmul(sxy, iszh[z]), inv_h2), c6 = cscale(cmul(sxy, iszh[z + 1]), inv_h2);
        if (b) {   // variable density: b at the half nodes
            const long long pl_ = (long long)nx * ny;
            c1 = cscale(c1, bhalf(b, i, x, nx, 1, -1)); c2 = cscale(c2, bhalf(b, i, x, nx, 1, +1));
            c3 = cscale(c3, bhalf(b, i, y, ny, nx, -1)); c4 = cscale(c4, bhalf(b, i, y, ny, nx, +1));
            c5 = cscale(c5, bhalf(b, i, z, nz, pl_, -1)); c6 = cscale(c6, bhalf(b, i, z, nz, pl_, +1));
        }
        const double2 sxyz = cmul(sxy, sz);
        double2 dg = cscale(sxyz, omega2 * m[i]);
        dg = csub(dg, cadd(cadd(cadd(c1, c2), cadd(c3, c4)), cadd(c5, c6)));
        // absent neighbours (outside the box) take a zero coefficient and the cell's own index
        const long long pl = (long long)nx * ny;
        const double2 zero = make_double2(0.0, 0.0);
        const long long ix0 = x > 0 ? i - 1 : i, ix1 = x < nx - 1 ? i + 1 : i;
        const long long iy0 = y > 0 ? i - nx : i, iy1 = y < ny - 1 ? i + nx : i;
        const long long iz0 = z > 0 ? i - pl : i, iz1 = z < nz - 1 ? i + pl : i;
        if (x == 0) c1 = zero;
        if (x == nx - 1) c2 = zero;
        if (y == 0) c3 = zero;
        if (y == ny - 1) c4 = zero;
        if (z == 0) c5 = zero;
        if (z == nz - 1) c6 = zero;
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            const int r = r0 + j;
            if (r >= R) break;
            const double2* ur = u + (long long)r * N3;
            double2 au = cmul(dg, ur[i]);
            au = cadd(au, cmul(c1, ur[ix0]));
            au = cadd(au, cmul(c2, ur[ix1]));
            au = cadd(au, cmul(c3, ur[iy0]));
            au = cadd(au, cmul(c4, ur[iy1]));
            au = cadd(au, cmul(c5, ur[iz0]));
            au = cadd(au, cmul(c6, ur[iz1]));
            double2 g = f[(long long)r * N3 + i];
            if (scale) g = cmul(sxyz, g);
            const double2 res = csub(g, au);
            if (rout) rout[(long long)r * N3 + i] = res;
            rr[j] = res.x * res.x + res.y * res.y;
            gg[j] = g.x * g.x + g.y * g.y;
        }
    }
    // block reductions of the RB column pairs, one atomic pair per column and block
    __shared__ double sr[RB][8], sg[RB][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        for (int o = 16; o > 0; o >>= 1) {
            rr[j] += __shfl_down_sync(0xffffffffu, rr[j], o);
            gg[j] += __shfl_down_sync(0xffffffffu, gg[j], o);
        }
        if (lane == 0) { sr[j][w] = rr[j]; sg[j][w] = gg[j]; }
    }
    __syncthreads();
    if (threadIdx.x < RB && r0 + (int)threadIdx.x < R) {
        const int j = threadIdx.x;
        double a = 0.0, c = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += sr[j][k]; c += sg[j][k]; }
        atomicAdd(&norms[2 * (r0 + j)], a);
        atomicAdd(&norms[2 * (r0 + j) + 1], c);
    }
}

// ------------------------------------------------------------------------------------------
// batched FP64 GMRES kernels: one Krylov space per right-hand-side column
// ------------------------------------------------------------------------------------------
__device__ inline double2 block_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    __shared__ double2 sh[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (w == 0) {
        int nw = blockDim.x >> 5;
        s = lane < nw ? sh[lane] : make_double2(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_down_sync(0xffffffffu, s.x, o);
            s.y += __shfl_down_sync(0xffffffffu, s.y, o);
        }
    }
    return s;  // valid in thread 0
}

// dots[r*ld + i] += <V_i[r], w[r]> (conjugated first argument), i < nv
__global__ void k_mdot(const double2* V, long long vstride, const double2* w, long long n, int nv,
                       double2* dots, int ld) {
    const int r = blockIdx.y;
    const double2* wr = w + (long long)r * n;
    for (int i = 0; i < nv; ++i) {
        const double2* vr = V + (long long)i * vstride + (long long)r * n;
        double2 s = make_double2(0.0, 0.0);
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
             e += (long long)gridDim.x * blockDim.x) {
            double2 a = vr[e], b = wr[e];
            s.x += a.x * b.x + a.y * b.y;
            s.y += a.x * b.y - a.y * b.x;
        }
        s = block_sum2(s);
        if (threadIdx.x == 0) {
            atomicAdd(&dots[(long long)r * ld + i].x, s.x);
            atomicAdd(&dots[(long long)r * ld + i].y, s.y);
        }
    }
}

// w[r] -= sum_i h[r*ld + i] V_i[r]
__global__ void k_maxpy(const double2* V, long long vstride, double2* w, long long n, int nv,
                        const double2* h, int ld) {
    const int r = blockIdx.y;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 acc = w[(long long)r * n + e];
    for (int i = 0; i < nv; ++i) acc = csub(acc, cmul(h[(long long)r * ld + i], V[(long long)i * vstride + (long long)r * n + e]));
    w[(long long)r * n + e] = acc;
}

// x[r] += sum_i y[r*ld + i] V_i[r]
__global__ void k_maxpy_plus(const double2* V, long long vstride, double2* x, long long n, int nv,
                             const double2* y, int ld) {
    const int r = blockIdx.y;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double2 acc = x[(long long)r * n + e];
    for (int i = 0; i < nv; ++i) acc = cadd(acc, cmul(y[(long long)r * ld + i], V[(long long)i * vstride + (long long)r * n + e]));
    x[(long long)r * n + e] = acc;
}

__global__ void k_nrm2(const double2* w, long long n, double* out) {
    const int r = blockIdx.y;
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        double2 a = w[(long long)r * n + e];
        s += a.x * a.x + a.y * a.y;
    }
    double2 t = block_sum2(make_double2(s, 0.0));
    if (threadIdx.x == 0) atomicAdd(&out[r], t.x);
}

__global__ void k_scale_vec(double2* dst, const double2* src, long long n, const double* scale) {
    const int r = blockIdx.y;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    dst[(long long)r * n + e] = cscale(src[(long long)r * n + e], scale[r]);
}

// y[r] = a x[r] + b z[r] over len elements per column (strided per column)
__global__ void k_lincomb(double2* y, long long ys, double a, const double2* x, long long xs, double b,
                          const double2* z, long long zs, long long len) {
    const int r = blockIdx.y;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double2 v = cscale(x[(long long)r * xs + e], a);
    if (z) v = cadd(v, cscale(z[(long long)r * zs + e], b));
    y[(long long)r * ys + e] = v;
}

// dots[r*(m+1) + i] += y[r*m + i], i < nv
__global__ void k_accum_dots(double2* dots, const double2* y, int R, int m, int nv) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R * nv) return;
    int r = q / nv, i = q % nv;
    dots[(long long)r * (m + 1) + i] = cadd(dots[(long long)r * (m + 1) + i], y[(long long)r * m + i]);
}

struct GmresState {
    double2* H;      // [R][(m+1)*m], H[i + j*(m+1)]
    double2* cs_sn;  // [R][m] pairs: (c, 0) and s stored as two arrays
    double2* sn;
    double2* g;      // [R][m+1]
    double2* dots;   // [R][m+1] scratch (sum of both CGS passes)
    double* nrm;     // [R]
    double* invb;    // [R] 1/beta used to normalise the next basis vector (0 = frozen)
    double* resid;   // [R] |g_{j+1}|
    int* active;     // [R]
    int* kused;      // [R] basis vectors used by each column in this cycle
    double2* y;      // [R][m]
};

// start of a cycle: beta = sqrt(nrm), g = (beta, 0, ...), invb = 1/beta
__global__ void k_gmres_start(GmresState s, int R, int m, double tiny) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double b = sqrt(s.nrm[r]);
    for (int i = 0; i <= m; ++i) s.g[(long long)r * (m + 1) + i] = make_double2(0.0, 0.0);
    s.g[(long long)r * (m + 1)] = make_double2(b, 0.0);
    s.resid[r] = b;
    s.kused[r] = 0;
    bool act = s.active[r] && b > tiny;
    s.active[r] = act;
    s.invb[r] = act ? 1.0 / b : 0.0;
}

// column j of the Hessenberg matrix: h(0..j) from dots, h(j+1) = ||w||; Givens update
__global__ void k_gmres_arnoldi(GmresState s, int R, int m, int j, double tol_abs_scale, const double* b0,
                                double tol, double tiny) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (!s.active[r]) { s.invb[r] = 0.0; return; }
    double2* H = s.H + (long long)r * (m + 1) * m;
    double2* cs = s.cs_sn + (long long)r * m;
    double2* sn = s.sn + (long long)r * m;
    double2* g = s.g + (long long)r * (m + 1);
    const double2* d = s.dots + (long long)r * (m + 1);
    for (int i = 0; i <= j; ++i) H[i + j * (m + 1)] = d[i];
    double beta = sqrt(s.nrm[r]);
    H[j + 1 + j * (m + 1)] = make_double2(beta, 0.0);
    // previous rotations
    for (int i = 0; i < j; ++i) {
        double2 a = H[i + j * (m + 1)], bb = H[i + 1 + j * (m + 1)];
        double c = cs[i].x;
        double2 sv = sn[i];
        double2 na = cadd(cscale(a, c), cmul(sv, bb));
        double2 nb = csub(cscale(bb, c), cmul(make_double2(sv.x, -sv.y), a));
        H[i + j * (m + 1)] = na;
        H[i + 1 + j * (m + 1)] = nb;
    }
    double2 h1 = H[j + j * (m + 1)];
    double2 h2 = H[j + 1 + j * (m + 1)];
    double a1 = sqrt(h1.x * h1.x + h1.y * h1.y), a2 = sqrt(h2.x * h2.x + h2.y * h2.y);
    double rho = sqrt(a1 * a1 + a2 * a2);
    double c;
    double2 sv;
    if (rho == 0.0) { c = 1.0; sv = make_double2(0.0, 0.0); }
    else if (a1 == 0.0) { c = 0.0; sv = make_double2(h2.x / a2, -h2.y / a2); }
    else {
        c = a1 / rho;
        double2 ph = make_double2(h1.x / a1, h1.y / a1);
        sv = cscale(cmul(ph, make_double2(h2.x, -h2.y)), 1.0 / rho);
    }
    cs[j] = make_double2(c, 0.0);
    sn[j] = sv;
    H[j + j * (m + 1)] = cadd(cscale(h1, c), cmul(sv, h2));
    H[j + 1 + j * (m + 1)] = make_double2(0.0, 0.0);
    double2 gj = g[j];
    g[j] = cscale(gj, c);
    g[j + 1] = cneg(cmul(make_double2(sv.x, -sv.y), gj));
    double res = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y);
    s.resid[r] = res;
    s.kused[r] = j + 1;
    if (res <= tol * sqrt(b0[r]) || beta <= tiny) {
        s.active[r] = 0;
        s.invb[r] = 0.0;
    } else {
        s.invb[r] = 1.0 / beta;
    }
    (void)tol_abs_scale;
}

// back substitution H(0:k,0:k) y = g(0:k) per column
__global__ void k_gmres_lsq(GmresState s, int R, int m) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double2* H = s.H + (long long)r * (m + 1) * m;
    const double2* g = s.g + (long long)r * (m + 1);
    double2* y = s.y + (long long)r * m;
    int k = s.kused[r];
    for (int i = 0; i < m; ++i) y[i] = make_double2(0.0, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double2 v = g[i];
        for (int q = i + 1; q < k; ++q) v = csub(v, cmul(H[i + q * (m + 1)], y[q]));
        y[i] = cmul(v, crecip(H[i + i * (m + 1)]));
    }
}

// ------------------------------------------------------------------------------------------
// host-side helpers: every operator is recorded into a Rec (descriptors uploaded once, stream
// operations as closures) so that it can run directly or be replayed as a CUDA graph
// ------------------------------------------------------------------------------------------
inline const double2* pair_ptr(const double2* base, const Ctx& c, int dir, int j) {
    return base + (long long)dir * c.K * 2 * c.P + (long long)j * 2 * c.P;
}
inline double2* pair_ptr(double2* base, const Ctx& c, int dir, int j) {
    return base + (long long)dir * c.K * 2 * c.P + (long long)j * 2 * c.P;
}

template <class C>
void rec_zero_slots(Ctx& ctx, Rec& rec, const std::vector<int>& layers, int ldc) {
    for (int l : layers) {
        void* p = ctx.slot_acc[l];
        const size_t bytes = (size_t)ctx.shapes[ctx.layers[l].shape].N * ldc * sizeof(C);
        rec.add([p, bytes](cudaStream_t st) { HZ_CUDA(cudaMemsetAsync(p, 0, bytes, st)); });
    }
}

// approx: the substitution serves the preconditioner, whose tensor-core products then run with
// the handle's precond_split TF32 terms
// sparse: sparsity code of the batch (sparse_code(fwd, bwd), see get_batch); the handle's
// sparse_subst switch masks it (HZ_SPARSE: 3 forward and backward, 2 backward only, 0 never)
// A per-block code (blocked_code) needs blocks of whole 64-column chunks; otherwise, or when
// every block has the same code, the batch runs as one job per layer with the union of the codes.
template <class C>
void rec_subst(Ctx& ctx, Rec& rec, const std::vector<int>& layers, int ncols, bool approx = false, int sparse = 0) {
    const int split = approx ? ctx.precond_split : 3;
    auto mask = [&](int code) {
        if (!(ctx.sparse_subst & 1)) code &= ~3;          // forward products everywhere
        if (!(ctx.sparse_subst & 2)) code &= ~(3 << 2);   // backward products everywhere
        return code;
    };
    // plane set covering two: SP_ALL absorbs, two different pairs make SP_BOTH
    auto join = [](int a, int b) { return (a == SP_ALL || b == SP_ALL) ? SP_ALL : (a == b ? a : SP_BOTH); };
    const int nblk = block_count(sparse);
    if (nblk > 1) {
        int codes[4], fu = -1, bu = -1;
        bool same = true;
        for (int q = 0; q < nblk; ++q) {
            codes[q] = mask(block_code(sparse, q));
            same = same && codes[q] == codes[0];
            fu = fu < 0 ? (codes[q] & 3) : join(fu, codes[q] & 3);
            bu = bu < 0 ? ((codes[q] >> 2) & 3) : join(bu, (codes[q] >> 2) & 3);
        }
        const bool whole = ncols % nblk == 0 && (ncols / nblk) % 64 == 0;
        sparse = (whole && !same) ? blocked_code(nblk, codes) : sparse_code(fu, bu);
    } else {
        sparse = mask(sparse);
    }
    ensure_tuned<C>(ctx, layers, ncols, split, sparse);  // at record time, before any capture
    const Batch* b = &get_batch<C>(ctx, layers, ncols, split, sparse);
    Ctx* cp = &ctx;
    rec.add([cp, b, ncols](cudaStream_t st) { substitute<C>(*cp, *b, ncols, st); });
}

// S_top on layer l (source pair of interface l-1) / S_bot on layer l (pair of interface l)
template <class C>
Inject<C> make_inject(Ctx& ctx, int l, bool top, const double2* pair, long long rstride, int ldc, int col0) {
    const Layer& ly = ctx.layers[l];
    const Shape& sh = ctx.shapes[ly.shape];
    Inject<C> q;
    q.acc = (C*)ctx.slot_acc[l];
    q.pos = sh.d_pos;
    q.src = pair;
    q.rstride = rstride;
    q.ldc = ldc;
    q.col0 = col0;
    q.b = ly.d_b;
    const int Pl = (int)ctx.P;
    if (top) {  // Q_{l-1} = lo gets -c t(P); P_{l-1} = lo-1 gets +c t(Q)
        q.zl_m = ly.lo - ly.zlo; q.off_m = 0;
        q.zl_p = ly.lo - 1 - ly.zlo; q.off_p = Pl;
    } else {    // P_l = hi gets -c t(Q); Q_l = hi+1 gets +c t(P)
        q.zl_m = ly.hi - ly.zlo; q.off_m = Pl;
        q.zl_p = ly.hi + 1 - ly.zlo; q.off_p = 0;
    }
    return q;
}

template <class C>
Extract<C> make_extract(Ctx& ctx, int l, bool bottom, int pl, const std::vector<int>& cols, double2* dst,
                        long long rstride, int ldc, double sign) {
    const Layer& ly = ctx.layers[l];
    const Shape& sh = ctx.shapes[ly.shape];
    Extract<C> e;
    e.x = (const C*)ctx.slot_x[l];
    e.pos = sh.d_pos;
    e.dst = dst;
    e.rstride = rstride;
    e.ldc = ldc;
    // bottom: planes (P_l, Q_l) = (hi, hi+1); top: (P_{l-1}, Q_{l-1}) = (lo-1, lo)
    int z = bottom ? (ly.hi + pl) : (ly.lo - 1 + pl);
    e.zl = z - ly.zlo;
    e.nblk = (int)cols.size();
    for (int b = 0; b < 4; ++b) e.cols[b] = b < e.nblk ? cols[b] : 0;
    e.sign = sign;
    return e;
}

template <class C>
void rec_inject(Ctx& ctx, Rec& rec, const std::vector<Inject<C>>& v, int R) {
    if (v.empty()) return;
    const Inject<C>* d = rec.up(v);
    dim3 grid(cdiv(ctx.P, IO_T), cdiv(R, IO_T), (unsigned)v.size());
    const double2 *sx = ctx.d_sx_n, *sy = ctx.d_sy_n;
    const double ih2 = 1.0 / (ctx.h * ctx.h);
    const int nx = ctx.nx, ny = ctx.ny;
    rec.add([=](cudaStream_t st) {
        k_inject<C><<<grid, 256, 0, st>>>(d, sx, sy, ih2, nx, ny, R);
        HZ_CHECK_LAUNCH();
    });
}

template <class C>
void rec_extract(Ctx& ctx, Rec& rec, const std::vector<Extract<C>>& v, int R) {
    if (v.empty()) return;
    const Extract<C>* d = rec.up(v);
    dim3 grid(cdiv(ctx.P, IO_T), cdiv(R, IO_T), (unsigned)v.size());
    const int P = (int)ctx.P;
    rec.add([=](cudaStream_t st) {
        k_extract<C><<<grid, 256, 0, st>>>(d, P, R);
        HZ_CHECK_LAUNCH();
    });
}

void rec_pairs_axpy(Ctx& ctx, Rec& rec, double2* y, long long ys, const double2* x, long long xs, double a,
                    const double2* z, long long zs, double b, int zplane, int npairs, int R) {
    const long long n = (long long)npairs * 2 * ctx.P;
    dim3 grid(cdiv(n, 256), R);
    const int P = (int)ctx.P;
    rec.add([=](cudaStream_t st) {
        k_pairs_axpy<<<grid, 256, 0, st>>>(y, ys, x, xs, a, z, zs, b, zplane, npairs, P);
        HZ_CHECK_LAUNCH();
    });
}

std::vector<int> all_layers(const Ctx& ctx) {
    std::vector<int> v(ctx.L);
    for (int l = 0; l < ctx.L; ++l) v[l] = l;
    return v;
}

// g: the volume right-hand side; with gslot != nullptr the kernel reads it from that device slot
// instead (plans recorded once and replayed for every call)
template <class C>
void rec_volume_sources(Ctx& ctx, Rec& rec, const std::vector<int>& layers, const double2* g, bool scale, int R,
                        int ldc, const double2* const* gslot = nullptr) {
    std::vector<VolIO<C>> io;
    int maxpl = 0;
    for (int l : layers) {
        const Layer& ly = ctx.layers[l];
        VolIO<C> q;
        q.vec = (C*)ctx.slot_acc[l];
        q.pos = ctx.shapes[ly.shape].d_pos;
        q.ldc = ldc; q.col0 = 0; q.lo = ly.lo; q.hi = ly.hi; q.zlo = ly.zlo;
        io.push_back(q);
        maxpl = std::max(maxpl, ly.hi - ly.lo + 1);
    }
    const VolIO<C>* d = rec.up(io);
    const int nrt = (int)cdiv(R, IO_T);
    dim3 grid(cdiv(ctx.P, IO_T), (unsigned)(maxpl * nrt), (unsigned)io.size());
    const long long N3 = (long long)ctx.nz * ctx.P;
    const int nx = ctx.nx, ny = ctx.ny;
    const double2 *sx = ctx.d_sx_n, *sy = ctx.d_sy_n, *sz = ctx.d_sz_n;
    const int sc = scale ? 1 : 0;
    rec.add([=](cudaStream_t st) {
        k_volume_source<C><<<grid, 256, 0, st>>>(d, g, gslot, R, nrt, N3, nx, ny, sx, sy, sz, sc);
        HZ_CHECK_LAUNCH();
    });
}

// run a freshly recorded operator once and release its descriptors
inline void run_now(Ctx& ctx, Rec& rec) {
    rec.run(ctx.stream);
    HZ_CUDA(cudaStreamSynchronize(ctx.stream));
}

// ------------------------------------------------------------------------------------------
// operators on the explicit trace-to-trace blocks
// ------------------------------------------------------------------------------------------
template <class C>
bool use_trace_blocks(const Ctx& ctx, int R) {
    return ctx.tb.base && ctx.tb.elem == sizeof(C) && R <= ctx.tb.max_cols;
}

// E_rs of layer l (r, s: 0 top, 1 bottom); the caller only asks for blocks that exist
template <class C>
const C* trace_block(const Ctx& ctx, int l, int r, int s) {
    const long long o = ctx.tb.off[l][2 * r + s];
    if (o < 0) throw Error{HZ_ERR_STATE, "explicit trace block missing"};
    return (const C*)ctx.tb.base + o;
}

template <class C, int NC>
void launch_trace_block(const TBJob<C>* d, unsigned njobs, int n2, int R, long long xs, long long ys, int ksplit,
                        int kslice, int ncg, cudaStream_t st) {
    dim3 grid(cdiv(n2, TB_ROWS), (unsigned)(ncg * ksplit), njobs);
    k_trace_block<C, NC><<<grid, TB_ROWS, 0, st>>>(d, n2, R, xs, ys, kslice, ncg);
    HZ_CHECK_LAUNCH();
}

// k_trace_block2 takes more than the default 48 KiB of dynamic shared memory; set at record time
// (never inside a stream capture), on the current device
inline void tb2_allow_smem() {
    HZ_CUDA(cudaFuncSetAttribute(k_trace_block2<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb2_smem(8)));
    HZ_CUDA(cudaFuncSetAttribute(k_trace_block2<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb2_smem(16)));
}

template <int NC>
void launch_trace_block2(const TBJob<float2>* d, unsigned njobs, int n2, int R, long long xs, long long ys, int ksplit,
                         int kslice, int ncg, cudaStream_t st) {
    dim3 grid(cdiv(n2, TB2_ROWS), (unsigned)(ncg * ksplit), njobs);
    k_trace_block2<NC><<<grid, TB2_THREADS, tb2_smem(NC), st>>>(d, n2, R, xs, ys, kslice, ncg);
    HZ_CHECK_LAUNCH();
}

inline void launch_tb_kind(const TBJob<float2>* d, unsigned nj, int n2, int R, long long xs, long long ys, int ksplit,
                           int kslice, int ncg, int NC, cudaStream_t st) {
    if (NC == 8) launch_trace_block2<8>(d, nj, n2, R, xs, ys, ksplit, kslice, ncg, st);
    else launch_trace_block2<16>(d, nj, n2, R, xs, ys, ksplit, kslice, ncg, st);
}
inline void launch_tb_kind(const TBJob<double2>* d, unsigned nj, int n2, int R, long long xs, long long ys, int ksplit,
                           int kslice, int ncg, int NC, cudaStream_t st) {
    if (NC == 8) launch_trace_block<double2, 8>(d, nj, n2, R, xs, ys, ksplit, kslice, ncg, st);
    else launch_trace_block<double2, 16>(d, nj, n2, R, xs, ys, ksplit, kslice, ncg, st);
}

// One launch of block products over independent jobs (distinct outputs), on trace pairs of
// vectors with the trace-vector stride.  Outputs must hold their other terms already.  The source
// range is split into K slices (partial sums added with FP64 atomics) when that fills the GPU's
// block slots with less wave quantization.
template <class C>
void rec_trace_blocks(Ctx& ctx, Rec& rec, const std::vector<TBJob<C>>& jobs, int R) {
    if (jobs.empty()) return;
    const bool dbl = sizeof(C) == 16;
    const int n2 = (int)(2 * ctx.P);
    // complex64: k_trace_block2 with 8 or 16 columns per pass; complex128: k_trace_block
    const int NC = R <= 8 ? 8 : 16;
    const int ncg = cdiv(R, NC);
    const int rows = dbl ? TB_ROWS : TB2_ROWS;
    int sms = 0;
    HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx.device));
    // resident blocks per launch: k_trace_block2 one per SM (210 registers x 256 threads), k_trace_block two
    const long long slots = (dbl ? 2LL : 1LL) * sms;
    const long long base = (long long)cdiv(n2, rows) * ncg * (long long)jobs.size();
    const int kmax = std::max(1, n2 / (4 * TB_KC));
    // smallest split whose blocks fill at least 90 % of the slots of their last wave, else the best one
    int ksplit = 1;
    double best = -1.0;
    for (int k = 1; k <= kmax; ++k) {
        const int ksl = cdiv(cdiv(n2, k), TB_KC) * TB_KC;
        const long long blocks = base * cdiv(n2, ksl);
        const double waves = (double)blocks / slots;
        const double eff = blocks < slots ? waves : waves / std::ceil(waves);
        if (eff > best + 1e-9) { best = eff; ksplit = k; }
        if (eff >= 0.9) break;
    }
    const int kslice = cdiv(cdiv(n2, ksplit), TB_KC) * TB_KC;
    ksplit = cdiv(n2, kslice);
    if (!dbl) tb2_allow_smem();
    const TBJob<C>* d = rec.up(jobs);
    const unsigned nj = (unsigned)jobs.size();
    const long long xs = ctx.ntr, ys = ctx.ntr;
    // algorithmic work of the launch: every block entry read once; 8 real flops per entry and column
    long long terms = 0;
    for (const auto& j : jobs) terms += j.nterm;
    const double lbytes = (double)terms * n2 * (double)n2 * sizeof(C);
    const double lflops = 8.0 * terms * n2 * (double)n2 * R;
    Ctx* cp = &ctx;
    rec.add([=](cudaStream_t st) {
        ProfRec pr{};
        const bool timed = cp->prof && cp->prof_detail;   // never during a graph capture (prof off)
        if (timed) {
            HZ_CUDA(cudaEventCreate(&pr.e0));
            HZ_CUDA(cudaEventCreate(&pr.e1));
            HZ_CUDA(cudaEventRecord(pr.e0, st));
        }
        launch_tb_kind(d, nj, n2, R, xs, ys, ksplit, kslice, ncg, NC, st);
        if (timed) {
            HZ_CUDA(cudaEventRecord(pr.e1, st));
            pr.kind = 2;
            pr.mode = 0;
            pr.level = 0;
            pr.tasks = nj;
            pr.bytes = lbytes;
            pr.flops = lflops;
            cp->prof_launch.push_back(pr);
        }
    });
}

template <class C>
TBJob<C> tb_job(double2* y, double sign) {
    TBJob<C> j;
    j.t[0] = j.t[1] = TBTerm<C>{nullptr, nullptr, nullptr};
    j.y = y;
    j.nterm = 0;
    j.sign = sign;
    return j;
}
template <class C>
void tb_term(TBJob<C>& j, const C* E, const double2* x0, const double2* x1 = nullptr) {
    j.t[j.nterm++] = TBTerm<C>{E, x0, x1};
}

// y = M_pol x with the local solves replaced by block products: down row j gets
// E^j_bt (x_down + x_up)_{j-1} + E^j_bb x_up_j, up row j gets E^{j+1}_tt x_down_j +
// E^{j+1}_tb (x_down + x_up)_{j+1} (the read-outs the stacked solve of rec_apply_mpol sums).
template <class C>
void rec_apply_mpol_blocks(Ctx& ctx, Rec& rec, const double2* x, int R, double2* y) {
    const int K = ctx.K, L = ctx.L;
    const long long ntr = ctx.ntr;
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 0, 0), ntr, pair_ptr(x, ctx, 0, 0), ntr, -1.0, pair_ptr(x, ctx, 1, 0), ntr,
                   -1.0, 0, K, R);
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 1, 0), ntr, pair_ptr(x, ctx, 1, 0), ntr, -1.0, pair_ptr(x, ctx, 0, 0), ntr,
                   -1.0, 1, K, R);
    std::vector<TBJob<C>> jobs;
    for (int j = 0; j < K; ++j) {
        TBJob<C> dn = tb_job<C>(pair_ptr(y, ctx, 0, j), 1.0);
        if (j >= 1) tb_term(dn, trace_block<C>(ctx, j, 1, 0), pair_ptr(x, ctx, 0, j - 1), pair_ptr(x, ctx, 1, j - 1));
        tb_term(dn, trace_block<C>(ctx, j, 1, 1), pair_ptr(x, ctx, 1, j));
        jobs.push_back(dn);
        TBJob<C> up = tb_job<C>(pair_ptr(y, ctx, 1, j), 1.0);
        tb_term(up, trace_block<C>(ctx, j + 1, 0, 0), pair_ptr(x, ctx, 0, j));
        if (j + 1 <= L - 2)
            tb_term(up, trace_block<C>(ctx, j + 1, 0, 1), pair_ptr(x, ctx, 0, j + 1), pair_ptr(x, ctx, 1, j + 1));
        jobs.push_back(up);
    }
    rec_trace_blocks<C>(ctx, rec, jobs, R);
}

// y = P x (Eq. 16) on the blocks: down sweep y_down_j = E^j_bt y_down_{j-1} - x_down_j; reflections
// s_j = x_up_j + [Q] y_down_j - E^{j+1}_tt y_down_j - E^{j+1}_tb y_down_{j+1}; up sweep
// y_up_j = E^{j+1}_tb y_up_{j+1} - s_j.  tmp: one trace vector of scratch (s in its up half).
template <class C>
void rec_apply_precond_blocks(Ctx& ctx, Rec& rec, const double2* x, int R, double2* y, double2* tmp) {
    const int K = ctx.K, L = ctx.L;
    const long long ntr = ctx.ntr;
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 0, 0), ntr, pair_ptr(x, ctx, 0, 0), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
    for (int j = 1; j < K; ++j) {
        rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 0, j), ntr, pair_ptr(x, ctx, 0, j), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
        TBJob<C> jb = tb_job<C>(pair_ptr(y, ctx, 0, j), 1.0);
        tb_term(jb, trace_block<C>(ctx, j, 1, 0), pair_ptr(y, ctx, 0, j - 1));
        rec_trace_blocks<C>(ctx, rec, {jb}, R);
    }
    double2* s = tmp;
    rec_pairs_axpy(ctx, rec, pair_ptr(s, ctx, 1, 0), ntr, pair_ptr(x, ctx, 1, 0), ntr, 1.0, pair_ptr(y, ctx, 0, 0), ntr,
                   1.0, 1, K, R);
    {
        std::vector<TBJob<C>> jobs;
        for (int j = 0; j < K; ++j) {
            TBJob<C> jb = tb_job<C>(pair_ptr(s, ctx, 1, j), -1.0);
            tb_term(jb, trace_block<C>(ctx, j + 1, 0, 0), pair_ptr(y, ctx, 0, j));
            if (j + 1 <= L - 2) tb_term(jb, trace_block<C>(ctx, j + 1, 0, 1), pair_ptr(y, ctx, 0, j + 1));
            jobs.push_back(jb);
        }
        rec_trace_blocks<C>(ctx, rec, jobs, R);
    }
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 1, K - 1), ntr, pair_ptr(s, ctx, 1, K - 1), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
    for (int j = K - 2; j >= 0; --j) {
        rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 1, j), ntr, pair_ptr(s, ctx, 1, j), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
        TBJob<C> jb = tb_job<C>(pair_ptr(y, ctx, 1, j), 1.0);
        tb_term(jb, trace_block<C>(ctx, j + 1, 0, 1), pair_ptr(y, ctx, 1, j + 1));
        rec_trace_blocks<C>(ctx, rec, {jb}, R);
    }
}

}  // namespace

// Explicit blocks of every layer: unit source traces, `chunk` at a time, injected through S_top
// (column block 0) and S_bot (column block 1) of every layer at once, solved, and read at the
// layer's top and bottom pairs; the read-outs of the chunk become columns k0 .. k0 + chunk - 1 of
// the blocks.
template <class C>
void build_trace_blocks(Ctx& ctx, int chunk) {
    const bool dbl = sizeof(C) == 16;
    const int L = ctx.L;
    const int n2 = (int)(2 * ctx.P);
    if (chunk < 64 || chunk % 64 || padded_ldc(dbl, 2 * chunk) > ctx.slot_cap)
        throw Error{HZ_ERR_ARG, "trace block chunk does not fit the layer workspace"};
    const int ldc = padded_ldc(dbl, 2 * chunk);
    TraceBlocks tb;
    tb.elem = sizeof(C);
    tb.off.assign(L, {-1, -1, -1, -1});
    struct Blk { int l, r, s; };
    std::vector<Blk> blks;
    long long nb = 0;
    for (int l = 0; l < L; ++l)
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s) {
                if ((r == 0 || s == 0) && l == 0) continue;       // no top interface
                if ((r == 1 || s == 1) && l == L - 1) continue;   // no bottom interface
                tb.off[l][2 * r + s] = nb * (long long)n2 * n2;
                blks.push_back({l, r, s});
                ++nb;
            }
    tb.bytes = nb * (long long)n2 * n2 * (long long)sizeof(C);
    if (cudaMalloc(&tb.base, std::max<long long>(tb.bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        tb.base = nullptr;
        throw Error{HZ_ERR_OOM, "explicit trace blocks (" + std::to_string(tb.bytes >> 20) + " MiB) do not fit"};
    }
    double2 *U = nullptr, *T = nullptr;
    long long* d_off = nullptr;
    auto cleanup = [&]() {
        if (U) cudaFree(U);
        if (T) cudaFree(T);
        if (d_off) cudaFree(d_off);
    };
    try {
        const size_t ubytes = (size_t)chunk * n2 * sizeof(double2);
        const size_t tbytes = (size_t)nb * chunk * n2 * sizeof(double2);
        if (cudaMalloc((void**)&U, ubytes) != cudaSuccess || cudaMalloc((void**)&T, tbytes) != cudaSuccess ||
            cudaMalloc((void**)&d_off, nb * sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            throw Error{HZ_ERR_OOM, "trace block staging does not fit"};
        }
        std::vector<long long> h_off;
        for (const Blk& b : blks) h_off.push_back(tb.off[b.l][2 * b.r + b.s]);
        HZ_CUDA(cudaMemcpyAsync(d_off, h_off.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, ctx.stream));
        Rec rec;
        rec.upload_stream = ctx.stream;
        auto layers = all_layers(ctx);
        rec_zero_slots<C>(ctx, rec, layers, ldc);
        std::vector<Inject<C>> inj;
        for (int l = 0; l < L; ++l) {
            if (l >= 1) inj.push_back(make_inject<C>(ctx, l, true, U, n2, ldc, 0));
            if (l <= L - 2) inj.push_back(make_inject<C>(ctx, l, false, U, n2, ldc, chunk));
        }
        rec_inject<C>(ctx, rec, inj, chunk);
        const int codes[2] = {sparse_code(SP_TOP, SP_BOTH), sparse_code(SP_BOT, SP_BOTH)};
        rec_subst<C>(ctx, rec, layers, 2 * chunk, false, blocked_code(2, codes));
        rec.add([T, tbytes](cudaStream_t st) { HZ_CUDA(cudaMemsetAsync(T, 0, tbytes, st)); });
        std::vector<Extract<C>> ex;
        for (long long b = 0; b < nb; ++b)
            for (int pl = 0; pl < 2; ++pl)
                ex.push_back(make_extract<C>(ctx, blks[b].l, blks[b].r == 1, pl, {blks[b].s == 0 ? 0 : chunk},
                                             T + b * chunk * n2 + pl * ctx.P, n2, ldc, 1.0));
        rec_extract<C>(ctx, rec, ex, chunk);
        const dim3 g1(cdiv((long long)chunk * n2, 256)), g2(cdiv((long long)chunk * n2, 256), (unsigned)nb);
        for (int k0 = 0; k0 < n2; k0 += chunk) {
            k_unit_traces<<<g1, 256, 0, ctx.stream>>>(U, n2, chunk, k0);
            HZ_CHECK_LAUNCH();
            rec.run(ctx.stream);
            k_store_blocks<C><<<g2, 256, 0, ctx.stream>>>((C*)tb.base, d_off, T, n2, chunk, k0);
            HZ_CHECK_LAUNCH();
        }
        HZ_CUDA(cudaStreamSynchronize(ctx.stream));
    } catch (...) {
        cudaStreamSynchronize(ctx.stream);
        cleanup();
        cudaFree(tb.base);
        throw;
    }
    cleanup();
    ctx.tb.release();
    ctx.tb = tb;
}

// ------------------------------------------------------------------------------------------
// operators (recorders)
// ------------------------------------------------------------------------------------------
template <class C>
void rec_polarized_rhs(Ctx& ctx, Rec& rec, const double2* g, bool scale, int R, double2* fpol,
                       const double2* const* gslot = nullptr) {
    const bool dbl = sizeof(C) == 16;
    const int ldc = padded_ldc(dbl, R);
    if (ldc > ctx.slot_cap) throw Error{HZ_ERR_ADMISSION, "too many columns for the layer workspace"};
    auto layers = all_layers(ctx);
    rec_zero_slots<C>(ctx, rec, layers, ldc);
    rec_volume_sources<C>(ctx, rec, layers, g, scale, R, ldc, gslot);
    rec_subst<C>(ctx, rec, layers, R, false, sparse_code(SP_ALL, SP_BOTH));   // read-outs on the interface planes only
    const size_t bytes = (size_t)R * ctx.ntr * sizeof(double2);
    rec.add([fpol, bytes](cudaStream_t st) { HZ_CUDA(cudaMemsetAsync(fpol, 0, bytes, st)); });
    std::vector<Extract<C>> ex;
    for (int j = 0; j < ctx.K; ++j)
        for (int pl = 0; pl < 2; ++pl) {
            // f_down_j = -(v^j(P_j), v^j(Q_j)); f_up_j = -(v^{j+1}(P_j), v^{j+1}(Q_j))
            ex.push_back(make_extract<C>(ctx, j, true, pl, {0}, pair_ptr(fpol, ctx, 0, j) + pl * ctx.P, ctx.ntr, ldc, -1.0));
            ex.push_back(make_extract<C>(ctx, j + 1, false, pl, {0}, pair_ptr(fpol, ctx, 1, j) + pl * ctx.P, ctx.ntr, ldc, -1.0));
        }
    rec_extract<C>(ctx, rec, ex, R);
}

// y = M_pol x: u_down = D_down x_down + U x_up,  u_up = D_up x_up + L x_down.
template <class C>
void rec_apply_mpol(Ctx& ctx, Rec& rec, const double2* x, int R, double2* y) {
    if (use_trace_blocks<C>(ctx, R)) {
        rec_apply_mpol_blocks<C>(ctx, rec, x, R, y);
        return;
    }
    const bool dbl = sizeof(C) == 16;
    const int K = ctx.K, L = ctx.L;
    const long long ntr = ctx.ntr;
    // identity terms: u_down_j = -x_down_j - [P plane] x_up_j ; u_up_j = -x_up_j - [Q plane] x_down_j
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 0, 0), ntr, pair_ptr(x, ctx, 0, 0), ntr, -1.0, pair_ptr(x, ctx, 1, 0), ntr,
                   -1.0, 0, K, R);
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 1, 0), ntr, pair_ptr(x, ctx, 1, 0), ntr, -1.0, pair_ptr(x, ctx, 0, 0), ntr,
                   -1.0, 1, K, R);
    // source blocks: 0 = S_top x_down_{l-1}, 1 = S_bot x_down_l, 2 = S_top x_up_{l-1}, 3 = S_bot x_up_l
    int per_pass = 4;
    while (per_pass > 1 && padded_ldc(dbl, per_pass * R) > ctx.slot_cap) per_pass /= 2;
    if (padded_ldc(dbl, R) > ctx.slot_cap) throw Error{HZ_ERR_ADMISSION, "too many columns for the layer workspace"};
    auto layers = all_layers(ctx);
    for (int p0 = 0; p0 < 4; p0 += per_pass) {
        const int nbk = per_pass;
        const int ncols = nbk * R;
        const int ldc = padded_ldc(dbl, ncols);
        rec_zero_slots<C>(ctx, rec, layers, ldc);
        std::vector<Inject<C>> inj;
        int colof[4] = {-1, -1, -1, -1};
        for (int q = 0; q < nbk; ++q) colof[p0 + q] = q * R;
        for (int l = 0; l < L; ++l)
            for (int q = 0; q < nbk; ++q) {
                int blk = p0 + q;
                bool top = (blk == 0 || blk == 2);
                int dir = (blk < 2) ? 0 : 1;
                if (top && l >= 1)
                    inj.push_back(make_inject<C>(ctx, l, true, pair_ptr(x, ctx, dir, l - 1), ntr, ldc, q * R));
                if (!top && l <= L - 2)
                    inj.push_back(make_inject<C>(ctx, l, false, pair_ptr(x, ctx, dir, l), ntr, ldc, q * R));
            }
        rec_inject<C>(ctx, rec, inj, R);
        // sources and read-outs on the interface planes, per block: its source pair, and the pairs
        // read from it (bottom of layer j -> u_down_j, top of layer j+1 -> u_up_j, as extracted below)
        const int blk_code[4] = {sparse_code(SP_TOP, SP_BOTH), sparse_code(SP_BOT, SP_TOP),
                                 sparse_code(SP_TOP, SP_BOT), sparse_code(SP_BOT, SP_BOTH)};
        rec_subst<C>(ctx, rec, layers, ncols, false,
                     nbk > 1 ? blocked_code(nbk, blk_code + p0) : blk_code[p0]);
        std::vector<Extract<C>> ex;
        for (int j = 0; j < K; ++j) {
            // bottom of layer j -> u_down_j: blocks {0 (l>=1), 2 (l>=1), 3}
            std::vector<int> cb, ct;
            if (j >= 1 && colof[0] >= 0) cb.push_back(colof[0]);
            if (j >= 1 && colof[2] >= 0) cb.push_back(colof[2]);
            if (colof[3] >= 0) cb.push_back(colof[3]);
            // top of layer j+1 -> u_up_j: blocks {0, 1 (l<=L-2), 3 (l<=L-2)}
            if (colof[0] >= 0) ct.push_back(colof[0]);
            if (j + 1 <= L - 2 && colof[1] >= 0) ct.push_back(colof[1]);
            if (j + 1 <= L - 2 && colof[3] >= 0) ct.push_back(colof[3]);
            for (int pl = 0; pl < 2; ++pl) {
                if (!cb.empty())
                    ex.push_back(make_extract<C>(ctx, j, true, pl, cb, pair_ptr(y, ctx, 0, j) + pl * ctx.P, ntr, ldc, 1.0));
                if (!ct.empty())
                    ex.push_back(make_extract<C>(ctx, j + 1, false, pl, ct, pair_ptr(y, ctx, 1, j) + pl * ctx.P, ntr, ldc, 1.0));
            }
        }
        rec_extract<C>(ctx, rec, ex, R);
    }
}

// y = P x (Eq. 16): y_down = sweep_down(x_down); s = x_up - L y_down; y_up = sweep_up(s).
// tmp: one trace vector [R][ntr] of scratch.
template <class C>
void rec_apply_precond(Ctx& ctx, Rec& rec, const double2* x, int R, double2* y, double2* tmp) {
    if (use_trace_blocks<C>(ctx, R)) {
        rec_apply_precond_blocks<C>(ctx, rec, x, R, y, tmp);
        return;
    }
    const bool dbl = sizeof(C) == 16;
    const int K = ctx.K, L = ctx.L;
    const long long ntr = ctx.ntr;
    const int ldc = padded_ldc(dbl, R);
    if (ldc > ctx.slot_cap) throw Error{HZ_ERR_ADMISSION, "too many columns for the layer workspace"};
    // downward sweep (Algorithm 4)
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 0, 0), ntr, pair_ptr(x, ctx, 0, 0), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
    for (int j = 1; j < K; ++j) {
        std::vector<int> one{j};
        rec_zero_slots<C>(ctx, rec, one, ldc);
        rec_inject<C>(ctx, rec, {make_inject<C>(ctx, j, true, pair_ptr(y, ctx, 0, j - 1), ntr, ldc, 0)}, R);
        rec_subst<C>(ctx, rec, one, R, true, sparse_code(SP_TOP, SP_BOT));   // source on top, read at the bottom
        rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 0, j), ntr, pair_ptr(x, ctx, 0, j), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
        std::vector<Extract<C>> ex;
        for (int pl = 0; pl < 2; ++pl)
            ex.push_back(make_extract<C>(ctx, j, true, pl, {0}, pair_ptr(y, ctx, 0, j) + pl * ctx.P, ntr, ldc, 1.0));
        rec_extract<C>(ctx, rec, ex, R);
    }
    // upward reflections (Algorithm 6): s_j = x_up_j - ([w]_P, [w]_Q - y_down_j(Q)),
    // w = G^{j+1} (S_top y_down_j + S_bot y_down_{j+1}); s lives in the up half of tmp
    double2* s = tmp;
    rec_pairs_axpy(ctx, rec, pair_ptr(s, ctx, 1, 0), ntr, pair_ptr(x, ctx, 1, 0), ntr, 1.0, pair_ptr(y, ctx, 0, 0), ntr,
                   1.0, 1, K, R);
    {
        std::vector<int> layers;
        for (int l = 1; l < L; ++l) layers.push_back(l);
        rec_zero_slots<C>(ctx, rec, layers, ldc);
        std::vector<Inject<C>> inj;
        for (int l = 1; l < L; ++l) {
            inj.push_back(make_inject<C>(ctx, l, true, pair_ptr(y, ctx, 0, l - 1), ntr, ldc, 0));
            if (l <= L - 2) inj.push_back(make_inject<C>(ctx, l, false, pair_ptr(y, ctx, 0, l), ntr, ldc, 0));
        }
        rec_inject<C>(ctx, rec, inj, R);
        rec_subst<C>(ctx, rec, layers, R, true, sparse_code(SP_BOTH, SP_TOP));   // read at the top only
        std::vector<Extract<C>> ex;
        for (int j = 0; j < K; ++j)
            for (int pl = 0; pl < 2; ++pl)
                ex.push_back(make_extract<C>(ctx, j + 1, false, pl, {0}, pair_ptr(s, ctx, 1, j) + pl * ctx.P, ntr, ldc, -1.0));
        rec_extract<C>(ctx, rec, ex, R);
    }
    // upward sweep (Algorithm 5)
    rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 1, K - 1), ntr, pair_ptr(s, ctx, 1, K - 1), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
    for (int j = K - 2; j >= 0; --j) {
        std::vector<int> one{j + 1};
        rec_zero_slots<C>(ctx, rec, one, ldc);
        rec_inject<C>(ctx, rec, {make_inject<C>(ctx, j + 1, false, pair_ptr(y, ctx, 1, j + 1), ntr, ldc, 0)}, R);
        rec_subst<C>(ctx, rec, one, R, true, sparse_code(SP_BOT, SP_TOP));   // source at the bottom, read on top
        rec_pairs_axpy(ctx, rec, pair_ptr(y, ctx, 1, j), ntr, pair_ptr(s, ctx, 1, j), ntr, -1.0, nullptr, 0, 0.0, 0, 1, R);
        std::vector<Extract<C>> ex;
        for (int pl = 0; pl < 2; ++pl)
            ex.push_back(make_extract<C>(ctx, j + 1, false, pl, {0}, pair_ptr(y, ctx, 1, j) + pl * ctx.P, ntr, ldc, 1.0));
        rec_extract<C>(ctx, rec, ex, R);
    }
}

// u = reconstruction from f and traces t [R][K][2][P] (Algorithm 2, inner solves).
template <class C>
void rec_reconstruct(Ctx& ctx, Rec& rec, const double2* g, bool scale, const double2* t, int R, double2* u,
                     bool accumulate, const double2* const* gslot = nullptr, double2* const* uslot = nullptr) {
    const bool dbl = sizeof(C) == 16;
    const int L = ctx.L;
    const int ldc = padded_ldc(dbl, R);
    if (ldc > ctx.slot_cap) throw Error{HZ_ERR_ADMISSION, "too many columns for the layer workspace"};
    auto layers = all_layers(ctx);
    rec_zero_slots<C>(ctx, rec, layers, ldc);
    rec_volume_sources<C>(ctx, rec, layers, g, scale, R, ldc, gslot);
    const long long ts = (long long)ctx.K * 2 * ctx.P;
    std::vector<Inject<C>> inj;
    for (int l = 0; l < L; ++l) {
        if (l >= 1) inj.push_back(make_inject<C>(ctx, l, true, t + (long long)(l - 1) * 2 * ctx.P, ts, ldc, 0));
        if (l <= L - 2) inj.push_back(make_inject<C>(ctx, l, false, t + (long long)l * 2 * ctx.P, ts, ldc, 0));
    }
    rec_inject<C>(ctx, rec, inj, R);
    rec_subst<C>(ctx, rec, layers, R);
    std::vector<VolIO<C>> io;
    int maxpl = 0;
    for (int l : layers) {
        const Layer& ly = ctx.layers[l];
        VolIO<C> q;
        q.vec = (C*)ctx.slot_x[l];
        q.pos = ctx.shapes[ly.shape].d_pos;
        q.ldc = ldc; q.col0 = 0; q.lo = ly.lo; q.hi = ly.hi; q.zlo = ly.zlo;
        io.push_back(q);
        maxpl = std::max(maxpl, ly.hi - ly.lo + 1);
    }
    const VolIO<C>* d = rec.up(io);
    dim3 grid(cdiv(ctx.P, 256), maxpl, (unsigned)io.size());
    const long long N3 = (long long)ctx.nz * ctx.P;
    const int P = (int)ctx.P, acc = accumulate ? 1 : 0;
    rec.add([=](cudaStream_t st) {
        k_volume_out<C><<<grid, 256, 0, st>>>(d, u, uslot, R, N3, P, acc);
        HZ_CHECK_LAUNCH();
    });
}

// ------------------------------------------------------------------------------------------
// one-shot operators (stage entry points)
// ------------------------------------------------------------------------------------------
template <class C>
void op_layer_solve(Ctx& ctx, int ell, const double2* g, int ncols, double2* w) {
    const bool dbl = sizeof(C) == 16;
    const int ldc = padded_ldc(dbl, ncols);
    if (ldc > ctx.slot_cap) throw Error{HZ_ERR_ADMISSION, "too many columns for the layer workspace"};
    const Layer& ly = ctx.layers[ell];
    const Shape& sh = ctx.shapes[ly.shape];
    std::vector<int> one{ell};
    Rec rec;
    rec.upload_stream = ctx.stream;
    rec_zero_slots<C>(ctx, rec, one, ldc);
    dim3 grid(cdiv(sh.N, 256), ncols);
    C* acc = (C*)ctx.slot_acc[ell];
    const C* xv = (const C*)ctx.slot_x[ell];
    const int* pos = sh.d_pos;
    const long long N = sh.N;
    rec.add([=](cudaStream_t st) {
        k_gather_local<C><<<grid, 256, 0, st>>>(acc, pos, ldc, g, N, ncols);
        HZ_CHECK_LAUNCH();
    });
    rec_subst<C>(ctx, rec, one, ncols);
    rec.add([=](cudaStream_t st) {
        k_scatter_local<C><<<grid, 256, 0, st>>>(xv, pos, ldc, w, N, ncols);
        HZ_CHECK_LAUNCH();
    });
    run_now(ctx, rec);
}

template <class C>
void op_polarized_rhs(Ctx& ctx, const double2* g, bool scale, int R, double2* fpol) {
    Rec rec;
    rec.upload_stream = ctx.stream;
    rec_polarized_rhs<C>(ctx, rec, g, scale, R, fpol);
    run_now(ctx, rec);
}

template <class C>
void op_apply_mpol(Ctx& ctx, const double2* x, int R, double2* y) {
    Rec rec;
    rec.upload_stream = ctx.stream;
    rec_apply_mpol<C>(ctx, rec, x, R, y);
    run_now(ctx, rec);
}

template <class C>
void op_apply_precond(Ctx& ctx, const double2* x, int R, double2* y, double2* tmp) {
    Rec rec;
    rec.upload_stream = ctx.stream;
    rec_apply_precond<C>(ctx, rec, x, R, y, tmp);
    run_now(ctx, rec);
}

template <class C>
void op_reconstruct(Ctx& ctx, const double2* g, bool scale, const double2* t, int R, double2* u, bool accumulate) {
    Rec rec;
    rec.upload_stream = ctx.stream;
    rec_reconstruct<C>(ctx, rec, g, scale, t, R, u, accumulate);
    run_now(ctx, rec);
}

void op_volume_residual(Ctx& ctx, const double2* f, bool scale, const double2* u, int R, double2* r, double* norms) {
    long long N3 = (long long)ctx.nx * ctx.ny * ctx.nz;
    HZ_CUDA(cudaMemsetAsync(norms, 0, 2 * R * sizeof(double), ctx.stream));
    constexpr int RB = 8;   // columns per thread
    dim3 grid(cdiv(N3, 256), cdiv(R, RB));
    k_residual<RB><<<grid, 256, 0, ctx.stream>>>(f, u, r, norms, scale ? 1 : 0, R, ctx.nx, ctx.ny, ctx.nz,
                                                 ctx.d_sx_n, ctx.d_isx_h, ctx.d_sy_n, ctx.d_isy_h, ctx.d_sz_n,
                                                 ctx.d_isz_h, ctx.d_m, ctx.d_b, ctx.omega * ctx.omega,
                                                 1.0 / (ctx.h * ctx.h));
    HZ_CHECK_LAUNCH();
}

// ------------------------------------------------------------------------------------------
// GMRES on P M_pol u = P f_pol (Eq. 15), x0 = 0, one Krylov space per column, CGS2.
// Then traces t = u_down + u_up and the volume reconstruction.  Writes u (not accumulated).
// The workspace persists in the handle; the matrix-vector product P M_pol (fixed input and
// output buffers) is recorded once per column count and replayed as a CUDA graph.
// ------------------------------------------------------------------------------------------
namespace {

void ensure_gmres_work(Ctx& ctx, int R, int m) {
    GmresWork& g = ctx.gw;
    if (g.cap_R >= R && g.m == m) return;
    g.release();
    ctx.plans.clear();
    ctx.setup_plans.clear();
    ctx.recon_plans.clear();
    const long long n = ctx.ntr;
    const long long vs = (long long)R * n;
    auto alloc = [&](size_t bytes) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            g.release();
            throw Error{HZ_ERR_ADMISSION, "GMRES workspace does not fit in device memory"};
        }
        g.bufs.push_back(p);
        return p;
    };
    g.V = (double2*)alloc((size_t)(m + 1) * vs * sizeof(double2));
    g.in = (double2*)alloc((size_t)vs * sizeof(double2));
    g.out = (double2*)alloc((size_t)vs * sizeof(double2));
    g.w2 = (double2*)alloc((size_t)vs * sizeof(double2));
    g.tmp = (double2*)alloc((size_t)vs * sizeof(double2));
    g.b = (double2*)alloc((size_t)vs * sizeof(double2));
    g.xs = (double2*)alloc((size_t)vs * sizeof(double2));
    g.H = (double2*)alloc((size_t)R * (m + 1) * m * sizeof(double2));
    g.cs = (double2*)alloc((size_t)R * m * sizeof(double2));
    g.sn = (double2*)alloc((size_t)R * m * sizeof(double2));
    g.g = (double2*)alloc((size_t)R * (m + 1) * sizeof(double2));
    g.dots = (double2*)alloc((size_t)R * (m + 1) * sizeof(double2));
    g.y = (double2*)alloc((size_t)R * m * sizeof(double2));
    g.t = (double2*)alloc((size_t)R * ctx.K * 2 * ctx.P * sizeof(double2));
    g.nrm = (double*)alloc(R * sizeof(double));
    g.invb = (double*)alloc(R * sizeof(double));
    g.resid = (double*)alloc(R * sizeof(double));
    g.b0 = (double*)alloc(R * sizeof(double));
    g.active = (int*)alloc(R * sizeof(int));
    g.kused = (int*)alloc(R * sizeof(int));
    g.cap_R = R;
    g.m = m;
}

template <class C>
Rec& matvec_plan(Ctx& ctx, int R) {
    auto it = ctx.plans.find(R);
    if (it != ctx.plans.end()) return *it->second;
    auto rec = std::make_unique<Rec>();
    rec->upload_stream = ctx.stream;
    rec_apply_mpol<C>(ctx, *rec, ctx.gw.in, R, ctx.gw.w2);
    rec_apply_precond<C>(ctx, *rec, ctx.gw.w2, R, ctx.gw.out, ctx.gw.tmp);
    return *ctx.plans.emplace(R, std::move(rec)).first->second;
}

// Device slots holding the current call's volume pointers (right-hand side, solution), read by the
// recorded set-up and reconstruction plans; written before each run on the handle's stream.
inline void set_io(Ctx& ctx, const double2* g, double2* u) {
    if (!ctx.d_io) {
        void* p = nullptr;
        if (cudaMalloc(&p, 2 * sizeof(void*)) != cudaSuccess) {
            cudaGetLastError();
            throw Error{HZ_ERR_OOM, "pointer slots"};
        }
        ctx.d_io = (void**)p;
        HZ_CUDA(cudaMallocHost((void**)&ctx.h_io, 2 * sizeof(void*)));
    }
    HZ_CUDA(cudaStreamSynchronize(ctx.stream));   // the pinned staging pair is reused by every call
    ctx.h_io[0] = (void*)g;
    ctx.h_io[1] = (void*)u;
    HZ_CUDA(cudaMemcpyAsync(ctx.d_io, ctx.h_io, 2 * sizeof(void*), cudaMemcpyHostToDevice, ctx.stream));
}

// b = P f_pol for the volume right-hand side in slot 0 (Algorithm 2 up to the trace system), into
// the Krylov workspace's b; recorded once per (column count, scaling)
template <class C>
Rec& setup_plan(Ctx& ctx, int R, bool scale) {
    const long long key = 2LL * R + (scale ? 1 : 0);
    auto it = ctx.setup_plans.find(key);
    if (it != ctx.setup_plans.end()) return *it->second;
    auto rec = std::make_unique<Rec>();
    rec->upload_stream = ctx.stream;
    const double2* const* gslot = (const double2* const*)ctx.d_io;
    rec_polarized_rhs<C>(ctx, *rec, nullptr, scale, R, ctx.gw.w2, gslot);
    rec_apply_precond<C>(ctx, *rec, ctx.gw.w2, R, ctx.gw.b, ctx.gw.tmp);
    return *ctx.setup_plans.emplace(key, std::move(rec)).first->second;
}

// u (slot 1) from the volume right-hand side (slot 0) and the traces in the workspace's t
// (Algorithm 2, reconstruction); recorded once per (column count, scaling)
template <class C>
Rec& recon_plan(Ctx& ctx, int R, bool scale) {
    const long long key = 2LL * R + (scale ? 1 : 0);
    auto it = ctx.recon_plans.find(key);
    if (it != ctx.recon_plans.end()) return *it->second;
    auto rec = std::make_unique<Rec>();
    rec->upload_stream = ctx.stream;
    rec_reconstruct<C>(ctx, *rec, nullptr, scale, ctx.gw.t, R, nullptr, false,
                       (const double2* const*)ctx.d_io, (double2* const*)ctx.d_io + 1);
    return *ctx.recon_plans.emplace(key, std::move(rec)).first->second;
}

template <class C>
void run_plan(Ctx& ctx, Rec& rec) {
    if (ctx.use_graphs && !ctx.prof) rec.run_graph(ctx.stream);
    else rec.run(ctx.stream);
}

}  // namespace

template <class C>
void gmres_solve(Ctx& ctx, const double2* g, bool scale, int R, double2* u, const hz_solve_opts& o,
                 hz_solve_info* info) {
    cudaStream_t st = ctx.stream;
    const long long n = ctx.ntr;
    if (ctx.L == 1 || n == 0) {
        op_reconstruct<C>(ctx, g, scale, nullptr, R, u, false);
        if (info) for (int r = 0; r < R; ++r) { info[r].iters = 0; info[r].trace_relres = 0.0; }
        return;
    }
    const int m = std::max(1, std::min(o.restart, o.max_iter));
    ensure_gmres_work(ctx, R, m);
    GmresWork& W = ctx.gw;
    const long long vs = (long long)R * n;  // stride between Krylov vectors
    GmresState s;
    s.H = W.H; s.cs_sn = W.cs; s.sn = W.sn; s.g = W.g; s.dots = W.dots; s.y = W.y;
    s.nrm = W.nrm; s.invb = W.invb; s.resid = W.resid; s.active = W.active; s.kused = W.kused;
    double* b0 = W.b0;
    const long long half = (long long)ctx.K * 2 * ctx.P;
    const int TB = 256;
    const int gblocks = (int)std::min<long long>(1024, std::max<long long>(1, (n + TB - 1) / TB));
    const dim3 gvec(cdiv(n, TB), R);
    Rec& mv = matvec_plan<C>(ctx, R);
    auto matvec = [&](const double2* in, double2* out) {
        HZ_CUDA(cudaMemcpyAsync(W.in, in, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        if (ctx.use_graphs && !ctx.prof) mv.run_graph(st);
        else mv.run(st);
        if (out != W.out) HZ_CUDA(cudaMemcpyAsync(out, W.out, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    };
    auto norms = [&](const double2* v, double* out) {
        HZ_CUDA(cudaMemsetAsync(out, 0, R * sizeof(double), st));
        k_nrm2<<<dim3(gblocks, R), TB, 0, st>>>(v, n, out);
        HZ_CHECK_LAUNCH();
    };
    std::vector<int> hact(R);
    auto any_active = [&]() {
        HZ_CUDA(cudaMemcpyAsync(hact.data(), s.active, R * sizeof(int), cudaMemcpyDeviceToHost, st));
        HZ_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) if (hact[r]) return true;
        return false;
    };
    const double tiny = 1e-300;
    std::vector<double> h_resid(R), h_b0(R);
    int total_it = 0;
    // b = P f_pol ; x = 0
    set_io(ctx, g, u);
    run_plan<C>(ctx, setup_plan<C>(ctx, R, scale));
    HZ_CUDA(cudaMemsetAsync(W.xs, 0, (size_t)vs * sizeof(double2), st));
    norms(W.b, b0);
    {
        std::vector<int> ones(R, 1);
        HZ_CUDA(cudaMemcpyAsync(s.active, ones.data(), R * sizeof(int), cudaMemcpyHostToDevice, st));
        HZ_CUDA(cudaStreamSynchronize(st));
    }
    double2* w = W.out;  // the matvec writes its result here
    bool first = true;
    for (;;) {
        // residual of the preconditioned system: r0 = b - P M x
        if (first) {
            HZ_CUDA(cudaMemcpyAsync(w, W.b, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        } else {
            matvec(W.xs, w);
            k_lincomb<<<gvec, TB, 0, st>>>(w, n, 1.0, W.b, n, -1.0, w, n, n);
            HZ_CHECK_LAUNCH();
        }
        first = false;
        norms(w, s.nrm);
        k_gmres_start<<<cdiv(R, 128), 128, 0, st>>>(s, R, m, tiny);
        HZ_CHECK_LAUNCH();
        k_scale_vec<<<gvec, TB, 0, st>>>(W.V, w, n, s.invb);
        HZ_CHECK_LAUNCH();
        if (!any_active()) break;
        for (int j = 0; j < m && total_it < o.max_iter; ++j) {
            matvec(W.V + (long long)j * vs, w);
            HZ_CUDA(cudaMemsetAsync(s.dots, 0, (size_t)R * (m + 1) * sizeof(double2), st));
            for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
                HZ_CUDA(cudaMemsetAsync(s.y, 0, (size_t)R * m * sizeof(double2), st));
                k_mdot<<<dim3(gblocks, R), TB, 0, st>>>(W.V, vs, w, n, j + 1, s.y, m);
                HZ_CHECK_LAUNCH();
                k_maxpy<<<gvec, TB, 0, st>>>(W.V, vs, w, n, j + 1, s.y, m);
                HZ_CHECK_LAUNCH();
                k_accum_dots<<<cdiv(R * (j + 1), 128), 128, 0, st>>>(s.dots, s.y, R, m, j + 1);
                HZ_CHECK_LAUNCH();
            }
            norms(w, s.nrm);
            k_gmres_arnoldi<<<cdiv(R, 128), 128, 0, st>>>(s, R, m, j, 0.0, b0, o.gmres_tol, tiny);
            HZ_CHECK_LAUNCH();
            k_scale_vec<<<gvec, TB, 0, st>>>(W.V + (long long)(j + 1) * vs, w, n, s.invb);
            HZ_CHECK_LAUNCH();
            ++total_it;
            if (!any_active()) break;
        }
        // x += V y for this cycle
        k_gmres_lsq<<<cdiv(R, 128), 128, 0, st>>>(s, R, m);
        HZ_CHECK_LAUNCH();
        k_maxpy_plus<<<gvec, TB, 0, st>>>(W.V, vs, W.xs, n, m, s.y, m);
        HZ_CHECK_LAUNCH();
        if (!any_active() || total_it >= o.max_iter) break;
        // columns still active restart from their current iterate
    }
    HZ_CUDA(cudaMemcpyAsync(h_resid.data(), s.resid, R * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(h_b0.data(), b0, R * sizeof(double), cudaMemcpyDeviceToHost, st));
    // traces t = x_down + x_up, laid out [R][K][2][P]
    k_lincomb<<<dim3(cdiv(half, TB), R), TB, 0, st>>>(W.t, half, 1.0, W.xs, n, 1.0, W.xs + half, n, half);
    HZ_CHECK_LAUNCH();
    run_plan<C>(ctx, recon_plan<C>(ctx, R, scale));
    HZ_CUDA(cudaStreamSynchronize(st));
    if (info) {
        for (int r = 0; r < R; ++r) {
            info[r].iters = total_it;
            double nb = sqrt(std::max(h_b0[r], 0.0));
            info[r].trace_relres = nb > 0 ? h_resid[r] / nb : 0.0;
        }
    }
}

template void op_layer_solve<float2>(Ctx&, int, const double2*, int, double2*);
template void op_layer_solve<double2>(Ctx&, int, const double2*, int, double2*);
template void op_polarized_rhs<float2>(Ctx&, const double2*, bool, int, double2*);
template void op_polarized_rhs<double2>(Ctx&, const double2*, bool, int, double2*);
template void op_apply_mpol<float2>(Ctx&, const double2*, int, double2*);
template void op_apply_mpol<double2>(Ctx&, const double2*, int, double2*);
template void op_apply_precond<float2>(Ctx&, const double2*, int, double2*, double2*);
template void op_apply_precond<double2>(Ctx&, const double2*, int, double2*, double2*);
template void op_reconstruct<float2>(Ctx&, const double2*, bool, const double2*, int, double2*, bool);
template void op_reconstruct<double2>(Ctx&, const double2*, bool, const double2*, int, double2*, bool);
template void build_trace_blocks<float2>(Ctx&, int);
template void build_trace_blocks<double2>(Ctx&, int);
// ------------------------------------------------------------------------------------------
// Bi-CGSTAB on the same left-preconditioned trace system P M_pol x = P f_pol (the paper's
// remark on Krylov solvers in its Parallelization Strategies section: Bi-CGSTAB keeps a fixed,
// small number of vectors where GMRES keeps its whole basis).  One process per column, FP64,
// x0 = 0, shadow residual r^ = r0; per iteration two matrix-vector products:
//   rho = <r^, r>;  beta = (rho / rho_old)(alpha / omega);  p = r + beta (p - omega v);
//   v = A p;  alpha = rho / <r^, v>;  s = r - alpha v;  t = A s;  omega = <t, s> / <t, t>;
//   x += alpha p + omega s;  r = s - omega t
// with <a, b> = a^H b.  A column stops when ||r|| <= tol ||b|| or on a breakdown (a vanishing
// <r^, r> or <r^, v>); stopped columns are no longer updated.
// ------------------------------------------------------------------------------------------
struct BicgScalars {
    double2* dots;     // [R][4]: <r^, r>, <r^, v>, <t, s>, <t, t>
    double2* rho_old;  // [R]
    double2* alpha;    // [R]
    double2* omega;    // [R]
    double2* beta;     // [R]
    double* nrm;       // [R] ||r||^2
    double* resid;     // [R] ||r||
    const double* b0;  // [R] ||b||^2
    int* active;       // [R]
};

__device__ inline double2 cdivc(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__global__ void k_bicg_init(BicgScalars s, int R, double tiny) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    s.rho_old[r] = make_double2(1.0, 0.0);
    s.alpha[r] = make_double2(1.0, 0.0);
    s.omega[r] = make_double2(1.0, 0.0);
    s.resid[r] = sqrt(s.b0[r]);
    s.active[r] = s.b0[r] > tiny * tiny;
}

// stage 0: beta from rho = <r^, r>; stage 1: alpha = rho / <r^, v>; stage 2: omega = <t,s>/<t,t>
__global__ void k_bicg_scalars(BicgScalars s, int R, int stage, double tiny) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !s.active[r]) return;
    const double2* d = s.dots + 4LL * r;
    if (stage == 0) {
        const double2 rho = d[0];
        if (!(sqrt(rho.x * rho.x + rho.y * rho.y) > tiny)) { s.active[r] = 0; return; }
        s.beta[r] = cmul(cdivc(rho, s.rho_old[r]), cdivc(s.alpha[r], s.omega[r]));
        s.rho_old[r] = rho;
    } else if (stage == 1) {
        const double2 rv = d[1];
        if (!(sqrt(rv.x * rv.x + rv.y * rv.y) > tiny)) { s.active[r] = 0; return; }
        s.alpha[r] = cdivc(s.rho_old[r], rv);
    } else {
        const double tt = d[3].x;
        s.omega[r] = tt > 0.0 ? cscale(d[2], 1.0 / tt) : make_double2(0.0, 0.0);
    }
}

// op 0: p = r + beta (p - omega v); op 1: s = r - alpha v; op 2: x += alpha p + omega s, r = s - omega t
__global__ void k_bicg_update(BicgScalars s, int op, double2* x, double2* rv, double2* p, const double2* v,
                              double2* sv, const double2* t, long long n) {
    const int r = blockIdx.y;
    if (!s.active[r]) return;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long i = (long long)r * n + e;
    if (op == 0) {
        p[i] = cadd(rv[i], cmul(s.beta[r], csub(p[i], cmul(s.omega[r], v[i]))));
    } else if (op == 1) {
        sv[i] = csub(rv[i], cmul(s.alpha[r], v[i]));
    } else {
        x[i] = cadd(x[i], cadd(cmul(s.alpha[r], p[i]), cmul(s.omega[r], sv[i])));
        rv[i] = csub(sv[i], cmul(s.omega[r], t[i]));
    }
}

__global__ void k_bicg_check(BicgScalars s, int R, double tol) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !s.active[r]) return;
    const double res = sqrt(s.nrm[r]);
    s.resid[r] = res;
    if (!(res > tol * sqrt(s.b0[r]))) s.active[r] = 0;
}

template <class C>
void bicgstab_solve(Ctx& ctx, const double2* g, bool scale, int R, double2* u, const hz_solve_opts& o,
                    hz_solve_info* info) {
    cudaStream_t st = ctx.stream;
    const long long n = ctx.ntr;
    if (ctx.L == 1 || n == 0) {
        op_reconstruct<C>(ctx, g, scale, nullptr, R, u, false);
        if (info) for (int r = 0; r < R; ++r) { info[r].iters = 0; info[r].trace_relres = 0.0; }
        return;
    }
    // six vectors of the Krylov process (r, r^, p, v, s, t) in the workspace's basis slots; a
    // larger basis already allocated for GMRES is reused as it is
    const int m = (ctx.gw.cap_R >= R && ctx.gw.m >= 5) ? ctx.gw.m : 5;
    ensure_gmres_work(ctx, R, m);
    GmresWork& W = ctx.gw;
    const long long vs = (long long)R * n;
    double2 *rv = W.V, *rh = W.V + vs, *p = W.V + 2 * vs, *v = W.V + 3 * vs, *sv = W.V + 4 * vs, *t = W.V + 5 * vs;
    BicgScalars sc;
    sc.dots = W.g;   // R x (m + 1) >= R x 4
    sc.rho_old = W.H;
    sc.alpha = W.H + R;
    sc.omega = W.H + 2 * R;
    sc.beta = W.H + 3 * R;
    sc.nrm = W.nrm;
    sc.resid = W.resid;
    sc.b0 = W.b0;
    sc.active = W.active;
    const long long half = (long long)ctx.K * 2 * ctx.P;
    const int TB = 256;
    const int gblocks = (int)std::min<long long>(1024, std::max<long long>(1, (n + TB - 1) / TB));
    const dim3 gvec(cdiv(n, TB), R);
    Rec& mv = matvec_plan<C>(ctx, R);
    auto matvec = [&](const double2* in, double2* out) {
        HZ_CUDA(cudaMemcpyAsync(W.in, in, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        if (ctx.use_graphs && !ctx.prof) mv.run_graph(st);
        else mv.run(st);
        HZ_CUDA(cudaMemcpyAsync(out, W.out, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    };
    auto dot = [&](const double2* a, const double2* b, int slot) {   // dots[r][slot] = <a_r, b_r>
        k_mdot<<<dim3(gblocks, R), TB, 0, st>>>(a, vs, b, n, 1, sc.dots + slot, 4);
        HZ_CHECK_LAUNCH();
    };
    std::vector<int> hact(R);
    auto any_active = [&]() {
        HZ_CUDA(cudaMemcpyAsync(hact.data(), sc.active, R * sizeof(int), cudaMemcpyDeviceToHost, st));
        HZ_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) if (hact[r]) return true;
        return false;
    };
    const double tiny = 1e-300;
    // b = P f_pol; x = 0; r = r^ = b; p = v = 0
    set_io(ctx, g, u);
    run_plan<C>(ctx, setup_plan<C>(ctx, R, scale));
    HZ_CUDA(cudaMemsetAsync(W.xs, 0, (size_t)vs * sizeof(double2), st));
    HZ_CUDA(cudaMemsetAsync(p, 0, (size_t)vs * sizeof(double2), st));
    HZ_CUDA(cudaMemsetAsync(v, 0, (size_t)vs * sizeof(double2), st));
    HZ_CUDA(cudaMemcpyAsync(rv, W.b, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    HZ_CUDA(cudaMemcpyAsync(rh, W.b, (size_t)vs * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    HZ_CUDA(cudaMemsetAsync(W.b0, 0, R * sizeof(double), st));
    k_nrm2<<<dim3(gblocks, R), TB, 0, st>>>(W.b, n, W.b0);
    HZ_CHECK_LAUNCH();
    k_bicg_init<<<cdiv(R, 128), 128, 0, st>>>(sc, R, tiny);
    HZ_CHECK_LAUNCH();
    int it = 0;
    while (it < o.max_iter && any_active()) {
        HZ_CUDA(cudaMemsetAsync(sc.dots, 0, (size_t)R * 4 * sizeof(double2), st));
        dot(rh, rv, 0);
        k_bicg_scalars<<<cdiv(R, 128), 128, 0, st>>>(sc, R, 0, tiny);
        HZ_CHECK_LAUNCH();
        k_bicg_update<<<gvec, TB, 0, st>>>(sc, 0, W.xs, rv, p, v, sv, t, n);
        HZ_CHECK_LAUNCH();
        matvec(p, v);
        dot(rh, v, 1);
        k_bicg_scalars<<<cdiv(R, 128), 128, 0, st>>>(sc, R, 1, tiny);
        HZ_CHECK_LAUNCH();
        k_bicg_update<<<gvec, TB, 0, st>>>(sc, 1, W.xs, rv, p, v, sv, t, n);
        HZ_CHECK_LAUNCH();
        matvec(sv, t);
        dot(t, sv, 2);
        dot(t, t, 3);
        k_bicg_scalars<<<cdiv(R, 128), 128, 0, st>>>(sc, R, 2, tiny);
        HZ_CHECK_LAUNCH();
        k_bicg_update<<<gvec, TB, 0, st>>>(sc, 2, W.xs, rv, p, v, sv, t, n);
        HZ_CHECK_LAUNCH();
        HZ_CUDA(cudaMemsetAsync(sc.nrm, 0, R * sizeof(double), st));
        k_nrm2<<<dim3(gblocks, R), TB, 0, st>>>(rv, n, sc.nrm);
        HZ_CHECK_LAUNCH();
        k_bicg_check<<<cdiv(R, 128), 128, 0, st>>>(sc, R, o.gmres_tol);
        HZ_CHECK_LAUNCH();
        ++it;
    }
    std::vector<double> h_resid(R), h_b0(R);
    HZ_CUDA(cudaMemcpyAsync(h_resid.data(), sc.resid, R * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(h_b0.data(), W.b0, R * sizeof(double), cudaMemcpyDeviceToHost, st));
    // traces t = x_down + x_up, laid out [R][K][2][P]
    k_lincomb<<<dim3(cdiv(half, TB), R), TB, 0, st>>>(W.t, half, 1.0, W.xs, n, 1.0, W.xs + half, n, half);
    HZ_CHECK_LAUNCH();
    run_plan<C>(ctx, recon_plan<C>(ctx, R, scale));
    HZ_CUDA(cudaStreamSynchronize(st));
    if (info) {
        for (int r = 0; r < R; ++r) {
            info[r].iters = it;
            const double nb = sqrt(std::max(h_b0[r], 0.0));
            info[r].trace_relres = nb > 0 ? h_resid[r] / nb : 0.0;
        }
    }
}

template <class C>
void krylov_solve(Ctx& ctx, const double2* g, bool scale, int R, double2* u, const hz_solve_opts& o,
                  hz_solve_info* info) {
    if (o.krylov == 1) bicgstab_solve<C>(ctx, g, scale, R, u, o, info);
    else gmres_solve<C>(ctx, g, scale, R, u, o, info);
}

template void gmres_solve<float2>(Ctx&, const double2*, bool, int, double2*, const hz_solve_opts&, hz_solve_info*);
template void gmres_solve<double2>(Ctx&, const double2*, bool, int, double2*, const hz_solve_opts&, hz_solve_info*);
template void krylov_solve<float2>(Ctx&, const double2*, bool, int, double2*, const hz_solve_opts&, hz_solve_info*);
template void krylov_solve<double2>(Ctx&, const double2*, bool, int, double2*, const hz_solve_opts&, hz_solve_info*);

}  // namespace hz
