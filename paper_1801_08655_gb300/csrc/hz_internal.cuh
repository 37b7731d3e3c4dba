// Internal declarations shared by the translation units of libhz.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "hz.h"

namespace hz {

constexpr int TILE = 32;           // factor tiles are TILE x TILE, column-major inside
constexpr int TILE2 = TILE * TILE;

// ------------------------------------------------------------------------------------------
// complex helpers on float2 / double2 (interleaved re, im)
// ------------------------------------------------------------------------------------------
template <class T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <class R> using cx = typename cplx<R>::type;

template <class C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }

template <class C> __host__ __device__ inline C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class C> __host__ __device__ inline C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class C> __host__ __device__ inline C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a += b * c
template <class C> __host__ __device__ inline void cfma(C& a, C b, C c) {
    a.x = fma(b.x, c.x, a.x); a.x = fma(-b.y, c.y, a.x);
    a.y = fma(b.x, c.y, a.y); a.y = fma(b.y, c.x, a.y);
}
template <class C> __host__ __device__ inline C cscale(C a, typename real_of<C>::type s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
template <class C> __host__ __device__ inline C cneg(C a) { C r; r.x = -a.x; r.y = -a.y; return r; }
template <class C> __host__ __device__ inline C czero() { C r; r.x = 0; r.y = 0; return r; }
// 1/a = conj(a) / |a|^2 (definition of the complex reciprocal)
__host__ __device__ inline double2 crecip(double2 a) {
    double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}
__host__ __device__ inline float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ inline double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ inline double2 to_d(double2 a) { return a; }
template <class C> __host__ __device__ inline C from_d(double2 a);
template <> __host__ __device__ inline float2 from_d<float2>(double2 a) { return to_f(a); }
template <> __host__ __device__ inline double2 from_d<double2>(double2 a) { return a; }

// Coefficient b of div(b grad u) (b = 1/rho) at the half node between cell i (coordinate `coord`
// of `n` along an axis of element stride `stride`) and its neighbour in direction d = -1 / +1:
// the average of the two nodes, the cell itself standing in for a neighbour beyond the grid.
// b == nullptr means constant density (b = 1).
__host__ __device__ inline double bhalf(const double* b, long long i, int coord, int n, long long stride, int d) {
    if (!b) return 1.0;
    const int c2 = coord + d;
    const double v2 = (c2 >= 0 && c2 < n) ? b[i + d * stride] : b[i];
    return 0.5 * (b[i] + v2);
}

// ------------------------------------------------------------------------------------------
// symbolic structures (host), built once per distinct slab shape
// ------------------------------------------------------------------------------------------
struct NodeDev {            // device copy of what the solve kernels need per tree node
    int own0, nown, nupd, own_t, upd_t;
    int pad_;
    long long upd_off;      // into the shape's upd_idx array
    long long linv_off;     // tile offset of packed lower-triangular L^{-1} (own_t*(own_t+1)/2 tiles)
    long long l21_off;      // tile offset of L21 (upd_t x own_t tiles, row-tile major)
};

struct Node {
    int own0 = 0, nown = 0, nupd = 0;
    int parent = -1, child[2] = {-1, -1}, nchild = 0;
    int height = 0;
    int box[6] = {0, 0, 0, 0, 0, 0};       // x0,x1,y0,y1,z0,z1 (half open) of the subtree box
    int sep[6] = {0, 0, 0, 0, 0, 0};       // box of the own cells
    long long upd_off = 0;
    long long front_off = 0;               // element offset of the dense front in a layer's arena
    int m = 0;                             // front dimension nown + nupd
    int own_t = 0, upd_t = 0;
    long long linv_off = 0, l21_off = 0;   // tile offsets in the layer's factor storage
    long long asm_off = 0; int nasm = 0;   // assembly entries
    long long emap_off = 0;                // extend-add map into the parent front (nupd entries)
};

struct AsmEntry {            // one original-matrix entry of a front (lower triangle, own columns)
    long long foff;          // element offset inside the node's front (row + col*m)
    int cell;                // natural local cell index of the column unknown
    int dir;                 // 0 diagonal, 1..6 = x-, x+, y-, y+, z-, z+ neighbour (row unknown)
};

struct Shape {
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    std::vector<Node> nodes;
    std::vector<int> perm;                 // elimination index -> natural local cell
    std::vector<int> pos;                  // natural local cell -> elimination index
    std::vector<int> upd_idx;              // elimination indices of every node's update set
    std::vector<AsmEntry> asm_entries;
    std::vector<int> emap;
    std::vector<std::vector<int>> levels;  // node ids by height (0 = leaves)
    long long front_total = 0;             // sum of m^2 (elements)
    long long factor_tiles = 0;            // packed tiles (Linv + L21)
    double factor_flops = 0;               // real flops of the numeric factorization
    double solve_flops_per_col = 0;        // real flops of one forward+backward substitution, one column
    int max_m = 0;
    // device copies
    NodeDev* d_nodes = nullptr;
    int* d_pos = nullptr;
    int* d_upd_idx = nullptr;
    AsmEntry* d_asm = nullptr;
    int* d_emap = nullptr;
    long long* d_front_off = nullptr;
    int* d_front_m = nullptr;
};

void build_shape(Shape& s, int nx, int ny, int nz, int leaf);

// ------------------------------------------------------------------------------------------
// per-layer data
// ------------------------------------------------------------------------------------------
struct Layer {
    int shape = 0;
    int lo = 0, hi = 0;        // owned global planes
    int zlo = 0, zhi = 0;      // extended local grid
    int nzl = 0;
    // FP64 coefficient inputs (device): 1D stretch profiles and local m
    double2* d_sz_n = nullptr;     // s_z at local nodes (nzl)
    double2* d_isz_h = nullptr;    // 1/s_z at local half nodes (nzl+1), index k <-> k - 1/2
    double* d_m = nullptr;         // m on the local grid (nzl*ny*nx)
    double* d_b = nullptr;         // b = 1/rho on the local grid (owned planes and one plane beyond
                                   // each internal interface as they are globally, copied further
                                   // into the pads), or nullptr for constant density
    void* d_fac = nullptr;         // packed factor tiles (complex T)
    void* d_dinv = nullptr;        // D^{-1} by elimination index (complex T, N)
};

// Job of a batched local solve: which layer and which vectors (elimination order, row-major,
// leading dimension ldc complex elements).
template <class C> struct JobDev {
    const C* fac;
    const C* dinv;
    const NodeDev* nodes;
    const int* upd_idx;
    C* acc;   // accumulator (forward) / scratch (backward)
    C* x;     // solution
};

struct Task { int job, node, tile, pad_; };

// ------------------------------------------------------------------------------------------
// error handling
// ------------------------------------------------------------------------------------------
struct Error {
    hz_status st;
    std::string msg;
};

#define HZ_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            throw ::hz::Error{HZ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
        }                                                                                     \
    } while (0)

// every kernel launch of the library goes through this check, which also counts it
extern std::atomic<long long> g_launch_count;
#define HZ_CHECK_LAUNCH()                                                   \
    do {                                                                    \
        ::hz::g_launch_count.fetch_add(1, std::memory_order_relaxed);       \
        HZ_CUDA(cudaGetLastError());                                        \
    } while (0)

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace hz
