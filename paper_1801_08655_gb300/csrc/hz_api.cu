// C ABI of the solver (declared in include/hz.h): problem set-up, offline factorization,
// online solves with FP64 volume-residual defect correction, and stage entry points.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <cstdlib>
#include <new>
#include <thread>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"
#include "hz_solve.cuh"

using hz::Ctx;
using hz::Error;

namespace hz {
std::atomic<long long> g_launch_count{0};
namespace {

thread_local std::string g_create_error;

// Quadratic PML profile (Formulation section, Eq. 5): sigma = (C/delta)(d/delta)^2 with d the
// distance into the pad measured from the first physical node (index npml), delta = npml*h.
double sigma_global(double x, int n, int npml, double C, double h) {
    if (npml <= 0) return 0.0;
    const double lo = npml, hi = n - 1 - npml, delta = npml * h;
    double d = x < lo ? lo - x : (x > hi ? x - hi : 0.0);
    d *= h;
    return (C / delta) * (d / delta) * (d / delta);
}

// Internal layer pads start half a cell past the owned planes [lo, hi] (npml_loc nodes thick),
// the global profile is inherited at the outer faces.
double sigma_local_z(double z, int ell, int L, int lo, int hi, int n, int npml, int npml_loc, double C,
                     double h) {
    double s = sigma_global(z, n, npml, C, h);
    if (npml_loc > 0) {
        const double dl = npml_loc * h;
        if (ell > 0 && z < lo - 0.5) {
            double d = (lo - 0.5 - z) * h;
            s = (C / dl) * (d / dl) * (d / dl);
        }
        if (ell < L - 1 && z > hi + 0.5) {
            double d = (z - hi - 0.5) * h;
            s = (C / dl) * (d / dl) * (d / dl);
        }
    }
    return s;
}

// s = 1 + i sigma/omega (inverse of the stretching factor beta of Eq. 4)
double2 s_of(double sigma, double omega) { return make_double2(1.0, sigma / omega); }
double2 inv_s(double sigma, double omega) {
    std::complex<double> v(1.0, sigma / omega);
    v = 1.0 / v;
    return make_double2(v.real(), v.imag());
}

// A failed cudaMalloc is HZ_ERR_OOM when the device ran out of memory and HZ_ERR_CUDA otherwise
// (no device, driver missing, a sticky error from earlier work), with the runtime's message.
[[noreturn]] void alloc_failed(cudaError_t e, size_t bytes) {
    cudaGetLastError();
    const std::string what = "device allocation of " + std::to_string(bytes) + " bytes failed: ";
    if (e == cudaErrorMemoryAllocation) throw Error{HZ_ERR_OOM, what + cudaGetErrorString(e)};
    throw Error{HZ_ERR_CUDA, what + cudaGetErrorString(e)};
}

template <class T> T* dev_copy(const std::vector<T>& v) {
    T* d = nullptr;
    const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
    const cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) alloc_failed(e, bytes);
    HZ_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

void* dev_alloc(size_t bytes) {
    void* d = nullptr;
    const cudaError_t e = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) alloc_failed(e, bytes);
    return d;
}

// Device-to-host copy ordered after the work queued on the handle's stream (which may be a
// non-blocking stream that the legacy default stream does not wait for).
void d2h(Ctx& c, void* dst, const void* src, size_t bytes) {
    HZ_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.stream));
    HZ_CUDA(cudaStreamSynchronize(c.stream));
}

size_t elem_size(const Ctx& c) { return c.prec == HZ_PREC_FP64 ? sizeof(double2) : sizeof(float2); }

__global__ void k_demote(float2* dst, const double2* src, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

// FP64 factorization into temporary complex128 storage, then rounding to the complex64 factors.
void factor_fp64_demote(Ctx& c) {
    std::vector<void*> tmp_fac, tmp_dinv;
    try {
        for (auto& ly : c.layers) {
            const Shape& sh = c.shapes[ly.shape];
            tmp_fac.push_back(dev_alloc((size_t)sh.factor_tiles * TILE2 * sizeof(double2)));
            tmp_dinv.push_back(dev_alloc((size_t)sh.N * sizeof(double2)));
        }
        std::vector<std::pair<void*, void*>> keep;
        for (size_t l = 0; l < c.layers.size(); ++l) {
            keep.push_back({c.layers[l].d_fac, c.layers[l].d_dinv});
            c.layers[l].d_fac = tmp_fac[l];
            c.layers[l].d_dinv = tmp_dinv[l];
        }
        try {
            factor_layers<double2>(c);
        } catch (...) {
            for (size_t l = 0; l < c.layers.size(); ++l) { c.layers[l].d_fac = keep[l].first; c.layers[l].d_dinv = keep[l].second; }
            throw;
        }
        for (size_t l = 0; l < c.layers.size(); ++l) {
            c.layers[l].d_fac = keep[l].first;
            c.layers[l].d_dinv = keep[l].second;
            const Shape& sh = c.shapes[c.layers[l].shape];
            k_demote<<<4096, 256, 0, c.stream>>>((float2*)c.layers[l].d_fac, (const double2*)tmp_fac[l],
                                                 sh.factor_tiles * TILE2);
            HZ_CHECK_LAUNCH();
            k_demote<<<1024, 256, 0, c.stream>>>((float2*)c.layers[l].d_dinv, (const double2*)tmp_dinv[l], sh.N);
            HZ_CHECK_LAUNCH();
        }
        HZ_CUDA(cudaStreamSynchronize(c.stream));
    } catch (...) {
        for (void* p : tmp_fac) cudaFree(p);
        for (void* p : tmp_dinv) cudaFree(p);
        throw;
    }
    for (void* p : tmp_fac) cudaFree(p);
    for (void* p : tmp_dinv) cudaFree(p);
}

void release_slots(Ctx& c) {
    c.plans.clear();  // recorded plans point into the slot batches
    c.setup_plans.clear();
    c.recon_plans.clear();
    free_batches(c);
    for (void* p : c.slot_acc) cudaFree(p);
    for (void* p : c.slot_x) cudaFree(p);
    c.slot_acc.clear();
    c.slot_x.clear();
    c.slot_cap = 0;
}

// Make sure every layer has acc/x slot vectors for `want` columns (at least `need`).
void ensure_slots(Ctx& c, int need, int want) {
    if (c.slot_cap >= want) return;
    if (c.slot_cap >= need && c.slot_cap > 0) {
        // keep the smaller slots unless the larger ones fit comfortably
        size_t fr = 0, tot = 0;
        HZ_CUDA(cudaMemGetInfo(&fr, &tot));
        long long sumN = 0;
        for (auto& ly : c.layers) sumN += c.shapes[ly.shape].N;
        double extra = 2.0 * sumN * (double)(want - c.slot_cap) * elem_size(c);
        if (extra > 0.5 * fr) return;
    }
    release_slots(c);
    size_t fr = 0, tot = 0;
    HZ_CUDA(cudaMemGetInfo(&fr, &tot));
    long long sumN = 0;
    for (auto& ly : c.layers) sumN += c.shapes[ly.shape].N;
    int cap = want;
    while (cap > need && 2.0 * sumN * (double)cap * elem_size(c) > 0.6 * fr) cap = std::max(need, cap / 2);
    if (2.0 * sumN * (double)cap * elem_size(c) > 0.8 * fr)
        throw Error{HZ_ERR_ADMISSION, "layer solve workspace for this many right-hand sides does not fit"};
    for (auto& ly : c.layers) {
        size_t bytes = (size_t)c.shapes[ly.shape].N * cap * elem_size(c);
        c.slot_acc.push_back(dev_alloc(bytes));
        c.slot_x.push_back(dev_alloc(bytes));
    }
    c.slot_cap = cap;
}

void prepare_for(Ctx& c, int R) {
    const bool dbl = c.prec == HZ_PREC_FP64;
    ensure_slots(c, padded_ldc(dbl, R), padded_ldc(dbl, 4 * R));
}

__global__ void k_axpy_vol(double2* u, const double2* d, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = cadd(u[i], d[i]);
}

void do_solve(Ctx& c, const double2* rhs, int R, double2* u, const hz_solve_opts& o, hz_solve_info* info,
              hz_status& st_out) {
    if (!c.factored) throw Error{HZ_ERR_STATE, "hz_solve before hz_factor"};
    if (R < 1 || !rhs || !u) throw Error{HZ_ERR_ARG, "bad rhs/u/R"};
    prepare_for(c, R);
    cudaEvent_t e0, e1;
    HZ_CUDA(cudaEventCreate(&e0));
    HZ_CUDA(cudaEventCreate(&e1));
    HZ_CUDA(cudaEventRecord(e0, c.stream));
    std::vector<hz_solve_info> inf(R);
    for (auto& x : inf) std::memset(&x, 0, sizeof(x));
    const long long N3 = (long long)c.nx * c.ny * c.nz;
    // persistent per-handle buffers (grown as needed): per-column norms and, in mixed precision,
    // the volume residual and correction of the defect-correction passes; reusing them keeps
    // allocations (and the device-wide synchronisation of cudaFree) out of the solve
    if (c.norms_cap < R) {
        if (c.d_norms) cudaFree(c.d_norms);
        c.d_norms = nullptr;
        c.norms_cap = 0;
        c.d_norms = (double*)dev_alloc(2 * (size_t)R * sizeof(double));
        c.norms_cap = R;
    }
    double* norms = c.d_norms;
    std::vector<double> hn(2 * R);
    st_out = HZ_OK;
    try {
        if (c.prec == HZ_PREC_FP64) {
            krylov_solve<double2>(c, rhs, true, R, u, o, inf.data());
            for (auto& x : inf) x.iters_total = x.iters;
            op_volume_residual(c, rhs, true, u, R, nullptr, norms);
            d2h(c, hn.data(), norms, 2 * R * sizeof(double));
            for (int r = 0; r < R; ++r) {
                inf[r].volume_relres = hn[2 * r + 1] > 0 ? std::sqrt(hn[2 * r] / hn[2 * r + 1]) : 0.0;
                if (!(inf[r].trace_relres <= o.gmres_tol * 1.0001)) st_out = HZ_ERR_NO_CONVERGENCE;
                if (!std::isfinite(inf[r].volume_relres)) st_out = HZ_ERR_NONFINITE;
            }
        } else {
            krylov_solve<float2>(c, rhs, true, R, u, o, inf.data());
            for (auto& x : inf) x.iters_total = x.iters;
            if (c.vol_cap < R) {
                if (c.d_vol_res) cudaFree(c.d_vol_res);
                if (c.d_vol_du) cudaFree(c.d_vol_du);
                c.d_vol_res = c.d_vol_du = nullptr;
                c.vol_cap = 0;
                c.d_vol_res = (double2*)dev_alloc((size_t)R * N3 * sizeof(double2));
                c.d_vol_du = (double2*)dev_alloc((size_t)R * N3 * sizeof(double2));
                c.vol_cap = R;
            }
            double2* res = c.d_vol_res;
            double2* du = c.d_vol_du;
            {
                std::vector<double> g2(R);
                op_volume_residual(c, rhs, true, u, R, res, norms);
                d2h(c, hn.data(), norms, 2 * R * sizeof(double));
                for (int r = 0; r < R; ++r) g2[r] = hn[2 * r + 1];
                auto relres = [&](int r) { return g2[r] > 0 ? std::sqrt(hn[2 * r] / g2[r]) : 0.0; };
                int passes = 0;
                for (;;) {
                    double worst = 0.0;
                    for (int r = 0; r < R; ++r) worst = std::max(worst, relres(r));
                    if (!std::isfinite(worst)) { st_out = HZ_ERR_NONFINITE; break; }
                    if (worst <= o.refine_tol || passes >= o.max_refine) break;
                    // defect correction: A du = r with the mixed path, u += du.  The correction
                    // needs the digits that bring the residual below refine_tol, with a factor 10
                    // to spare: its Krylov tolerance is 0.1 refine_tol / (current residual), never
                    // looser than 1e-1, whatever gmres_tol (which sets the first pass's) is.
                    std::vector<hz_solve_info> inf2(R);
                    hz_solve_opts o2 = o;
                    o2.gmres_tol = std::min(1e-1, 0.1 * o.refine_tol / std::max(worst, 1e-300));
                    krylov_solve<float2>(c, res, false, R, du, o2, inf2.data());
                    k_axpy_vol<<<cdiv((long long)R * N3, 256), 256, 0, c.stream>>>(u, du, (long long)R * N3);
                    HZ_CHECK_LAUNCH();
                    ++passes;
                    for (int r = 0; r < R; ++r) {
                        inf[r].iters = inf2[r].iters;
                        inf[r].iters_total += inf2[r].iters;
                    }
                    op_volume_residual(c, rhs, true, u, R, res, norms);
                    d2h(c, hn.data(), norms, 2 * R * sizeof(double));
                }
                for (int r = 0; r < R; ++r) {
                    inf[r].refinements = passes;
                    inf[r].volume_relres = relres(r);
                    if (st_out == HZ_OK && inf[r].volume_relres > o.refine_tol) st_out = HZ_ERR_NO_CONVERGENCE;
                }
            }
        }
    } catch (...) {
        throw;
    }
    int flags[4];
    d2h(c, flags, c.d_flag, sizeof(flags));
    if (flags[1]) {
        HZ_CUDA(cudaMemset(c.d_flag + 1, 0, sizeof(int)));
        throw Error{HZ_ERR_TIMEOUT, "a tensor-core substitution block gave up waiting on its MMAs"};
    }
    HZ_CUDA(cudaEventRecord(e1, c.stream));
    HZ_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto& x : inf) x.ms_total = ms;
    if (info) std::memcpy(info, inf.data(), R * sizeof(hz_solve_info));
}

hz_status fail(hz_handle* h, const Error& e) {
    if (h) h->ctx.last_error = e.msg;
    else g_create_error = e.msg;
    return e.st;
}

}  // namespace
}  // namespace hz

using namespace hz;

#define HZ_TRY(h, ...)                                                   \
    try {                                                                \
        __VA_ARGS__                                                      \
    } catch (const hz::Error& e) {                                       \
        return hz::fail(h, e);                                           \
    } catch (const std::bad_alloc&) {                                    \
        return hz::fail(h, hz::Error{HZ_ERR_OOM, "host allocation failed"}); \
    }

extern "C" {

void hz_default_opts(hz_precision prec, hz_solve_opts* o) {
    if (!o) return;
    o->gmres_tol = prec == HZ_PREC_FP64 ? 1e-10 : 1e-7;  // mixed modes: 1e-7
    o->restart = 12;
    o->max_iter = 100;
    o->refine_tol = 1e-9;
    o->max_refine = 3;
    o->krylov = 0;
}

hz_status hz_create(const hz_grid* grid, const double* m, double omega, const hz_pml* pml, int32_t n_layers,
                    hz_precision prec, void* stream, hz_handle** out) {
    return hz_create_ex(grid, m, nullptr, omega, pml, n_layers, prec, stream, out);
}

hz_status hz_create_ex(const hz_grid* grid, const double* m, const double* b, double omega, const hz_pml* pml,
                       int32_t n_layers, hz_precision prec, void* stream, hz_handle** out) {
    if (out) *out = nullptr;
    hz_handle* h = nullptr;
    try {
        if (!grid || !m || !pml || !out) throw Error{HZ_ERR_ARG, "null argument"};
        if (grid->nx < 3 || grid->ny < 3 || grid->nz < 3 || !(grid->h > 0)) throw Error{HZ_ERR_ARG, "grid"};
        if (!(omega > 0) || !std::isfinite(omega)) throw Error{HZ_ERR_ARG, "omega must be > 0"};
        if (pml->npml < 0 || !(pml->C >= 0)) throw Error{HZ_ERR_ARG, "pml"};
        if (prec != HZ_PREC_FP64 && prec != HZ_PREC_MIXED && prec != HZ_PREC_MIXED_FP64_FACTOR)
            throw Error{HZ_ERR_ARG, "precision"};
        const int nz = grid->nz;
        const int nphys = nz - 2 * pml->npml;
        if (n_layers < 1 || nphys < n_layers) throw Error{HZ_ERR_ARG, "n_layers out of range"};
        const long long N3 = (long long)grid->nx * grid->ny * grid->nz;
        // m and b may live in host or device (or managed) memory: device arrays are copied to the
        // host once here (the checks and the per-layer extensions below read them on the host)
        std::vector<double> m_copy, b_copy;
        auto to_host = [&](const double* p, std::vector<double>& buf) -> const double* {
            cudaPointerAttributes at{};
            const cudaError_t e = cudaPointerGetAttributes(&at, p);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return p;
            }
            if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return p;
            buf.resize((size_t)N3);
            HZ_CUDA(cudaMemcpy(buf.data(), p, (size_t)N3 * sizeof(double), cudaMemcpyDefault));
            return buf.data();
        };
        m = to_host(m, m_copy);
        if (b) b = to_host(b, b_copy);
        for (long long i = 0; i < N3; ++i)
            if (!std::isfinite(m[i])) throw Error{HZ_ERR_NONFINITE, "m has a non-finite entry"};
        if (b)
            for (long long i = 0; i < N3; ++i) {
                if (!std::isfinite(b[i])) throw Error{HZ_ERR_NONFINITE, "b has a non-finite entry"};
                if (!(b[i] > 0)) throw Error{HZ_ERR_ARG, "b = 1/rho must be positive"};
            }
        h = new hz_handle();
        Ctx& c = h->ctx;
        c.nx = grid->nx; c.ny = grid->ny; c.nz = grid->nz; c.h = grid->h;
        c.omega = omega; c.C = pml->C; c.npml = pml->npml;
        c.npml_loc = pml->npml_local < 0 ? pml->npml : pml->npml_local;
        c.L = n_layers; c.K = n_layers - 1; c.prec = prec;
        c.stream = (cudaStream_t)stream;
        c.P = (long long)c.nx * c.ny;
        c.ntr = 4LL * c.K * c.P;
        // global profiles: nodes and reciprocal at half nodes (index i <-> i - 1/2)
        auto prof = [&](int n, std::vector<double2>& sn, std::vector<double2>& ish) {
            sn.resize(n);
            ish.resize(n + 1);
            for (int i = 0; i < n; ++i) sn[i] = s_of(sigma_global(i, n, c.npml, c.C, c.h), omega);
            for (int i = 0; i <= n; ++i) ish[i] = inv_s(sigma_global(i - 0.5, n, c.npml, c.C, c.h), omega);
        };
        std::vector<double2> sxn, isxh, syn, isyh, szn, iszh;
        prof(c.nx, sxn, isxh);
        prof(c.ny, syn, isyh);
        prof(c.nz, szn, iszh);
        c.d_sx_n = dev_copy(sxn); c.d_isx_h = dev_copy(isxh);
        c.d_sy_n = dev_copy(syn); c.d_isy_h = dev_copy(isyh);
        c.d_sz_n = dev_copy(szn); c.d_isz_h = dev_copy(iszh);
        c.d_m = dev_copy(std::vector<double>(m, m + N3));
        if (b) c.d_b = dev_copy(std::vector<double>(b, b + N3));
        c.d_flag = (int*)dev_alloc(4 * sizeof(int));
        HZ_CUDA(cudaMemset(c.d_flag, 0, 4 * sizeof(int)));
        // layer partition: physical planes split evenly, earlier layers take the remainder;
        // layer 0 also owns the top PML planes, layer L-1 the bottom ones
        // nested-dissection leaf size (cells); HZ_LEAF overrides.  256-cell leaves give the
        // tensor-core kernel full 128-row work items at the bottom of the tree: measured at 128^3,
        // R = 128, 28.4 solves/s against 23.5 with 64-cell leaves (more leaf flops, at 5-7x the rate)
        int leaf = 256;
        if (const char* e = std::getenv("HZ_LEAF")) leaf = std::max(8, std::atoi(e));
        const int q = nphys / n_layers, rem = nphys % n_layers;
        int start = c.npml;
        std::vector<LayerCoef> coefs;
        std::map<int, int> shape_of_nz;
        for (int l = 0; l < n_layers; ++l) {
            Layer ly;
            int size = q + (l < rem ? 1 : 0);
            ly.lo = start;
            ly.hi = start + size - 1;
            start += size;
            if (l == 0) ly.lo = 0;
            if (l == n_layers - 1) ly.hi = nz - 1;
            ly.zlo = l > 0 ? ly.lo - c.npml_loc : ly.lo;
            ly.zhi = l < n_layers - 1 ? ly.hi + c.npml_loc : ly.hi;
            ly.nzl = ly.zhi - ly.zlo + 1;
            if (l > 0 && c.npml_loc < 1) throw Error{HZ_ERR_ARG, "npml_local must be >= 1 with several layers"};
            auto it = shape_of_nz.find(ly.nzl);
            if (it == shape_of_nz.end()) {
                Shape sh;
                build_shape(sh, c.nx, c.ny, ly.nzl, leaf);
                std::vector<NodeDev> nds;
                std::vector<long long> foff;
                std::vector<int> fm;
                for (auto& nd : sh.nodes) {
                    NodeDev d;
                    d.own0 = nd.own0; d.nown = nd.nown; d.nupd = nd.nupd; d.own_t = nd.own_t; d.upd_t = nd.upd_t;
                    d.pad_ = 0; d.upd_off = nd.upd_off; d.linv_off = nd.linv_off; d.l21_off = nd.l21_off;
                    nds.push_back(d);
                }
                sh.d_nodes = dev_copy(nds);
                sh.d_pos = dev_copy(sh.pos);
                sh.d_upd_idx = dev_copy(sh.upd_idx);
                sh.d_asm = dev_copy(sh.asm_entries);
                sh.d_emap = dev_copy(sh.emap);
                c.shapes.push_back(std::move(sh));
                it = shape_of_nz.emplace(ly.nzl, (int)c.shapes.size() - 1).first;
            }
            ly.shape = it->second;
            // local z profile and m (extended into the pads by copying the nearest owned plane)
            std::vector<double2> lzn(ly.nzl), lzh(ly.nzl + 1);
            for (int k = 0; k < ly.nzl; ++k)
                lzn[k] = s_of(sigma_local_z(ly.zlo + k, l, n_layers, ly.lo, ly.hi, nz, c.npml, c.npml_loc, c.C, c.h),
                              omega);
            for (int k = 0; k <= ly.nzl; ++k)
                lzh[k] = inv_s(sigma_local_z(ly.zlo + k - 0.5, l, n_layers, ly.lo, ly.hi, nz, c.npml, c.npml_loc,
                                             c.C, c.h), omega);
            std::vector<double> lm((size_t)ly.nzl * c.P);
            for (int k = 0; k < ly.nzl; ++k) {
                int zg = std::min(std::max(ly.zlo + k, ly.lo), ly.hi);
                std::memcpy(&lm[(size_t)k * c.P], m + (size_t)zg * c.P, c.P * sizeof(double));
            }
            ly.d_sz_n = dev_copy(lzn);
            ly.d_isz_h = dev_copy(lzh);
            ly.d_m = dev_copy(lm);
            if (b) {
                // b on the local grid: the owned planes and the plane beyond each internal interface
                // as they are globally (the owned rows' half-node couplings are then the global
                // ones), copied further into the pads
                std::vector<double> lb((size_t)ly.nzl * c.P);
                for (int k = 0; k < ly.nzl; ++k) {
                    int zg = std::min(std::max(ly.zlo + k, std::max(ly.lo - 1, 0)), std::min(ly.hi + 1, nz - 1));
                    std::memcpy(&lb[(size_t)k * c.P], b + (size_t)zg * c.P, c.P * sizeof(double));
                }
                ly.d_b = dev_copy(lb);
            }
            LayerCoef lc;
            lc.sx_n = c.d_sx_n; lc.isx_h = c.d_isx_h; lc.sy_n = c.d_sy_n; lc.isy_h = c.d_isy_h;
            lc.sz_n = ly.d_sz_n; lc.isz_h = ly.d_isz_h; lc.m = ly.d_m; lc.b = ly.d_b;
            lc.nx = c.nx; lc.ny = c.ny; lc.nzl = ly.nzl; lc.omega2 = omega * omega; lc.inv_h2 = 1.0 / (c.h * c.h);
            coefs.push_back(lc);
            c.layers.push_back(ly);
        }
        c.d_coefs = dev_copy(coefs);
        HZ_CUDA(cudaGetDevice(&c.device));
        if (const char* e = std::getenv("HZ_SUBST_TC")) c.tc_mode = std::max(0, std::min(2, std::atoi(e)));
        if (const char* e = std::getenv("HZ_TC_KS")) c.tc_ks = std::max(1, std::atoi(e));
        if (const char* e = std::getenv("HZ_AUTOTUNE")) c.autotune = std::atoi(e) != 0;
        if (const char* e = std::getenv("HZ_GRAPHS")) c.use_graphs = std::atoi(e) != 0;
        if (const char* e = std::getenv("HZ_TC_MIN_TILES")) c.tc_min_tiles = std::max(1, std::atoi(e));
        // HZ_PRECOND_SPLIT=1: single-term TF32 tensor-core products inside the preconditioner
        if (const char* e = std::getenv("HZ_PRECOND_SPLIT")) c.precond_split = std::atoi(e) == 1 ? 1 : 3;
        if (const char* e = std::getenv("HZ_TC_CFG")) c.tc_cfg = std::atoi(e) == 0 ? 0 : 1;
        if (const char* e = std::getenv("HZ_FACTOR_TC_MIN")) c.factor_tc_min_upd = std::max(0, std::atoi(e));
        if (const char* e = std::getenv("HZ_FACTOR_PROFILE")) c.factor_prof = std::atoi(e) != 0;
        if (const char* e = std::getenv("HZ_SPARSE")) c.sparse_subst = std::max(0, std::min(3, std::atoi(e)));
        if (const char* e = std::getenv("HZ_TC_WAIT_POLLS")) c.tc_wait_polls = std::max(1LL, std::atoll(e));
        HZ_CUDA(cudaDeviceSynchronize());  // uploads complete before any work on the stream
        *out = h;
        return HZ_OK;
    } catch (const Error& e) {
        if (h) hz_destroy(h);
        g_create_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        if (h) hz_destroy(h);
        g_create_error = "host allocation failed";
        return HZ_ERR_OOM;
    }
}

hz_status hz_factor(hz_handle* h) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (c.tb.base) {   // explicit trace blocks of the previous factors are stale
            c.tb.release();
            c.plans.clear();
            c.setup_plans.clear();
        }
        const size_t es = elem_size(c);
        for (auto& ly : c.layers) {
            if (!ly.d_fac) {
                const Shape& sh = c.shapes[ly.shape];
                ly.d_fac = dev_alloc((size_t)sh.factor_tiles * TILE2 * es);
                ly.d_dinv = dev_alloc((size_t)sh.N * es);
            }
        }
        HZ_CUDA(cudaMemset(c.d_flag, 0, 4 * sizeof(int)));
        cudaEvent_t e0, e1;
        HZ_CUDA(cudaEventCreate(&e0));
        HZ_CUDA(cudaEventCreate(&e1));
        HZ_CUDA(cudaEventRecord(e0, c.stream));
        if (c.prec == HZ_PREC_FP64) factor_layers<double2>(c);
        else if (c.prec == HZ_PREC_MIXED_FP64_FACTOR) factor_fp64_demote(c);
        else factor_layers<float2>(c);
        HZ_CUDA(cudaEventRecord(e1, c.stream));
        HZ_CUDA(cudaEventSynchronize(e1));
        HZ_CUDA(cudaEventElapsedTime(&c.factor_ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int flag[4];
        d2h(c, flag, c.d_flag, sizeof(flag));
        if (flag[1]) {
            HZ_CUDA(cudaMemset(c.d_flag + 1, 0, sizeof(int)));
            throw Error{HZ_ERR_TIMEOUT, "a tensor-core factorization block gave up waiting on its MMAs"};
        }
        if (flag[0]) throw Error{HZ_ERR_PIVOT, "tiny or non-finite pivot in the unpivoted LDL^T"};
        c.factored = true;
        return HZ_OK;
    })
}

hz_status hz_solve(hz_handle* h, const double* rhs, int32_t R, double* u, const hz_solve_opts* opts,
                   hz_solve_info* info) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        hz_solve_opts o;
        if (opts) o = *opts; else hz_default_opts(h->ctx.prec, &o);
        if (o.restart < 1 || o.max_iter < 1 || !(o.gmres_tol > 0) || (o.krylov != 0 && o.krylov != 1))
            throw Error{HZ_ERR_ARG, "solve options"};
        hz_status st = HZ_OK;
        do_solve(h->ctx, (const double2*)rhs, R, (double2*)u, o, info, st);
        if (st != HZ_OK) h->ctx.last_error = st == HZ_ERR_NONFINITE ? "non-finite result" : "did not converge";
        return st;
    })
}

hz_status hz_solve_host(hz_handle* h, const double* rhs_host, int32_t R, double* u_host, const hz_solve_opts* opts,
                        hz_solve_info* info) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (R < 1 || !rhs_host || !u_host) throw Error{HZ_ERR_ARG, "bad rhs/u/R"};
        const size_t bytes = (size_t)R * c.nx * c.ny * c.nz * sizeof(double2);
        // device copies of the two volumes, kept by the handle (grown as needed) so that a
        // repeated call neither allocates nor frees (cudaFree synchronises the device)
        if (c.stage_cap < R) {
            if (c.d_stage_rhs) cudaFree(c.d_stage_rhs);
            if (c.d_stage_u) cudaFree(c.d_stage_u);
            c.d_stage_rhs = c.d_stage_u = nullptr;
            c.stage_cap = 0;
            c.d_stage_rhs = (double2*)dev_alloc(bytes);
            c.d_stage_u = (double2*)dev_alloc(bytes);
            c.stage_cap = R;
        }
        HZ_CUDA(cudaMemcpyAsync(c.d_stage_rhs, rhs_host, bytes, cudaMemcpyHostToDevice, c.stream));
        const hz_status st = hz_solve(h, (const double*)c.d_stage_rhs, R, (double*)c.d_stage_u, opts, info);
        if (st == HZ_OK || st == HZ_ERR_NO_CONVERGENCE) {
            HZ_CUDA(cudaMemcpyAsync(u_host, c.d_stage_u, bytes, cudaMemcpyDeviceToHost, c.stream));
            HZ_CUDA(cudaStreamSynchronize(c.stream));
        }
        return st;
    })
}

hz_status hz_destroy(hz_handle* h) {
    if (!h) return HZ_OK;
    Ctx& c = h->ctx;
    if (c.stream) cudaStreamSynchronize(c.stream);
    else cudaDeviceSynchronize();
    release_slots(c);
    c.gw.release();
    c.tb.release();
    cudaFree(c.d_flag);
    if (c.d_io) cudaFree(c.d_io);
    if (c.h_io) cudaFreeHost(c.h_io);
    if (c.d_norms) cudaFree(c.d_norms);
    if (c.d_vol_res) cudaFree(c.d_vol_res);
    if (c.d_vol_du) cudaFree(c.d_vol_du);
    if (c.d_stage_rhs) cudaFree(c.d_stage_rhs);
    if (c.d_stage_u) cudaFree(c.d_stage_u);
    if (c.owns_shared) {
        for (auto& sh : c.shapes) {
            cudaFree(sh.d_nodes); cudaFree(sh.d_pos); cudaFree(sh.d_upd_idx); cudaFree(sh.d_asm); cudaFree(sh.d_emap);
        }
        for (auto& ly : c.layers) {
            cudaFree(ly.d_sz_n); cudaFree(ly.d_isz_h); cudaFree(ly.d_m); cudaFree(ly.d_b); cudaFree(ly.d_fac);
            cudaFree(ly.d_dinv);
        }
        cudaFree(c.d_coefs);
        cudaFree(c.d_sx_n); cudaFree(c.d_isx_h); cudaFree(c.d_sy_n); cudaFree(c.d_isy_h);
        cudaFree(c.d_sz_n); cudaFree(c.d_isz_h); cudaFree(c.d_m); cudaFree(c.d_b);
    }
    delete h;
    return HZ_OK;
}

hz_status hz_create_shared(hz_handle* src, void* stream, hz_handle** out) {
    if (out) *out = nullptr;
    if (!src || !out) return HZ_ERR_ARG;
    if (!src->ctx.factored) {
        src->ctx.last_error = "hz_create_shared: the source handle is not factored";
        return HZ_ERR_STATE;
    }
    hz_handle* h = nullptr;
    try {
        h = new hz_handle();
        Ctx& c = h->ctx;
        const Ctx& s = src->ctx;
        c.nx = s.nx; c.ny = s.ny; c.nz = s.nz; c.h = s.h; c.omega = s.omega; c.C = s.C;
        c.npml = s.npml; c.npml_loc = s.npml_loc; c.L = s.L; c.K = s.K; c.prec = s.prec;
        c.P = s.P; c.ntr = s.ntr; c.device = s.device;
        c.shapes = s.shapes;    // host copies; device arrays borrowed
        c.layers = s.layers;    // factors borrowed
        c.d_coefs = s.d_coefs;
        c.d_sx_n = s.d_sx_n; c.d_isx_h = s.d_isx_h; c.d_sy_n = s.d_sy_n; c.d_isy_h = s.d_isy_h;
        c.d_sz_n = s.d_sz_n; c.d_isz_h = s.d_isz_h; c.d_m = s.d_m; c.d_b = s.d_b;
        c.tc_mode = s.tc_mode; c.tc_ks = s.tc_ks; c.tc_min_tiles = s.tc_min_tiles; c.precond_split = s.precond_split; c.tc_cfg = s.tc_cfg;
        c.sparse_subst = s.sparse_subst;
        c.tc_wait_polls = s.tc_wait_polls;
        c.autotune = s.autotune; c.use_graphs = s.use_graphs;
        c.tuned = s.tuned;
        c.factored = true;
        c.owns_shared = false;
        c.stream = (cudaStream_t)stream;
        c.d_flag = (int*)dev_alloc(4 * sizeof(int));
        HZ_CUDA(cudaMemset(c.d_flag, 0, 4 * sizeof(int)));
        HZ_CUDA(cudaDeviceSynchronize());
        *out = h;
        return HZ_OK;
    } catch (const Error& e) {
        if (h) { h->ctx.owns_shared = false; hz_destroy(h); }
        src->ctx.last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        if (h) { h->ctx.owns_shared = false; hz_destroy(h); }
        return HZ_ERR_OOM;
    }
}

hz_status hz_trace_blocks(hz_handle* h, int32_t max_cols, int64_t* bytes) {
    if (bytes) *bytes = 0;
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (max_cols < 0) throw Error{HZ_ERR_ARG, "hz_trace_blocks: max_cols must be >= 0"};
        if (max_cols > 0 && !c.factored) throw Error{HZ_ERR_STATE, "hz_trace_blocks before hz_factor"};
        HZ_CUDA(cudaStreamSynchronize(c.stream));
        c.plans.clear();        // recorded M_pol / P applications follow the new setting
        c.setup_plans.clear();
        if (max_cols == 0) {
            c.tb.release();
            return HZ_OK;
        }
        if (c.L >= 2 && !c.tb.base) {
            const bool dbl = c.prec == HZ_PREC_FP64;
            const int n2 = (int)(2 * c.P);
            const int chunk = std::min(256, (n2 + 63) / 64 * 64);
            ensure_slots(c, padded_ldc(dbl, 2 * chunk), padded_ldc(dbl, 2 * chunk));
            if (dbl) build_trace_blocks<double2>(c, chunk);
            else build_trace_blocks<float2>(c, chunk);
        }
        c.tb.max_cols = max_cols;
        if (bytes) *bytes = c.tb.bytes;
        return HZ_OK;
    })
}

hz_status hz_symbolic_shape(int32_t nx, int32_t ny, int32_t nz, int32_t leaf, int64_t* n_nodes, int64_t* n_upd,
                            int32_t* perm, int32_t* own0, int32_t* nown, int32_t* parent, int64_t* upd_off,
                            int32_t* upd_idx) {
    try {
        if (nx < 1 || ny < 1 || nz < 1 || leaf < 1 || (long long)nx * ny * nz > (1LL << 30))
            throw Error{HZ_ERR_ARG, "hz_symbolic_shape: box sizes or leaf out of range"};
        Shape sh;
        build_shape(sh, nx, ny, nz, leaf);
        if (n_nodes) *n_nodes = (int64_t)sh.nodes.size();
        if (n_upd) *n_upd = (int64_t)sh.upd_idx.size();
        if (perm) std::memcpy(perm, sh.perm.data(), sh.perm.size() * sizeof(int32_t));
        for (size_t i = 0; i < sh.nodes.size(); ++i) {
            const Node& nd = sh.nodes[i];
            if (own0) own0[i] = nd.own0;
            if (nown) nown[i] = nd.nown;
            if (parent) parent[i] = nd.parent;
            if (upd_off) upd_off[i] = nd.upd_off;
        }
        if (upd_idx) std::memcpy(upd_idx, sh.upd_idx.data(), sh.upd_idx.size() * sizeof(int32_t));
        return HZ_OK;
    } catch (const Error& e) {
        g_create_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        g_create_error = "host allocation failed";
        return HZ_ERR_OOM;
    }
}

const char* hz_last_error(const hz_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->ctx.last_error.c_str();
}

hz_status hz_layer_info(const hz_handle* h, int32_t ell, int32_t* lo, int32_t* hi, int32_t* zlo, int32_t* zhi) {
    if (!h || ell < 0 || ell >= h->ctx.L) return HZ_ERR_ARG;
    const Layer& ly = h->ctx.layers[ell];
    if (lo) *lo = ly.lo;
    if (hi) *hi = ly.hi;
    if (zlo) *zlo = ly.zlo;
    if (zhi) *zhi = ly.zhi;
    return HZ_OK;
}

hz_status hz_factor_stats(const hz_handle* h, int64_t* nodes, int64_t* factor_entries, double* factor_flops,
                          int64_t* workspace_bytes, float* factor_ms) {
    if (!h) return HZ_ERR_ARG;
    const Ctx& c = h->ctx;
    long long nn = 0, fe = 0;
    double ff = 0;
    for (auto& ly : c.layers) {
        const Shape& sh = c.shapes[ly.shape];
        nn += (long long)sh.nodes.size();
        fe += sh.factor_tiles * TILE2;
        ff += sh.factor_flops;
    }
    if (nodes) *nodes = nn;
    if (factor_entries) *factor_entries = fe;
    if (factor_flops) *factor_flops = ff;
    if (workspace_bytes) *workspace_bytes = c.workspace_bytes;
    if (factor_ms) *factor_ms = c.factor_ms;
    return HZ_OK;
}

hz_status hz_layer_solve_cost(const hz_handle* h, int32_t ell, double* bytes, double* flops_per_col) {
    if (!h || ell < 0 || ell >= h->ctx.L) return HZ_ERR_ARG;
    const Ctx& c = h->ctx;
    const Shape& sh = c.shapes[c.layers[ell].shape];
    double entries = 0;
    for (auto& nd : sh.nodes) entries += (double)nd.nown * (nd.nown + 1) / 2.0 + (double)nd.nown * nd.nupd;
    if (bytes) *bytes = 2.0 * entries * (double)elem_size(c);
    if (flops_per_col) *flops_per_col = sh.solve_flops_per_col;
    return HZ_OK;
}

hz_status hz_layer_solve(hz_handle* h, int32_t ell, const double* g, int32_t ncols, double* w) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (!c.factored) throw Error{HZ_ERR_STATE, "not factored"};
        if (ell < 0 || ell >= c.L || ncols < 1 || !g || !w) throw Error{HZ_ERR_ARG, "layer solve args"};
        const bool dbl = c.prec == HZ_PREC_FP64;
        ensure_slots(c, padded_ldc(dbl, ncols), padded_ldc(dbl, ncols));
        if (dbl) op_layer_solve<double2>(c, ell, (const double2*)g, ncols, (double2*)w);
        else op_layer_solve<float2>(c, ell, (const double2*)g, ncols, (double2*)w);
        HZ_CUDA(cudaStreamSynchronize(c.stream));
        return HZ_OK;
    })
}

hz_status hz_polarized_rhs(hz_handle* h, const double* rhs, int32_t R, double* fpol) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (!c.factored) throw Error{HZ_ERR_STATE, "not factored"};
        if (R < 1 || !rhs || !fpol || c.K < 1) throw Error{HZ_ERR_ARG, "polarized rhs args"};
        prepare_for(c, R);
        if (c.prec == HZ_PREC_FP64) op_polarized_rhs<double2>(c, (const double2*)rhs, true, R, (double2*)fpol);
        else op_polarized_rhs<float2>(c, (const double2*)rhs, true, R, (double2*)fpol);
        HZ_CUDA(cudaStreamSynchronize(c.stream));
        return HZ_OK;
    })
}

hz_status hz_apply_mpol(hz_handle* h, const double* x, int32_t R, double* y) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (!c.factored) throw Error{HZ_ERR_STATE, "not factored"};
        if (R < 1 || !x || !y || c.K < 1) throw Error{HZ_ERR_ARG, "mpol args"};
        prepare_for(c, R);
        if (c.prec == HZ_PREC_FP64) op_apply_mpol<double2>(c, (const double2*)x, R, (double2*)y);
        else op_apply_mpol<float2>(c, (const double2*)x, R, (double2*)y);
        HZ_CUDA(cudaStreamSynchronize(c.stream));
        return HZ_OK;
    })
}

hz_status hz_apply_precond(hz_handle* h, const double* x, int32_t R, double* y) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (!c.factored) throw Error{HZ_ERR_STATE, "not factored"};
        if (R < 1 || !x || !y || c.K < 1) throw Error{HZ_ERR_ARG, "precond args"};
        prepare_for(c, R);
        double2* tmp = (double2*)dev_alloc((size_t)R * c.ntr * sizeof(double2));
        try {
            if (c.prec == HZ_PREC_FP64) op_apply_precond<double2>(c, (const double2*)x, R, (double2*)y, tmp);
            else op_apply_precond<float2>(c, (const double2*)x, R, (double2*)y, tmp);
            HZ_CUDA(cudaStreamSynchronize(c.stream));
        } catch (...) {
            cudaFree(tmp);
            throw;
        }
        cudaFree(tmp);
        return HZ_OK;
    })
}

hz_status hz_reconstruct(hz_handle* h, const double* rhs, const double* t, int32_t R, double* u) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (!c.factored) throw Error{HZ_ERR_STATE, "not factored"};
        if (R < 1 || !rhs || !u || (c.K > 0 && !t)) throw Error{HZ_ERR_ARG, "reconstruct args"};
        prepare_for(c, R);
        if (c.prec == HZ_PREC_FP64)
            op_reconstruct<double2>(c, (const double2*)rhs, true, (const double2*)t, R, (double2*)u, false);
        else
            op_reconstruct<float2>(c, (const double2*)rhs, true, (const double2*)t, R, (double2*)u, false);
        HZ_CUDA(cudaStreamSynchronize(c.stream));
        return HZ_OK;
    })
}

hz_status hz_volume_residual(hz_handle* h, const double* rhs, const double* u, int32_t R, double* r,
                             double* relres_host) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        if (R < 1 || !rhs || !u) throw Error{HZ_ERR_ARG, "residual args"};
        double* norms = (double*)dev_alloc(2 * R * sizeof(double));
        std::vector<double> hn(2 * R);
        try {
            op_volume_residual(c, (const double2*)rhs, true, (const double2*)u, R, (double2*)r, norms);
            d2h(c, hn.data(), norms, 2 * R * sizeof(double));
        } catch (...) {
            cudaFree(norms);
            throw;
        }
        cudaFree(norms);
        if (relres_host)
            for (int q = 0; q < R; ++q) relres_host[q] = hn[2 * q + 1] > 0 ? std::sqrt(hn[2 * q] / hn[2 * q + 1]) : 0.0;
        return HZ_OK;
    })
}

static hz_status profile_begin(hz_handle* h, bool detail) {
    if (!h) return HZ_ERR_ARG;
    Ctx& c = h->ctx;
    for (auto* v : {&c.prof_recs, &c.prof_launch}) {
        for (auto& r : *v) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        v->clear();
    }
    for (auto& k : c.kern_stat) k = KernStat{};
    c.kern_lvl.clear();
    c.prof = true;
    c.prof_detail = detail;
    return HZ_OK;
}

hz_status hz_profile_begin(hz_handle* h) { return profile_begin(h, false); }
hz_status hz_profile_begin_detail(hz_handle* h) { return profile_begin(h, true); }

hz_status hz_profile_end(hz_handle* h, int64_t* calls, double* total_ms, double* alg_bytes, double* alg_flops) {
    if (!h) return HZ_ERR_ARG;
    HZ_TRY(h, {
        Ctx& c = h->ctx;
        c.prof = false;
        c.prof_detail = false;
        HZ_CUDA(cudaStreamSynchronize(c.stream));
        double ms = 0, by = 0, fl = 0;
        for (auto& r : c.prof_recs) {
            float t = 0.f;
            HZ_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
            ms += t;
            by += r.bytes;
            fl += r.flops;
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
        for (auto& r : c.prof_launch) {
            float t = 0.f;
            HZ_CUDA(cudaEventElapsedTime(&t, r.e0, r.e1));
            KernStat& k = c.kern_stat[r.kind];
            k.launches += 1;
            k.ms += t;
            k.bytes += r.bytes;
            k.flops += r.flops;
            KernStat& kl = c.kern_lvl[std::make_tuple(r.kind, r.mode, r.level)];
            kl.launches += 1;
            kl.ms += t;
            kl.bytes += r.bytes;
            kl.flops += r.flops;
            kl.tasks += r.tasks;
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
        if (calls) *calls = (int64_t)c.prof_recs.size();
        c.prof_recs.clear();
        c.prof_launch.clear();
        if (total_ms) *total_ms = ms;
        if (alg_bytes) *alg_bytes = by;
        if (alg_flops) *alg_flops = fl;
        return HZ_OK;
    })
}

hz_status hz_profile_kernel(hz_handle* h, int32_t kind, int64_t* launches, double* total_ms, double* alg_bytes,
                            double* alg_flops) {
    if (!h) return HZ_ERR_ARG;
    if (kind < 0 || kind > 2) {
        h->ctx.last_error = "hz_profile_kernel: kind must be 0 (CUDA-core), 1 (tensor-core) or 2 (trace-block)";
        return HZ_ERR_ARG;
    }
    const KernStat& k = h->ctx.kern_stat[kind];
    if (launches) *launches = k.launches;
    if (total_ms) *total_ms = k.ms;
    if (alg_bytes) *alg_bytes = k.bytes;
    if (alg_flops) *alg_flops = k.flops;
    return HZ_OK;
}

int64_t hz_kernel_launches(void) { return (int64_t)hz::g_launch_count.load(); }

hz_status hz_solve_group(hz_handle* const* hs, int32_t n, const double* const* rhs, const int32_t* R,
                         double* const* u, const hz_solve_opts* opts, hz_solve_info* const* info,
                         hz_status* statuses) {
    if (!hs || n < 1 || !rhs || !R || !u) return HZ_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return HZ_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (hs[i] == hs[j]) return HZ_ERR_ARG;  // a handle is not shared between threads
    }
    std::vector<hz_status> st(n, HZ_OK);
    std::vector<std::thread> th;
    th.reserve(n);
    for (int i = 0; i < n; ++i) {
        th.emplace_back([&, i]() {
            if (cudaSetDevice(hs[i]->ctx.device) != cudaSuccess) {
                cudaGetLastError();
                st[i] = HZ_ERR_CUDA;
                return;
            }
            st[i] = hz_solve(hs[i], rhs[i], R[i], u[i], opts, info ? info[i] : nullptr);
        });
    }
    for (auto& t : th) t.join();
    hz_status worst = HZ_OK;
    for (int i = 0; i < n; ++i) {
        if (statuses) statuses[i] = st[i];
        if (worst == HZ_OK && st[i] != HZ_OK) worst = st[i];
    }
    return worst;
}

const char* hz_factor_report(hz_handle* h) {
    if (!h) return "";
    return h->ctx.factor_text.c_str();
}

const char* hz_profile_report(hz_handle* h) {
    if (!h) return "";
    Ctx& c = h->ctx;
    static const char* kinds[3] = {"cuda-core", "tensor-core", "trace-block"};
    static const char* modes[4] = {"FA", "FB", "BA", "BB"};
    c.prof_text = "kind phase level launches tasks ms alg_TFLOP/s\n";
    for (auto& kv : c.kern_lvl) {
        const KernStat& k = kv.second;
        char line[160];
        std::snprintf(line, sizeof line, "%s %s %d %lld %lld %.3f %.2f\n", kinds[std::get<0>(kv.first)],
                      modes[std::get<1>(kv.first)], std::get<2>(kv.first), k.launches, k.tasks, k.ms,
                      k.ms > 0 ? k.flops / (k.ms * 1e-3) / 1e12 : 0.0);
        c.prof_text += line;
    }
    return c.prof_text.c_str();
}

const char* hz_tuning_report(hz_handle* h) {
    if (!h) return "";
    h->ctx.last_error.clear();
    for (auto& s : h->ctx.tune_log) h->ctx.last_error += s + "\n";
    return h->ctx.last_error.c_str();
}

}  // extern "C"
