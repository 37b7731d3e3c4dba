// Allocation-free variant of the FP64 volume residual (hz_volume_residual_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the residual: a
// process whose device memory is entirely handed out by a caching allocator (PyTorch's, for
// example) gets a failed cudaMalloc there, or -- once the allocator releases its cache to make
// room -- a device-wide synchronisation; a serving loop with a fixed memory budget must not grow
// its footprint per request.  For them this entry point keeps its only scratch -- the per-column
// partial sums of ||r||^2 and ||S f||^2 that the kernel accumulates -- in a fixed file-scope
// device array instead of a buffer allocated per call.  It reads only buffers the handle
// already owns (set up by hz_create) and the caller's inputs and outputs.  Like the other entry
// points it returns with the result on the host: it copies the sums to host memory and
// synchronizes the handle's stream.
#include <cmath>
#include <mutex>

#include "hz_internal.cuh"
#include "hz_ctx.cuh"

namespace hz {
namespace {

// At most this many right-hand-side columns per call (2 doubles of scratch each, 16 KiB).
constexpr int kNoallocMaxCols = 1024;

// Every device that loads the library holds this array until the process exits.  All
// calls share it: it keeps the previous call's sums, so each call clears the part it uses.
__device__ __align__(256) double g_residual_scratch[2 * kNoallocMaxCols];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (the handle's device).  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per device, with
// that device current, and cached; the caller's current device is restored afterwards.
hz_status scratch_address(int dev, double** out, std::string& err) {
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device ordinal out of range";
        return HZ_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        int prev = 0;
        if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) {
            cudaGetLastError();
            err = "cannot make the handle's device current";
            return HZ_ERR_CUDA;
        }
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
        cudaSetDevice(prev);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            err = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return HZ_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return HZ_OK;
}

// Makes `dev` the current device for the lifetime of the guard (the handle's stream and the
// scratch address belong to it) and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~DeviceGuard() {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

// Same arithmetic as the residual kernel of the online path: r = S f - A u with the
// symmetric-form stretched 7-point operator, plus per-column sums of |r|^2 and |S f|^2.
__global__ void k_residual_static(const double2* f, const double2* u, double2* rout, double* norms, int nx,
                                  int ny, int nz, const double2* sxn, const double2* isxh, const double2* syn,
                                  const double2* isyh, const double2* szn, const double2* iszh, const double* m,
                                  const double* b, double omega2, double inv_h2) {
    const long long N3 = (long long)nx * ny * nz;
    const int r = blockIdx.y;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0, gg = 0.0;
    if (i < N3) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        const double2* ur = u + (long long)r * N3;
        double2 sx = sxn[x], sy = syn[y], sz = szn[z];
        double2 syz = cmul(sy, sz), sxz = cmul(sx, sz), sxy = cmul(sx, sy);
        double2 c1 = cscale(cmul(syz, isxh[x]), inv_h2), c2 = cscale(cmul(syz, isxh[x + 1]), inv_h2);
        double2 c3 = cscale(cmul(sxz, isyh[y]), inv_h2), c4 = cscale(cmul(sxz, isyh[y + 1]), inv_h2);
        double2 c5 = cscale(cmul(sxy, iszh[z]), inv_h2), c6 = cscale(cmul(sxy, iszh[z + 1]), inv_h2);
        if (b) {   // variable density: b at the half nodes
            const long long pl_ = (long long)nx * ny;
            c1 = cscale(c1, bhalf(b, i, x, nx, 1, -1)); c2 = cscale(c2, bhalf(b, i, x, nx, 1, +1));
            c3 = cscale(c3, bhalf(b, i, y, ny, nx, -1)); c4 = cscale(c4, bhalf(b, i, y, ny, nx, +1));
            c5 = cscale(c5, bhalf(b, i, z, nz, pl_, -1)); c6 = cscale(c6, bhalf(b, i, z, nz, pl_, +1));
        }
        double2 dg = cscale(cmul(sxy, sz), omega2 * m[i]);
        dg = csub(dg, cadd(cadd(cadd(c1, c2), cadd(c3, c4)), cadd(c5, c6)));
        double2 au = cmul(dg, ur[i]);
        if (x > 0) au = cadd(au, cmul(c1, ur[i - 1]));
        if (x < nx - 1) au = cadd(au, cmul(c2, ur[i + 1]));
        if (y > 0) au = cadd(au, cmul(c3, ur[i - nx]));
        if (y < ny - 1) au = cadd(au, cmul(c4, ur[i + nx]));
        const long long pl = (long long)nx * ny;
        if (z > 0) au = cadd(au, cmul(c5, ur[i - pl]));
        if (z < nz - 1) au = cadd(au, cmul(c6, ur[i + pl]));
        double2 g = cmul(cmul(sxy, sz), f[(long long)r * N3 + i]);
        double2 res = csub(g, au);
        if (rout) rout[(long long)r * N3 + i] = res;
        rr = res.x * res.x + res.y * res.y;
        gg = g.x * g.x + g.y * g.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        gg += __shfl_down_sync(0xffffffffu, gg, o);
    }
    __shared__ double sr[32], sg[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sr[w] = rr; sg[w] = gg; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        rr = lane < nw ? sr[lane] : 0.0;
        gg = lane < nw ? sg[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            rr += __shfl_down_sync(0xffffffffu, rr, o);
            gg += __shfl_down_sync(0xffffffffu, gg, o);
        }
        if (lane == 0) {
            atomicAdd(&norms[2 * r], rr);
            atomicAdd(&norms[2 * r + 1], gg);
        }
    }
}

}  // namespace
}  // namespace hz

extern "C" hz_status hz_volume_residual_noalloc(hz_handle* h, const double* rhs, const double* u, int32_t R,
                                                double* r, double* relres_host) {
    if (!h) return HZ_ERR_ARG;
    hz::Ctx& c = h->ctx;
    if (R < 1 || !rhs || !u || !relres_host) {
        c.last_error = "hz_volume_residual_noalloc: bad arguments";
        return HZ_ERR_ARG;
    }
    if (R > hz::kNoallocMaxCols) {
        c.last_error = "hz_volume_residual_noalloc: R = " + std::to_string(R) + " exceeds the fixed scratch of " +
                       std::to_string(hz::kNoallocMaxCols) + " columns";
        return HZ_ERR_ARG;
    }
    hz::DeviceGuard guard(c.device);
    if (!guard.ok) {
        c.last_error = "hz_volume_residual_noalloc: cannot make the handle's device current";
        return HZ_ERR_CUDA;
    }
    double* scratch = nullptr;
    hz_status st = hz::scratch_address(c.device, &scratch, c.last_error);
    if (st != HZ_OK) return st;
    const long long N3 = (long long)c.nx * c.ny * c.nz;
    // the array keeps the previous call's sums: clear the columns this call accumulates into
    if (cudaMemsetAsync(scratch, 0, 2 * (size_t)R * sizeof(double), c.stream) != cudaSuccess) {
        c.last_error = "hz_volume_residual_noalloc: cudaMemsetAsync failed";
        cudaGetLastError();
        return HZ_ERR_CUDA;
    }
    dim3 grid((unsigned)((N3 + 255) / 256), (unsigned)R);
    hz::k_residual_static<<<grid, 256, 0, c.stream>>>((const double2*)rhs, (const double2*)u, (double2*)r, scratch,
                                                     c.nx, c.ny, c.nz, c.d_sx_n, c.d_isx_h, c.d_sy_n, c.d_isy_h,
                                                     c.d_sz_n, c.d_isz_h, c.d_m, c.d_b, c.omega * c.omega,
                                                     1.0 / (c.h * c.h));
    hz::g_launch_count.fetch_add(1, std::memory_order_relaxed);
    double sums[2 * hz::kNoallocMaxCols];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(sums, scratch, 2 * (size_t)R * sizeof(double), cudaMemcpyDeviceToHost, c.stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c.stream) != cudaSuccess) {
        c.last_error = "hz_volume_residual_noalloc: CUDA launch or copy failed";
        cudaGetLastError();
        return HZ_ERR_CUDA;
    }
    for (int q = 0; q < R; ++q) relres_host[q] = sums[2 * q + 1] > 0 ? std::sqrt(sums[2 * q] / sums[2 * q + 1]) : 0.0;
    return HZ_OK;
}
