// Solver context shared by the translation units (the object behind hz_handle).
#pragma once

#include <array>
#include <functional>
#include <map>
#include <tuple>
#include <memory>
#include <string>
#include <vector>

#include "hz_internal.cuh"

namespace hz {

__device__ __host__ inline int cdiv_dev(int a, int b) { return (a + b - 1) / b; }

// FP64 inputs of the stencil coefficients of one layer's local operator.
struct LayerCoef {
    const double2* sx_n;   // s_x at nodes (nx)
    const double2* isx_h;  // 1/s_x at half nodes (nx+1), index i <-> i - 1/2
    const double2* sy_n;
    const double2* isy_h;
    const double2* sz_n;   // local z profile (nzl)
    const double2* isz_h;  // (nzl+1)
    const double* m;       // local m (nzl*ny*nx)
    const double* b;       // local b = 1/rho (nzl*ny*nx) or nullptr (constant density)
    int nx, ny, nzl;
    double omega2, inv_h2;
};

// A set of layers solved together (one job per layer) with its per-level task lists.
struct Batch {
    std::vector<int> layers;
    int H = 0;
    int KS = 1 << 30;                           // max reduction tiles per task (split-K)
    int CC = 0;                                 // right-hand-side columns per block (0: default)
    bool tc = false;                            // holds tensor-core task lists (large nodes)
    std::vector<long long> off[4], cnt[4];      // per phase (FA, FB, BA, BB) and level, into d_tasks
    int KS_tc = 1 << 30;                        // split-K of the tensor-core tasks (tiles)
    int min_t = 8;                              // output tiles a node product needs for the tensor cores
    int split = 3;                              // TF32 terms per real product on the tensor cores (3 or 1)
    int tc_cfg = 0;                             // tensor-core kernel: 0 one block per work item, 1 persistent
    int sparse = 0;                             // products skipped away from the interface planes (get_batch)
    int job_cols = 0;                           // columns per job when per-block sparsity splits each
                                                // layer's columns into jobs (0: one job per layer, ldc wide)
    long long wait_polls = 1LL << 26;           // poll limit of the tensor-core kernels' pipeline waits
    std::vector<long long> pair_off[4], pair_cnt[4];  // tensor-core tasks: two output tiles each
    Task* d_tasks = nullptr;
    void* d_jobs = nullptr;                     // JobDev<C>[njobs]
    std::vector<std::pair<void*, void*>> vec_ptrs;  // (acc, x) of each job
    std::vector<long long> vec_rows;
    double alg_bytes = 0;       // factor bytes one forward+backward substitution streams (all jobs)
    double flops_per_col = 0;   // real flops per right-hand-side column (all jobs)
    // algorithmic factor bytes and real flops per column of each launch, by kernel kind
    // (0 CUDA-core, 1 tensor-core), phase and level
    std::vector<double> lvl_bytes[2][4], lvl_flops[2][4];
};

// Event-timed record of a substitution call (hz_profile_begin) or, in detail mode, of one
// kernel launch of it (kind 0 CUDA-core, 1 tensor-core).
struct ProfRec { cudaEvent_t e0, e1; double bytes, flops; int kind, mode, level; long long tasks; };
struct KernStat { long long launches = 0, tasks = 0; double ms = 0, bytes = 0, flops = 0; };

// Recorded sequence of stream operations with the device descriptors it owns.  run() issues
// the operations on a stream; run_graph() captures them once into a CUDA graph and replays it.
struct Rec {
    std::vector<std::function<void(cudaStream_t)>> ops;
    std::vector<void*> owned;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t upload_stream = 0;
    long long graph_kernels = 0;   // kernels in the captured graph (counted again at every replay)
    Rec() = default;
    Rec(const Rec&) = delete;
    Rec& operator=(const Rec&) = delete;
    ~Rec() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void* p : owned) cudaFree(p);
    }
    template <class T> T* up(const std::vector<T>& v) {
        T* d = nullptr;
        if (cudaMalloc((void**)&d, std::max<size_t>(1, v.size()) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            throw Error{HZ_ERR_OOM, "descriptor upload"};
        }
        owned.push_back(d);
        if (!v.empty()) {
            HZ_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, upload_stream));
            HZ_CUDA(cudaStreamSynchronize(upload_stream));
        }
        return d;
    }
    void add(std::function<void(cudaStream_t)> f) { ops.push_back(std::move(f)); }
    void run(cudaStream_t st) { for (auto& f : ops) f(st); }
    void run_graph(cudaStream_t st) {
        if (!exec) {
            // capture on a private stream (the legacy default stream cannot be captured); the
            // instantiated graph is then launched on the caller's stream
            cudaStream_t cs = nullptr;
            HZ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaStreamDestroy(cs);
                throw Error{HZ_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e)};
            }
            const long long k0 = g_launch_count.load();
            try {
                run(cs);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(cs, &g);
                if (g) cudaGraphDestroy(g);
                cudaStreamDestroy(cs);
                cudaGetLastError();
                throw;
            }
            e = cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) throw Error{HZ_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e)};
            HZ_CUDA(cudaGraphInstantiate(&exec, graph, 0));
            // the capture counted the kernels once (as launched by this first replay)
            graph_kernels = g_launch_count.load() - k0;
        } else {
            g_launch_count.fetch_add(graph_kernels, std::memory_order_relaxed);
        }
        HZ_CUDA(cudaGraphLaunch(exec, st));
    }
};

// Persistent GMRES workspace of a handle (sized for up to cap_R columns).
struct GmresWork {
    int cap_R = 0, m = 0;
    std::vector<void*> bufs;
    double2 *V = nullptr, *in = nullptr, *out = nullptr, *w2 = nullptr, *tmp = nullptr, *b = nullptr, *xs = nullptr;
    double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *dots = nullptr, *y = nullptr, *t = nullptr;
    double *nrm = nullptr, *invb = nullptr, *resid = nullptr, *b0 = nullptr;
    int *active = nullptr, *kused = nullptr;
    void release() {
        for (void* p : bufs) cudaFree(p);
        bufs.clear();
        cap_R = 0;
        m = 0;
    }
};

// Explicit trace-to-trace Green's blocks of the layers (hz_trace_blocks): per layer up to four
// dense 2P x 2P blocks E_rs, r the read-out pair and s the source pair (0 top, 1 bottom), stored
// column-major (a unit source trace's 2P read-outs contiguous) in the complex type of the
// handle's local solves.
struct TraceBlocks {
    void* base = nullptr;
    size_t elem = 0;                             // sizeof the complex type of the blocks
    long long bytes = 0;
    std::vector<std::array<long long, 4>> off;   // per layer: element offset of E_rs at [2 r + s], -1 absent
    int max_cols = 0;                            // M_pol and P use the blocks for at most this many columns
    void release() {
        if (base) cudaFree(base);
        base = nullptr;
        elem = 0;
        bytes = 0;
        off.clear();
        max_cols = 0;
    }
};

struct Ctx {
    // problem
    int nx = 0, ny = 0, nz = 0;
    double h = 1.0, omega = 0.0, C = 0.0;
    int npml = 0, npml_loc = 0, L = 1, K = 0;
    hz_precision prec = HZ_PREC_FP64;
    cudaStream_t stream = 0;
    int device = 0;
    long long P = 0;     // plane size nx*ny
    long long ntr = 0;   // polarized trace vector length per RHS: 2*K*2*P
    // decomposition and symbolic data
    std::vector<Shape> shapes;
    std::vector<Layer> layers;
    LayerCoef* d_coefs = nullptr;
    // global FP64 profiles and medium (volume residual, source scaling, interface weights)
    double2 *d_sx_n = nullptr, *d_isx_h = nullptr, *d_sy_n = nullptr, *d_isy_h = nullptr;
    double2 *d_sz_n = nullptr, *d_isz_h = nullptr;
    double* d_m = nullptr;
    double* d_b = nullptr;   // b = 1/rho on the global grid, nullptr for constant density
    int* d_flag = nullptr;   // device error flags: [0] tiny pivot
    bool factored = false;
    bool owns_shared = true;  // false for handles that borrow another handle's factors (hz_create_shared)
    long long workspace_bytes = 0;
    float factor_ms = 0.f;
    // solve workspaces
    int slot_cap = 0;        // columns per layer slot
    std::vector<void*> slot_acc, slot_x;   // per layer, N_layer * slot_cap complex
    std::map<std::string, Batch> batches;
    std::string last_error;
    bool prof = false;
    bool use_graphs = true;   // replay the GMRES matrix-vector product as a captured CUDA graph
    GmresWork gw;
    std::map<long long, std::unique_ptr<Rec>> plans;   // matvec plans by column count
    std::map<long long, std::unique_ptr<Rec>> setup_plans, recon_plans;  // by (column count, scaling)
    void** d_io = nullptr;   // device slots: the current call's volume right-hand side and solution
    void** h_io = nullptr;   // pinned staging of the two slots
    double* d_norms = nullptr;           // per-column norm pairs of the volume residual (2 x norms_cap)
    int norms_cap = 0;
    double2 *d_vol_res = nullptr, *d_vol_du = nullptr;   // defect correction: residual, correction
    int vol_cap = 0;                                      // (vol_cap columns of nx*ny*nz each)
    double2 *d_stage_rhs = nullptr, *d_stage_u = nullptr; // device copies of hz_solve_host's host
    int stage_cap = 0;                                    // buffers (stage_cap columns each)
    // autotuner: (shape signature, ldc) -> chosen split-K depth and column chunk
    bool autotune = true;
    struct TuneChoice { int KS, CC, tc, KS_tc, min_t, tc_cfg; };
    std::map<std::string, TuneChoice> tuned;
    std::vector<std::string> tune_log;
    int tc_mode = 2;        // tensor-core substitution (complex64, >= 64 columns): 0 never, 1 always,
                            // 2 when the autotuner measures it faster for the batch signature
    int tc_ks = 4;          // split-K (factor tiles per block) of small tensor-core batches
    int tc_min_tiles = 8;   // output tiles a node product needs to run on the tensor cores
    int tc_cfg = 0;         // untuned tensor-core kernel: 0 one block per work item, 1 persistent (HZ_TC_CFG)
    int precond_split = 3;  // TF32 terms of the tensor-core products inside the preconditioner (3 or 1)
    long long tc_wait_polls = 1LL << 26;  // poll limit of the tensor-core pipeline waits (HZ_TC_WAIT_POLLS:
                                          // a small value makes the waits give up, to test that path)
    int sparse_subst = 3;   // skip substitution products away from the interface planes where the
                            // operator allows it (bit 0 forward, bit 1 backward; HZ_SPARSE)
    bool factor_prof = false;     // time every factorization launch by kernel kind (HZ_FACTOR_PROFILE=1)
    std::string factor_text;      // per-kind table of the last profiled factorization
    int factor_tc_min_upd = 128;  // complex64 fronts with at least this many update unknowns (and a
                                  // full tile of own unknowns) get their L21 and Schur products on
                                  // the tensor cores; 0 switches this off (HZ_FACTOR_TC_MIN)
    std::vector<ProfRec> prof_recs;
    bool prof_detail = false;                 // also time every substitution launch by kernel kind
    std::vector<ProfRec> prof_launch;
    KernStat kern_stat[3];                    // per kind (CUDA-core, tensor-core substitution;
                                              // explicit trace-block products), from the last hz_profile_end
    std::map<std::tuple<int, int, int>, KernStat> kern_lvl;  // per (kind, phase, tree level)
    std::string prof_text;
    TraceBlocks tb;
};

template <class C> void factor_layers(Ctx& ctx);

// Tensor-core products of the factorization of complex64 fronts (factor_tc.cu): L21 = F21 L11^{-T}
// D^{-1} into the packed factor tiles, then F22 -= L21 D L21^T in the front.
struct FrontGemmDesc {
    float2* F;             // dense front (m x m, column-major)
    float2* fac;           // layer's packed factor tiles
    const float2* dinv;    // layer's D^{-1} by elimination index
    long long linv_off, l21_off;
    int m, nown, nupd, own0, own_t, upd_t;
};
struct GemmItem { int front, ti, tj, nst; };   // 128 x 128 output tile (ti, tj), pipeline stages
bool front_gemm_eligible(int nown, int nupd, int min_upd);
void front_gemm_items(const std::vector<FrontGemmDesc>& fronts, std::vector<GemmItem>& l21,
                      std::vector<GemmItem>& schur);
void launch_front_gemm(int mode, const GemmItem* d_items, long long n, const FrontGemmDesc* d_fronts, int* flag,
                       long long polls, cudaStream_t st);

}  // namespace hz

struct hz_handle {
    hz::Ctx ctx;
};
