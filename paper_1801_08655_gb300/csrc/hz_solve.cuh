// Declarations of the batched local-solve driver (solve.cu) and the online-phase
// operators (polarized.cu).
#pragma once

#include "hz_ctx.cuh"

namespace hz {

int chunk_cols(bool is_double, int ncols);
int tc_columns(int ldc);   // tensor-core column tile for this leading dimension (0: not usable)
void launch_level_tc(const Batch& b, int h, int mode, int ldc, int* flag, cudaStream_t st);
int padded_ldc(bool is_double, int ncols);

// Sparsity of a batch: which planes of each layer carry the sources (forward code, bits 0-1) and
// the read-outs (backward code, bits 2-3).  SP_ALL: anywhere (no product skipped); SP_BOTH: the
// plane pairs next to both internal interfaces; SP_TOP / SP_BOT: the pair next to the top /
// bottom interface only.  Forward products of nodes whose subtree holds none of the source planes
// are skipped (their right-hand side, and so their forward result, is zero), and backward
// products of nodes whose subtree holds none of the read-out planes (nothing below them is read).
enum { SP_ALL = 0, SP_BOTH = 1, SP_TOP = 2, SP_BOT = 3 };
constexpr int sparse_code(int fwd, int bwd) { return fwd | (bwd << 2); }

// Per-block sparsity: the batch's columns split into nblk (2-4) equal blocks, each with its own
// sparsity code (block q in bits 4q..4q+3; SP_BLOCKS marks the form, the block count sits in bits
// 17-19).  Each block is then a job of its own, so that a node product runs only on the column
// blocks that need it.
constexpr int SP_BLOCKS = 1 << 16;
inline int blocked_code(int nblk, const int* codes) {
    int s = SP_BLOCKS | (nblk << 17);
    for (int q = 0; q < nblk; ++q) s |= (codes[q] & 15) << (4 * q);
    return s;
}
inline int block_count(int sparse) { return (sparse & SP_BLOCKS) ? (sparse >> 17) & 7 : 1; }
inline int block_code(int sparse, int q) { return (sparse & SP_BLOCKS) ? (sparse >> (4 * q)) & 15 : sparse; }

// Job set with per-level task lists, cached by layer list and sparsity code.
template <class C> Batch& get_batch(Ctx& ctx, const std::vector<int>& layers, int ncols, int split = 3, int sparse = 0);
// Build (or fetch) a batch with an explicit split-K depth and column chunk.
template <class C> Batch& get_batch_cfg(Ctx& ctx, const std::vector<int>& layers, int ncols, int KS, int CC, bool tc,
                                       int KS_tc, int min_t, int split = 3, int tc_cfg = 0, int sparse = 0);
// Autotune the substitution of this batch signature (times candidate split-K depths and column
// chunks on zeroed slot vectors); a no-op once the signature is tuned or when tuning is off.
template <class C> void ensure_tuned(Ctx& ctx, const std::vector<int>& layers, int ncols, int split = 3,
                                     int sparse = 0);
void free_batches(Ctx& ctx);

// Forward/backward substitution for every job of the batch on ncols columns of the
// layers' slot vectors (acc holds the right-hand side in elimination order on entry and
// is clobbered; x receives the solution).
template <class C> void substitute(Ctx& ctx, const Batch& b, int ncols, cudaStream_t st);

// Online operators on polarized trace vectors [R][2][K][2][P] (complex128, device).
template <class C> void op_polarized_rhs(Ctx& ctx, const double2* g, bool scale, int R, double2* fpol);
template <class C> void op_apply_mpol(Ctx& ctx, const double2* x, int R, double2* y);
template <class C> void op_apply_precond(Ctx& ctx, const double2* x, int R, double2* y, double2* tmp);
template <class C> void op_reconstruct(Ctx& ctx, const double2* g, bool scale, const double2* t, int R,
                                       double2* u, bool accumulate);
template <class C> void op_layer_solve(Ctx& ctx, int ell, const double2* g, int ncols, double2* w);
void op_volume_residual(Ctx& ctx, const double2* f, bool scale, const double2* u, int R, double2* r,
                        double* norms /* device, 2R: ||r||^2, ||g||^2 */);

// Explicit trace-to-trace Green's blocks of every layer (into ctx.tb), computed by local solves of
// unit source traces in chunks of at most `chunk` columns per source pair (a multiple of 64; the
// layer slots must hold 2 * chunk columns).
template <class C> void build_trace_blocks(Ctx& ctx, int chunk);

struct GmresOut { int iters; double relres; };
template <class C> void gmres_solve(Ctx& ctx, const double2* g, bool scale, int R, double2* u,
                                    const hz_solve_opts& o, hz_solve_info* info);
// GMRES (o.krylov == 0) or Bi-CGSTAB (1) on the trace system
template <class C> void krylov_solve(Ctx& ctx, const double2* g, bool scale, int R, double2* u,
                                     const hz_solve_opts& o, hz_solve_info* info);

}  // namespace hz
