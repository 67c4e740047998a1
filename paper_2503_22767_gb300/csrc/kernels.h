// Host-side launchers of the substep kernels (implemented in kernels_*.cu).
// Each returns the cudaError_t of its launch; all work goes on `st`.
#pragma once

#include <cuda_runtime.h>

#include "mpm_device.cuh"

namespace mpm {

// Buffers one particle kernel touches; unused members stay null.
struct StepArgs {
    const float* s_in = nullptr;     // state read by the kernel (SoA, stride np)
    // initial positions in the current order (stride np): the X slot of the
    // state holds the displacement u = x - x0 and positions are x0 + u; null:
    // the X slot holds x itself
    const float* x0 = nullptr;
    float* s_out = nullptr;          // state written by G2P
    const float* s_aux = nullptr;    // adjoint: state of the G2P^T substep (x, F)
    const float4* V = nullptr;       // grid velocity of the G2P (or G2P^T) substep
    float4* acc = nullptr;           // P2G accumulator
    float4* Vbar = nullptr;          // G2P^T scatter target
    const float4* gadj = nullptr;    // grid adjoint (mbar, mvbar) of the P2G^T substep
    float* adj = nullptr;            // particle adjoint (SoA, stride np)
    const float* phi = nullptr;      // current-order design (stride np)
    const float* mag = nullptr;
    float* gphi = nullptr;           // current-order design gradients
    float* gmag = nullptr;
    const float* field = nullptr;    // [inst][n_steps][D]
    float* gfield = nullptr;
    float* mom = nullptr;            // [n_steps][n_inst] sum_p m_p v_x after each substep
    const float* Minst = nullptr;    // [n_inst] instance mass
    const float* dloss = nullptr;    // [n_inst]
    const int* inst_off = nullptr;   // [n_inst + 1]
    int* err = nullptr;
    int n_p2g = 0;                   // substep index of the P2G (or P2G^T) part
    int n_g2p = 0;                   // substep index of the G2P part (momentum row)
    // fused grid operation: the particle kernels evaluate Eq. 16-18 (and its
    // reverse) per stencil node from the accumulators instead of reading V /
    // gadj written by a separate grid kernel
    const float4* accG = nullptr;    // accumulator of the G2P (or G2P^T) substep
    const float4* accP = nullptr;    // accumulator of the P2G^T substep
    const float4* VbarIn = nullptr;  // Vbar of the P2G^T substep
    float4* zero4 = nullptr;         // buffer the kernel clears for a later substep
    long long zero_n = 0;            // its length in float4
    // 3D: the P2G part marks the node blocks its stencils touch (null: no marking)
    ActiveBlocks blk;
};

// forward particle kernel: G2P of substep n_g2p and/or P2G of n_p2g.
// write_all: also store v and C (needed at checkpoints and in the store pass).
// fuse: take the grid velocity from a.accG through the grid operation.
cudaError_t launch_forward(int dim, bool g2p, bool p2g, bool write_all, bool fuse,
                           const Params& P, const StepArgs& a, int block, cudaStream_t st);
// adjoint particle kernel: P2G^T of substep n_p2g and/or G2P^T of n_p2g - 1
// (or, without P2G^T, of substep n_p2g).
// fuse: grid adjoint from (a.accP, a.VbarIn); fuse_v: grid velocity of the
// G2P^T substep from a.accG through the grid operation (fuse implies fuse_v).
cudaError_t launch_adjoint(int dim, bool p2gt, bool g2pt, bool fuse, bool fuse_v, const Params& P,
                           const StepArgs& a, int block, cudaStream_t st);
// Per-dimension instantiations (D = 2, 3) of the two calls above, each in a
// translation unit of its own.
template <int D>
cudaError_t launch_forward_dim(bool g2p, bool p2g, bool write_all, bool fuse, const Params& P,
                               const StepArgs& a, int block, cudaStream_t st);
template <int D>
cudaError_t launch_adjoint_dim(bool p2gt, bool g2pt, bool fuse, bool fuse_v, const Params& P,
                               const StepArgs& a, int block, cudaStream_t st);
extern template cudaError_t launch_forward_dim<2>(bool, bool, bool, bool, const Params&, const StepArgs&,
                                                  int, cudaStream_t);
extern template cudaError_t launch_forward_dim<3>(bool, bool, bool, bool, const Params&, const StepArgs&,
                                                  int, cudaStream_t);
extern template cudaError_t launch_adjoint_dim<2>(bool, bool, bool, bool, const Params&, const StepArgs&,
                                                  int, cudaStream_t);
extern template cudaError_t launch_adjoint_dim<3>(bool, bool, bool, bool, const Params&, const StepArgs&,
                                                  int, cudaStream_t);
// grid operation on every node of every instance: acc -> V; clears acc
// (lean) or clears acc_next (store pass).
cudaError_t launch_grid(int dim, const Params& P, float4* acc, float4* V, float4* acc_next,
                        bool clear_acc, int step, cudaStream_t st);
// grid adjoint: Vbar -> gadj (clears Vbar).
cudaError_t launch_grid_adjoint(int dim, const Params& P, const float4* acc, float4* Vbar,
                                float4* gadj, int step, cudaStream_t st);
// 3D, over the listed node blocks only (ctas persistent CTAs walk the list).
// Grid operation: acc -> V; with clear_acc, also zeroes acc (the forward
// pass, whose next P2G reuses it).
cudaError_t launch_grid_blocks(const Params& P, float4* acc, float4* V, ActiveBlocks blk, bool clear_acc,
                               int step, int ctas, cudaStream_t st);
// Grid adjoint: Vbar -> gadj, zeroing Vbar.
cudaError_t launch_grid_adjoint_blocks(const Params& P, const float4* acc, float4* Vbar, float4* gadj,
                                       ActiveBlocks blk, int step, int ctas, cudaStream_t st);
// Zeroes the flags of the listed blocks and, with acc, the n_sub
// accumulators acc + k * acc_stride over them (the count and the warps'
// boxes are left to the caller).
cudaError_t launch_clear_blocks(const Params& P, float4* acc, long long acc_stride, ActiveBlocks blk, int n_sub,
                                cudaStream_t st);

// initial state from x0 / v0 (input order): u = x - x0 = 0, C = 0, F = I,
// id = p, and the current-order initial positions x0c (stride np).
cudaError_t launch_init_state(int dim, const Params& P, const float* x0, const float* v0,
                              float* s, int* id, float* x0c, cudaStream_t st);
// dst[c][p] = src[c][perm[p]] for every component, id_dst[p] = id_src[perm[p]].
cudaError_t launch_reorder(int ncomp, const Params& P, const float* src, float* dst,
                           const int* perm, const int* id_src, int* id_dst, cudaStream_t st);
// adj_old[c][perm[p]] = adj_new[c][p]
cudaError_t launch_unpermute(int ncomp, const Params& P, const float* src, float* dst,
                             const int* perm, cudaStream_t st);
// out[c][id[p]] = s[c][p] (+ add[c][p] when add is set, stride np) for
// components [c0, c0 + ncomp), out stride n_total; diag > 0 marks a diag x
// diag block stored as E = F - I (F is written).
cudaError_t launch_to_input_order(int ncomp, const Params& P, const float* s, int c0,
                                  const int* id, float* out, cudaStream_t st, int diag = 0,
                                  const float* add = nullptr);
// current-order design from the per-design arrays, and the current-order
// initial positions x0c[c][p] = x0[c][id[p]] (x0 in input order, stride N)
cudaError_t launch_gather_design(int dim, const Params& P, const int* id, const int* inst_off,
                                 const int* dbase, const float* phi_d, const float* mag_d,
                                 long long nd, float* phi, float* mag, const float* x0, float* x0c,
                                 cudaStream_t st);
// per-design gradients += current-order gradients
cudaError_t launch_scatter_design_grad(int dim, const Params& P, const int* id,
                                       const int* inst_off, const int* dbase, const float* gphi,
                                       const float* gmag, long long nd, float* g_phi,
                                       float* g_mag, cudaStream_t st);
cudaError_t launch_instance_mass(const Params& P, const float* phi, const int* inst_off,
                                 float* Minst, cudaStream_t st);
// (x0: current-order initial positions; the state holds displacements)
cudaError_t launch_loss(int dim, const Params& P, const float* s, const float* x0, const float* target,
                        const int* id, const int* inst_off, const float* Minst, const float* mom,
                        float* loss_acc, float* loss_out, cudaStream_t st);
cudaError_t launch_seed(int dim, const Params& P, const float* s, const float* x0, const float* target,
                        const int* id, const int* inst_off, const float* phi, const float* Minst,
                        const float* mom, const float* dloss, float* adj, float* gphi,
                        cudaStream_t st);

// ---- persistent passes (kernels_persist.cuh) ----
enum class PersistKind { kLean, kStore, kAdjoint };
// One checkpoint segment [s0, s1) of a pass in one cooperative launch.
struct PersistArgs {
    StepArgs base;                      // the fields every substep shares
    int s0 = 0, s1 = 0, T = 0;          // segment and horizon
    bool first_p2g = false;             // lean: start with the P2G of substep s0
    float* st[2] = {nullptr, nullptr};  // lean: the two state buffers (st[0] holds state s0)
    float* state = nullptr;             // store / adjoint: state k of the segment at state + k S
    long long S = 0;
    float4* acc = nullptr;              // lean: the accumulator; store / adjoint: that of substep s0 (+ k G)
    float4* V = nullptr;                // the same for the grid velocity
    long long G = 0;
    ActiveBlocks blk;                   // 3D: the segment's node-block list
    ActiveBlocks blk_next;              // lean: the next segment's list (the last P2G)
    unsigned* bar = nullptr;            // grid barrier {arrivals, generation}, zero at launch
    long long spin_limit = 0;           // polls before a barrier wait gives up (kErrTimeout)
};
// lists must be true in 3D and false in 2D; at most max_ctas CTAs (0: as
// many as are resident at once, capped by the particles).
cudaError_t launch_persist(int dim, PersistKind kind, bool lists, const Params& P, const PersistArgs& pa, int block,
                           int max_ctas, cudaStream_t st);
template <int D>
cudaError_t launch_persist_dim(PersistKind kind, bool lists, const Params& P, const PersistArgs& pa, int block,
                               int max_ctas, cudaStream_t st);
extern template cudaError_t launch_persist_dim<2>(PersistKind, bool, const Params&, const PersistArgs&, int, int,
                                                  cudaStream_t);
extern template cudaError_t launch_persist_dim<3>(PersistKind, bool, const Params&, const PersistArgs&, int, int,
                                                  cudaStream_t);

// ---- sort (kernels_sort.cu) ----
struct SortBuffers {
    int* keys = nullptr;       // [N]
    int* slot = nullptr;       // [N]
    int* counts = nullptr;     // [n_keys]
    int* offsets = nullptr;    // [n_keys]
    int* scan_tmp = nullptr;   // block sums of the recursive scan
    long long scan_tmp_len = 0;
    long long n_keys = 0;
};
long long sort_key_space(int dim, int res, int n_inst);
// exclusive prefix sum of n ints (in == out allowed); tmp holds
// sort_scan_tmp_len(n) ints
cudaError_t launch_scan_exclusive(const int* in, int* out, long long n, int* tmp, cudaStream_t st);
long long sort_scan_tmp_len(long long n_keys);
// keys, stable permutation perm[new] = old for positions x (component stride
// xstride), or x0 + x when x0 is set (same stride: x holds displacements);
// flags kErrDomain for stencils outside the grid (keys clamp).
cudaError_t launch_sort(int dim, const Params& P, const float* x, long long xstride,
                        const int* inst_off, SortBuffers& sb, int* perm, int* err,
                        cudaStream_t st, const float* x0 = nullptr);

}  // namespace mpm
