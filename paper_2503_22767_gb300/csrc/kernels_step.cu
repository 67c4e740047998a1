// Grid kernels of the magneto-elastic MLS-MPM substep and its reverse, and
// the per-particle helpers around them (arxiv 2503.22767, Section 2.2-2.3).
//
// The grid kernel applies Eq. 16-18; the grid adjoint kernel reverses them
// with the forward branches replayed.  The particle kernels are in
// particle_kernels.cuh; launch_forward / launch_adjoint pick their
// per-dimension instantiation here.
// Grids are float4 per node ([inst][node]): accumulators (m, mv), velocities
// (v, 0), adjoints (mbar, mvbar).  Particle arrays are structure-of-arrays
// with component stride P.np: x[D], v[D], C[D][D], E[D][D] with E = F - I.
#include "kernels.h"
#include "mpm_device.cuh"
#include "grid_phase.cuh"
#include "particle_io.cuh"

namespace mpm {

namespace {

// ---------------------------------------------------------------------------
// grid operation (Eq. 16-18)
// ---------------------------------------------------------------------------
// One block row per instance (blockIdx.y), so node indices stay 32-bit.
// Nodes without mass (most of a 3D grid) skip the node arithmetic: Eq. 16
// gives them no velocity, and the reverse gives them no gradient.
template <int D>
__global__ void __launch_bounds__(256) k_grid(Params P, float4* __restrict__ acc,
                                              float4* __restrict__ V, float4* __restrict__ acc_next,
                                              bool clear_acc, int step) {
    pdl_wait();
    pdl_trigger();
    const int local = blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= P.nodes) return;
    int c[D];
    node_coords<D>(local, P.res, c);
    grid_node<D>(P, acc, V, acc_next, clear_acc, step, (long long)blockIdx.y * P.nodes + local, c);
}

template <int D>
__global__ void __launch_bounds__(256) k_grid_adjoint(Params P, const float4* __restrict__ acc,
                                                      float4* __restrict__ Vbar,
                                                      float4* __restrict__ gadj, int step) {
    pdl_wait();
    pdl_trigger();
    const int local = blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= P.nodes) return;
    int c[D];
    node_coords<D>(local, P.res, c);
    grid_adjoint_node<D>(P, acc, Vbar, gadj, step, (long long)blockIdx.y * P.nodes + local, c);
}

// ---------------------------------------------------------------------------
// the same over the listed node blocks only (3D)
// ---------------------------------------------------------------------------
// Persistent CTAs of 256 threads walk the list, four blocks of 64 nodes at a
// time (one thread per node).  The list holds block ids, instance-major.
__global__ void __launch_bounds__(256) k_grid_blocks(Params P, float4* __restrict__ acc, float4* __restrict__ V,
                                                     ActiveBlocks blk, bool clear, int step) {
    pdl_wait();
    pdl_trigger();
    const int n = *blk.count;
    const int t = threadIdx.x & 63;
    for (int e = blockIdx.x * 4 + (threadIdx.x >> 6); e < n; e += gridDim.x * 4) {
        const BlockNode nd = block_node(P, blk.list[e], t);
        if (nd.in) grid_node<3>(P, acc, V, nullptr, clear, step, nd.i, nd.c);
    }
}

__global__ void __launch_bounds__(256) k_grid_adjoint_blocks(Params P, const float4* __restrict__ acc,
                                                             float4* __restrict__ Vbar, float4* __restrict__ gadj,
                                                             ActiveBlocks blk, int step) {
    pdl_wait();
    pdl_trigger();
    const int n = *blk.count;
    const int t = threadIdx.x & 63;
    for (int e = blockIdx.x * 4 + (threadIdx.x >> 6); e < n; e += gridDim.x * 4) {
        const BlockNode nd = block_node(P, blk.list[e], t);
        if (nd.in) grid_adjoint_node<3>(P, acc, Vbar, gadj, step, nd.i, nd.c);
    }
}

// blockIdx.y: the accumulator (substep) this CTA clears over the listed
// blocks; the CTAs of accumulator 0 also zero the flags
__global__ void __launch_bounds__(256) k_clear_blocks(Params P, float4* __restrict__ acc, long long acc_stride,
                                                      ActiveBlocks blk) {
    const int k = blockIdx.y;
    const int n = *blk.count;
    const int t = threadIdx.x & 63;
    for (int e = blockIdx.x * 4 + (threadIdx.x >> 6); e < n; e += gridDim.x * 4) {
        const int b = blk.list[e];
        if (acc) {
            const BlockNode nd = block_node(P, b, t);
            if (nd.in) acc[acc_stride * k + nd.i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (k == 0 && t == 0) blk.flag[b] = 0;
    }
}

// ---------------------------------------------------------------------------
// helpers: init, permutations, design, loss and seeds
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_init_state(Params P, const float* __restrict__ x0, const float* __restrict__ v0,
                             float* __restrict__ s, int* __restrict__ id, float* __restrict__ x0c) {
    using L = Layout<D>;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    const long long np = P.np, n = P.n_total;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        s[(L::X + i) * np + p] = 0.0f;  // displacement u = x - x0
        x0c[i * np + p] = x0[i * n + p];
        s[(L::V + i) * np + p] = v0 ? v0[i * n + p] : 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            s[(L::C + i * D + j) * np + p] = 0.0f;
            s[(L::F + i * D + j) * np + p] = 0.0f;  // E = F - I = 0 at rest
        }
    }
    id[p] = p;
}

__global__ void k_reorder(Params P, int ncomp, const float* __restrict__ src, float* __restrict__ dst,
                          const int* __restrict__ perm, const int* __restrict__ id_src,
                          int* __restrict__ id_dst) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    int q = perm[p];
    for (int c = 0; c < ncomp; ++c) dst[c * P.np + p] = src[c * P.np + q];
    if (id_dst) id_dst[p] = id_src[q];
}

__global__ void k_unpermute(Params P, int ncomp, const float* __restrict__ src,
                            float* __restrict__ dst, const int* __restrict__ perm) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    int q = perm[p];
    for (int c = 0; c < ncomp; ++c) dst[c * P.np + q] = src[c * P.np + p];
}

// diag > 0: the components are a diag x diag block stored as E = F - I;
// write F (add the identity on the diagonal).  add: a current-order array
// added component by component (x0 to displacements).
__global__ void k_to_input_order(Params P, int ncomp, const float* __restrict__ s, int c0,
                                 const int* __restrict__ id, float* __restrict__ out, int diag,
                                 const float* __restrict__ add) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    int q = id[p];
    for (int c = 0; c < ncomp; ++c) {
        float val = s[(c0 + c) * P.np + p];
        if (add) val = __fadd_rn(val, add[c * P.np + p]);
        if (diag > 0 && c % (diag + 1) == 0) val += 1.0f;
        out[(long long)c * P.n_total + q] = val;
    }
}

__device__ __forceinline__ long long design_index(int g, const int* __restrict__ inst_off,
                                                  const int* __restrict__ dbase, int n_inst) {
    int inst = find_instance(inst_off, n_inst, g);
    return (long long)dbase[inst] + (g - inst_off[inst]);
}

template <int D>
__global__ void k_gather_design(Params P, const int* __restrict__ id, const int* __restrict__ inst_off,
                                const int* __restrict__ dbase, const float* __restrict__ phi_d,
                                const float* __restrict__ mag_d, long long nd,
                                float* __restrict__ phi, float* __restrict__ mag,
                                const float* __restrict__ x0, float* __restrict__ x0c) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    const int q = id[p];
    long long di = design_index(q, inst_off, dbase, P.n_inst);
    phi[p] = phi_d[di];
#pragma unroll
    for (int i = 0; i < D; ++i) mag[i * P.np + p] = mag_d[i * nd + di];
    if (x0c) {
#pragma unroll
        for (int i = 0; i < D; ++i) x0c[i * P.np + p] = x0[(long long)i * P.n_total + q];
    }
}

template <int D>
__global__ void k_scatter_design_grad(Params P, const int* __restrict__ id,
                                      const int* __restrict__ inst_off,
                                      const int* __restrict__ dbase, const float* __restrict__ gphi,
                                      const float* __restrict__ gmag, long long nd,
                                      float* __restrict__ g_phi, float* __restrict__ g_mag) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    long long di = design_index(id[p], inst_off, dbase, P.n_inst);
    if (g_phi) atomicAdd(g_phi + di, gphi[p]);
    if (g_mag) {
#pragma unroll
        for (int i = 0; i < D; ++i) atomicAdd(g_mag + i * nd + di, gmag[i * P.np + p]);
    }
}

__global__ void k_instance_mass(Params P, const float* __restrict__ phi,
                                const int* __restrict__ inst_off, float* __restrict__ Minst) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = p < P.n_total;
    int inst = active ? find_instance(inst_off, P.n_inst, p) : -1;
    float m[1] = {active ? phi[p] * P.rho0 * P.p_vol : 0.0f};
    warp_add_per_instance<1>(m, inst, Minst, 1);
}

template <int D>
__global__ void k_loss_mse(Params P, const float* __restrict__ s, const float* __restrict__ x0,
                           const float* __restrict__ target, const int* __restrict__ id,
                           const int* __restrict__ inst_off, float* __restrict__ loss_acc) {
    using L = Layout<D>;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = p < P.n_total;
    int inst = active ? find_instance(inst_off, P.n_inst, p) : -1;
    float e2[1] = {0.0f};
    if (active) {
        int q = id[p];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float x = __fadd_rn(s[(L::X + i) * P.np + p], x0[i * P.np + p]);
            float e = x - target[(long long)i * P.n_total + q];
            e2[0] += e * e;
        }
    }
    warp_add_per_instance<1>(e2, inst, loss_acc, 1);
}

__global__ void k_loss_finalize(Params P, const int* __restrict__ inst_off,
                                const float* __restrict__ Minst, const float* __restrict__ mom,
                                const float* __restrict__ loss_acc, float* __restrict__ loss_out) {
    int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= P.n_inst) return;
    if (P.loss_kind == 1) {
        float M = Minst[inst];
        double acc = 0.0;
        for (int n = 0; n < P.n_steps; ++n) acc += mom[(long long)n * P.n_inst + inst];
        loss_out[inst] = M > 0.0f ? (float)(-(double)P.dt * acc / M) : 0.0f;
    } else {
        int cnt = inst_off[inst + 1] - inst_off[inst];
        loss_out[inst] = cnt > 0 ? loss_acc[inst] / (float)cnt : 0.0f;
    }
}

template <int D>
__global__ void k_seed(Params P, const float* __restrict__ s, const float* __restrict__ x0,
                       const float* __restrict__ target,
                       const int* __restrict__ id, const int* __restrict__ inst_off,
                       const float* __restrict__ phi, const float* __restrict__ Minst,
                       const float* __restrict__ mom, const float* __restrict__ dloss,
                       float* __restrict__ adj, float* __restrict__ gphi) {
    using L = Layout<D>;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    int inst = find_instance(inst_off, P.n_inst, p);
    const long long np = P.np;
    for (int c = 0; c < L::N; ++c) adj[c * np + p] = 0.0f;
    float dl = dloss[inst];
    if (P.loss_kind == 1) {
        float M = Minst[inst];
        if (M > 0.0f && P.n_steps > 0) {
            float rM = 1.0f / M;
            float mp = phi[p] * P.rho0 * P.p_vol;
            float vx = s[L::V * np + p];
            float vbar = mom[(long long)(P.n_steps - 1) * P.n_inst + inst] * rM;
            adj[L::V * np + p] = -P.dt * mp * rM * dl;
            gphi[p] -= P.dt * (vx - vbar) * rM * dl * P.rho0 * P.p_vol;
        }
    } else {
        int cnt = inst_off[inst + 1] - inst_off[inst];
        int q = id[p];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float x = __fadd_rn(s[(L::X + i) * np + p], x0[i * np + p]);
            float e = x - target[(long long)i * P.n_total + q];
            adj[(L::X + i) * np + p] = 2.0f * e / (float)cnt * dl;
        }
    }
}

inline int blocks_for(long long n, int block) { return (int)((n + block - 1) / block); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_forward(int dim, bool g2p, bool p2g, bool write_all, bool fuse,
                           const Params& P, const StepArgs& a, int block, cudaStream_t st) {
    return dim == 2 ? launch_forward_dim<2>(g2p, p2g, write_all, fuse, P, a, block, st)
                    : launch_forward_dim<3>(g2p, p2g, write_all, fuse, P, a, block, st);
}

cudaError_t launch_adjoint(int dim, bool p2gt, bool g2pt, bool fuse, bool fuse_v, const Params& P,
                           const StepArgs& a, int block, cudaStream_t st) {
    return dim == 2 ? launch_adjoint_dim<2>(p2gt, g2pt, fuse, fuse_v, P, a, block, st)
                    : launch_adjoint_dim<3>(p2gt, g2pt, fuse, fuse_v, P, a, block, st);
}

cudaError_t launch_persist(int dim, PersistKind kind, bool lists, const Params& P, const PersistArgs& pa, int block,
                           int max_ctas, cudaStream_t st) {
    return dim == 2 ? launch_persist_dim<2>(kind, lists, P, pa, block, max_ctas, st)
                    : launch_persist_dim<3>(kind, lists, P, pa, block, max_ctas, st);
}

cudaError_t launch_grid(int dim, const Params& P, float4* acc, float4* V, float4* acc_next,
                        bool clear_acc, int step, cudaStream_t st) {
    dim3 grid(blocks_for(P.nodes, 256), P.n_inst);
    if (dim == 2) return launch_chain(P, k_grid<2>, grid, dim3(256), st, P, acc, V, acc_next, clear_acc, step);
    return launch_chain(P, k_grid<3>, grid, dim3(256), st, P, acc, V, acc_next, clear_acc, step);
}

cudaError_t launch_grid_adjoint(int dim, const Params& P, const float4* acc, float4* Vbar,
                                float4* gadj, int step, cudaStream_t st) {
    dim3 grid(blocks_for(P.nodes, 256), P.n_inst);
    if (dim == 2) return launch_chain(P, k_grid_adjoint<2>, grid, dim3(256), st, P, acc, Vbar, gadj, step);
    return launch_chain(P, k_grid_adjoint<3>, grid, dim3(256), st, P, acc, Vbar, gadj, step);
}

cudaError_t launch_grid_blocks(const Params& P, float4* acc, float4* V, ActiveBlocks blk, bool clear_acc,
                               int step, int ctas, cudaStream_t st) {
    return launch_chain(P, k_grid_blocks, dim3(ctas), dim3(256), st, P, acc, V, blk, clear_acc, step);
}

cudaError_t launch_grid_adjoint_blocks(const Params& P, const float4* acc, float4* Vbar, float4* gadj,
                                       ActiveBlocks blk, int step, int ctas, cudaStream_t st) {
    return launch_chain(P, k_grid_adjoint_blocks, dim3(ctas), dim3(256), st, P, acc, Vbar, gadj, blk, step);
}

cudaError_t launch_clear_blocks(const Params& P, float4* acc, long long acc_stride, ActiveBlocks blk, int n_sub,
                                cudaStream_t st) {
    if (n_sub <= 0) return cudaSuccess;
    k_clear_blocks<<<dim3(32, n_sub), 256, 0, st>>>(P, acc, acc_stride, blk);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int dim, const Params& P, const float* x0, const float* v0, float* s,
                              int* id, float* x0c, cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    dim3 grid(blocks_for(P.n_total, 256));
    if (dim == 2) k_init_state<2><<<grid, 256, 0, st>>>(P, x0, v0, s, id, x0c);
    else k_init_state<3><<<grid, 256, 0, st>>>(P, x0, v0, s, id, x0c);
    return cudaGetLastError();
}

cudaError_t launch_reorder(int ncomp, const Params& P, const float* src, float* dst,
                           const int* perm, const int* id_src, int* id_dst, cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    k_reorder<<<blocks_for(P.n_total, 256), 256, 0, st>>>(P, ncomp, src, dst, perm, id_src, id_dst);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(int ncomp, const Params& P, const float* src, float* dst,
                             const int* perm, cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    k_unpermute<<<blocks_for(P.n_total, 256), 256, 0, st>>>(P, ncomp, src, dst, perm);
    return cudaGetLastError();
}

cudaError_t launch_to_input_order(int ncomp, const Params& P, const float* s, int c0,
                                  const int* id, float* out, cudaStream_t st, int diag, const float* add) {
    if (P.n_total == 0) return cudaSuccess;
    k_to_input_order<<<blocks_for(P.n_total, 256), 256, 0, st>>>(P, ncomp, s, c0, id, out, diag, add);
    return cudaGetLastError();
}

cudaError_t launch_gather_design(int dim, const Params& P, const int* id, const int* inst_off,
                                 const int* dbase, const float* phi_d, const float* mag_d,
                                 long long nd, float* phi, float* mag, const float* x0, float* x0c,
                                 cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    dim3 grid(blocks_for(P.n_total, 256));
    if (dim == 2)
        k_gather_design<2><<<grid, 256, 0, st>>>(P, id, inst_off, dbase, phi_d, mag_d, nd, phi, mag, x0, x0c);
    else
        k_gather_design<3><<<grid, 256, 0, st>>>(P, id, inst_off, dbase, phi_d, mag_d, nd, phi, mag, x0, x0c);
    return cudaGetLastError();
}

cudaError_t launch_scatter_design_grad(int dim, const Params& P, const int* id,
                                       const int* inst_off, const int* dbase, const float* gphi,
                                       const float* gmag, long long nd, float* g_phi,
                                       float* g_mag, cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    dim3 grid(blocks_for(P.n_total, 256));
    if (dim == 2)
        k_scatter_design_grad<2><<<grid, 256, 0, st>>>(P, id, inst_off, dbase, gphi, gmag, nd, g_phi, g_mag);
    else
        k_scatter_design_grad<3><<<grid, 256, 0, st>>>(P, id, inst_off, dbase, gphi, gmag, nd, g_phi, g_mag);
    return cudaGetLastError();
}

cudaError_t launch_instance_mass(const Params& P, const float* phi, const int* inst_off,
                                 float* Minst, cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    k_instance_mass<<<blocks_for(P.n_total, 256), 256, 0, st>>>(P, phi, inst_off, Minst);
    return cudaGetLastError();
}

cudaError_t launch_loss(int dim, const Params& P, const float* s, const float* x0, const float* target,
                        const int* id, const int* inst_off, const float* Minst, const float* mom,
                        float* loss_acc, float* loss_out, cudaStream_t st) {
    if (P.loss_kind == 0 && P.n_total > 0) {
        dim3 grid(blocks_for(P.n_total, 256));
        if (dim == 2) k_loss_mse<2><<<grid, 256, 0, st>>>(P, s, x0, target, id, inst_off, loss_acc);
        else k_loss_mse<3><<<grid, 256, 0, st>>>(P, s, x0, target, id, inst_off, loss_acc);
    }
    k_loss_finalize<<<blocks_for(P.n_inst, 64), 64, 0, st>>>(P, inst_off, Minst, mom, loss_acc, loss_out);
    return cudaGetLastError();
}

cudaError_t launch_seed(int dim, const Params& P, const float* s, const float* x0, const float* target,
                        const int* id, const int* inst_off, const float* phi, const float* Minst,
                        const float* mom, const float* dloss, float* adj, float* gphi,
                        cudaStream_t st) {
    if (P.n_total == 0) return cudaSuccess;
    dim3 grid(blocks_for(P.n_total, 256));
    if (dim == 2) k_seed<2><<<grid, 256, 0, st>>>(P, s, x0, target, id, inst_off, phi, Minst, mom, dloss, adj, gphi);
    else k_seed<3><<<grid, 256, 0, st>>>(P, s, x0, target, id, inst_off, phi, Minst, mom, dloss, adj, gphi);
    return cudaGetLastError();
}

}  // namespace mpm
