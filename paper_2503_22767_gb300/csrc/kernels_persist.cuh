// Persistent passes: one cooperative launch runs every substep of one
// checkpoint segment of a pass (Section 2.2; its reverse, Section 2.3).
//
// The chained form launches, per substep, a grid kernel and a particle
// kernel (and the same two in reverse), each a dependent launch.  Here a
// grid of CTAs that are all resident at once (a cooperative launch) walks the
// substeps itself: grid phase, grid-wide barrier, particle phase, barrier.
// For a small body (the 2D locomotion workload's 30,000 particles) the
// per-substep cost is the chain of dependent launches, which the barriers
// replace.  The phases run the same per-node and per-particle code as the
// chained kernels (grid_phase.cuh, forward_particle / adjoint_particle), so
// results do not depend on the form.
//
// Every barrier wait is bounded: a CTA that has spun spin_limit times without
// the barrier opening sets kErrTimeout and returns (the host reports
// MPM_ERR_TIMEOUT); the CTAs that still wait give up the same way.
#pragma once

#include <algorithm>

#include "grid_phase.cuh"
#include "particle_kernels.cuh"

namespace mpm {

namespace {

// Resident 256-thread blocks per SM the persistent kernels are compiled for
// (<= 128 registers).  Their CTAs stay resident for the whole segment, and
// for the small bodies they serve the work per phase is a few particles per
// thread, so registers are spent on avoiding spills rather than on
// occupancy (at the chained kernels' 48-register 2D budget the forward pass
// spilled 196 bytes).
constexpr int kPersistBlocks = 2;

// Grid-wide barrier over all CTAs of a cooperative launch.  bar = {arrivals,
// generation}, both zero at launch.  Thread 0 of each CTA reads the
// generation, arrives, and the last arrival resets the count and opens the
// next generation; the others wait for it, at most spin_limit polls.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, long long spin_limit, int* err) {
    __shared__ int s_open;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        int open = 1;
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > spin_limit) {
                    open = 0;
                    atomicOr(err, kErrTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_open = open;
    }
    __syncthreads();
    return s_open != 0;
}

// Particle phase: every thread takes particles tid, tid + threads, ...; all
// lanes of a warp run each round together (the bodies use warp collectives).
template <typename Body>
__device__ __forceinline__ void particle_phase(const Params& P, Body body) {
    const int threads = gridDim.x * blockDim.x;
    for (int p0 = 0; p0 < P.n_total; p0 += threads) body(p0 + blockIdx.x * blockDim.x + threadIdx.x);
}

// Grid phase over every node of every instance grid, or (LISTS, 3D) over the
// listed node blocks, 64 threads per block.
template <int D, bool LISTS, typename Node>
__device__ __forceinline__ void grid_phase(const Params& P, const ActiveBlocks& blk, Node node) {
    if constexpr (LISTS) {
        const int n = *(volatile int*)blk.count;
        const int t = threadIdx.x & 63;
        const int groups = gridDim.x * (blockDim.x >> 6);
        for (int e = blockIdx.x * (blockDim.x >> 6) + (threadIdx.x >> 6); e < n; e += groups) {
            const BlockNode nd = block_node(P, blk.list[e], t);
            if (nd.in) node(nd.i, nd.c);
        }
    } else {
        const long long total = P.nodes * P.n_inst;
        const long long threads = (long long)gridDim.x * blockDim.x;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += threads) {
            int c[D];
            node_coords<D>((int)(i % P.nodes), P.res, c);
            node(i, c);
        }
    }
}

// ---------------------------------------------------------------------------
// forward pass, lean (between checkpoints only x and E are stored)
// ---------------------------------------------------------------------------
// Substeps [s0, s1): grid operation of n, then G2P of n with P2G of n + 1
// (the state alternates between st[0] and st[1], st[0] holding state s0).
// The last substep stores the full state (the next checkpoint) and, within
// the horizon, lists its P2G blocks in blk_next.
template <int D, bool LISTS>
__global__ void __launch_bounds__(256, kPersistBlocks)
    k_persist_lean(Params P, PersistArgs pa) {
    extern __shared__ float4 s_warp[];
    float4* sm = s_warp + (threadIdx.x >> 5) * warp_slots<D, true>();
    int* err = pa.base.err;
    if (pa.first_p2g) {  // P2G of substep s0 (the start of the pass)
        StepArgs a = pa.base;
        a.s_in = pa.st[0];
        a.acc = pa.acc;
        a.n_p2g = pa.s0;
        if (LISTS) a.blk = pa.blk;
        particle_phase(P, [&](int p) { forward_particle<D, false, true, false, false, false, false>(P, a, p, sm); });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
    }
    for (int n = pa.s0; n < pa.s1; ++n) {
        const int k = n - pa.s0;
        grid_phase<D, LISTS>(P, pa.blk, [&](long long i, const int (&c)[D]) {
            grid_node<D>(P, pa.acc, pa.V, nullptr, true, n, i, c);
        });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
        StepArgs a = pa.base;
        a.s_in = pa.st[k & 1];
        a.s_out = pa.st[(k + 1) & 1];
        a.V = pa.V;
        a.n_g2p = n;
        a.n_p2g = n + 1;
        const bool p2g = n + 1 < pa.T;
        a.acc = p2g ? pa.acc : nullptr;
        if (LISTS && p2g) a.blk = n + 1 < pa.s1 ? pa.blk : pa.blk_next;
        if (n + 1 < pa.s1)
            particle_phase(P, [&](int p) { forward_particle<D, true, true, false, false, false, false>(P, a, p, sm); });
        else if (p2g)
            particle_phase(P, [&](int p) { forward_particle<D, true, true, true, false, false, false>(P, a, p, sm); });
        else
            particle_phase(P, [&](int p) { forward_particle<D, true, false, true, false, false, false>(P, a, p, sm); });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
    }
}

// ---------------------------------------------------------------------------
// recomputation of a segment, storing every state and grid
// ---------------------------------------------------------------------------
// state k at state + k S, accumulator and velocity of substep s0 + k at
// acc + k G and V + k G.
template <int D, bool LISTS>
__global__ void __launch_bounds__(256, kPersistBlocks)
    k_persist_store(Params P, PersistArgs pa) {
    extern __shared__ float4 s_warp[];
    float4* sm = s_warp + (threadIdx.x >> 5) * warp_slots<D, true>();
    int* err = pa.base.err;
    const int Ks = pa.s1 - pa.s0;
    {
        StepArgs a = pa.base;
        a.s_in = pa.state;
        a.acc = pa.acc;
        a.n_p2g = pa.s0;
        if (LISTS) a.blk = pa.blk;
        particle_phase(P, [&](int p) { forward_particle<D, false, true, false, false, false, false>(P, a, p, sm); });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
    }
    for (int k = 0; k < Ks; ++k) {
        const int n = pa.s0 + k;
        const bool p2g = k + 1 < Ks;
        float4* acc_k = pa.acc + pa.G * k;
        float4* V_k = pa.V + pa.G * k;
        float4* acc_next = p2g ? acc_k + pa.G : nullptr;
        // over every node, the next accumulator is cleared here; the lists
        // find it zero already
        grid_phase<D, LISTS>(P, pa.blk, [&](long long i, const int (&c)[D]) {
            grid_node<D>(P, acc_k, V_k, LISTS ? nullptr : acc_next, false, n, i, c);
        });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
        StepArgs a = pa.base;
        a.s_in = pa.state + pa.S * k;
        a.s_out = pa.state + pa.S * (k + 1);
        a.V = V_k;
        a.n_g2p = n;
        a.n_p2g = n + 1;
        a.acc = acc_next;
        if (LISTS && p2g) a.blk = pa.blk;
        if (p2g)
            particle_phase(P, [&](int p) { forward_particle<D, true, true, true, false, false, false>(P, a, p, sm); });
        else
            particle_phase(P, [&](int p) { forward_particle<D, true, false, true, false, false, false>(P, a, p, sm); });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
    }
}

// ---------------------------------------------------------------------------
// adjoint of a segment (its recomputation stored every state and grid)
// ---------------------------------------------------------------------------
// G2P^T of the last substep; then per substep in reverse the grid adjoint and
// P2G^T of n with G2P^T of n - 1; then the grid adjoint and P2G^T of s0.  The
// particle adjoint of the segment end is in pa.base.adj on entry.
template <int D, bool LISTS>
__global__ void __launch_bounds__(256, kPersistBlocks) k_persist_adjoint(Params P, PersistArgs pa) {
    extern __shared__ float4 s_warp[];
    float4* sm = s_warp + (threadIdx.x >> 5) * warp_slots<D, true>();
    int* err = pa.base.err;
    const int Ks = pa.s1 - pa.s0;
    {
        StepArgs a = pa.base;
        a.s_in = pa.state + pa.S * Ks;
        a.s_aux = pa.state + pa.S * (Ks - 1);
        a.n_p2g = pa.s1;
        a.V = pa.V + pa.G * (Ks - 1);
        particle_phase(P, [&](int p) { adjoint_particle<D, false, true, false, false, false, false, false>(P, a, p, sm); });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
    }
    for (int k = Ks - 1; k >= 0; --k) {
        const int n = pa.s0 + k;
        const float4* acc_k = pa.acc + pa.G * k;
        grid_phase<D, LISTS>(P, pa.blk, [&](long long i, const int (&c)[D]) {
            grid_adjoint_node<D>(P, acc_k, pa.base.Vbar, const_cast<float4*>(pa.base.gadj), n, i, c);
        });
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
        StepArgs a = pa.base;
        a.s_in = pa.state + pa.S * k;
        a.n_p2g = n;
        if (k >= 1) {
            a.s_aux = pa.state + pa.S * (k - 1);
            a.V = pa.V + pa.G * (k - 1);
            particle_phase(P, [&](int p) { adjoint_particle<D, true, true, false, false, false, false, false>(P, a, p, sm); });
        } else {
            particle_phase(P, [&](int p) { adjoint_particle<D, true, false, false, false, false, false, false>(P, a, p, sm); });
        }
        if (!grid_barrier(pa.bar, pa.spin_limit, err)) return;
    }
}

// Resident CTAs per SM of a persistent kernel, for `block` threads with the
// dynamic shared memory it takes.
template <typename K>
int resident(K kernel, int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <typename K>
cudaError_t launch_cooperative(K kernel, int ctas, int block, size_t smem, cudaStream_t st, const Params& P,
                               const PersistArgs& pa) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, P, pa);
}

}  // namespace

template <int D>
cudaError_t launch_persist_dim(PersistKind kind, bool lists, const Params& P, const PersistArgs& pa, int block,
                               int max_ctas, cudaStream_t st) {
    const size_t smem = (size_t)((block + 31) / 32) * warp_slots<D, true>() * sizeof(float4);
    auto go = [&](auto kernel) -> cudaError_t {
        const int per_sm = resident(kernel, block, smem);
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long cap = (long long)per_sm * sms;
        if (cap < 1) return cudaErrorCooperativeLaunchTooLarge;
        const long long want = std::max<long long>(1, (P.n_total + block - 1) / block);
        const int ctas = (int)std::min<long long>(std::min<long long>(cap, want), max_ctas > 0 ? max_ctas : cap);
        if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch_cooperative(kernel, ctas, block, smem, st, P, pa);
    };
    // 3D walks the node-block lists, 2D every node (its grids are small)
    constexpr bool L = D == 3;
    if (lists != L) return cudaErrorInvalidValue;
    switch (kind) {
        case PersistKind::kLean: return go(k_persist_lean<D, L>);
        case PersistKind::kStore: return go(k_persist_store<D, L>);
        default: return go(k_persist_adjoint<D, L>);
    }
}

}  // namespace mpm
