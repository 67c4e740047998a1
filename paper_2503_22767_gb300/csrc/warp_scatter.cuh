// Warp-aggregated stencil scatter of the 3D particle kernels (the P2G of the
// forward kernel, the G2P^T of the adjoint kernel).
#pragma once

#include "mpm_device.cuh"

namespace mpm {

// ---------------------------------------------------------------------------
// Aggregated stencil scatter (the P2G of the forward kernel, the G2P^T of the
// adjoint kernel).
//
// The cell-sorted particles of one cell (8 per cell in 3D at the
// configurations' densities) share their base node, and so every stencil
// node; issued one per lane, their float4 atomics reach L2 as separate
// same-address updates.  Here the lanes of one base node (a group, found with
// one __match_any_sync) sum their contributions in shared memory first, slab
// by slab of kAggSlab stencil nodes: every lane writes its node values, then
// each quarter-warp takes one group and sums the group's value of one slab
// node per lane (in lane order), and issues one atomic per node.  A warp with
// G groups thus needs ceil(G / 4) passes per slab, whatever the group sizes:
// once a deforming body leaves cells with uneven particle counts, a warp holds
// groups of 1 to 15 lanes, and the pass count no longer follows the smallest
// group (with a group of one lane, one lane summing every node of the slab
// for its group took eight passes).  A group of one issues exactly the
// per-lane atomics.
// ---------------------------------------------------------------------------
// Nodes per slab: 8, one per lane of a quarter-warp (27 = 8 + 8 + 8 + 3).  A
// lane's slots are 9 float4 apart (144 bytes, 36 banks), so the 8 lanes of a
// quarter-warp storing their values hit disjoint banks, and a quarter-warp
// summing one group reads 8 consecutive float4 of one lane's slots.
constexpr int kAggSlab = 8;
constexpr int kAggStride = 9;
constexpr int kAggValueSlots = kAggStride * 32;  // float4 of node values per warp
// after the values: per group, its lanes (32 x unsigned) and the element
// offset of its base node from grid0 (32 x long long): 384 bytes = 24 float4
constexpr int kAggTableSlots = 24;
constexpr int kAggSlots = kAggValueSlots + kAggTableSlots;  // float4 per warp

// Always in 3D (the forward kernel went from 98 to 59 us per launch on
// 600,000 particles).  In 2D, with 4 particles per cell, it pays only for
// large launches: the forward P2G of the 64-walker batch (1.5M particles) went
// from 81 to 72 us, while the single 30,000-particle walker lost 10% per
// design iteration and the 2D G2P^T lost on both.  2D P2G takes it per handle
// (Params::agg2, chosen by the autotuner); 2D G2P^T never does.
template <int D>
__host__ __device__ constexpr bool aggregate_scatter() {
    return D == 3;
}

// float4 slots of dynamic shared memory per warp of a particle kernel whose
// scatter is aggregated (AGG), none otherwise
template <int D, bool SCATTER, bool AGG = aggregate_scatter<D>()>
__host__ __device__ constexpr int warp_slots() {
    return SCATTER && AGG ? kAggSlots : 0;
}

// Offset of stencil node k (last axis fastest, k < 3^D) from the base node on
// a grid of res nodes per axis (res2 = res^2): k / 9, (k / 3) % 3 and k % 3
// by multiply and shift (exact for k < 27).
template <int D>
__device__ __forceinline__ int stencil_node_offset(int k, int res, int res2) {
    if (D == 3) {
        const int a0 = (k * 57) >> 9, r = k - 9 * a0;
        const int a1 = (r * 11) >> 5;
        return a0 * res2 + a1 * res + (r - 3 * a1);
    }
    const int a0 = (k * 11) >> 5;
    return a0 * res + (k - 3 * a0);
}

// Every lane of the warp calls this; a lane without a particle passes
// active = false (its values are not read).  value(k) gives the float4 that
// stencil node k (last axis fastest) receives from this lane's particle; it
// is called with every k < 3^D.  grid0 is instance 0's grid (instance i's
// starts nodes further on each), nb the base node, sm this warp's kAggSlots
// slots.  (The atomics address grid0 plus an offset read from the group
// table, so that they stay global-memory atomics.)
template <int D, typename Value>
__device__ __forceinline__ void scatter_aggregated(int nb, int inst, bool active, float4* __restrict__ grid0,
                                                   long long nodes, int res, float4* sm, Value value) {
    const int lane = threadIdx.x & 31;
    // instances are < 2^16 and node indices < 2^31, so no active key is ~0 - lane
    const unsigned long long key =
        active ? (((unsigned long long)(unsigned)inst << 32) | (unsigned)nb) : ~0ull - (unsigned)lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    // the groups of active lanes, numbered by their lowest lane
    const bool leader = active && lane == __ffs(peers) - 1;
    const unsigned leaders = __ballot_sync(0xffffffffu, leader);
    const int G = __popc(leaders);
    unsigned* g_lanes = reinterpret_cast<unsigned*>(sm + kAggValueSlots);
    long long* g_base = reinterpret_cast<long long*>(g_lanes + 32);
    __syncwarp();  // the table's readers in an earlier call are done
    if (leader) {
        const int gi = __popc(leaders & ((1u << lane) - 1u));
        g_lanes[gi] = peers;
        g_base[gi] = (long long)inst * nodes + nb;
    }
    float4* mine = sm + lane * kAggStride;
    constexpr int kNodes = D == 3 ? 27 : 9;
    const int res2 = res * res;
#pragma unroll
    for (int k0 = 0; k0 < kNodes; k0 += kAggSlab) {
        const int nk = kNodes - k0 < kAggSlab ? kNodes - k0 : kAggSlab;  // nodes in this slab
        __syncwarp();  // the slots' earlier readers are done
#pragma unroll
        for (int n = 0; n < kAggSlab; ++n)
            if (n < nk) mine[n] = value(k0 + n);
        __syncwarp();
        // item t = (group t / nk, slab node t % nk): a quarter-warp per group
        // in full slabs
        for (int t = lane; t < G * nk; t += 32) {
            const int gi = t / nk, n = t - gi * nk;
            const unsigned pm = g_lanes[gi];
            // the sum in lane order, two components per packed add
            float2 a01 = make_float2(0.0f, 0.0f), a23 = make_float2(0.0f, 0.0f);
            for (unsigned q = pm; q; q &= q - 1u) {
                const float4 c = sm[(__ffs(q) - 1) * kAggStride + n];
                a01 = __fadd2_rn(a01, make_float2(c.x, c.y));
                a23 = __fadd2_rn(a23, make_float2(c.z, c.w));
            }
            atomicAdd(grid0 + (g_base[gi] + stencil_node_offset<D>(k0 + n, res, res2)),
                      make_float4(a01.x, a01.y, a23.x, a23.y));
        }
    }
}

}  // namespace mpm
