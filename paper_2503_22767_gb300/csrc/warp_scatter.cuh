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
// same-address updates.  Here the lanes of one base node (found with one
// __match_any_sync) sum their contributions in shared memory first, slab by
// slab of kAggSlab stencil nodes: every lane writes its node values, then the
// j-th lane of a group of g sums nodes j, j + g, ... of the slab over the
// group (in lane order) and issues one atomic per node.  A group of one
// issues exactly the per-lane atomics.
// ---------------------------------------------------------------------------
// Nodes per slab: 8, so that a group of 8 lanes (8 particles per cell in 3D)
// sums one node per lane and slab (27 = 8 + 8 + 8 + 3).  A lane's slots are 9
// float4 apart (144 bytes, 36 banks): the 8 lanes of one quarter-warp store
// then hit disjoint banks, where a 128-byte stride would put all on the same 4.
constexpr int kAggSlab = 8;
constexpr int kAggStride = 9;
constexpr int kAggSlots = kAggStride * 32;  // float4 per warp

// 3D only: with 4 particles per cell in 2D the exchange cost more than the
// atomics it saved on every 2D workload measured (2D locomotion 15.8 -> 17.4
// ms per design iteration); in 3D it took the forward kernel from 98 to 59 us
// per launch (600,000 particles).
template <int D>
__host__ __device__ constexpr bool aggregate_scatter() {
    return D == 3;
}

// float4 slots of dynamic shared memory per warp of a particle kernel that
// runs the aggregated scatter (none otherwise)
template <int D, bool SCATTER>
__host__ __device__ constexpr int warp_slots() {
    return SCATTER && aggregate_scatter<D>() ? kAggSlots : 0;
}

// Every lane of the warp calls this; a lane without a particle passes
// active = false (its values are not read).  value(k) gives the float4 that
// stencil node k (last axis fastest) receives from this lane's particle; it
// is called with every k < 3^D.  grid is the instance's grid, nb the base
// node, sm this warp's kAggSlots slots.
template <int D, typename Value>
__device__ __forceinline__ void scatter_aggregated(int nb, int inst, bool active, float4* __restrict__ grid, int res,
                                                   float4* sm, Value value) {
    const int lane = threadIdx.x & 31;
    // instances are < 2^16 and node indices < 2^31, so no active key is ~0 - lane
    const unsigned long long key =
        active ? (((unsigned long long)(unsigned)inst << 32) | (unsigned)nb) : ~0ull - (unsigned)lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int g = __popc(peers);
    const int j = __popc(peers & ((1u << lane) - 1u));
    float4* mine = sm + lane * kAggStride;
    constexpr int kNodes = D == 3 ? 27 : 9;
#pragma unroll
    for (int k0 = 0; k0 < kNodes; k0 += kAggSlab) {
        const int nk = kNodes - k0 < kAggSlab ? kNodes - k0 : kAggSlab;  // nodes in this slab
        __syncwarp();  // the slots' earlier readers are done
#pragma unroll
        for (int n = 0; n < kAggSlab; ++n)
            if (n < nk) mine[n] = value(k0 + n);
        __syncwarp();
        if (active) {
            for (int n = j; n < nk; n += g) {
                // the sum in lane order, two components per packed add
                float2 a01 = make_float2(0.0f, 0.0f), a23 = make_float2(0.0f, 0.0f);
                auto add = [&](const float4& c) {
                    a01 = __fadd2_rn(a01, make_float2(c.x, c.y));
                    a23 = __fadd2_rn(a23, make_float2(c.z, c.w));
                };
                // (a version that summed consecutive-lane groups at fixed offsets,
                // unrolled, ran 7 us slower per 3D forward launch)
                for (unsigned q = peers; q; q &= q - 1u) add(sm[(__ffs(q) - 1) * kAggStride + n]);
                const float4 acc = make_float4(a01.x, a01.y, a23.x, a23.y);
                const int k = k0 + n;
                const int off = D == 3 ? ((k / 9) * res + (k / 3) % 3) * res + k % 3 : (k / 3) * res + k % 3;
                atomicAdd(grid + nb + off, acc);
            }
        }
    }
}

}  // namespace mpm
