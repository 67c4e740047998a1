// Warp-cooperative staging of grid nodes for the particle gathers (G2P,
// P2G^T, G2P^T).
//
// The 32 cell-sorted particles of a warp have base cells in a small box: the
// sort orders cells block by block, with the last axis fastest.  A warp
// typically holds one row of 4 (3D) or 8 (2D) cells, so its 27- / 9-node
// stencils touch ~54 / ~30 distinct nodes instead of 864 / 288 node reads.
// The warp loads the box's nodes once into its own shared-memory slots, four
// float4 loads per lane that are all in flight together.  Each lane then reads
// its stencil from shared memory.  A thread otherwise pays one L2 round trip
// per few gathers, limited by the registers that in-flight loads need.
//
// The box has a fixed shape of 2^box_log(a) nodes per axis, 128 nodes in all:
// 8 x 16 in 2D and 4 x 4 x 8 in 3D.  A warp whose stencils do not fit it, or
// whose particles belong to more than one instance, gathers directly from
// global memory, with the same results.
#pragma once

#include <climits>

#include "mpm_device.cuh"

namespace mpm {

template <int D>
__host__ __device__ constexpr int box_log(int a) {
    return D == 2 ? (a == 0 ? 3 : 4) : (a == D - 1 ? 3 : 2);
}

template <int D>
__host__ __device__ constexpr int box_nodes() {
    return 128;
}

constexpr int kBoxWarps = 8;  // warps per block (blocks of at most 256 threads)

template <int D>
struct WarpBox {
    int lo[D];   // first node per axis
    int ext[D];  // nodes per axis that some stencil of the warp touches
    int inst;    // instance of every active lane (when use)
    bool use;    // warp-uniform: stage the box, else gather directly
};

// With enable, every lane of the warp must call this (base cells of active
// lanes count).  enable must be warp-uniform; without it nothing is exchanged
// and the box is not used, so a partly active warp may call it inside a branch.
template <int D>
__device__ __forceinline__ WarpBox<D> warp_box(const int (&base)[D], bool active, int inst, bool enable) {
    const unsigned full = 0xffffffffu;
    WarpBox<D> b;
    b.use = false;
    b.inst = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) b.lo[a] = b.ext[a] = 0;
    if (!enable) return b;
    bool fit = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int lo = __reduce_min_sync(full, active ? base[a] : INT_MAX);
        const int hi = __reduce_max_sync(full, active ? base[a] : INT_MIN);
        const bool any = lo <= hi;
        b.lo[a] = any ? lo : 0;
        b.ext[a] = any ? hi - lo + 3 : 0;
        fit = fit && any && b.ext[a] <= (1 << box_log<D>(a));
    }
    const int i0 = __reduce_min_sync(full, active ? inst : INT_MAX);
    const int i1 = __reduce_max_sync(full, active ? inst : INT_MIN);
    b.inst = i0;
    b.use = fit && i0 == i1;
    return b;
}

// Slot of node coordinates c in the box (c inside the box).
template <int D>
__device__ __forceinline__ int box_slot(const WarpBox<D>& b, const int (&c)[D]) {
    int i = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) i = (i << box_log<D>(a)) | (c[a] - b.lo[a]);
    return i;
}

// Slot of stencil node k relative to the slot of the stencil's base node
// (every stencil node of a lane lies inside the box when it is used, so the
// per-axis fields never carry into each other).
template <int D>
__device__ __forceinline__ constexpr int box_offset(int k) {
    return D == 2 ? ((k / 3) << box_log<D>(1)) + k % 3
                  : ((k / 9) << (box_log<D>(1) + box_log<D>(2))) + (((k / 3) % 3) << box_log<D>(2)) + k % 3;
}

// Every lane of the warp: fill this warp's slots `sm` with load(c, node) for
// the box nodes inside the touched extent.  node is the index within the
// instance grid.  The other slots are left as they are and never read.
template <int D, typename Load>
__device__ __forceinline__ void stage_box(const WarpBox<D>& b, int res, float4* sm, Load load) {
    const int lane = threadIdx.x & 31;
    __syncwarp();  // earlier reads of these slots are done
#pragma unroll
    for (int t0 = 0; t0 < box_nodes<D>(); t0 += 32) {
        const int t = t0 + lane;
        int c[D], rem = t;
        bool in = true;
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
            const int r = rem & ((1 << box_log<D>(a)) - 1);
            rem >>= box_log<D>(a);
            c[a] = b.lo[a] + r;
            in = in && r < b.ext[a];
        }
        if (in) {
            int node = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) node = node * res + c[a];
            sm[t] = load(c, node);
        }
    }
    __syncwarp();
}

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
// stages gather boxes and, with scatter, runs the aggregated scatter
template <int D, bool SCATTER>
__host__ __device__ constexpr int warp_slots() {
    return SCATTER && aggregate_scatter<D>() ? kAggSlots : box_nodes<D>();
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
                float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                for (unsigned q = peers; q; q &= q - 1u) {
                    const float4 c = sm[(__ffs(q) - 1) * kAggStride + n];
                    acc.x += c.x;
                    acc.y += c.y;
                    acc.z += c.z;
                    acc.w += c.w;
                }
                const int k = k0 + n;
                const int off = D == 3 ? ((k / 9) * res + (k / 3) % 3) * res + k % 3 : (k / 3) * res + k % 3;
                atomicAdd(grid + nb + off, acc);
            }
        }
    }
}

}  // namespace mpm
