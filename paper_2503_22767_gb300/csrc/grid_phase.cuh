// Per-node grid operation (Eq. 16-18) and its reverse, shared by the grid
// kernels (kernels_step.cu) and the persistent passes (kernels_persist.cuh).
// Grids are one float4 per node, [inst][node]: accumulators (m, m v),
// velocities (v, 0), adjoints (mbar, mvbar).
#pragma once

#include "particle_io.cuh"

namespace mpm {

// Node i of the [inst][node] grids, local index `local` within its instance
// grid: V = the grid operation of acc (zero without mass: Eq. 16 gives no
// velocity); clear_acc zeroes acc, acc_next (or null) is zeroed too.
template <int D>
__device__ __forceinline__ void grid_node(const Params& P, float4* __restrict__ acc, float4* __restrict__ V,
                                          float4* __restrict__ acc_next, bool clear_acc, int step, long long i,
                                          const int (&c)[D]) {
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 g = acc[i];
    float4 out = zero;
    if (g.x > 0.0f) {
        float mv[D], v[D];
        unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mv);
        grid_velocity<D>(P, c, g.x, mv, v, step);
        out = make_float4(v[0], v[1 % D], D == 3 ? v[2 % D] : 0.0f, 0.0f);
    }
    V[i] = out;
    if (clear_acc) acc[i] = zero;
    if (acc_next) acc_next[i] = zero;
}

// The reverse at node i: Vbar -> (mbar, mvbar) in gadj, Vbar zeroed (nodes
// without mass pass no gradient).
template <int D>
__device__ __forceinline__ void grid_adjoint_node(const Params& P, const float4* __restrict__ acc,
                                                  float4* __restrict__ Vbar, float4* __restrict__ gadj, int step,
                                                  long long i, const int (&c)[D]) {
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 g = acc[i];
    float4 out = zero;
    if (g.x > 0.0f) {
        float mv[D], vb[D], mvb[D], mb;
        unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mv);
        unpack3<D>(Vbar[i], vb);
        grid_velocity_adjoint<D>(P, c, g.x, mv, vb, mb, mvb, step);
        out = pack4<D>(mb, mvb);
    }
    Vbar[i] = zero;
    gadj[i] = out;
}

// Node t (0..63) of listed block b (3D, blocks of kBlockEdge^3 nodes).
struct BlockNode {
    long long i;  // node index in the [inst][node] grid
    int c[3];     // node coordinates
    bool in;      // inside the grid (res need not be a multiple of the block edge)
};

__device__ __forceinline__ BlockNode block_node(const Params& P, int b, int t) {
    const int nb = blocks_per_axis(P.res);
    const int bpi = nb * nb * nb;
    const int inst = b / bpi, lb = b - inst * bpi;
    BlockNode n;
    n.c[0] = (lb / (nb * nb)) * kBlockEdge + (t >> 4);
    n.c[1] = ((lb / nb) % nb) * kBlockEdge + ((t >> 2) & 3);
    n.c[2] = (lb % nb) * kBlockEdge + (t & 3);
    n.in = n.c[0] < P.res && n.c[1] < P.res && n.c[2] < P.res;
    n.i = (long long)inst * P.nodes + ((long long)n.c[0] * P.res + n.c[1]) * P.res + n.c[2];
    return n;
}

}  // namespace mpm
