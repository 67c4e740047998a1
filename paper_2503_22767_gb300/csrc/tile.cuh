// Shared-memory grid tiles for the transfer kernels.
//
// A CTA processes a contiguous range of cell-sorted particles, so their
// stencils cover a small box of grid nodes. The CTA stages that box in
// shared memory:
//   - gathers (G2P, P2G^T) read node values from the tile instead of 9 / 27
//     scattered L2 loads per particle, and the grid operation (or its
//     reverse) runs once per tile node instead of once per particle-node pair;
//   - scatters (P2G, G2P^T) first sum the contributions of lanes that share a
//     cell with warp shuffles, then add them into the tile with shared-memory
//     atomics, and finally flush every non-zero tile node to global memory with
//     one float4 atomic.
// A CTA whose box exceeds kTileMax nodes, or whose particles belong to more
// than one instance, uses the direct global path (same results).
#pragma once

#include <climits>

#include "mpm_device.cuh"

namespace mpm {

constexpr int kTileMax = 1024;  // nodes per tile (16 KB of float4)

template <int D>
struct TileBox {
    int lo[D];   // first node coordinate per axis
    int ext[D];  // node extent per axis (cell range + 2)
    int n;       // nodes in the box
    int use;     // 1: tile path; 0: direct global path
    int inst;    // instance of every particle in the CTA (tile path)
};

// Block-wide box of the stencils whose base cells are `base` (active lanes).
// Every thread of the block must call it; `red` holds (2D + 2) * 32 ints.
template <int D>
__device__ __forceinline__ void block_box(const int (&base)[D], bool active, int inst,
                                          TileBox<D>& box, int* red, TileBox<D>* s_box) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int vmin[D + 1], vmax[D + 1];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        vmin[a] = active ? base[a] : INT_MAX;
        vmax[a] = active ? base[a] : INT_MIN;
    }
    vmin[D] = active ? inst : INT_MAX;
    vmax[D] = active ? inst : INT_MIN;
#pragma unroll
    for (int a = 0; a <= D; ++a) {
        vmin[a] = __reduce_min_sync(full, vmin[a]);
        vmax[a] = __reduce_max_sync(full, vmax[a]);
    }
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a <= D; ++a) {
            red[a * 32 + warp] = vmin[a];
            red[(D + 1 + a) * 32 + warp] = vmax[a];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int lo[D + 1], hi[D + 1];
#pragma unroll
        for (int a = 0; a <= D; ++a) {
            lo[a] = INT_MAX;
            hi[a] = INT_MIN;
            for (int w = 0; w < nw; ++w) {
                lo[a] = min(lo[a], red[a * 32 + w]);
                hi[a] = max(hi[a], red[(D + 1 + a) * 32 + w]);
            }
        }
        TileBox<D> b;
        if (lo[D] > hi[D]) {  // no active particle
            b.n = 0;
            b.use = 1;
            b.inst = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                b.lo[a] = 0;
                b.ext[a] = 0;
            }
        } else {
            long long n = 1;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                b.lo[a] = lo[a];
                b.ext[a] = hi[a] - lo[a] + 3;
                n *= b.ext[a];
            }
            b.use = (n <= kTileMax && lo[D] == hi[D]) ? 1 : 0;
            b.n = b.use ? (int)n : 0;
            b.inst = lo[D];
        }
        *s_box = b;
    }
    __syncthreads();
    box = *s_box;
}

// position of node coordinates c inside the box
template <int D>
__device__ __forceinline__ int box_index(const TileBox<D>& b, const int (&c)[D]) {
    int i = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) i = i * b.ext[a] + (c[a] - b.lo[a]);
    return i;
}

// node coordinates of box position t
template <int D>
__device__ __forceinline__ void box_coords(const TileBox<D>& b, int t, int (&c)[D]) {
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
        c[a] = b.lo[a] + t % b.ext[a];
        t /= b.ext[a];
    }
}

template <int D>
__device__ __forceinline__ long long grid_index(const int (&c)[D], int res) {
    long long i = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) i = i * res + c[a];
    return i;
}

// Runs of consecutive lanes with equal keys (cell-sorted particles sharing a
// base cell).  After seg_sum, the first lane of every run holds the run total.
struct Segments {
    int end;     // last lane of this lane's run
    int rounds;  // shuffle rounds covering the longest run in the warp
    bool head;   // first lane of its run
};

__device__ __forceinline__ Segments make_segments(int key) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(full, key, 1);
    Segments s;
    s.head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(full, s.head);
    const unsigned after = heads & ~((2u << lane) - 1u);  // heads after this lane
    const int next = after ? __ffs(after) - 1 : 32;
    s.end = next - 1;
    const int len = s.head ? next - lane : 0;
    const int maxlen = __reduce_max_sync(full, len);
    int r = 0;
    while ((1 << r) < maxlen) ++r;
    s.rounds = r;
    return s;
}

__device__ __forceinline__ float seg_sum(float v, const Segments& s) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < s.rounds; ++r) {
        const int off = 1 << r;
        const float y = __shfl_down_sync(0xffffffffu, v, off);
        if (lane + off <= s.end) v += y;
    }
    return v;
}

// every thread of the block: add tile nodes [0, box.n) into grid (float4 atomics)
template <int D>
__device__ __forceinline__ void flush_tile(const TileBox<D>& box, const float4* tile, float4* grid,
                                           const Params& P) {
    float4* g = grid + (long long)box.inst * P.nodes;
    for (int t = threadIdx.x; t < box.n; t += blockDim.x) {
        const float4 v = tile[t];
        if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f) {
            int c[D];
            box_coords<D>(box, t, c);
            atomicAdd(g + grid_index<D>(c, P.res), v);
        }
    }
}

}  // namespace mpm
