// Particle-array access shared by the transfer kernels.
//
// Particle arrays are structure-of-arrays with component stride P.np:
// x[D], v[D], C[D][D], E[D][D] (row-major), 2D + 2D^2 components, where
// E = F - I is the strain form of the deformation gradient.  Grids are one
// float4 per node.
#pragma once

#include <utility>

#include "kernels.h"

namespace mpm {

// Launch a per-substep kernel; with P.pdl the launch allows programmatic
// dependent launch (the kernel begins with pdl_wait()).
// launch_chain_smem also gives the launch smem bytes of dynamic shared memory.
template <typename... KArgs, typename... Args>
cudaError_t launch_chain_smem(const Params& P, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = P.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chain(const Params& P, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                         cudaStream_t st, Args&&... args) {
    return launch_chain_smem(P, kernel, grid, block, 0, st, std::forward<Args>(args)...);
}

template <int D>
struct Layout {
    // F slot holds E = F - I
    static constexpr int X = 0, V = D, C = 2 * D, F = 2 * D + D * D, N = 2 * D + 2 * D * D;
};

template <int D>
__device__ __forceinline__ float4 pack4(float a, const float (&v)[D]) {
    return make_float4(a, v[0], v[1 % D], D == 3 ? v[2 % D] : 0.0f);
}

template <int D>
__device__ __forceinline__ void unpack3(const float4& g, float (&v)[D]) {
    v[0] = g.x;
    v[1 % D] = g.y;
    if (D == 3) v[2 % D] = g.z;
}

// A load that stays where it is written (asm volatile, so it is neither
// merged with an earlier load of the same address nor moved): reloading a
// value after a long stretch of code frees its registers in between.
__device__ __forceinline__ float reload(const float* p) {
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <int D>
__device__ __forceinline__ void reload_mat(const float* __restrict__ s, int base, long long np, int p,
                                           float (&M)[D][D]) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) M[a][b] = reload(s + (long long)(base + a * D + b) * np + p);
}

// The particle state is read once per kernel (a streaming read, evict-first),
// so that it does not push the stencil nodes the gathers reuse out of L1
// (3D locomotion, 1M particles: forward 97.6 -> 95.2 us per launch).
template <int D>
__device__ __forceinline__ void load_vec(const float* __restrict__ s, int base, long long np, int p,
                                         float (&v)[D]) {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = __ldcs(s + (long long)(base + a) * np + p);
}

// Position of particle p: the X slot of the state plus x0 (the state holds
// the displacement u = x - x0; x0 null: the slot holds x itself).
template <int D>
__device__ __forceinline__ void load_position(const float* __restrict__ s, const float* __restrict__ x0,
                                              long long np, int p, float (&x)[D]) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float u = __ldcs(s + (long long)a * np + p);
        x[a] = x0 ? __fadd_rn(u, __ldg(x0 + (long long)a * np + p)) : u;
    }
}

template <int D>
__device__ __forceinline__ void load_mat(const float* __restrict__ s, int base, long long np, int p,
                                         float (&M)[D][D]) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) M[a][b] = __ldcs(s + (long long)(base + a * D + b) * np + p);
}

template <int D>
__device__ __forceinline__ void store_vec(float* __restrict__ s, int base, long long np, int p,
                                          const float (&v)[D]) {
#pragma unroll
    for (int a = 0; a < D; ++a) s[(long long)(base + a) * np + p] = v[a];
}

template <int D>
__device__ __forceinline__ void store_mat(float* __restrict__ s, int base, long long np, int p,
                                          const float (&M)[D][D]) {
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) s[(long long)(base + a * D + b) * np + p] = M[a][b];
}

constexpr int kStencil2 = 9, kStencil3 = 27;
template <int D>
constexpr int stencil_size() { return D == 2 ? kStencil2 : kStencil3; }

// ---------------------------------------------------------------------------
// forward particle kernel
// ---------------------------------------------------------------------------
// Clears a.zero4 (grid-stride over the whole launch); fused mode only.
__device__ __forceinline__ void clear_buffer(const StepArgs& a) {
    if (a.zero4 == nullptr) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.zero_n; i += stride)
        a.zero4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Grid velocity at a stencil node: read V (separate grid kernel) or apply
// the grid operation (Eq. 16-18) to the node's accumulator (fused).
template <int D, bool FUSE, bool BOXES = true>
__device__ __forceinline__ void node_velocity(const float4* __restrict__ grid, const NodeTerm<D>& t,
                                              const Params& P, float (&gv)[D], int step) {
    const float4 g = __ldg(grid + t.node);
    if (FUSE) {
        float mv[D];
        unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mv);
        grid_velocity<D, BOXES>(P, t.c, g.x, mv, gv, step);
    } else {
        unpack3<D>(g, gv);
    }
}

}  // namespace mpm
