// Device building blocks of the magneto-elastic MLS-MPM substep (sm_103a).
//
// Templated on the spatial dimension D (2 or 3).  Everything here is
// single-precision and register-resident; the kernels that use it live in
// particle_kernels.cuh and kernels_step.cu.  Equations refer to arxiv 2503.22767.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

namespace mpm {

constexpr float kMu0 = 1.25663706143591729e-6f;  // vacuum permeability 4 pi 1e-7

enum ErrBits : int { kErrNumeric = 1, kErrDomain = 2, kErrTimeout = 4 };

// Scalar parameters every kernel receives by value.
struct Params {
    int res;         // nodes per axis
    int bound;       // wall band width in nodes
    int wall_mode;   // 0 all non-slip, 1 Coulomb floor on axis 1 (low side)
    int loss_kind;   // 0 shape MSE (Eq. 38), 1 locomotion (Eq. 40)
    int simp_q;      // SIMP exponent (Eq. 31)
    int n_inst;      // instances
    int n_steps;     // horizon N
    int n_total;     // particles (all instances)
    long long np;    // stride between SoA components of particle arrays
    long long nodes; // nodes per instance grid (res^D)
    float dx, inv_dx, dt, kappa;  // kappa = 4/dx^2 (inverse B-spline inertia)
    float p_vol, rho0, G, K, eps, damping, mu;
    float gravity[3];
    int pdl;  // per-substep kernels launched with programmatic dependent launch
    int adj_blocks;  // register budget of the adjoint particle kernel: 256-thread blocks per SM (2 or 3)
    int agg2;        // 2D: the fused forward kernel's P2G scatter is aggregated over same-node lanes
    // solid boxes of Eq. 18 beyond the walls and a non-uniform applied field
    // (device memory), or null for neither.  One pointer keeps the parameter
    // block (and the transfer kernels' register allocation) as small as
    // without them.
    const struct Extras* ext;
};

constexpr int kMaxBoundaries = 8;
constexpr int kBoundaryCoulomb = 0, kBoundaryNonSlip = 1, kBoundaryAttached = 2;

struct Boundary {
    int kind;  // kBoundary*
    float mu;  // friction coefficient (Coulomb)
    float lo[3], hi[3];  // axis-aligned box at t = 0
};

struct Extras {
    int n;                        // boxes in use (<= kMaxBoundaries)
    Boundary box[kMaxBoundaries];
    const float* motion;          // per box and substep: offset, velocity v_b
                                  // ([b][n_steps][2][D]), or null for static boxes
    // non-uniform applied field B(x, t_n) = B_a[n] + G[n] (x - x_c), x_c the
    // domain centre: G per instance and substep, [inst][n_steps][D][D]
    // (dB_i/dx_j), or null for a uniform field; gfgrad receives dL/dG
    const float* fgrad;
    float* gfgrad;
};

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor drains; it must wait (here,
// before any global access) until the predecessor's writes are visible.
// Without a programmatic predecessor both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// A hint to bring the line holding *p into L2 (the point of coherence, so it
// is safe for data another kernel may still write); no register is used.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// The same into L1 (data no kernel writes while this one runs).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// ---------------------------------------------------------------------------
// active node blocks (3D): the grid operation and its reverse run only over
// the blocks of kBlockEdge^3 nodes that some particle's stencil touches.
// A list holds the blocks touched during the current checkpoint segment (it
// only grows within the segment).  Each warp of 32 particles keeps the box of
// base cells whose stencils it has listed (wbox); a substep whose particles
// stay inside that box lists nothing, so most substeps cost the warp a few
// reductions and one load.  Warps whose particles moved out of their box
// list the blocks of the enlarged box.
// ---------------------------------------------------------------------------
constexpr int kBlockEdge = 4;

struct ActiveBlocks {
    int* flag = nullptr;   // [n_inst * blocks per instance]: 1 while the block is listed
    int* list = nullptr;   // listed block ids (instance * blocks per instance + block)
    int* count = nullptr;  // number of listed blocks
    int4* wbox = nullptr;  // per warp: lo | (hi + 1) << 16 of the listed base cells per
                           // axis (x, y, z); all zero = nothing listed yet
};

__host__ __device__ __forceinline__ int blocks_per_axis(int res) { return (res + kBlockEdge - 1) / kBlockEdge; }

// Lists block b (on its first marking); every lane of the warp calls this,
// with want = false where it has no block.  The warp appends its new blocks
// with one atomic on the count.
__device__ __forceinline__ void list_blocks(const ActiveBlocks& ab, bool want, int b) {
    // a stale 0 from L1 only costs an atomic; the atomic swap decides
    const bool mine = want && __ldcg(ab.flag + b) == 0 && atomicExch(ab.flag + b, 1) == 0;
    const unsigned m = __ballot_sync(0xffffffffu, mine);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    int first = 0;
    if (lane == __ffs(m) - 1) first = atomicAdd(ab.count, __popc(m));
    first = __shfl_sync(0xffffffffu, first, __ffs(m) - 1);
    if (mine) ab.list[first + __popc(m & ((1u << lane) - 1u))] = b;
}

// The rare part of mark_blocks: list the blocks of the box lo..hi of base
// cells (instance inst, or per lane when the warp spans two instances) and
// record the box as this warp's.  (Inlined: as an out-of-line call its
// calling convention cost the 3D forward kernel 18 us per launch on 1M
// particles, although the call itself is rare.)
__device__ __forceinline__ void mark_blocks_slow(const ActiveBlocks& ab, long long w, bool active, int inst, int i_lo, int i_hi,
                                              const int (&base)[3], const int (&lo)[3], const int (&hi)[3],
                                              int res) {
    const int nb = blocks_per_axis(res);
    if (i_lo != i_hi) {
        // a warp across two instances: each lane lists its own stencil's blocks
        // (one or two blocks per axis), every substep
        for (int c = 0; c < 8; ++c) {
            const int i0 = base[0] / kBlockEdge + (c >> 2), i1 = base[1] / kBlockEdge + ((c >> 1) & 1);
            const int i2 = base[2] / kBlockEdge + (c & 1);
            const bool want = active && i0 <= (base[0] + 2) / kBlockEdge && i1 <= (base[1] + 2) / kBlockEdge &&
                              i2 <= (base[2] + 2) / kBlockEdge;
            list_blocks(ab, want, want ? (inst * nb + i0) * nb * nb + i1 * nb + i2 : 0);
        }
        return;
    }
    const int b0 = lo[0] / kBlockEdge, n0 = (hi[0] + 2) / kBlockEdge - b0 + 1;
    const int b1 = lo[1] / kBlockEdge, n1 = (hi[1] + 2) / kBlockEdge - b1 + 1;
    const int b2 = lo[2] / kBlockEdge, n2 = (hi[2] + 2) / kBlockEdge - b2 + 1;
    const int total = n0 * n1 * n2;
    const int lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        const int i2 = j % n2, i1 = (j / n2) % n1, i0 = j / (n1 * n2);
        list_blocks(ab, j < total, ((i_lo * nb + b0 + i0) * nb + b1 + i1) * nb + b2 + i2);
    }
    if (lane == 0) {
        ab.wbox[w] = make_int4(lo[0] | (hi[0] + 1) << 16, lo[1] | (hi[1] + 1) << 16, lo[2] | (hi[2] + 1) << 16, 0);
    }
}

// Every lane of a warp calls this after its P2G, with the base node of its
// stencil (active: the lane has a particle).  w: the warp's index (its
// particles are 32w .. 32w + 31); stored: its wbox entry.
__device__ __forceinline__ void mark_blocks(const ActiveBlocks& ab, long long w, bool active, int inst,
                                            const int (&base)[3], int res, int4 stored) {
    const unsigned full = 0xffffffffu;
    const int i_lo = __reduce_min_sync(full, active ? inst : INT_MAX);
    const int i_hi = __reduce_max_sync(full, active ? inst : INT_MIN);
    if (i_lo > i_hi) return;  // no particle in this warp
    int lo[3], hi[3];
    const int st[3] = {stored.x, stored.y, stored.z};
    bool covered = i_lo == i_hi;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(full, active ? base[a] : INT_MAX);
        hi[a] = __reduce_max_sync(full, active ? base[a] : INT_MIN);
        covered = covered && st[a] != 0 && lo[a] >= (st[a] & 0xffff) && hi[a] + 1 <= (st[a] >> 16);
    }
    if (covered) return;
    // the box grows to hold the old and the new cells
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (st[a] != 0) {
            lo[a] = min(lo[a], st[a] & 0xffff);
            hi[a] = max(hi[a], (st[a] >> 16) - 1);
        }
    }
    mark_blocks_slow(ab, w, active, inst, i_lo, i_hi, base, lo, hi, res);
}

// Index of the instance owning particle p (instance ranges are contiguous
// and survive the cell sort, whose key starts with the instance).
__device__ __forceinline__ int find_instance(const int* __restrict__ inst_off, int n_inst, int p) {
    int lo = 0, hi = n_inst;  // inst_off[lo] <= p < inst_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(inst_off + mid) <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// quadratic B-spline stencil (Section 2.2 step 1): base = floor(x/dx - 0.5)
// ---------------------------------------------------------------------------
template <int D>
struct Stencil {
    int base[D];
    float r[D];       // x/dx - base, in [0.5, 1.5) for a particle inside the grid
    float w[D][3];    // 1D weights per axis
    float dw[D][3];   // their derivatives with respect to x/dx
};

// Returns false (and clamps the base so every node index stays in range) when
// the particle's stencil leaves the grid or its position is not finite.
template <int D>
__device__ __forceinline__ bool make_stencil(const float (&x)[D], const Params& P, Stencil<D>& s) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float fx = __fmul_rn(x[a], P.inv_dx);
        float fb = floorf(__fsub_rn(fx, 0.5f));
        int b;
        if (fb >= 0.0f && fb <= (float)(P.res - 3)) {
            b = (int)fb;
        } else {
            ok = false;
            b = (fb > 0.0f) ? P.res - 3 : 0;  // NaN lands here too
        }
        float r = fx - (float)b;
        s.base[a] = b;
        s.r[a] = r;
        float u0 = 1.5f - r, u1 = r - 1.0f, u2 = r - 0.5f;
        s.w[a][0] = 0.5f * u0 * u0;
        s.w[a][1] = 0.75f - u1 * u1;
        s.w[a][2] = 0.5f * u2 * u2;
        s.dw[a][0] = -u0;
        s.dw[a][1] = -2.0f * u1;
        s.dw[a][2] = u2;
    }
    return ok;
}

template <int D>
struct NodeTerm {
    int node;        // node index within the instance grid (< 2^31 by configuration check)
    int c[D];        // node coordinates
    float w;         // weight N(x_p - x_i)
    float gw[D];     // d w / d x_p
    float dpos[D];   // x_i - x_p
};

template <int D>
__device__ __forceinline__ void node_term(const Stencil<D>& s, int k, const Params& P, NodeTerm<D>& t) {
    int o[D];
    if (D == 2) {
        o[0] = k / 3;
        o[D - 1] = k % 3;
    } else {
        o[0] = k / 9;
        o[1 % D] = (k / 3) % 3;
        o[D - 1] = k % 3;
    }
    float w = 1.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) w *= s.w[a][o[a]];
    t.w = w;
    int idx = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        float g = s.dw[c][o[c]] * P.inv_dx;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (a != c) g *= s.w[a][o[a]];
        t.gw[c] = g;
        t.dpos[c] = ((float)o[c] - s.r[c]) * P.dx;
        t.c[c] = s.base[c] + o[c];
        idx = idx * P.res + t.c[c];
    }
    t.node = idx;
}

// offset along axis b of stencil node k (node k = (o0, o1[, o2]), last axis fastest);
// a compile-time constant inside unrolled loops over k
template <int D>
__device__ __forceinline__ constexpr int stencil_offset(int k, int b) {
    return D == 2 ? (b == 0 ? k / 3 : k % 3) : (b == 0 ? k / 9 : (b == 1 ? (k / 3) % 3 : k % 3));
}

// a + o d for a stencil offset o in {0, 1, 2}: with o a compile-time
// constant (unrolled stencil loops) this is no instruction, one add or one FMA.
__device__ __forceinline__ float add_offset(float a, int o, float d) {
    return o == 0 ? a : (o == 1 ? a + d : fmaf(2.0f, d, a));
}

// Index of the stencil's base node within the instance grid, and the offset
// of stencil node k from it (last axis fastest).
template <int D>
__device__ __forceinline__ int base_node(const Stencil<D>& s, int res) {
    int idx = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) idx = idx * res + s.base[a];
    return idx;
}

template <int D>
__device__ __forceinline__ int node_offset(int k, int res) {
    return D == 2 ? stencil_offset<D>(k, 0) * res + stencil_offset<D>(k, 1)
                  : (stencil_offset<D>(k, 0) * res + stencil_offset<D>(k, 1)) * res + stencil_offset<D>(k, 2);
}

// ---------------------------------------------------------------------------
// small dense algebra
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ float frob(const float (&A)[D][D], const float (&B)[D][D]) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) s += A[i][j] * B[i][j];
    return s;
}

__device__ __forceinline__ float int_pow(float x, int q) {
    float r = 1.0f;
    for (int i = 0; i < q; ++i) r *= x;
    return r;
}

// det(I + E) - 1, expanded so that small strains keep their digits:
// tr E + (sum of principal 2x2 minors of E) + det E.
template <int D>
__device__ __forceinline__ float det_minus_one(const float (&E)[D][D]) {
    if (D == 2) return E[0][0] + E[1 % D][1 % D] + (E[0][0] * E[1 % D][1 % D] - E[0][1 % D] * E[1 % D][0]);
    const float m2 = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) +
                     (E[0][0] * E[2 % D][2 % D] - E[0][2 % D] * E[2 % D][0]) +
                     (E[1][1] * E[2 % D][2 % D] - E[1][2 % D] * E[2 % D][1]);
    const float d3 = E[0][0] * (E[1][1] * E[2 % D][2 % D] - E[1][2 % D] * E[2 % D][1]) -
                     E[0][1] * (E[1][0] * E[2 % D][2 % D] - E[1][2 % D] * E[2 % D][0]) +
                     E[0][2 % D] * (E[1][0] * E[2 % D][1] - E[1][1] * E[2 % D][0]);
    return E[0][0] + E[1][1] + E[2 % D][2 % D] + m2 + d3;
}

// H = F^{-T} = cofactor(I + E) / J
template <int D>
__device__ __forceinline__ void inv_transpose_of(const float (&E)[D][D], float J, float (&H)[D][D]) {
    float F[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) F[i][j] = E[i][j] + (i == j ? 1.0f : 0.0f);
    const float rJ = 1.0f / J;
    if (D == 2) {
        H[0][0] = F[1 % D][1 % D] * rJ;
        H[0][1 % D] = -F[1 % D][0] * rJ;
        H[1 % D][0] = -F[0][1 % D] * rJ;
        H[1 % D][1 % D] = F[0][0] * rJ;
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                int i1 = (i + 1) % D, i2 = (i + 2) % D, j1 = (j + 1) % D, j2 = (j + 2) % D;
                H[i][j] = (F[i1][j1] * F[i2][j2] - F[i1][j2] * F[i2][j1]) * rJ;
            }
    }
}

// ---------------------------------------------------------------------------
// constitutive model: Piola stress of Eq. 7 under the SIMP weights of Eq. 31.
//
// The kernels keep the deformation gradient as its strain E = F - I.  In
// float32, F itself near I holds a strain of 1e-4 with three significant
// digits; J - 1, I1 - 3 and the deviatoric term F - (I1/3) F^{-T} computed
// from F lose the rest.  From E they are formed without cancellation:
//   J - 1                = det_minus_one(E)
//   I1 - 3               = 2 tr E + |E|^2      (2D plane strain: the same,
//                                               F3 = diag(F, 1), I1 = |F|^2 + 1)
//   F - (I1/3) F^{-T}    = H E^T + E - ((I1 - 3)/3) H,   since I - H = H E^T.
// ---------------------------------------------------------------------------
template <int D>
struct StressParts {
    float J, Jm1, I1, a, b;  // a = G J^{-2/3}, b = K J (J - 1)
    float H[D][D];           // F^{-T}
    float dev[D][D];         // F - (I1/3) F^{-T}
    float s, sE;             // phi^q and eps + (1 - eps) phi^q
};

template <int D>
__device__ __forceinline__ void stress_parts(const float (&E)[D][D], float phi, const Params& P,
                                             StressParts<D>& S) {
    S.Jm1 = det_minus_one<D>(E);
    S.J = 1.0f + S.Jm1;
    inv_transpose_of<D>(E, S.J, S.H);
    float trE = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) trE += E[i][i];
    const float q3 = (2.0f * trE + frob<D>(E, E)) * (1.0f / 3.0f);  // (I1 - 3)/3
    S.I1 = 3.0f + 3.0f * q3;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float hEt = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) hEt += S.H[i][k] * E[j][k];
            S.dev[i][j] = hEt + E[i][j] - q3 * S.H[i][j];
        }
    const float r13 = rcbrtf(S.J);
    S.a = P.G * r13 * r13;
    S.b = P.K * S.J * S.Jm1;
    S.s = int_pow(phi, P.simp_q);
    S.sE = P.eps + (1.0f - P.eps) * S.s;
}

template <int D>
__device__ __forceinline__ void piola(const StressParts<D>& S, const float (&Br)[D],
                                      const float (&Ba)[D], float (&Pk)[D][D]) {
    const float sm = S.s * (1.0f / kMu0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float pe = S.a * S.dev[i][j] + S.b * S.H[i][j];
            Pk[i][j] = S.sE * pe - sm * Ba[i] * Br[j];
        }
}

// Reverse of piola(): given Pbar, accumulate dL/dF (= dL/dE) into Fbar and
// the phi, B~_r and B_applied cotangents into phib, brb, bab.
//   dJ = J H:dF, dI1 = 2F:dF, d(F^{-T}) = -H dF^T H, d a = -(2/3) a H:dF,
//   d b = K (2J - 1) J H:dF.
template <int D>
__device__ __forceinline__ void piola_adjoint(const float (&E)[D][D], float phi,
                                              const StressParts<D>& S, const float (&Br)[D],
                                              const float (&Ba)[D], const float (&Pbar)[D][D],
                                              const Params& P, float (&Fbar)[D][D], float& phib,
                                              float (&brb)[D], float (&bab)[D]) {
    const float third = S.I1 * (1.0f / 3.0f);
    // phi: d s / d phi = q phi^(q-1)
    const float ds = P.simp_q > 0 ? (float)P.simp_q * int_pow(phi, P.simp_q - 1) : 0.0f;
    float pe_dot = 0.0f, pm_dot = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            pe_dot += Pbar[i][j] * (S.a * S.dev[i][j] + S.b * S.H[i][j]);
            pm_dot -= Pbar[i][j] * Ba[i] * Br[j];
        }
    phib += ds * ((1.0f - P.eps) * pe_dot + pm_dot * (1.0f / kMu0));
    // magnetic part  -(s/mu0) Ba (x) Br
    const float sm = S.s * (1.0f / kMu0);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            bab[i] -= sm * Pbar[i][j] * Br[j];
            brb[j] -= sm * Pbar[i][j] * Ba[i];
        }
    // elastic part scaled by sE
    float Pb[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) Pb[i][j] = S.sE * Pbar[i][j];
    const float PbDev = frob<D>(Pb, S.dev);  // Pb : (F - (I1/3) H), without cancellation
    const float PbH = frob<D>(Pb, S.H);
    float HPt[D][D];  // H Pb^T
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < D; ++l) acc += S.H[i][l] * Pb[k][l];
            HPt[i][k] = acc;
        }
    const float cH = -(2.0f / 3.0f) * S.a * PbDev + P.K * (2.0f * S.J - 1.0f) * S.J * PbH;
    const float cF = -(2.0f / 3.0f) * S.a * PbH;
    const float cX = S.a * third - S.b;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float X = 0.0f;  // (H Pb^T H)_ij
#pragma unroll
            for (int k = 0; k < D; ++k) X += HPt[i][k] * S.H[k][j];
            const float Fij = E[i][j] + (i == j ? 1.0f : 0.0f);
            Fbar[i][j] += S.a * Pb[i][j] + cH * S.H[i][j] + cF * Fij + cX * X;
        }
}

// ---------------------------------------------------------------------------
// grid operation on one node (Eq. 16-18).  Bands are applied axis by axis,
// low side before high side; a band whose wall the velocity points into
// projects it: Coulomb friction on the floor in wall mode 1, otherwise v = 0.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void node_coords(int local, int res, int (&c)[D]) {
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
        c[a] = local % res;
        local /= res;
    }
}

// Non-uniform applied field, linear about the domain centre x_c = (1/2, ...):
// B at the particle is B_a + G (x - x_c), with G row-major dB_i/dx_j.
template <int D>
__device__ __forceinline__ void field_at_particle(const float* __restrict__ Gn, const float (&x)[D],
                                                  float (&B)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) B[i] += __ldg(Gn + i * D + j) * (x[j] - 0.5f);
}

// Body force of the non-uniform field: minus the position derivative of the
// SIMP-scaled magnetic energy (Eq. 31-32), f = (s V / mu0) G^T (F B~_r), with
// F = I + E and s = phi^q.
template <int D>
__device__ __forceinline__ void magnetic_force(const float* __restrict__ Gn, const float (&E)[D][D],
                                               const float (&Br)[D], float s, const Params& P, float (&f)[D]) {
    float FB[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        FB[i] = Br[i];
#pragma unroll
        for (int k = 0; k < D; ++k) FB[i] += E[i][k] * Br[k];
    }
    const float c = s * P.p_vol * (1.0f / kMu0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < D; ++i) acc += __ldg(Gn + i * D + j) * FB[i];
        f[j] = c * acc;
    }
}

// Solid box b at substep `step` and node c: true when the node lies inside
// the (moved) box, with the box velocity vb and the outward normal sgn e_axis
// of the face nearest to the node (ties: lowest axis, low face first).
template <int D>
__device__ __forceinline__ bool box_contact(const Extras* ext, float dx, int n_steps, int b, int step,
                                            const int* c, float (&vb)[D], int& axis, float& sgn) {
    const Boundary B = ext->box[b];
    const float* mo = ext->motion ? ext->motion + ((long long)b * n_steps + step) * 2 * D : nullptr;
    bool inside = true;
    float best = 3.0e38f;
    axis = 0;
    sgn = -1.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float off = mo ? mo[a] : 0.0f;
        vb[a] = mo ? mo[D + a] : 0.0f;
        const float x = (float)c[a] * dx, lo = B.lo[a] + off, hi = B.hi[a] + off;
        if (x < lo || x > hi) inside = false;
        if (x - lo < best) {
            best = x - lo;
            axis = a;
            sgn = -1.0f;
        }
        if (hi - x < best) {
            best = hi - x;
            axis = a;
            sgn = 1.0f;
        }
    }
    return inside;
}

// Eq. 18 on the velocity relative to a boundary moving at vb, outward
// normal sgn e_a: the normal part becomes vb's, the tangential part shrinks
// by mu |vn| (to zero at most).
template <int D>
__device__ __forceinline__ void coulomb_project(int a, float sgn, float mu, const float (&vb)[D], float (&v)[D]) {
    float vr[D], t2 = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        vr[i] = v[i] - vb[i];
        if (i != a) t2 += vr[i] * vr[i];
    }
    const float vn = sgn * vr[a];
    const float u = sqrtf(t2);
    const float sp = u + mu * vn;
    const float f = (u > 0.0f && sp > 0.0f) ? sp / u : 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = vb[i] + (i == a ? 0.0f : vr[i] * f);
}

// The solid boxes of the grid operation and their reverse.  Not inlined:
// every grid-operation call site would otherwise carry the box loops, which
// multiplies compile time and costs the fused particle kernels registers
// even without boxes; they are called only when boxes are set.
//
// apply_boxes: boxes act after the walls, in order; attached boxes set
// v = v_b, the others act when the velocity relative to the box points into
// it (Eq. 18 relative to the box).
template <int D>
__device__ __forceinline__ void apply_boxes(const Extras* ext, float dx, int n_steps, int step, const int* c,
                                         float* v) {
    float w[D];
#pragma unroll
    for (int i = 0; i < D; ++i) w[i] = v[i];
    for (int b = 0; b < ext->n; ++b) {
        float vb[D], sgn;
        int axis;
        if (!box_contact<D>(ext, dx, n_steps, b, step, c, vb, axis, sgn)) continue;
        const int kind = ext->box[b].kind;
        if (kind != kBoundaryAttached && !(sgn * (w[axis] - vb[axis]) < 0.0f)) continue;
        if (kind == kBoundaryCoulomb) {
            coulomb_project<D>(axis, sgn, ext->box[b].mu, vb, w);
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) w[i] = vb[i];
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = w[i];
}

// reverse_boxes: Vbar through the boxes, last first, given the velocity v
// that entered the first box (the walls' output).  The velocity entering box
// b is recomputed by replaying boxes 0..b-1 (at most 8 boxes, no per-box
// arrays).  The box velocity is a constant, so the Coulomb Jacobian acts on
// the relative velocity r = v - v_b: out_t = r_t (1 + mu vn / u), out_n = 0,
// vn = sgn r_a, u = |r_t|.
template <int D>
__device__ __noinline__ void reverse_boxes(const Extras* ext, float dx, int n_steps, int step, const int* c,
                                           const float* v, float* vbar) {
    float vb[D];
#pragma unroll
    for (int i = 0; i < D; ++i) vb[i] = vbar[i];
    const int nb = min(ext->n, kMaxBoundaries);
    for (int b = nb - 1; b >= 0; --b) {
        float ve[D];
#pragma unroll
        for (int i = 0; i < D; ++i) ve[i] = v[i];
        for (int e = 0; e <= b; ++e) {
            float vbx[D], sgn;
            int axis;
            if (!box_contact<D>(ext, dx, n_steps, e, step, c, vbx, axis, sgn)) continue;
            const int kind = ext->box[e].kind;
            if (kind != kBoundaryAttached && !(sgn * (ve[axis] - vbx[axis]) < 0.0f)) continue;
            if (e < b) {  // replay an earlier box
                if (kind == kBoundaryCoulomb) {
                    coulomb_project<D>(axis, sgn, ext->box[e].mu, vbx, ve);
                } else {
#pragma unroll
                    for (int i = 0; i < D; ++i) ve[i] = vbx[i];
                }
                continue;
            }
            // box b fired on the entering velocity ve
            if (kind != kBoundaryCoulomb) {
#pragma unroll
                for (int i = 0; i < D; ++i) vb[i] = 0.0f;
                continue;
            }
            const float mu = ext->box[e].mu;
            float r[D], t2 = 0.0f, tdot = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i) r[i] = ve[i] - vbx[i];
            const float vn = sgn * r[axis];
#pragma unroll
            for (int i = 0; i < D; ++i)
                if (i != axis) {
                    t2 += r[i] * r[i];
                    tdot += vb[i] * r[i];
                }
            const float u = sqrtf(t2);
            if (u > 0.0f && u + mu * vn > 0.0f) {
                const float ru = 1.0f / u;
                const float f = 1.0f + mu * vn * ru;
                const float g = mu * vn * tdot * ru * ru * ru;
                const float out_n = sgn * mu * tdot * ru;
#pragma unroll
                for (int i = 0; i < D; ++i) vb[i] = (i == axis) ? out_n : vb[i] * f - g * r[i];
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) vb[i] = 0.0f;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) vbar[i] = vb[i];
}

// BOXES: the caller may run with solid boxes (P.ext set).  Kernels launched
// without them pass false and carry no box code, which the fused particle
// kernels (one grid operation per stencil node) need for their registers.
template <int D, bool BOXES = true>
__device__ __forceinline__ void grid_velocity(const Params& P, const int (&c)[D], float m,
                                              const float (&mv)[D], float (&v)[D], int step) {
    if (!(m > 0.0f)) {
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = 0.0f;
        return;
    }
    float rm = 1.0f / m;
    float keep = 1.0f - P.dt * P.damping;
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = keep * (mv[i] * rm) + P.dt * P.gravity[i];
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            bool band = side == 0 ? (c[a] < P.bound) : (c[a] >= P.res - P.bound);
            float vn = side == 0 ? v[a] : -v[a];
            if (!band || !(vn < 0.0f)) continue;
            if (P.wall_mode == 1 && a == 1 && side == 0) {
                float t2 = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i)
                    if (i != a) t2 += v[i] * v[i];
                float u = sqrtf(t2);
                float sp = u + P.mu * vn;
                float f = (u > 0.0f && sp > 0.0f) ? sp / u : 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i) v[i] = (i == a) ? 0.0f : v[i] * f;
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) v[i] = 0.0f;
            }
        }
    }
    // solid boxes after the walls (only when set)
    if (BOXES && P.ext && P.ext->n > 0) apply_boxes<D>(P.ext, P.dx, P.n_steps, step, c, v);
}

// Reverse of grid_velocity: Vbar -> (mbar, mvbar).  The forward branches are
// replayed from (m, mv); overwritten components pass no gradient.
template <int D, bool BOXES = true>
__device__ __forceinline__ void grid_velocity_adjoint(const Params& P, const int (&c)[D], float m,
                                                      const float (&mv)[D], const float (&Vbar)[D],
                                                      float& mbar, float (&mvbar)[D], int step) {
    mbar = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) mvbar[i] = 0.0f;
    if (!(m > 0.0f)) return;
    float rm = 1.0f / m;
    float keep = 1.0f - P.dt * P.damping;
    float v0[D], v[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        v0[i] = mv[i] * rm;
        v[i] = keep * v0[i] + P.dt * P.gravity[i];
    }
    // replay, remembering the input of every projection that fired
    float vin[2 * D][D];
    int kind[2 * D];
    int nops = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            bool band = side == 0 ? (c[a] < P.bound) : (c[a] >= P.res - P.bound);
            float vn = side == 0 ? v[a] : -v[a];
            int op = 2 * a + side;
            kind[op] = 0;
            if (!band || !(vn < 0.0f)) continue;
#pragma unroll
            for (int i = 0; i < D; ++i) vin[op][i] = v[i];
            ++nops;
            if (P.wall_mode == 1 && a == 1 && side == 0) {
                kind[op] = 2;
                float t2 = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i)
                    if (i != a) t2 += v[i] * v[i];
                float u = sqrtf(t2);
                float sp = u + P.mu * vn;
                float f = (u > 0.0f && sp > 0.0f) ? sp / u : 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i) v[i] = (i == a) ? 0.0f : v[i] * f;
            } else {
                kind[op] = 1;
#pragma unroll
                for (int i = 0; i < D; ++i) v[i] = 0.0f;
            }
        }
    }
    float vb[D];
#pragma unroll
    for (int i = 0; i < D; ++i) vb[i] = Vbar[i];
    // reverse of the solid boxes (only when set), from the walls' output v
    if (BOXES && P.ext && P.ext->n > 0) reverse_boxes<D>(P.ext, P.dx, P.n_steps, step, c, v, vb);
    if (nops > 0) {
#pragma unroll
        for (int op = 2 * D - 1; op >= 0; --op) {
            if (kind[op] == 1) {
#pragma unroll
                for (int i = 0; i < D; ++i) vb[i] = 0.0f;
            } else if (kind[op] == 2) {
                const int a = op >> 1;
                float vn = vin[op][a];
                float t2 = 0.0f, tdot = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i)
                    if (i != a) {
                        t2 += vin[op][i] * vin[op][i];
                        tdot += vb[i] * vin[op][i];
                    }
                float u = sqrtf(t2);
                float sp = u + P.mu * vn;
                if (u > 0.0f && sp > 0.0f) {
                    float ru = 1.0f / u;
                    float f = 1.0f + P.mu * vn * ru;
                    float g = P.mu * vn * tdot * ru * ru * ru;
                    float out_n = P.mu * tdot * ru;
#pragma unroll
                    for (int i = 0; i < D; ++i) vb[i] = (i == a) ? out_n : vb[i] * f - g * vin[op][i];
                } else {
#pragma unroll
                    for (int i = 0; i < D; ++i) vb[i] = 0.0f;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float v0b = keep * vb[i];
        mvbar[i] = v0b * rm;
        mbar -= v0b * v0[i] * rm;
    }
}

// Warp-aggregated add of per-lane values into dst[inst * stride + c]: lanes
// of one instance are summed with shuffles first (the common case), mixed
// warps fall back to per-lane atomics.  Every lane of the warp must call it.
template <int NC>
__device__ __forceinline__ void warp_add_per_instance(const float (&val)[NC], int inst,
                                                      float* __restrict__ dst, long long stride) {
    const unsigned full = 0xffffffffu;
    int inst0 = __shfl_sync(full, inst, 0);
    bool uniform = __all_sync(full, inst == inst0 || inst < 0) && inst0 >= 0;
    if (uniform) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float s = val[c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(full, s, off);
            if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(dst + (long long)inst0 * stride + c, s);
        }
    } else if (inst >= 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (val[c] != 0.0f) atomicAdd(dst + (long long)inst * stride + c, val[c]);
    }
}

}  // namespace mpm
