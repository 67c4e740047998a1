// Particle kernels of the magneto-elastic MLS-MPM substep and its reverse.
//
// Forward (arxiv 2503.22767, Section 2.2): the particle kernel fuses the G2P
// of substep n (Eq. 19-22) with the P2G of substep n+1 (Eq. 14-15 with the
// SIMP-scaled stress of Eq. 7/31-33), so between substeps a particle's state
// is read once and written once.  Reverse (Section 2.3): the particle kernel
// fuses the P2G^T of substep n with the G2P^T of substep n-1.
//
// Particle arrays are structure-of-arrays with component stride P.np:
// x[D], v[D], C[D][D], E[D][D] (row-major), i.e. 2D + 2D^2 components, where
// E = F - I is the strain form of the deformation gradient (see
// mpm_device.cuh: it keeps small strains exact to float32 precision).
// Grids are float4 per node ([inst][node]): accumulators (m, mv), velocities
// (v, 0), adjoints (mbar, mvbar).
//
// The kernels are templates over the dimension and the fused stages; each
// dimension and direction is instantiated in a translation unit of its own
// (kernels_particle2.cu, kernels_forward3.cu, kernels_adjoint3.cu), so they
// compile in parallel.
#pragma once

#include <type_traits>

#include "kernels.h"
#include "particle_io.cuh"
#include "warp_scatter.cuh"

namespace mpm {

// Resident 256-thread blocks per SM that the register allocation must allow
// (the compiler caps registers at 65536 / (256 x this)).  The transfer kernels
// are latency-bound, so occupancy is traded against spills: the 3D forward
// kernel is held to 64 registers, and the adjoint kernel is compiled for 2
// (<= 128 registers), 3 (<= 80) and, in 2D, 4 (<= 64) blocks, chosen per
// launch (Params::adj_blocks; 4 acts as 3 in 3D).
constexpr int kMinBlocksForward3 = 4;
// 2D: at most 48 registers (40 warps per SM, no spills); the 2D batch's
// forward launch went from 83 to 79 us, the single 2D locomotion body is
// unchanged (its 469 blocks of 64 threads are far from filling the GPU)
constexpr int kMinBlocksForward2 = 5;

namespace {

inline int particle_blocks(long long n, int block) { return (int)((n + block - 1) / block); }

// The forward step of particle p (G2P of substep a.n_g2p and/or P2G of
// a.n_p2g); every lane of a warp calls it together, with particles
// 32w .. 32w + 31 (w = p / 32).  sm: this warp's warp_slots<D, P2G>()
// float4 of shared memory (the scatter slab of P2G).
// EXT: P.ext is set (solid boxes or a non-uniform field); without it the
// code for them is left out.  CHAIN: the kernel is one launch of a chain
// with programmatic dependent launch (k_forward); a persistent kernel calls
// this between its own grid-wide barriers instead.  AGG_P2G: the P2G scatter
// is aggregated over the lanes of one base node (scatter_aggregated).
template <int D, bool G2P, bool P2G, bool WRITE_ALL, bool FUSE, bool EXT, bool CHAIN,
          bool AGG_P2G = aggregate_scatter<D>()>
__device__ __forceinline__ void forward_particle(const Params& P, const StepArgs& a, int p, float4* sm) {
    using L = Layout<D>;
    // Early loads: with the grid operation in its own kernel, this kernel's
    // predecessor is that grid kernel, which writes none of the particle
    // arrays read first here.  Every kernel of the chain waits before it
    // triggers its dependents, so when this kernel starts, the particle
    // kernel before the grid kernel has completed, and the state loads can
    // overlap the grid kernel's tail.
    constexpr bool kEarly = CHAIN && G2P && !FUSE;
    // the P2G scatter is aggregated over the lanes of one cell (scatter_aggregated)
    constexpr bool AGG = P2G && AGG_P2G;
    const bool active = p < P.n_total;
    const int inst = active ? find_instance(a.inst_off, P.n_inst, p) : -1;
    const long long np = P.np;
    int flags = 0;
    // x: the X slot (the displacement u = x - x0 when a.x0 is set); every
    // stencil and field evaluation uses the position x0 + u (pos below)
    // xo: x0 (0 without a.x0), loaded with the state for G2P and again after
    // the G2P node loop for P2G, so that it holds no registers in the loop
    float x[D], v[D], C[D][D], F[D][D], xo[D];
    float phi = 0.0f, mp = 0.0f;
    auto position = [&](float (&pos)[D]) {
#pragma unroll
        for (int i = 0; i < D; ++i) pos[i] = __fadd_rn(x[i], xo[i]);
    };
    auto load_state = [&]() {
        load_vec<D>(a.s_in, L::X, np, p, x);
#pragma unroll
        for (int i = 0; i < D; ++i) xo[i] = a.x0 ? __ldg(a.x0 + (long long)i * np + p) : 0.0f;
        load_mat<D>(a.s_in, L::F, np, p, F);
        phi = a.phi[p];
        mp = phi * P.rho0 * P.p_vol;  // Eq. 33
        if (!G2P) {
            load_vec<D>(a.s_in, L::V, np, p, v);
            load_mat<D>(a.s_in, L::C, np, p, C);
        }
    };
    if (kEarly && active) load_state();
    if (CHAIN) {
        pdl_wait();
        pdl_trigger();
        if (FUSE) clear_buffer(a);
    }
    if (!kEarly && active) load_state();
    if (G2P) {
        float mom_x[1] = {0.0f};
        Stencil<D> s;
#pragma unroll
        for (int i = 0; i < D; ++i) s.base[i] = 0;
        if (active) {
            float pos[D];
            position(pos);
            if (!make_stencil<D>(pos, P, s)) flags |= kErrDomain;
        }
        const float4* __restrict__ Vg = FUSE ? a.accG : a.V;
        if (active) {
            const float4* __restrict__ Vi = Vg + (long long)inst * P.nodes;
            // Eq. 19-20 with x_i - x_p = (o - r) dx for stencil offset o:
            //   v = sum w V,  C = (4/dx) (sum w V o^T - v r^T)
#pragma unroll
            for (int i = 0; i < D; ++i) {
                v[i] = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) C[i][j] = 0.0f;  // sum w V o^T
            }
            // The sums run axis by axis: over the last axis with its 1D weights
            // (hv = sum w_l V, hv2 = sum o_l w_l V), then each row is weighted
            // by the product pw of the other axes' weights.
            const int nb = base_node<D>(s, P.res);
            float hv[D], hv2[D];
#pragma unroll
            for (int i = 0; i < D; ++i) hv[i] = hv2[i] = 0.0f;
#pragma unroll
            for (int k = 0; k < stencil_size<D>(); ++k) {
                const int o0 = stencil_offset<D>(k, 0), om = stencil_offset<D>(k, 1 % D);
                const int ol = stencil_offset<D>(k, D - 1);
                float gv[D];
                NodeTerm<D> t;
                t.node = nb + node_offset<D>(k, P.res);
#pragma unroll
                for (int e = 0; e < D; ++e) t.c[e] = s.base[e] + stencil_offset<D>(k, e);
                node_velocity<D, FUSE, EXT>(Vi, t, P, gv, a.n_g2p);
                const float wl = s.w[D - 1][ol];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const float wv = wl * gv[i];
                    hv[i] = ol == 0 ? wv : hv[i] + wv;
                    if (ol == 0) hv2[i] = 0.0f;
                    else hv2[i] = add_offset(hv2[i], ol, wv);
                }
                if (ol == 2) {  // the row is complete
                    const float pw = D == 2 ? s.w[0][o0] : s.w[0][o0] * s.w[1 % D][om];
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        const float hp = pw * hv[i];
                        v[i] += hp;
                        C[i][D - 1] += pw * hv2[i];
                        C[i][0] = add_offset(C[i][0], o0, hp);
                        if (D == 3) C[i][1 % D] = add_offset(C[i][1 % D], om, hp);
                    }
                }
            }
            if (P2G && a.x0) {  // x0 again for the P2G position; the load overlaps the G2P tail
#pragma unroll
                for (int i = 0; i < D; ++i) xo[i] = reload(a.x0 + (long long)i * np + p);
            }
            float Fn[D][D];
            const float c4 = 4.0f * P.inv_dx;
#pragma unroll
            for (int i = 0; i < D; ++i) {
#pragma unroll
                for (int j = 0; j < D; ++j) C[i][j] = c4 * (C[i][j] - v[i] * s.r[j]);
                x[i] += P.dt * v[i];                              // Eq. 21 (on u = x - x0)
            }
            // Eq. 22 in strain form: E' = E + dt C (I + E)
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float acc = C[i][j];
#pragma unroll
                    for (int k = 0; k < D; ++k) acc += C[i][k] * F[k][j];
                    Fn[i][j] = F[i][j] + P.dt * acc;
                }
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) F[i][j] = Fn[i][j];
            float Jm1 = det_minus_one<D>(F);
            if (!(Jm1 > -1.0f) || !isfinite(Jm1)) flags |= kErrNumeric;
            store_vec<D>(a.s_out, L::X, np, p, x);
            store_mat<D>(a.s_out, L::F, np, p, F);
            if (WRITE_ALL) {
                // v and C of a stored state are read only by the adjoint, a
                // segment later (the next substep's G2P computes its own):
                // streaming stores keep them from evicting the grids from L2
                // (2D batch, store passes: forward 89.6 -> 84.0 us per launch)
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    __stcs(a.s_out + (long long)(L::V + i) * np + p, v[i]);
#pragma unroll
                    for (int j = 0; j < D; ++j) __stcs(a.s_out + (long long)(L::C + i * D + j) * np + p, C[i][j]);
                }
            }
            mom_x[0] = mp * v[0];
        }
        if (P.loss_kind == 1 && a.mom != nullptr)
            warp_add_per_instance<1>(mom_x, inst, a.mom + (long long)a.n_g2p * P.n_inst, 1);
    }
    if (P2G) {
        // this warp's box of listed cells, read after the scatter (3D)
        if (D == 3 && a.blk.flag != nullptr) prefetch_l1(a.blk.wbox + (p >> 5));
        Stencil<D> s;
        float A[D][D], u[D];
        int nb = 0;
        float4* __restrict__ ai = a.acc + (long long)(active ? inst : 0) * P.nodes;
        if (active) {
            float pos[D];
            position(pos);
            if (!make_stencil<D>(pos, P, s)) flags |= kErrDomain;
            StressParts<D> S;
            stress_parts<D>(F, phi, P, S);
            if (!(S.J > 0.0f)) flags |= kErrNumeric;
            float Br[D], Ba[D], Pk[D][D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                Br[i] = a.mag[(long long)i * np + p];
                Ba[i] = __ldg(a.field + ((long long)inst * P.n_steps + a.n_p2g) * D + i);
            }
            if (EXT && P.ext->fgrad) {
                const float* Gn = P.ext->fgrad + ((long long)inst * P.n_steps + a.n_p2g) * D * D;
                field_at_particle<D>(Gn, pos, Ba);
                // body force of the non-uniform field, folded into the momentum
                // m v (f and m both vanish with phi, so m > 0 whenever f != 0)
                float f[D];
                magnetic_force<D>(Gn, F, Br, S.s, P, f);
                if (mp > 0.0f) {
#pragma unroll
                    for (int i = 0; i < D; ++i) v[i] += P.dt * f[i] / mp;
                }
            }
            piola<D>(S, Br, Ba, Pk);
            const float sc = P.dt * P.kappa * P.p_vol;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float pft = Pk[i][j];  // (P F^T)_ij with F = I + E
#pragma unroll
                    for (int k = 0; k < D; ++k) pft += Pk[i][k] * F[j][k];
                    // MLS-MPM affine momentum (Eq. 15 with the time step and the
                    // x_i - x_p offset of the MLS-MPM form): m C - dt (4/dx^2) V P F^T
                    A[i][j] = mp * C[i][j] - sc * pft;
                }
            // Eq. 15 with x_i - x_p = (o - r) dx: node momentum w (u + dx A o),
            // u = m v - dx A r
#pragma unroll
            for (int i = 0; i < D; ++i) {
                float ar = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    A[i][j] *= P.dx;
                    ar += A[i][j] * s.r[j];
                }
                u[i] = mp * v[i] - ar;
            }
            nb = base_node<D>(s, P.res);
        } else {  // a lane past the end takes part in the aggregated scatter with zeros
#pragma unroll
            for (int i = 0; i < D; ++i) {
                u[i] = 0.0f;
                s.base[i] = 0;
#pragma unroll
                for (int j = 0; j < D; ++j) A[i][j] = 0.0f;
#pragma unroll
                for (int j = 0; j < 3; ++j) s.w[i][j] = 0.0f;
            }
        }
        if constexpr (AGG) {
            // node (o0, .., ol) receives w (mp, u + A o), w = (w0 w1) w2 as below
            scatter_aggregated<D>(nb, inst, active, a.acc, P.nodes, P.res, sm, [&](int k) {
                const int o0 = stencil_offset<D>(k, 0), om = stencil_offset<D>(k, 1 % D);
                const int ol = stencil_offset<D>(k, D - 1);
                const float pw = D == 2 ? s.w[0][o0] : s.w[0][o0] * s.w[1 % D][om];
                const float w = pw * s.w[D - 1][ol];
                float mv[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    float t = add_offset(u[i], o0, A[i][0]);
                    if (D == 3) t = add_offset(t, om, A[i][1 % D]);
                    mv[i] = w * add_offset(t, ol, A[i][D - 1]);
                }
                return pack4<D>(w * mp, mv);
            });
            // the warp lists the node blocks its stencils reach beyond its box
            // (a.blk is uniform over the launch, so the whole warp takes part)
            if constexpr (D == 3) {
                if (a.blk.flag != nullptr) mark_blocks(a.blk, p >> 5, active, inst, s.base, P.res, a.blk.wbox[p >> 5]);
            }
        } else if (active) {
            float pw = 0.0f, Ug[D];  // per row: product of the other axes' weights, u + dx A o
#pragma unroll
            for (int i = 0; i < D; ++i) Ug[i] = 0.0f;
#pragma unroll
            for (int k = 0; k < stencil_size<D>(); ++k) {
                const int ol = stencil_offset<D>(k, D - 1);
                if (ol == 0)
                    pw = D == 2 ? s.w[0][stencil_offset<D>(k, 0)]
                                : s.w[0][stencil_offset<D>(k, 0)] * s.w[1 % D][stencil_offset<D>(k, 1 % D)];
                const float w = pw * s.w[D - 1][ol];
                if (ol == 0) {  // a new row: u + dx A o over all but the last axis
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        float ug = add_offset(u[i], stencil_offset<D>(k, 0), A[i][0]);
                        if (D == 3) ug = add_offset(ug, stencil_offset<D>(k, 1 % D), A[i][1 % D]);
                        Ug[i] = ug;
                    }
                }
                float mv[D];
#pragma unroll
                for (int i = 0; i < D; ++i) mv[i] = w * add_offset(Ug[i], ol, A[i][D - 1]);
                atomicAdd(ai + nb + node_offset<D>(k, P.res), pack4<D>(w * mp, mv));  // Eq. 14 in .x
            }
        }
    }
    if (flags) atomicOr(a.err, flags);
}

// 3D: at most 64 registers (32 warps per SM) to keep more gathers in flight
template <int D, bool G2P, bool P2G, bool WRITE_ALL, bool FUSE, bool EXT, bool AGG = aggregate_scatter<D>()>
__global__ void __launch_bounds__(256, D == 3 ? kMinBlocksForward3 : kMinBlocksForward2)
    k_forward(Params P, StepArgs a) {
    extern __shared__ float4 s_warp[];
    forward_particle<D, G2P, P2G, WRITE_ALL, FUSE, EXT, true, AGG>(
        P, a, blockIdx.x * blockDim.x + threadIdx.x, s_warp + (threadIdx.x >> 5) * warp_slots<D, P2G, AGG>());
}


// ---------------------------------------------------------------------------
// adjoint particle kernel
//   P2GT: reverse of P2G at substep n = a.n_p2g; completes the particle
//         adjoint of state n (x, v, C, F), accumulates design gradients.
//   G2PT: reverse of G2P at substep m (= n-1 when fused, else n): consumes
//         the adjoint of state m+1, scatters Vbar, writes the partial
//         adjoint (x, F) of state m.
// ---------------------------------------------------------------------------
// FUSE: P2G^T evaluates the grid adjoint per stencil node from (accP, VbarIn);
// FUSE_V: G2P^T takes the grid velocity from accG through the grid operation.
// EXT: P.ext is set (solid boxes or a non-uniform field), as in k_forward.
// CHAIN and the calling convention as in forward_particle; sm: this warp's
// warp_slots<D, G2PT>() float4 (the scatter slab of G2P^T).  RELIEF: the
// register budget is tight (80 registers or fewer), so the state and stress
// of P2G^T are reloaded and recomputed after its node loop.
template <int D, bool P2GT, bool G2PT, bool FUSE, bool FUSE_V, bool EXT, bool CHAIN, bool RELIEF>
__device__ __forceinline__ void adjoint_particle(const Params& P, const StepArgs& a, int p, float4* sm) {
    using L = Layout<D>;
    // Early loads as in k_forward: the fused kernel without grid-adjoint
    // fusion follows the grid adjoint kernel, which writes none of the
    // particle arrays of state n, the partial adjoint or the design.
    constexpr bool kEarly = CHAIN && P2GT && G2PT && !FUSE;
    // The late P2G^T epilogue (kLate): under the 80-register budget of the 3D
    // kernel it cuts the spills from 188 to 88 bytes per thread (3D
    // locomotion, 1M particles: 198.1 -> 196.0 us per launch, 3 x 200,000
    // particles: 119.3 -> 117.4 us).  The 2D budgets spill nothing in the
    // plain order and lose with this one (2D batch: 108.3 -> 112.3 us).
    constexpr bool kLate = RELIEF && D == 3;
    const bool active = p < P.n_total;
    const int inst = active ? find_instance(a.inst_off, P.n_inst, p) : -1;
    const long long np = P.np;
    int flags = 0;
    // adjoint of the state between the two halves (state n if P2GT)
    float xb[D], vb[D], Cb[D][D], Fb[D][D];
    float Cn[D][D];  // C of state n (= m+1), needed by G2P^T
    float x_n[D], v_n[D], F_n[D][D], phi_n = 0.0f;  // state n and design (P2G^T)
    auto load_state_n = [&]() {
        load_position<D>(a.s_in, a.x0, np, p, x_n);  // the position x0 + u
        load_vec<D>(a.s_in, L::V, np, p, v_n);
        // C and E are read again after the P2G^T node loop under RELIEF:
        // plain loads, so that the second read finds them cached
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                Cn[i][j] = RELIEF ? __ldg(a.s_in + (long long)(L::C + i * D + j) * np + p)
                                  : __ldcs(a.s_in + (long long)(L::C + i * D + j) * np + p);
                F_n[i][j] = RELIEF ? __ldg(a.s_in + (long long)(L::F + i * D + j) * np + p)
                                   : __ldcs(a.s_in + (long long)(L::F + i * D + j) * np + p);
            }
        load_vec<D>(a.adj, L::X, np, p, xb);
        phi_n = a.phi[p];
    };
    if (kEarly && active) load_state_n();
    if (P2GT && G2PT && active) {
        // x and E of state m = n-1 (G2P^T) come from the segment store in HBM;
        // request them now so that their loads after P2G^T find them in L2
#pragma unroll
        for (int c = 0; c < D; ++c) prefetch_l2(a.s_aux + (long long)(L::X + c) * np + p);
#pragma unroll
        for (int c = 0; c < D * D; ++c) prefetch_l2(a.s_aux + (long long)(L::F + c) * np + p);
    }
    if (P2GT && active) {  // the design and its gradients, read late in P2G^T
        prefetch_l2(a.gphi + p);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            prefetch_l2(a.mag + (long long)c * np + p);
            prefetch_l2(a.gmag + (long long)c * np + p);
        }
    }
    if (CHAIN) {
        pdl_wait();
        pdl_trigger();
        clear_buffer(a);
    }
    if (P2GT && !kEarly && active) load_state_n();
    constexpr bool AGG = G2PT && aggregate_scatter<D>();
    float bab[D];
#pragma unroll
    for (int i = 0; i < D; ++i) bab[i] = 0.0f;
    // non-uniform field: G of this substep (uniform over the launch), and the
    // particle's contribution to dL/dG
    const bool has_fgrad = EXT && P2GT && P.ext->fgrad;
    float gG[D * D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) gG[i] = 0.0f;
    if (P2GT) {
        if (active) {
            const int n = a.n_p2g;
            const float* Gn = has_fgrad ? P.ext->fgrad + ((long long)inst * P.n_steps + n) * D * D : nullptr;
            float(&x)[D] = x_n;
            float(&v)[D] = v_n;
            float(&F)[D][D] = F_n;
            const float phi = phi_n;
            const float mp = phi * P.rho0 * P.p_vol;
            float Br[D], Ba[D], Pk[D][D], A[D][D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                Br[i] = a.mag[(long long)i * np + p];
                Ba[i] = __ldg(a.field + ((long long)inst * P.n_steps + n) * D + i);
            }
            if (Gn) field_at_particle<D>(Gn, x, Ba);
            Stencil<D> s;
            if (!make_stencil<D>(x, P, s)) flags |= kErrDomain;
            StressParts<D> S;
            stress_parts<D>(F, phi, P, S);
            piola<D>(S, Br, Ba, Pk);
            const float sc = P.dt * P.kappa * P.p_vol;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float pft = Pk[i][j];  // (P F^T)_ij with F = I + E
#pragma unroll
                    for (int k = 0; k < D; ++k) pft += Pk[i][k] * F[j][k];
                    A[i][j] = mp * Cn[i][j] - sc * pft;
                }
            // Node sums with x_i - x_p = (o - r) dx (o the stencil offset):
            //   S0 = sum w mvb,  T = sum w mvb o^T,  mbs = sum w mb
            // give vbar = mp S0, Abar = dx (T - S0 r^T) and
            // mbar_p = mbs + S0 . v + C : Abar.  The node's contribution to
            // the particle's momentum is
            //   inner = mb mp + mvb . (mp v + A dpos) = mb mp + mvb . (u + dx A o),
            // u = mp v - dx A r, and xbar += sum (grad w) inner - A^T S0.
            // Every stencil sum runs axis by axis: over the last axis with its
            // 1D weights, then the partial sums are weighted by the other
            // axes' weights, so no node forms a product of weights.
            float u[D], dA[D][D];  // dA[c][i] = dx A_ic
#pragma unroll
            for (int i = 0; i < D; ++i) {
                float ar = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    ar += A[i][j] * s.r[j];
                    dA[j][i] = P.dx * A[i][j];
                }
                u[i] = mp * v[i] - P.dx * ar;
            }
            if (Gn) {  // the body force is part of the particle's momentum term
                float f[D];
                magnetic_force<D>(Gn, F, Br, S.s, P, f);
#pragma unroll
                for (int i = 0; i < D; ++i) u[i] += P.dt * f[i];
            }
            const float4* __restrict__ gi = (FUSE ? a.accP : a.gadj) + (long long)inst * P.nodes;
            const float4* __restrict__ vbi = FUSE ? a.VbarIn + (long long)inst * P.nodes : nullptr;
            const int nb = base_node<D>(s, P.res);
            float S0[D], T[D][D], mbs = 0.0f, xg[D];
            // partial sums over the last axis (h*) and, in 3D, the middle axis (l*)
            float Ug[D], hv[D], hv2[D], hm = 0.0f, ha = 0.0f, hb = 0.0f, la = 0.0f, lb = 0.0f, lc = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                S0[i] = xg[i] = Ug[i] = hv[i] = hv2[i] = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) T[i][j] = 0.0f;
            }
            auto node_loop = [&]() {
#pragma unroll
                for (int k = 0; k < stencil_size<D>(); ++k) {
                    const int o0 = stencil_offset<D>(k, 0), om = stencil_offset<D>(k, 1 % D);
                    const int ol = stencil_offset<D>(k, D - 1);
                    if (ol == 0) {  // a new row along the last axis
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            float ug = add_offset(u[i], o0, dA[0][i]);
                            if (D == 3) ug = add_offset(ug, om, dA[1 % D][i]);
                            Ug[i] = ug;
                            hv[i] = hv2[i] = 0.0f;
                        }
                        hm = ha = hb = 0.0f;
                    }
                    float4 g;
                    float mvb[D];
                    if (FUSE) {
                        const int node = nb + node_offset<D>(k, P.res);
                        g = __ldg(gi + node);
                        // grid adjoint (reverse of Eq. 16-18) of this node, on the fly
                        int c[D];
#pragma unroll
                        for (int e = 0; e < D; ++e) c[e] = s.base[e] + stencil_offset<D>(k, e);
                        float mv[D], vbv[D], mbv;
                        unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mv);
                        unpack3<D>(__ldg(vbi + node), vbv);
                        grid_velocity_adjoint<D, EXT>(P, c, g.x, mv, vbv, mbv, mvb, a.n_p2g);
                        g.x = mbv;
                    } else {
                        g = __ldg(gi + nb + node_offset<D>(k, P.res));
                        unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mvb);
                    }
                    const float wl = s.w[D - 1][ol], dwl = s.dw[D - 1][ol];
                    float inner = g.x * mp;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        inner += mvb[i] * add_offset(Ug[i], ol, dA[D - 1][i]);
                        const float wm = wl * mvb[i];
                        hv[i] += wm;
                        if (ol == 1) hv2[i] += wm;
                        else if (ol == 2) hv2[i] += 2.0f * wm;
                    }
                    hm += wl * g.x;
                    ha += wl * inner;
                    hb += dwl * inner;
                    if (ol == 2) {  // the row is complete: weight it by the other axes
                        const float w0 = s.w[0][o0], dw0 = s.dw[0][o0];
                        float pw = w0;
                        if (D == 2) {
                            xg[0] += dw0 * ha;
                            xg[D - 1] += w0 * hb;
                        } else {
                            const float w1 = s.w[1 % D][om], dw1 = s.dw[1 % D][om];
                            if (om == 0) la = lb = lc = 0.0f;
                            la += w1 * ha;
                            lb += dw1 * ha;
                            lc += w1 * hb;
                            if (om == 2) {
                                xg[0] += dw0 * la;
                                xg[1 % D] += w0 * lb;
                                xg[D - 1] += w0 * lc;
                            }
                            pw = w0 * w1;
                        }
                        mbs += pw * hm;
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            const float hp = pw * hv[i];
                            S0[i] += hp;
                            T[i][D - 1] += pw * hv2[i];
                            if (o0 == 1) T[i][0] += hp;
                            else if (o0 == 2) T[i][0] += 2.0f * hp;
                            if (D == 3) {
                                if (om == 1) T[i][1 % D] += hp;
                                else if (om == 2) T[i][1 % D] += 2.0f * hp;
                            }
                        }
                    }
                }
            };
            node_loop();
            // The node loop needs none of C, E, the stress (all used for A
            // before it) and Fbar of state n.  Under a tight register budget
            // (RELIEF) they are read again, and the stress recomputed, here, so
            // their registers are free during the loop (the recomputation is
            // cheaper than the spills); with registers to spare they stay live.
            // kLate: E, the stress and Fbar are formed only where first used,
            // and P element by element.
            if (RELIEF) reload_mat<D>(a.s_in, L::C, np, p, Cn);
            if (RELIEF && !kLate) reload_mat<D>(a.s_in, L::F, np, p, F);
            if (!kLate) load_mat<D>(a.adj, L::F, np, p, Fb);
            if (RELIEF && !kLate) {
                stress_parts<D>(F, phi, P, S);
                piola<D>(S, Br, Ba, Pk);
            }
            // grad w is (dw along its own axis) / dx times the other weights;
            // A^T S0 = (dA S0) / dx
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float g = xg[c];
#pragma unroll
                for (int i = 0; i < D; ++i) g -= dA[c][i] * S0[i];
                xb[c] += P.inv_dx * g;
            }
            float Ab[D][D], mpb = mbs;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                vb[i] = mp * S0[i];
                mpb += S0[i] * v[i];
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    Ab[i][j] = P.dx * (T[i][j] - S0[i] * s.r[j]);
                    mpb += Cn[i][j] * Ab[i][j];
                }
            }
            // A = mp C - sc P F^T:  Pbar = -sc Abar F,  Fbar -= sc Abar^T P
            float Pb[D][D];
            if (!kLate) {
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) Cb[i][j] = mp * Ab[i][j];
            }
            if (kLate) reload_mat<D>(a.s_in, L::F, np, p, F);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float pb = Ab[i][j], fb = 0.0f;  // (Abar F)_ij with F = I + E
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        pb += Ab[i][k] * F[k][j];
                        if (!kLate) fb += Ab[k][i] * Pk[k][j];  // (Abar^T P)_ij
                    }
                    Pb[i][j] = -sc * pb;
                    if (!kLate) Fb[i][j] -= sc * fb;
                }
            if (kLate) {
                stress_parts<D>(F, phi, P, S);
                load_mat<D>(a.adj, L::F, np, p, Fb);
                // P_kj as piola() forms it, used by its three products at once
                const float smu = S.s * (1.0f / kMu0);
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const float pk = S.sE * (S.a * S.dev[k][j] + S.b * S.H[k][j]) - smu * Ba[k] * Br[j];
#pragma unroll
                        for (int i = 0; i < D; ++i) Fb[i][j] -= sc * (Ab[k][i] * pk);
                    }
            }
            float phib = 0.0f, brb[D];
#pragma unroll
            for (int i = 0; i < D; ++i) brb[i] = 0.0f;
            piola_adjoint<D>(F, phi, S, Br, Ba, Pb, P, Fb, phib, brb, bab);
            if (kLate) {
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) Cb[i][j] = mp * Ab[i][j];
            }
            float gph = phib + mpb * P.rho0 * P.p_vol;
            if (Gn) {
                // B at the particle = B_a + G (x - x_c): dL/dB_a stays in bab,
                // dL/dG += bab (x - x_c)^T, xbar += G^T bab
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        gG[i * D + j] += bab[i] * (x[j] - 0.5f);
                        xb[j] += __ldg(Gn + i * D + j) * bab[i];
                    }
                // body force f = c G^T (F B~_r), c = s V / mu0, whose adjoint is
                // fbar = dt sum_i w mvb_i = dt S0
                const float c = S.s * P.p_vol * (1.0f / kMu0);
                float FB[D], Gfb[D], fraw = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    FB[i] = Br[i];
                    Gfb[i] = 0.0f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        FB[i] += F[i][k] * Br[k];
                        Gfb[i] += __ldg(Gn + i * D + k) * (P.dt * S0[k]);
                    }
                }
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    fraw += Gfb[i] * FB[i];
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        Fb[i][k] += c * Gfb[i] * Br[k];
                        brb[k] += c * Gfb[i] * ((i == k ? 1.0f : 0.0f) + F[i][k]);
                        gG[i * D + k] += c * FB[i] * (P.dt * S0[k]);
                    }
                }
                const float ds = P.simp_q > 0 ? (float)P.simp_q * int_pow(phi, P.simp_q - 1) : 0.0f;
                gph += ds * P.p_vol * (1.0f / kMu0) * fraw;
            }
            // locomotion seed on state n (n >= 1), Eq. 40
            if (P.loss_kind == 1 && n >= 1) {
                const float M = a.Minst[inst];
                if (M > 0.0f) {
                    const float dl = a.dloss[inst];
                    const float rM = 1.0f / M;
                    const float vbar = a.mom[(long long)(n - 1) * P.n_inst + inst] * rM;
                    vb[0] -= P.dt * mp * rM * dl;
                    gph -= P.dt * (v[0] - vbar) * rM * dl * P.rho0 * P.p_vol;
                }
            }
            a.gphi[p] += gph;
#pragma unroll
            for (int i = 0; i < D; ++i) a.gmag[(long long)i * np + p] += brb[i];
        }
        warp_add_per_instance<D>(bab, inst, a.gfield + (long long)a.n_p2g * D,
                                 (long long)P.n_steps * D);
        if (has_fgrad)  // uniform over the launch: every lane takes part
            warp_add_per_instance<D * D>(gG, inst, P.ext->gfgrad + (long long)a.n_p2g * D * D,
                                         (long long)P.n_steps * D * D);
        if (!G2PT && active) {
            store_vec<D>(a.adj, L::X, np, p, xb);
            store_vec<D>(a.adj, L::V, np, p, vb);
            store_mat<D>(a.adj, L::C, np, p, Cb);
            store_mat<D>(a.adj, L::F, np, p, Fb);
        }
    }
    if (G2PT) {
        Stencil<D> s;
        float q[D], dC[D][D];  // dC[c][i] = kappa dx Ct_ic
        int nb = 0;
        float4* __restrict__ Vbi = a.Vbar + (long long)(active ? inst : 0) * P.nodes;
        if (active) {
            if (!P2GT) {
                // adjoint of state m+1 and C_{m+1} from memory
                load_vec<D>(a.adj, L::X, np, p, xb);
                load_vec<D>(a.adj, L::V, np, p, vb);
                load_mat<D>(a.adj, L::C, np, p, Cb);
                load_mat<D>(a.adj, L::F, np, p, Fb);
                load_mat<D>(a.s_in, L::C, np, p, Cn);
            }
            float x[D], F[D][D];
            load_position<D>(a.s_aux, a.x0, np, p, x);  // the position x0 + u
            load_mat<D>(a.s_aux, L::F, np, p, F);
            if (!make_stencil<D>(x, P, s)) flags |= kErrDomain;
            // x' = x + dt v',  F' = (I + dt C') F  (Eq. 21-22)
            float vt[D], Ct[D][D], Fo[D][D];
            if (kLate && P2GT) reload_mat<D>(a.s_in, L::C, np, p, Cn);  // C of state n, for (I + dt C')^T
#pragma unroll
            for (int i = 0; i < D; ++i) vt[i] = vb[i] + P.dt * xb[i];
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float fft = Fb[i][j], ctf = Fb[i][j];  // F = I + E
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        fft += Fb[i][k] * F[j][k];          // (Fbar F^T)_ij
                        ctf += P.dt * Cn[k][i] * Fb[k][j];  // ((I + dt C')^T Fbar)_ij
                    }
                    Ct[i][j] = Cb[i][j] + P.dt * fft;
                    Fo[i][j] = ctf;
                }
            store_mat<D>(a.adj, L::F, np, p, Fo);  // complete: the stencil sums add nothing to it
            const float4* __restrict__ Vi = (FUSE_V ? a.accG : a.V) + (long long)inst * P.nodes;
            // Eq. 19-20 reversed (v' = sum w V, C' = kappa sum w V dpos^T) with
            // dpos = (o - r) dx: the node's velocity adjoint is w sv,
            //   sv = vt + kappa Ct dpos = q + kappa dx Ct o,  q = vt - kappa dx Ct r,
            // and xbar += sum (grad w) (V . sv) - kappa Ct^T sum w V.  The stencil
            // sums run axis by axis as in P2G^T; only the scatter needs the
            // node's weight.
            const float kdx = P.kappa * P.dx;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                float cr = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    cr += Ct[i][j] * s.r[j];
                    dC[j][i] = kdx * Ct[i][j];
                }
                q[i] = vt[i] - kdx * cr;
            }
            nb = base_node<D>(s, P.res);
            float xg[D], vs[D], Sg[D], hv[D], pw = 0.0f, ha = 0.0f, hb = 0.0f, la = 0.0f, lb = 0.0f, lc = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i) xg[i] = vs[i] = Sg[i] = hv[i] = 0.0f;
            auto node_loop = [&]() {
#pragma unroll
                for (int k = 0; k < stencil_size<D>(); ++k) {
                    const int o0 = stencil_offset<D>(k, 0), om = stencil_offset<D>(k, 1 % D);
                    const int ol = stencil_offset<D>(k, D - 1);
                    if (ol == 0) {  // a new row along the last axis
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            float sg = add_offset(q[i], o0, dC[0][i]);
                            if (D == 3) sg = add_offset(sg, om, dC[1 % D][i]);
                            Sg[i] = sg;
                            hv[i] = 0.0f;
                        }
                        ha = hb = 0.0f;
                        pw = D == 2 ? s.w[0][o0] : s.w[0][o0] * s.w[1 % D][om];
                    }
                    const int node = nb + node_offset<D>(k, P.res);
                    float gv[D];
                    {
                        NodeTerm<D> t;
                        t.node = node;
#pragma unroll
                        for (int e = 0; e < D; ++e) t.c[e] = s.base[e] + stencil_offset<D>(k, e);
                        node_velocity<D, FUSE_V, EXT>(Vi, t, P, gv, a.n_p2g - 1);
                    }
                    const float wl = s.w[D - 1][ol], dwl = s.dw[D - 1][ol];
                    float sv[D], dot = 0.0f;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        sv[i] = add_offset(Sg[i], ol, dC[D - 1][i]);
                        dot += gv[i] * sv[i];  // V . (vt + kappa Ct dpos)
                        hv[i] += wl * gv[i];
                    }
                    ha += wl * dot;
                    hb += dwl * dot;
                    if constexpr (!AGG) {
                        const float w = pw * wl;
#pragma unroll
                        for (int i = 0; i < D; ++i) sv[i] *= w;
                        atomicAdd(Vbi + node, make_float4(sv[0], sv[1 % D], D == 3 ? sv[2 % D] : 0.0f, 0.0f));
                    }
                    if (ol == 2) {  // the row is complete: weight it by the other axes
                        const float w0 = s.w[0][o0], dw0 = s.dw[0][o0];
                        if (D == 2) {
                            xg[0] += dw0 * ha;
                            xg[D - 1] += w0 * hb;
                        } else {
                            const float w1 = s.w[1 % D][om], dw1 = s.dw[1 % D][om];
                            if (om == 0) la = lb = lc = 0.0f;
                            la += w1 * ha;
                            lb += dw1 * ha;
                            lc += w1 * hb;
                            if (om == 2) {
                                xg[0] += dw0 * la;
                                xg[1 % D] += w0 * lb;
                                xg[D - 1] += w0 * lc;
                            }
                        }
#pragma unroll
                        for (int i = 0; i < D; ++i) vs[i] += pw * hv[i];
                    }
                }
            };
            node_loop();
            // kappa Ct^T vs = (dC vs) / dx
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float g = xg[c];
#pragma unroll
                for (int i = 0; i < D; ++i) g -= dC[c][i] * vs[i];
                xb[c] += P.inv_dx * g;
            }
            store_vec<D>(a.adj, L::X, np, p, xb);
        } else {  // a lane past the end takes part in the aggregated scatter with zeros
#pragma unroll
            for (int i = 0; i < D; ++i) {
                q[i] = 0.0f;
                s.base[i] = 0;
#pragma unroll
                for (int j = 0; j < D; ++j) dC[i][j] = 0.0f;
#pragma unroll
                for (int j = 0; j < 3; ++j) s.w[i][j] = 0.0f;
            }
        }
        if constexpr (AGG) {
            // node (o0, .., ol) receives w sv, sv = q + kappa dx Ct o, as above
            scatter_aggregated<D>(nb, inst, active, a.Vbar, P.nodes, P.res, sm, [&](int k) {
                const int o0 = stencil_offset<D>(k, 0), om = stencil_offset<D>(k, 1 % D);
                const int ol = stencil_offset<D>(k, D - 1);
                const float pw = D == 2 ? s.w[0][o0] : s.w[0][o0] * s.w[1 % D][om];
                const float w = pw * s.w[D - 1][ol];
                float sv[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    float t = add_offset(q[i], o0, dC[0][i]);
                    if (D == 3) t = add_offset(t, om, dC[1 % D][i]);
                    sv[i] = w * add_offset(t, ol, dC[D - 1][i]);
                }
                return make_float4(sv[0], sv[1 % D], D == 3 ? sv[2 % D] : 0.0f, 0.0f);
            });
        }
    }
    if (flags) atomicOr(a.err, flags);
}

template <int D, bool P2GT, bool G2PT, bool FUSE, bool FUSE_V, int MINB, bool EXT>
__global__ void __launch_bounds__(256, MINB) k_adjoint(Params P, StepArgs a) {
    extern __shared__ float4 s_warp[];
    adjoint_particle<D, P2GT, G2PT, FUSE, FUSE_V, EXT, true, (MINB >= 3)>(
        P, a, blockIdx.x * blockDim.x + threadIdx.x, s_warp + (threadIdx.x >> 5) * warp_slots<D, G2PT>());
}


}  // namespace

template <int D, bool FUSE>
static cudaError_t forward_d(bool g2p, bool p2g, bool all, const Params& P, const StepArgs& a,
                             int block, cudaStream_t st) {
    // a fused launch also clears a.zero4, so it runs even without particles
    if (P.n_total == 0 && !(FUSE && a.zero4)) return cudaSuccess;
    long long threads = P.n_total > 0 ? P.n_total : block;
    dim3 grid(particle_blocks(threads, block));
    const bool ext = P.ext != nullptr;
    const size_t warps = (size_t)(block + 31) / 32;
    auto go = [&](auto kernel, size_t smem) { return launch_chain_smem(P, kernel, grid, block, smem, st, P, a); };
    const size_t smem_p2g = warps * warp_slots<D, true>() * sizeof(float4);
    const size_t smem_g2p = warps * warp_slots<D, false>() * sizeof(float4);
    if (g2p && p2g) {
        if (ext) {
            if (all) return go(k_forward<D, true, true, true, FUSE, true>, smem_p2g);
            return go(k_forward<D, true, true, false, FUSE, true>, smem_p2g);
        }
        if constexpr (D == 2) {
            if (P.agg2) {  // the aggregated 2D P2G (Params::agg2)
                const size_t smem_agg = warps * warp_slots<D, true, true>() * sizeof(float4);
                if (all) return go(k_forward<D, true, true, true, FUSE, false, true>, smem_agg);
                return go(k_forward<D, true, true, false, FUSE, false, true>, smem_agg);
            }
        }
        if (all) return go(k_forward<D, true, true, true, FUSE, false>, smem_p2g);
        return go(k_forward<D, true, true, false, FUSE, false>, smem_p2g);
    } else if (g2p) {
        // with grid fusion the G2P applies the grid operation, boxes included
        if (ext && FUSE) {
            if (all) return go(k_forward<D, true, false, true, FUSE, true>, smem_g2p);
            return go(k_forward<D, true, false, false, FUSE, true>, smem_g2p);
        }
        if (all) return go(k_forward<D, true, false, true, FUSE, false>, smem_g2p);
        return go(k_forward<D, true, false, false, FUSE, false>, smem_g2p);
    } else {
        if (ext) return go(k_forward<D, false, true, false, FUSE, true>, smem_p2g);
        return go(k_forward<D, false, true, false, FUSE, false>, smem_p2g);
    }
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_forward_dim(bool g2p, bool p2g, bool write_all, bool fuse, const Params& P,
                               const StepArgs& a, int block, cudaStream_t st) {
    return fuse ? forward_d<D, true>(g2p, p2g, write_all, P, a, block, st)
                : forward_d<D, false>(g2p, p2g, write_all, P, a, block, st);
}

template <int D, bool FUSE, bool FUSE_V>
static cudaError_t adjoint_d(bool p2gt, bool g2pt, const Params& P, const StepArgs& a, int block,
                             cudaStream_t st) {
    if (P.n_total == 0 && !a.zero4) return cudaSuccess;
    long long threads = P.n_total > 0 ? P.n_total : block;
    dim3 grid(particle_blocks(threads, block));
    // with solid boxes or a field gradient only the 128-register budget is built
    const bool ext = P.ext != nullptr;
    const size_t warps = (size_t)(block + 31) / 32;
    auto go = [&](auto kernel, size_t smem) { return launch_chain_smem(P, kernel, grid, block, smem, st, P, a); };
    const size_t sm_g2pt = warps * warp_slots<D, true>() * sizeof(float4);
    const size_t sm_p2gt = warps * warp_slots<D, false>() * sizeof(float4);
    if (p2gt && g2pt) {
        if (ext) return go(k_adjoint<D, true, true, FUSE, FUSE_V, 2, true>, sm_g2pt);
        if constexpr (D == 2) {
            if (P.adj_blocks == 4) return go(k_adjoint<D, true, true, FUSE, FUSE_V, 4, false>, sm_g2pt);
        }
        if (P.adj_blocks >= 3)
            return go(k_adjoint<D, true, true, FUSE, FUSE_V, 3, false>, sm_g2pt);
        return go(k_adjoint<D, true, true, FUSE, FUSE_V, 2, false>, sm_g2pt);
    }
    // the segment-edge halves run once per checkpoint segment
    if (p2gt) {
        if (ext) return go(k_adjoint<D, true, false, FUSE, FUSE_V, 2, true>, sm_p2gt);
        return go(k_adjoint<D, true, false, FUSE, FUSE_V, 2, false>, sm_p2gt);
    }
    if (ext) return go(k_adjoint<D, false, true, FUSE, FUSE_V, 2, true>, sm_g2pt);
    return go(k_adjoint<D, false, true, FUSE, FUSE_V, 2, false>, sm_g2pt);
}

template <int D>
cudaError_t launch_adjoint_dim(bool p2gt, bool g2pt, bool fuse, bool fuse_v, const Params& P,
                               const StepArgs& a, int block, cudaStream_t st) {
    if (fuse) return adjoint_d<D, true, true>(p2gt, g2pt, P, a, block, st);
    if (fuse_v) return adjoint_d<D, false, true>(p2gt, g2pt, P, a, block, st);
    return adjoint_d<D, false, false>(p2gt, g2pt, P, a, block, st);
}


}  // namespace mpm
