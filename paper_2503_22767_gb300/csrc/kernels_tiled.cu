// Shared-memory tiled versions of the two per-substep particle kernels.
//
//   k_forward_tiled  G2P of substep n (Eq. 19-22) + P2G of substep n+1
//                    (Eq. 14-15, stress Eq. 7 / 31-33)
//   k_adjoint_tiled  P2G^T of substep n + G2P^T of substep n-1 (Section 2.3)
//
// They compute exactly what k_forward / k_adjoint (particle_kernels.cuh)
// compute without solid boxes or a field gradient (with either set the runtime
// runs those instead);
// only the grid traffic differs (see tile.cuh): node values are staged once
// per CTA (with the grid operation, Eq. 16-18, or its reverse applied per tile
// node in fused-grid mode) and scatters are warp-aggregated into a
// shared-memory tile that is flushed with one float4 atomic per node.
#include "kernels.h"
#include "particle_io.cuh"
#include "tile.cuh"

namespace mpm {

namespace {

// value of a gather node: from the staged tile, or straight from global
// memory (direct path, through the grid operation in fused-grid mode)
template <int D, bool FUSE>
__device__ __forceinline__ float4 gather_node(const TileBox<D>& box, const float4* tile,
                                              const float4* __restrict__ direct,
                                              const NodeTerm<D>& t, const Params& P, int step) {
    if (box.use) return tile[box_index<D>(box, t.c)];
    float gv[D];
    node_velocity<D, FUSE, false>(direct, t, P, gv, step);
    return make_float4(gv[0], gv[1 % D], D == 3 ? gv[2 % D] : 0.0f, 0.0f);
}

// grid velocity of node c for the tile: V written by the grid kernel, or the
// grid operation applied to the accumulator (fused grid)
template <int D, bool FUSE>
__device__ __forceinline__ float4 stage_velocity(const float4* __restrict__ src, const int (&c)[D],
                                                 const Params& P, int step) {
    const float4 g = __ldg(src + grid_index<D>(c, P.res));
    if (!FUSE) return g;
    float mv[D], v[D];
    unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mv);
    grid_velocity<D, false>(P, c, g.x, mv, v, step);
    return make_float4(v[0], v[1 % D], D == 3 ? v[2 % D] : 0.0f, 0.0f);
}

// Adds the D+1 values of every lane into tile node `li`, after summing lanes of
// the same run.  All lanes of the warp call it (inactive lanes with zeros).
template <int NV>
__device__ __forceinline__ void scatter_tile(float (&val)[NV], const Segments& sg, bool write,
                                             float* tile, int li) {
#pragma unroll
    for (int c = 0; c < NV; ++c) val[c] = seg_sum(val[c], sg);
    if (write && sg.head) {
#pragma unroll
        for (int c = 0; c < NV; ++c)
            if (val[c] != 0.0f) atomicAdd(tile + 4 * li + c, val[c]);
    }
}

// ---------------------------------------------------------------------------
template <int D, bool WRITE_ALL, bool FUSE>
__global__ void __launch_bounds__(256) k_forward_tiled(Params P, StepArgs a) {
    using L = Layout<D>;
    __shared__ float4 tileV[kTileMax];
    __shared__ float4 tileA[kTileMax];
    __shared__ int red[(2 * D + 2) * 32];
    __shared__ TileBox<D> s_box;
    pdl_wait();
    pdl_trigger();
    if (FUSE) clear_buffer(a);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < P.n_total;
    const int inst = active ? find_instance(a.inst_off, P.n_inst, p) : -1;
    const long long np = P.np;
    int flags = 0;
    float x[D], v[D], C[D][D], F[D][D];
    float phi = 0.0f, mp = 0.0f;
    Stencil<D> s;
#pragma unroll
    for (int i = 0; i < D; ++i) s.base[i] = 0;
    if (active) {
        load_vec<D>(a.s_in, L::X, np, p, x);
        load_mat<D>(a.s_in, L::F, np, p, F);
        phi = a.phi[p];
        mp = phi * P.rho0 * P.p_vol;  // Eq. 33
        if (!make_stencil<D>(x, P, s)) flags |= kErrDomain;
    }
    // ---- G2P of substep n: stage the grid velocity of the CTA's box ----
    TileBox<D> box;
    block_box<D>(s.base, active, inst, box, red, &s_box);
    for (int t = threadIdx.x; t < kTileMax; t += blockDim.x) tileA[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    {
        const float4* src = (FUSE ? a.accG : a.V) + (long long)box.inst * P.nodes;
        for (int t = threadIdx.x; t < box.n; t += blockDim.x) {
            int c[D];
            box_coords<D>(box, t, c);
            tileV[t] = stage_velocity<D, FUSE>(src, c, P, a.n_g2p);
        }
    }
    __syncthreads();
    float mom_x[1] = {0.0f};
    if (active) {
        const float4* direct = (FUSE ? a.accG : a.V) + (long long)inst * P.nodes;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            v[i] = 0.0f;
#pragma unroll
            for (int j = 0; j < D; ++j) C[i][j] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < stencil_size<D>(); ++k) {
            NodeTerm<D> t;
            node_term<D>(s, k, P, t);
            float gv[D];
            unpack3<D>(gather_node<D, FUSE>(box, tileV, direct, t, P, a.n_g2p), gv);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                v[i] += t.w * gv[i];  // Eq. 19
#pragma unroll
                for (int j = 0; j < D; ++j) C[i][j] += t.w * gv[i] * t.dpos[j];  // Eq. 20
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int j = 0; j < D; ++j) C[i][j] *= P.kappa;
            x[i] += P.dt * v[i];  // Eq. 21
        }
        float Fn[D][D];  // Eq. 22 in strain form: E' = E + dt C (I + E)
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
        const float Jm1 = det_minus_one<D>(F);
        if (!(Jm1 > -1.0f) || !isfinite(Jm1)) flags |= kErrNumeric;
        store_vec<D>(a.s_out, L::X, np, p, x);
        store_mat<D>(a.s_out, L::F, np, p, F);
        if (WRITE_ALL) {
            store_vec<D>(a.s_out, L::V, np, p, v);
            store_mat<D>(a.s_out, L::C, np, p, C);
        }
        mom_x[0] = mp * v[0];
    }
    if (P.loss_kind == 1 && a.mom != nullptr)
        warp_add_per_instance<1>(mom_x, inst, a.mom + (long long)a.n_g2p * P.n_inst, 1);

    // ---- P2G of substep n+1 at the new positions ----
    const bool p2g = a.acc != nullptr;
    Stencil<D> s2;
#pragma unroll
    for (int i = 0; i < D; ++i) s2.base[i] = 0;
    float A[D][D];
    if (p2g && active) {
        if (!make_stencil<D>(x, P, s2)) flags |= kErrDomain;
        StressParts<D> S;
        stress_parts<D>(F, phi, P, S);
        if (!(S.J > 0.0f)) flags |= kErrNumeric;
        float Br[D], Ba[D], Pk[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            Br[i] = a.mag[(long long)i * np + p];
            Ba[i] = __ldg(a.field + ((long long)inst * P.n_steps + a.n_p2g) * D + i);
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
                A[i][j] = mp * C[i][j] - sc * pft;  // MLS-MPM affine momentum
            }
    }
    if (p2g) {
        TileBox<D> box2;
        block_box<D>(s2.base, active, inst, box2, red, &s_box);
        if (box2.use) {
            const int lane = threadIdx.x & 31;
            const Segments sg = make_segments(active ? box_index<D>(box2, s2.base) : -1 - lane);
            float* tA = reinterpret_cast<float*>(tileA);
#pragma unroll
            for (int k = 0; k < stencil_size<D>(); ++k) {
                NodeTerm<D> t;
                float val[D + 1];
                int li = 0;
#pragma unroll
                for (int c = 0; c <= D; ++c) val[c] = 0.0f;
                if (active) {
                    node_term<D>(s2, k, P, t);
                    li = box_index<D>(box2, t.c);
                    val[0] = t.w * mp;  // Eq. 14
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        float ad = 0.0f;
#pragma unroll
                        for (int j = 0; j < D; ++j) ad += A[i][j] * t.dpos[j];
                        val[1 + i] = t.w * (mp * v[i] + ad);  // Eq. 15
                    }
                }
                scatter_tile<D + 1>(val, sg, active, tA, li);
            }
            __syncthreads();
            flush_tile<D>(box2, tileA, a.acc, P);
        } else if (active) {
            float4* __restrict__ ai = a.acc + (long long)inst * P.nodes;
#pragma unroll
            for (int k = 0; k < stencil_size<D>(); ++k) {
                NodeTerm<D> t;
                node_term<D>(s2, k, P, t);
                float mv[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    float ad = 0.0f;
#pragma unroll
                    for (int j = 0; j < D; ++j) ad += A[i][j] * t.dpos[j];
                    mv[i] = t.w * (mp * v[i] + ad);
                }
                atomicAdd(ai + t.node, pack4<D>(t.w * mp, mv));
            }
        }
    }
    if (flags) atomicOr(a.err, flags);
}

// ---------------------------------------------------------------------------
// FUSE: grid adjoint staged from (accP, VbarIn); FUSE_V: grid velocity of
// substep n-1 staged from accG through the grid operation.
template <int D, bool FUSE, bool FUSE_V>
__global__ void __launch_bounds__(256) k_adjoint_tiled(Params P, StepArgs a) {
    using L = Layout<D>;
    __shared__ float4 tileG[kTileMax];  // grid adjoint of substep n, then V of n-1
    __shared__ float4 tileS[kTileMax];  // Vbar scatter of substep n-1
    __shared__ int red[(2 * D + 2) * 32];
    __shared__ TileBox<D> s_box;
    pdl_wait();
    pdl_trigger();
    clear_buffer(a);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < P.n_total;
    const int inst = active ? find_instance(a.inst_off, P.n_inst, p) : -1;
    const long long np = P.np;
    const int n = a.n_p2g;
    int flags = 0;
    float xb[D], vb[D], Cb[D][D], Fb[D][D], Cn[D][D];
    float x[D], v[D], F[D][D];
    float phi = 0.0f, mp = 0.0f;
    float bab[D];
#pragma unroll
    for (int i = 0; i < D; ++i) bab[i] = 0.0f;
    Stencil<D> s;
#pragma unroll
    for (int i = 0; i < D; ++i) s.base[i] = 0;
    if (active) {
        load_vec<D>(a.s_in, L::X, np, p, x);
        load_vec<D>(a.s_in, L::V, np, p, v);
        load_mat<D>(a.s_in, L::C, np, p, Cn);
        load_mat<D>(a.s_in, L::F, np, p, F);
        load_vec<D>(a.adj, L::X, np, p, xb);
        load_mat<D>(a.adj, L::F, np, p, Fb);
        phi = a.phi[p];
        mp = phi * P.rho0 * P.p_vol;
        if (!make_stencil<D>(x, P, s)) flags |= kErrDomain;
    }
    // ---- stage the grid adjoint of substep n ----
    TileBox<D> box;
    block_box<D>(s.base, active, inst, box, red, &s_box);
    for (int t = threadIdx.x; t < kTileMax; t += blockDim.x) tileS[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    {
        const long long off = (long long)box.inst * P.nodes;
        for (int t = threadIdx.x; t < box.n; t += blockDim.x) {
            int c[D];
            box_coords<D>(box, t, c);
            const long long gi = off + grid_index<D>(c, P.res);
            if (FUSE) {
                const float4 g = __ldg(a.accP + gi);
                float mv[D], vbv[D], mvb[D], mbv;
                unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mv);
                unpack3<D>(__ldg(a.VbarIn + gi), vbv);
                grid_velocity_adjoint<D, false>(P, c, g.x, mv, vbv, mbv, mvb, a.n_p2g);
                tileG[t] = pack4<D>(mbv, mvb);
            } else {
                tileG[t] = __ldg(a.gadj + gi);
            }
        }
    }
    __syncthreads();
    // ---- P2G^T of substep n ----
    if (active) {
        float Br[D], Ba[D], Pk[D][D], A[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            Br[i] = a.mag[(long long)i * np + p];
            Ba[i] = __ldg(a.field + ((long long)inst * P.n_steps + n) * D + i);
        }
        StressParts<D> S;
        stress_parts<D>(F, phi, P, S);
        piola<D>(S, Br, Ba, Pk);
        const float sc = P.dt * P.kappa * P.p_vol;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                float pft = Pk[i][j];
#pragma unroll
                for (int k = 0; k < D; ++k) pft += Pk[i][k] * F[j][k];
                A[i][j] = mp * Cn[i][j] - sc * pft;
            }
        float mpb = 0.0f, Ab[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            vb[i] = 0.0f;
#pragma unroll
            for (int j = 0; j < D; ++j) Ab[i][j] = 0.0f;
        }
        const long long off = (long long)inst * P.nodes;
#pragma unroll
        for (int k = 0; k < stencil_size<D>(); ++k) {
            NodeTerm<D> t;
            node_term<D>(s, k, P, t);
            float4 g;
            if (box.use) {
                g = tileG[box_index<D>(box, t.c)];
            } else if (FUSE) {
                const float4 g4 = __ldg(a.accP + off + t.node);
                float mv[D], vbv[D], mvb[D], mbv;
                unpack3<D>(make_float4(g4.y, g4.z, g4.w, 0.0f), mv);
                unpack3<D>(__ldg(a.VbarIn + off + t.node), vbv);
                grid_velocity_adjoint<D, false>(P, t.c, g4.x, mv, vbv, mbv, mvb, a.n_p2g);
                g = pack4<D>(mbv, mvb);
            } else {
                g = __ldg(a.gadj + off + t.node);
            }
            float mvb[D];
            unpack3<D>(make_float4(g.y, g.z, g.w, 0.0f), mvb);
            float inner = g.x * mp, vcd = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                float ad = 0.0f, cd = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    ad += A[i][j] * t.dpos[j];
                    cd += Cn[i][j] * t.dpos[j];
                }
                inner += mvb[i] * (mp * v[i] + ad);
                vcd += mvb[i] * (v[i] + cd);
            }
            mpb += t.w * (g.x + vcd);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                vb[i] += t.w * mp * mvb[i];
#pragma unroll
                for (int j = 0; j < D; ++j) Ab[i][j] += t.w * mvb[i] * t.dpos[j];
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float atm = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i) atm += A[i][c] * mvb[i];
                xb[c] += t.gw[c] * inner - t.w * atm;
            }
        }
        float Pb[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) Cb[i][j] = mp * Ab[i][j];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                float pb = Ab[i][j], fb = 0.0f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    pb += Ab[i][k] * F[k][j];
                    fb += Ab[k][i] * Pk[k][j];
                }
                Pb[i][j] = -sc * pb;
                Fb[i][j] -= sc * fb;
            }
        float phib = 0.0f, brb[D];
#pragma unroll
        for (int i = 0; i < D; ++i) brb[i] = 0.0f;
        piola_adjoint<D>(F, phi, S, Br, Ba, Pb, P, Fb, phib, brb, bab);
        float gph = phib + mpb * P.rho0 * P.p_vol;
        if (P.loss_kind == 1 && n >= 1) {  // locomotion seed on state n, Eq. 40
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
    warp_add_per_instance<D>(bab, inst, a.gfield + (long long)n * D, (long long)P.n_steps * D);

    // ---- G2P^T of substep n-1 ----
    Stencil<D> s2;
#pragma unroll
    for (int i = 0; i < D; ++i) s2.base[i] = 0;
    float Fm[D][D];
    if (active) {
        load_vec<D>(a.s_aux, L::X, np, p, x);
        load_mat<D>(a.s_aux, L::F, np, p, Fm);
        if (!make_stencil<D>(x, P, s2)) flags |= kErrDomain;
    }
    TileBox<D> box2;
    block_box<D>(s2.base, active, inst, box2, red, &s_box);  // all gathers from tileG are done
    {
        const float4* src = (FUSE_V ? a.accG : a.V) + (long long)box2.inst * P.nodes;
        for (int t = threadIdx.x; t < box2.n; t += blockDim.x) {
            int c[D];
            box_coords<D>(box2, t, c);
            tileG[t] = stage_velocity<D, FUSE_V>(src, c, P, a.n_p2g - 1);
        }
    }
    __syncthreads();
    float vt[D], Ct[D][D], Fo[D][D];
    if (active) {
#pragma unroll
        for (int i = 0; i < D; ++i) vt[i] = vb[i] + P.dt * xb[i];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                float fft = Fb[i][j], ctf = Fb[i][j];  // F = I + E
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    fft += Fb[i][k] * Fm[j][k];         // (Fbar F^T)_ij
                    ctf += P.dt * Cn[k][i] * Fb[k][j];  // ((I + dt C')^T Fbar)_ij
                }
                Ct[i][j] = Cb[i][j] + P.dt * fft;
                Fo[i][j] = ctf;
            }
    }
    const int lane = threadIdx.x & 31;
    const Segments sg = make_segments(active && box2.use ? box_index<D>(box2, s2.base) : -1 - lane);
    const float4* direct = (FUSE_V ? a.accG : a.V) + (long long)(active ? inst : 0) * P.nodes;
    float4* __restrict__ Vbi = a.Vbar + (long long)(active ? inst : 0) * P.nodes;
    float* tS = reinterpret_cast<float*>(tileS);
#pragma unroll
    for (int k = 0; k < stencil_size<D>(); ++k) {
        NodeTerm<D> t;
        float sv[D];
        int li = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) sv[i] = 0.0f;
        if (active) {
            node_term<D>(s2, k, P, t);
            float gv[D];
            unpack3<D>(gather_node<D, FUSE_V>(box2, tileG, direct, t, P, a.n_p2g - 1), gv);
            float vdot = 0.0f, vcd = 0.0f, cd[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                cd[i] = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) cd[i] += Ct[i][j] * t.dpos[j];
                vdot += gv[i] * vt[i];
                vcd += gv[i] * cd[i];
            }
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float ctv = 0.0f;
#pragma unroll
                for (int i = 0; i < D; ++i) ctv += Ct[i][c] * gv[i];
                xb[c] += t.gw[c] * (vdot + P.kappa * vcd) - P.kappa * t.w * ctv;
            }
#pragma unroll
            for (int i = 0; i < D; ++i) sv[i] = t.w * (vt[i] + P.kappa * cd[i]);
            if (box2.use) li = box_index<D>(box2, t.c);
        }
        if (box2.use) {
            float val[D];
#pragma unroll
            for (int i = 0; i < D; ++i) val[i] = sv[i];
            scatter_tile<D>(val, sg, active, tS, li);
        } else if (active) {
            atomicAdd(Vbi + t.node, make_float4(sv[0], sv[1 % D], D == 3 ? sv[2 % D] : 0.0f, 0.0f));
        }
    }
    if (active) {
        store_vec<D>(a.adj, L::X, np, p, xb);
        store_mat<D>(a.adj, L::F, np, p, Fo);
    }
    if (box2.use) {
        __syncthreads();
        flush_tile<D>(box2, tileS, a.Vbar, P);
    }
    if (flags) atomicOr(a.err, flags);
}

inline int blocks_for(long long n, int block) { return (int)((n + block - 1) / block); }

template <int D, bool FUSE>
cudaError_t forward_tiled_d(bool all, const Params& P, const StepArgs& a, int block, cudaStream_t st) {
    if (P.n_total == 0 && !(FUSE && a.zero4)) return cudaSuccess;
    dim3 grid(blocks_for(P.n_total > 0 ? P.n_total : block, block));
    if (all) return launch_chain(P, k_forward_tiled<D, true, FUSE>, grid, dim3(block), st, P, a);
    return launch_chain(P, k_forward_tiled<D, false, FUSE>, grid, dim3(block), st, P, a);
}

template <int D, bool FUSE, bool FUSE_V>
cudaError_t adjoint_tiled_d(const Params& P, const StepArgs& a, int block, cudaStream_t st) {
    if (P.n_total == 0 && !a.zero4) return cudaSuccess;
    dim3 grid(blocks_for(P.n_total > 0 ? P.n_total : block, block));
    return launch_chain(P, k_adjoint_tiled<D, FUSE, FUSE_V>, grid, dim3(block), st, P, a);
}

template <int D>
cudaError_t adjoint_tiled_dim(bool fuse, bool fuse_v, const Params& P, const StepArgs& a, int block,
                              cudaStream_t st) {
    if (fuse) return adjoint_tiled_d<D, true, true>(P, a, block, st);
    if (fuse_v) return adjoint_tiled_d<D, false, true>(P, a, block, st);
    return adjoint_tiled_d<D, false, false>(P, a, block, st);
}

}  // namespace

cudaError_t launch_forward_tiled(int dim, bool write_all, bool fuse, const Params& P,
                                 const StepArgs& a, int block, cudaStream_t st) {
    if (dim == 2)
        return fuse ? forward_tiled_d<2, true>(write_all, P, a, block, st)
                    : forward_tiled_d<2, false>(write_all, P, a, block, st);
    return fuse ? forward_tiled_d<3, true>(write_all, P, a, block, st)
                : forward_tiled_d<3, false>(write_all, P, a, block, st);
}

cudaError_t launch_adjoint_tiled(int dim, bool fuse, bool fuse_v, const Params& P, const StepArgs& a,
                                 int block, cudaStream_t st) {
    return dim == 2 ? adjoint_tiled_dim<2>(fuse, fuse_v, P, a, block, st)
                    : adjoint_tiled_dim<3>(fuse, fuse_v, P, a, block, st);
}

}  // namespace mpm
