// Design representation and optimiser step (arxiv 2503.22767, Sections
// 3.1-3.2): density filter (Eq. 23-24), Heaviside projection (Eq. 25),
// magnetisation maps (Eq. 26-28), harmonic stimulus (Eq. 29-30), their
// reverse modes, and Adam with box clipping (Eq. 34c-d).
//
// Readings of the paper: Eq. 23's numerator weights the neighbour's variable
// phi_{p'}.  The neighbourhood is |x_p'(0) - x_p(0)| < R, p included.  Eq. 25's
// parameter is beta.  The field is sampled at t_n = n dt.
//
// The filter bins x(0) once into cells whose edge is at least R, sorted by
// cell with the library's counting sort, so every neighbour of a particle
// lies in the 3^d cells around its own.  Forward and reverse are gathers
// over those cells, with no atomics.  The reverse reuses the symmetry
// w_pp' = w_p'p: dL/dphi_p' = sum_p w_p'p (g_p / W_p), with W_p = sum w_pp'.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <string>

#include "kernels.h"
#include "mpm_design.h"

namespace {

constexpr long long kMaxFilterCells = 1LL << 24;
constexpr int kSmemRegionFloats = 8192;  // region sums staged per block when they fit

struct FilterGrid {
    int nc;       // cells per axis
    float inv_h;  // cells per unit length
    float R;
};

template <int D>
__device__ __forceinline__ void cell_of(const float (&x)[D], const FilterGrid& g, int (&c)[D]) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int i = (int)floorf(x[a] * g.inv_h);
        c[a] = min(max(i, 0), g.nc - 1);
    }
}

template <int D>
__device__ __forceinline__ int cell_index(const int (&c)[D], int nc) {
    int k = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) k = k * nc + c[a];
    return k;
}

template <int D>
__global__ void k_filter_keys(const float* __restrict__ x0, int n, FilterGrid g, int* __restrict__ keys,
                              int* __restrict__ slot, int* __restrict__ counts) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float x[D];
    int c[D];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = x0[(long long)a * n + p];
    cell_of<D>(x, g, c);
    int k = cell_index<D>(c, g.nc);
    keys[p] = k;
    slot[p] = atomicAdd(counts + k, 1);
}

__global__ void k_filter_scatter(const int* __restrict__ keys, const int* __restrict__ slot,
                                 const int* __restrict__ offsets, int n, int* __restrict__ order) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) order[offsets[keys[p]] + slot[p]] = p;
}

// Cell members in increasing particle index, so every sum below runs in a
// fixed order.
__global__ void k_filter_order_cells(const int* __restrict__ counts, const int* __restrict__ offsets,
                                     int* __restrict__ order, long long n_cells) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_cells) return;
    int c = counts[k];
    int* v = order + offsets[k];
    for (int i = 1; i < c; ++i) {
        int key = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > key) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = key;
    }
}

// out_p = sum_{|x_p' - x_p| < R} (1 - |x_p' - x_p| / R) val_p'  (Eq. 23-24),
// divided by norm_p when norm is given; val == nullptr sums the weights
// alone (the normaliser W_p).  One thread per particle, in cell order.
template <int D>
__global__ void __launch_bounds__(256) k_filter_apply(const float* __restrict__ x0, int n, FilterGrid g,
                                                      const int* __restrict__ order,
                                                      const int* __restrict__ offsets,
                                                      const float* __restrict__ val,
                                                      const float* __restrict__ norm, float* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int p = order[t];
    float x[D];
    int c[D];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = x0[(long long)a * n + p];
    cell_of<D>(x, g, c);
    int lo[D], hi[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = max(c[a] - 1, 0);
        hi[a] = min(c[a] + 1, g.nc - 1);
    }
    const float rR = 1.0f / g.R;
    float acc = 0.0f;
    int cc[D];
    // visit the (up to) 3^d neighbour cells
    for (int k = 0; k < (D == 2 ? 9 : 27); ++k) {
        int r = k;
        bool in = true;
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
            cc[a] = c[a] - 1 + r % 3;
            r /= 3;
            in = in && cc[a] >= lo[a] && cc[a] <= hi[a];
        }
        if (!in) continue;
        const int cell = cell_index<D>(cc, g.nc);
        const int j1 = offsets[cell + 1];
        for (int j = offsets[cell]; j < j1; ++j) {
            const int q = order[j];
            float d2 = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float dx = x0[(long long)a * n + q] - x[a];
                d2 += dx * dx;
            }
            const float dist = sqrtf(d2);
            if (dist < g.R) {
                const float w = 1.0f - dist * rR;
                acc += val ? w * val[q] : w;
            }
        }
    }
    out[p] = norm ? acc / norm[p] : acc;
}

// Eq. 25 and its reverse
__device__ __forceinline__ float heaviside(float x, float beta, float t_half) {
    return (t_half + tanhf(beta * (x - 0.5f))) / (2.0f * t_half);
}

__global__ void k_heaviside(const float* __restrict__ phi_t, int n, float beta, float t_half,
                            float* __restrict__ phi_bar) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) phi_bar[p] = heaviside(phi_t[p], beta, t_half);
}

// u_p = (dL/dphi_bar_p) dH/dphi~ / W_p: the vector the transposed filter gathers
__global__ void k_heaviside_adjoint(const float* __restrict__ phi_t, const float* __restrict__ g, int n,
                                    float beta, float t_half, const float* __restrict__ norm,
                                    float* __restrict__ u) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float th = tanhf(beta * (phi_t[p] - 0.5f));
    u[p] = g[p] * beta * (1.0f - th * th) / (2.0f * t_half) / norm[p];
}

// Eq. 26-28
template <int D>
__global__ void k_magnetization(const float* __restrict__ Br, const float* __restrict__ zeta,
                                const int* __restrict__ region, int n, int n_m, float Br_max, float delta,
                                float* __restrict__ mag) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int r = region ? region[p] : p;
    float z[D], s2 = delta;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        z[i] = zeta[(long long)i * n_m + r];
        s2 += z[i] * z[i];
    }
    const float a = Br_max * Br[r] / sqrtf(s2);
#pragma unroll
    for (int i = 0; i < D; ++i) mag[(long long)i * n + p] = a * z[i];
}

// Reverse of Eq. 26-28.  With b = zeta / s, s = sqrt(|zeta|^2 + delta):
//   dL/dBr = Br_max g.b,  dL/dzeta = Br_max Br (g - b (g.b)) / s,
// summed over the particles of a region (block-staged in shared memory
// when the region table fits, else straight to global memory).
template <int D>
__global__ void __launch_bounds__(256) k_magnetization_adjoint(
    const float* __restrict__ Br, const float* __restrict__ zeta, const int* __restrict__ region, int n, int n_m,
    float Br_max, float delta, const float* __restrict__ g, float* __restrict__ g_Br, float* __restrict__ g_zeta,
    bool stage) {
    extern __shared__ float s_acc[];  // [n_m] Br, then [D][n_m] zeta
    if (stage) {
        for (int i = threadIdx.x; i < (1 + D) * n_m; i += blockDim.x) s_acc[i] = 0.0f;
        __syncthreads();
    }
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        const int r = region ? region[p] : p;
        float z[D], gp[D], s2 = delta;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            z[i] = zeta[(long long)i * n_m + r];
            gp[i] = g[(long long)i * n + p];
            s2 += z[i] * z[i];
        }
        const float s = sqrtf(s2);
        float gb = 0.0f;
#pragma unroll
        for (int i = 0; i < D; ++i) gb += gp[i] * (z[i] / s);
        const float a = Br_max * Br[r] / s;
        if (!region) {
            g_Br[r] = Br_max * gb;
#pragma unroll
            for (int i = 0; i < D; ++i) g_zeta[(long long)i * n_m + r] = a * (gp[i] - (z[i] / s) * gb);
        } else if (stage) {
            atomicAdd(s_acc + r, Br_max * gb);
#pragma unroll
            for (int i = 0; i < D; ++i) atomicAdd(s_acc + (1 + i) * n_m + r, a * (gp[i] - (z[i] / s) * gb));
        } else {
            atomicAdd(g_Br + r, Br_max * gb);
#pragma unroll
            for (int i = 0; i < D; ++i) atomicAdd(g_zeta + (long long)i * n_m + r, a * (gp[i] - (z[i] / s) * gb));
        }
    }
    if (stage) {
        __syncthreads();
        for (int i = threadIdx.x; i < (1 + D) * n_m; i += blockDim.x) {
            const float v = s_acc[i];
            if (v != 0.0f) atomicAdd(i < n_m ? g_Br + i : g_zeta + (i - n_m), v);
        }
    }
}

// Eq. 29-30: field[l][n][i] = B_max Ba_l sin(2 pi fbar_l t_n) b_l,i
template <int D>
__global__ void k_stimulus(const float* __restrict__ Ba, const float* __restrict__ f, const float* __restrict__ eta,
                           int n_tasks, int n_steps, float dt, float B_max, float f_min, float f_max, float delta,
                           float* __restrict__ field) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_tasks * n_steps) return;
    const int l = (int)(i / n_steps), s = (int)(i % n_steps);
    float e[D], s2 = delta;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        e[c] = eta[l * D + c];
        s2 += e[c] * e[c];
    }
    const float fbar = (f_max - f_min) * f[l] + f_min;
    const float amp = B_max * Ba[l] * sinf(2.0f * 3.14159265358979f * fbar * ((float)s * dt)) / sqrtf(s2);
#pragma unroll
    for (int c = 0; c < D; ++c) field[i * D + c] = amp * e[c];
}

// Reverse of Eq. 29-30: one block per task reduces over the substeps.
template <int D>
__global__ void __launch_bounds__(256) k_stimulus_adjoint(const float* __restrict__ Ba, const float* __restrict__ f,
                                                          const float* __restrict__ eta, int n_steps, float dt,
                                                          float B_max, float f_min, float f_max, float delta,
                                                          const float* __restrict__ g, float* __restrict__ g_Ba,
                                                          float* __restrict__ g_f, float* __restrict__ g_eta) {
    const int l = blockIdx.x;
    float e[D], b[D], s2 = delta;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        e[c] = eta[l * D + c];
        s2 += e[c] * e[c];
    }
    const float s = sqrtf(s2);
#pragma unroll
    for (int c = 0; c < D; ++c) b[c] = e[c] / s;
    const float fbar = (f_max - f_min) * f[l] + f_min;
    const float w = 2.0f * 3.14159265358979f;
    // per thread: sum sin (g.b), sum cos t (g.b), sum sin g_c
    float acc[2 + D];
#pragma unroll
    for (int c = 0; c < 2 + D; ++c) acc[c] = 0.0f;
    for (int n = threadIdx.x; n < n_steps; n += blockDim.x) {
        const float t = (float)n * dt;
        float sn, cs;
        sincosf(w * fbar * t, &sn, &cs);
        const float* gn = g + ((long long)l * n_steps + n) * D;
        float gb = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            gb += gn[c] * b[c];
            acc[2 + c] += sn * gn[c];
        }
        acc[0] += sn * gb;
        acc[1] += cs * w * t * gb;
    }
    __shared__ float red[2 + D][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < 2 + D; ++c) {
        float v = acc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot[2 + D];
#pragma unroll
        for (int c = 0; c < 2 + D; ++c) {
            tot[c] = 0.0f;
            for (int k = 0; k < nw; ++k) tot[c] += red[c][k];
        }
        const float Bl = B_max * Ba[l];
        g_Ba[l] = B_max * tot[0];
        g_f[l] = Bl * tot[1] * (f_max - f_min);
        // dL/db = Bl sum sin g; through b = eta / s
        float gbv[D], proj = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            gbv[c] = Bl * tot[2 + c];
            proj += gbv[c] * b[c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) g_eta[l * D + c] = (gbv[c] - b[c] * proj) / s;
    }
}

__global__ void k_adam(long long n, float* __restrict__ x, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2, float lo,
                       float hi) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float xi = x[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    x[i] = fminf(fmaxf(xi, lo), hi);
}

__global__ void k_check_regions(const int* __restrict__ region, int n, int n_m, int* __restrict__ bad) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && (region[p] < 0 || region[p] >= n_m)) atomicOr(bad, 1);
}

unsigned blocks(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct mpm_design {
    mpm_design_config cfg{};
    int n_m = 0;
    FilterGrid grid{};
    long long n_cells = 0;
    float* x0 = nullptr;       // [d][N]
    int* region = nullptr;     // [N] or null
    int* order = nullptr;      // particles in cell order
    int* offsets = nullptr;    // [n_cells + 1]
    float* norm = nullptr;     // W_p
    float* phi_t = nullptr;    // phi~ of the last forward
    float* u = nullptr;        // reverse scratch
    float* in_Br = nullptr;    // material and stimulus inputs of the last forward:
    float* in_zeta = nullptr;  //   Br [n_m], zeta [d][n_m], Ba, f [n_tasks],
    float* in_Ba = nullptr;    //   eta [n_tasks][d]
    float* in_f = nullptr;
    float* in_eta = nullptr;
    float beta = 0.0f;
    bool forward_done = false;
    std::string err;
};

namespace {

int fail(mpm_design* h, int code, const std::string& why) {
    if (h) h->err = why;
    return code;
}

#define DCUDA(h, call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return fail(h, MPM_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

void release(mpm_design* h) {
    for (void* ptr : {(void*)h->x0, (void*)h->region, (void*)h->order, (void*)h->offsets, (void*)h->norm,
                      (void*)h->phi_t, (void*)h->u, (void*)h->in_Br, (void*)h->in_zeta, (void*)h->in_Ba,
                      (void*)h->in_f, (void*)h->in_eta})
        if (ptr) cudaFree(ptr);
}

int create_impl(mpm_design* h, const mpm_design_config* c, const float* x0, const int* region, cudaStream_t st) {
    const int d = c->dim, n = c->n_particles;
    h->cfg = *c;
    h->n_m = c->n_regions > 0 ? c->n_regions : n;
    // cells of edge >= R: floor(1 / R) per axis, capped
    long long nc = (long long)std::floor(1.0 / c->filter_radius);
    if (nc < 1) nc = 1;
    const long long cap = d == 2 ? 4096 : 256;  // cap^d = kMaxFilterCells
    if (nc > cap) nc = cap;
    h->grid.nc = (int)nc;
    h->grid.inv_h = (float)nc;
    h->grid.R = (float)c->filter_radius;
    h->n_cells = 1;
    for (int a = 0; a < d; ++a) h->n_cells *= nc;
    if (h->n_cells > kMaxFilterCells) return fail(h, MPM_ERR_ARG, "filter grid too large");
    const long long tmp_len = mpm::sort_scan_tmp_len(h->n_cells + 1);
    int *keys = nullptr, *slot = nullptr, *counts = nullptr, *tmp = nullptr, *bad = nullptr;
    auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes > 0 ? bytes : 4) == cudaSuccess; };
    bool ok = alloc((void**)&h->x0, sizeof(float) * d * (size_t)n) && alloc((void**)&h->order, sizeof(int) * (size_t)n) &&
              alloc((void**)&h->offsets, sizeof(int) * (size_t)(h->n_cells + 1)) &&
              alloc((void**)&h->norm, sizeof(float) * (size_t)n) && alloc((void**)&h->phi_t, sizeof(float) * (size_t)n) &&
              alloc((void**)&h->u, sizeof(float) * (size_t)n) && alloc((void**)&keys, sizeof(int) * (size_t)n) &&
              alloc((void**)&slot, sizeof(int) * (size_t)n) &&
              alloc((void**)&counts, sizeof(int) * (size_t)(h->n_cells + 1)) &&
              alloc((void**)&tmp, sizeof(int) * (size_t)tmp_len) && alloc((void**)&bad, sizeof(int)) &&
              alloc((void**)&h->in_Br, sizeof(float) * (size_t)h->n_m) &&
              alloc((void**)&h->in_zeta, sizeof(float) * d * (size_t)h->n_m) &&
              alloc((void**)&h->in_Ba, sizeof(float) * (size_t)c->n_tasks) &&
              alloc((void**)&h->in_f, sizeof(float) * (size_t)c->n_tasks) &&
              alloc((void**)&h->in_eta, sizeof(float) * d * (size_t)c->n_tasks);
    if (ok && region) ok = alloc((void**)&h->region, sizeof(int) * (size_t)n);
    int rc = MPM_OK;
    if (!ok) {
        cudaGetLastError();
        rc = fail(h, MPM_ERR_OOM, "device allocation failed");
    }
    auto step = [&](cudaError_t e, const char* what) {
        if (rc == MPM_OK && e != cudaSuccess) rc = fail(h, MPM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    if (rc == MPM_OK) {
        step(cudaMemcpyAsync(h->x0, x0, sizeof(float) * d * (size_t)n, cudaMemcpyDeviceToDevice, st), "copy x0");
        if (region) {
            step(cudaMemcpyAsync(h->region, region, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st), "copy region");
            step(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset");
            if (n > 0) k_check_regions<<<blocks(n), 256, 0, st>>>(h->region, n, h->n_m, bad);
            step(cudaGetLastError(), "k_check_regions");
        }
        step(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)(h->n_cells + 1), st), "memset");
        if (n > 0) {
            if (d == 2) k_filter_keys<2><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, keys, slot, counts);
            else k_filter_keys<3><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, keys, slot, counts);
            step(cudaGetLastError(), "k_filter_keys");
        }
        // offsets over n_cells + 1 entries: the last one is the total
        step(mpm::launch_scan_exclusive(counts, h->offsets, h->n_cells + 1, tmp, st), "scan");
        if (n > 0) {
            k_filter_scatter<<<blocks(n), 256, 0, st>>>(keys, slot, h->offsets, n, h->order);
            step(cudaGetLastError(), "k_filter_scatter");
            k_filter_order_cells<<<blocks(h->n_cells), 256, 0, st>>>(counts, h->offsets, h->order, h->n_cells);
            step(cudaGetLastError(), "k_filter_order_cells");
            // normalisers W_p = sum_p' w_pp'
            if (d == 2)
                k_filter_apply<2><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, h->order, h->offsets, nullptr,
                                                             nullptr, h->norm);
            else
                k_filter_apply<3><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, h->order, h->offsets, nullptr,
                                                             nullptr, h->norm);
            step(cudaGetLastError(), "k_filter_apply");
        }
    }
    int bad_h = 0;
    if (rc == MPM_OK && region) step(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    if (rc == MPM_OK) step(cudaStreamSynchronize(st), "synchronize");
    if (rc == MPM_OK && bad_h) rc = fail(h, MPM_ERR_ARG, "a region index is outside [0, n_regions)");
    for (void* ptr : {(void*)keys, (void*)slot, (void*)counts, (void*)tmp, (void*)bad})
        if (ptr) cudaFree(ptr);
    return rc;
}

}  // namespace

extern "C" {

int mpm_design_create(const mpm_design_config* c, const float* x0, const int* region, mpm_design** out,
                      void* cuda_stream) {
    if (!out) return MPM_ERR_ARG;
    *out = nullptr;
    if (!c) return MPM_ERR_ARG;
    auto bad = [](const char* why) {
        std::fprintf(stderr, "mpm_design_create: %s\n", why);
        return (int)MPM_ERR_ARG;
    };
    if (c->dim != 2 && c->dim != 3) return bad("dim must be 2 or 3");
    if (c->n_particles < 0 || c->n_regions < 0 || c->n_tasks < 1 || c->n_steps < 1) return bad("sizes out of range");
    if (!(c->dt > 0.0) || !(c->filter_radius > 0.0) || !(c->delta >= 0.0) || !(c->f_max >= c->f_min))
        return bad("dt and filter_radius must be > 0, delta >= 0, f_max >= f_min");
    if (c->n_particles > 0 && !x0) return bad("x0 is required");
    if ((c->n_regions > 0) != (region != nullptr)) return bad("region must be given exactly when n_regions > 0");
    mpm_design* h = new (std::nothrow) mpm_design();
    if (!h) return MPM_ERR_OOM;
    int rc;
    try {
        rc = create_impl(h, c, x0, region, (cudaStream_t)cuda_stream);
    } catch (...) {
        rc = MPM_ERR_CUDA;
    }
    if (rc != MPM_OK) {
        std::fprintf(stderr, "mpm_design_create: %s\n", h->err.c_str());
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return MPM_OK;
}

int mpm_design_destroy(mpm_design* h) {
    if (!h) return MPM_ERR_ARG;
    release(h);
    delete h;
    return MPM_OK;
}

const char* mpm_design_last_error(const mpm_design* h) { return h ? h->err.c_str() : "null handle"; }

int mpm_design_forward(mpm_design* h, float beta, const float* phi, const float* Br, const float* zeta,
                       const float* Ba, const float* f, const float* eta, float* phi_bar, float* mag, float* field,
                       void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    const mpm_design_config& c = h->cfg;
    const int n = c.n_particles, d = c.dim;
    if (!(beta > 0.0f)) return fail(h, MPM_ERR_ARG, "beta must be > 0");
    if ((n > 0 && (!phi || !Br || !zeta || !phi_bar || !mag)) || !Ba || !f || !eta || !field)
        return fail(h, MPM_ERR_ARG, "missing array");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    h->forward_done = false;
    const float t_half = tanhf(0.5f * beta);
    if (n > 0) {
        if (d == 2)
            k_filter_apply<2><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, h->order, h->offsets, phi, h->norm, h->phi_t);
        else
            k_filter_apply<3><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, h->order, h->offsets, phi, h->norm, h->phi_t);
        DCUDA(h, cudaGetLastError());
        k_heaviside<<<blocks(n), 256, 0, st>>>(h->phi_t, n, beta, t_half, phi_bar);
        DCUDA(h, cudaGetLastError());
        if (d == 2) k_magnetization<2><<<blocks(n), 256, 0, st>>>(Br, zeta, h->region, n, h->n_m, (float)c.Br_max, (float)c.delta, mag);
        else k_magnetization<3><<<blocks(n), 256, 0, st>>>(Br, zeta, h->region, n, h->n_m, (float)c.Br_max, (float)c.delta, mag);
        DCUDA(h, cudaGetLastError());
    }
    const long long nf = (long long)c.n_tasks * c.n_steps;
    auto keep = [&](float* dst, const float* src, long long count) {
        return count > 0 ? cudaMemcpyAsync(dst, src, sizeof(float) * count, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
    };
    if (n > 0) {
        DCUDA(h, keep(h->in_Br, Br, h->n_m));
        DCUDA(h, keep(h->in_zeta, zeta, (long long)d * h->n_m));
    }
    DCUDA(h, keep(h->in_Ba, Ba, c.n_tasks));
    DCUDA(h, keep(h->in_f, f, c.n_tasks));
    DCUDA(h, keep(h->in_eta, eta, (long long)d * c.n_tasks));
    if (d == 2)
        k_stimulus<2><<<blocks(nf), 256, 0, st>>>(Ba, f, eta, c.n_tasks, c.n_steps, (float)c.dt, (float)c.B_max,
                                                  (float)c.f_min, (float)c.f_max, (float)c.delta, field);
    else
        k_stimulus<3><<<blocks(nf), 256, 0, st>>>(Ba, f, eta, c.n_tasks, c.n_steps, (float)c.dt, (float)c.B_max,
                                                  (float)c.f_min, (float)c.f_max, (float)c.delta, field);
    DCUDA(h, cudaGetLastError());
    h->beta = beta;
    h->forward_done = true;
    return MPM_OK;
}

int mpm_design_backward(mpm_design* h, const float* g_phi_bar, const float* g_mag, const float* g_field, float* g_phi,
                        float* g_Br, float* g_zeta, float* g_Ba, float* g_f, float* g_eta, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (!h->forward_done) return fail(h, MPM_ERR_STATE, "mpm_design_backward needs mpm_design_forward first");
    const mpm_design_config& c = h->cfg;
    const int n = c.n_particles, d = c.dim, n_m = h->n_m;
    if ((n > 0 && (!g_phi_bar || !g_mag || !g_phi || !g_Br || !g_zeta)) || !g_field || !g_Ba || !g_f || !g_eta)
        return fail(h, MPM_ERR_ARG, "missing array");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float t_half = tanhf(0.5f * h->beta);
    if (n > 0) {
        // topology: Eq. 25 reversed, then the transposed filter of Eq. 23
        k_heaviside_adjoint<<<blocks(n), 256, 0, st>>>(h->phi_t, g_phi_bar, n, h->beta, t_half, h->norm, h->u);
        DCUDA(h, cudaGetLastError());
        if (d == 2)
            k_filter_apply<2><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, h->order, h->offsets, h->u, nullptr, g_phi);
        else
            k_filter_apply<3><<<blocks(n), 256, 0, st>>>(h->x0, n, h->grid, h->order, h->offsets, h->u, nullptr, g_phi);
        DCUDA(h, cudaGetLastError());
        // material: Eq. 26-28 reversed, summed per region
        const bool regions = h->region != nullptr;
        const bool stage = regions && (1 + d) * n_m <= kSmemRegionFloats;
        if (regions) {
            DCUDA(h, cudaMemsetAsync(g_Br, 0, sizeof(float) * n_m, st));
            DCUDA(h, cudaMemsetAsync(g_zeta, 0, sizeof(float) * d * (size_t)n_m, st));
        }
        const size_t smem = stage ? sizeof(float) * (1 + d) * n_m : 0;
        if (d == 2)
            k_magnetization_adjoint<2><<<blocks(n), 256, smem, st>>>(h->in_Br, h->in_zeta, h->region, n, n_m,
                                                                     (float)c.Br_max, (float)c.delta, g_mag, g_Br,
                                                                     g_zeta, stage);
        else
            k_magnetization_adjoint<3><<<blocks(n), 256, smem, st>>>(h->in_Br, h->in_zeta, h->region, n, n_m,
                                                                     (float)c.Br_max, (float)c.delta, g_mag, g_Br,
                                                                     g_zeta, stage);
        DCUDA(h, cudaGetLastError());
    }
    // stimulus: Eq. 29-30 reversed, one block per task
    if (d == 2)
        k_stimulus_adjoint<2><<<c.n_tasks, 256, 0, st>>>(h->in_Ba, h->in_f, h->in_eta, c.n_steps, (float)c.dt,
                                                         (float)c.B_max, (float)c.f_min, (float)c.f_max,
                                                         (float)c.delta, g_field, g_Ba, g_f, g_eta);
    else
        k_stimulus_adjoint<3><<<c.n_tasks, 256, 0, st>>>(h->in_Ba, h->in_f, h->in_eta, c.n_steps, (float)c.dt,
                                                         (float)c.B_max, (float)c.f_min, (float)c.f_max,
                                                         (float)c.delta, g_field, g_Ba, g_f, g_eta);
    DCUDA(h, cudaGetLastError());
    return MPM_OK;
}

int mpm_adam_step(long long n, float* x, const float* g, float* m, float* v, int k, double lr, double beta1,
                  double beta2, double eps, double lo, double hi, void* cuda_stream) {
    if (n < 0 || k < 1 || !(lo <= hi) || (n > 0 && (!x || !g || !m || !v))) return MPM_ERR_ARG;
    if (n == 0) return MPM_OK;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, k)), c2 = 1.0 / (1.0 - std::pow(beta2, k));
    k_adam<<<blocks(n), 256, 0, (cudaStream_t)cuda_stream>>>(n, x, g, m, v, (float)lr, (float)beta1, (float)beta2,
                                                             (float)eps, (float)c1, (float)c2, (float)lo, (float)hi);
    return cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}

}  // extern "C"
