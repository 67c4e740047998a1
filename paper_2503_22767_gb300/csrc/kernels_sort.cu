// Stable counting sort of particles by grid cell.
//
// The paper does not sort (its Taichi kernels need none); the GPU path sorts
// so that consecutive threads touch neighbouring grid nodes, which keeps the
// P2G / G2P^T scatters and the G2P / P2G^T gathers local.
//
// Key (integer, exact): per axis base = floor(fl(fl(x*res) - 0.5)) in float32
// round-to-nearest, clamped to [0, res-3]; cells grouped in blocks of edge
// BS (8 in 2D, 4 in 3D); key = inst * nb^D * BS^D + block * BS^D + cell in
// block, blocks and cells row-major with the last axis fastest.
// Stable: equal keys keep their input order (ties ordered by old index).
#include "kernels.h"

namespace mpm {

namespace {

template <int D>
constexpr int block_edge() { return D == 2 ? 8 : 4; }

template <int D>
__global__ void __launch_bounds__(256) k_cell_key(Params P, const float* __restrict__ x,
                                                  long long xstride, const float* __restrict__ x0,
                                                  const int* __restrict__ inst_off,
                                                  int* __restrict__ keys, int* __restrict__ slot,
                                                  int* __restrict__ counts, int* __restrict__ err) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    constexpr int BS = block_edge<D>();
    const int nb = (P.res + BS - 1) / BS;
    long long blk = 0, cel = 0, per_block = 1, per_inst = 1;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        // the position (x0 + u in the displacement-form state, as the kernels form it)
        const float xa = x0 ? __fadd_rn(x[a * xstride + p], x0[a * xstride + p]) : x[a * xstride + p];
        float fx = __fmul_rn(xa, (float)P.res);
        float fb = floorf(__fsub_rn(fx, 0.5f));
        int b;
        if (fb >= 0.0f && fb <= (float)(P.res - 3)) {
            b = (int)fb;
        } else {
            ok = false;
            b = (fb > 0.0f) ? P.res - 3 : 0;
        }
        blk = blk * nb + b / BS;
        cel = cel * BS + b % BS;
        per_block *= BS;
        per_inst *= (long long)nb * BS;
    }
    int inst = find_instance(inst_off, P.n_inst, p);
    int key = (int)(inst * per_inst + blk * per_block + cel);
    keys[p] = key;
    slot[p] = atomicAdd(counts + key, 1);
    if (!ok) atomicOr(err, kErrDomain);
}

// Exclusive scan of 2048 ints per block; block totals to `sums`.
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 2 * kScanThreads;

__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int* __restrict__ in,
                                                            int* __restrict__ out,
                                                            int* __restrict__ sums, long long n) {
    __shared__ int warp_tot[kScanThreads / 32];
    long long base = (long long)blockIdx.x * kScanTile + 2 * threadIdx.x;
    int a = base < n ? in[base] : 0;
    int b = base + 1 < n ? in[base + 1] : 0;
    int t = a + b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
        int wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31 && sums) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int excl = warp_tot[warp] + incl - t;
    if (base < n) out[base] = excl;
    if (base + 1 < n) out[base + 1] = excl + a;
}

__global__ void k_scan_add(int* __restrict__ out, const int* __restrict__ tile_off, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

__global__ void __launch_bounds__(256) k_scatter_perm(Params P, const int* __restrict__ keys,
                                                      const int* __restrict__ slot,
                                                      const int* __restrict__ offsets,
                                                      int* __restrict__ perm) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_total) return;
    perm[offsets[keys[p]] + slot[p]] = p;
}

// Atomic slots give an arbitrary order inside a key; restore input order.
__global__ void __launch_bounds__(256) k_order_bins(const int* __restrict__ counts,
                                                    const int* __restrict__ offsets,
                                                    int* __restrict__ perm, long long n_keys) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_keys) return;
    int c = counts[k];
    if (c < 2) return;
    int* v = perm + offsets[k];
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

cudaError_t scan_exclusive(const int* in, int* out, long long n, int* tmp, cudaStream_t st) {
    long long tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles <= 1) {
        k_scan_tile<<<1, kScanThreads, 0, st>>>(in, out, nullptr, n);
        return cudaGetLastError();
    }
    int* sums = tmp;
    int* rest = tmp + tiles;
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, sums, n);
    cudaError_t e = scan_exclusive(sums, sums, tiles, rest, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, sums, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_exclusive(const int* in, int* out, long long n, int* tmp, cudaStream_t st) {
    return scan_exclusive(in, out, n, tmp, st);
}

long long sort_key_space(int dim, int res, int n_inst) {
    int bs = dim == 2 ? 8 : 4;
    long long nb = (res + bs - 1) / bs, per = 1;
    for (int a = 0; a < dim; ++a) per *= nb * bs;
    return per * n_inst;
}

long long sort_scan_tmp_len(long long n_keys) {
    long long total = 0, n = n_keys;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n;
    }
    return total + 1;
}

cudaError_t launch_sort(int dim, const Params& P, const float* x, long long xstride,
                        const int* inst_off, SortBuffers& sb, int* perm, int* err,
                        cudaStream_t st, const float* x0) {
    if (P.n_total == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(sb.counts, 0, sizeof(int) * sb.n_keys, st);
    if (e != cudaSuccess) return e;
    unsigned grid = (unsigned)((P.n_total + 255) / 256);
    if (dim == 2)
        k_cell_key<2><<<grid, 256, 0, st>>>(P, x, xstride, x0, inst_off, sb.keys, sb.slot, sb.counts, err);
    else
        k_cell_key<3><<<grid, 256, 0, st>>>(P, x, xstride, x0, inst_off, sb.keys, sb.slot, sb.counts, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(sb.counts, sb.offsets, sb.n_keys, sb.scan_tmp, st)) != cudaSuccess) return e;
    k_scatter_perm<<<grid, 256, 0, st>>>(P, sb.keys, sb.slot, sb.offsets, perm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_order_bins<<<(unsigned)((sb.n_keys + 255) / 256), 256, 0, st>>>(sb.counts, sb.offsets, perm,
                                                                      sb.n_keys);
    return cudaGetLastError();
}

}  // namespace mpm
