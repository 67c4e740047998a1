// mpm_substep_noalloc: one substep of one instance with no device allocation.
//
// Some callers cannot call cudaMalloc. One example is a framework whose own
// pool allocator owns the whole device-memory budget. Another is a latency-
// critical path where an allocation could block or fail. For them this entry
// point keeps its grid scratch in a file-scope device array. Every call reuses
// the same array, so two calls that overlap on the GPU (different streams,
// threads or processes sharing a context) race on it. Serialise them.
//
// The array belongs to the library's CUDA module. With lazy module loading
// (the CUDA default) the module, and with it the array, is loaded on a device
// by the first call there: that call looks up the array's device address
// with cudaGetSymbolAddress (host code cannot use the symbol's name as a
// device pointer), which reserves the array's 8 MiB. A failure there comes
// back as MPM_ERR_OOM or MPM_ERR_CUDA. The address is cached per device and
// context: a context created anew (after cudaDeviceReset, say) has a new
// context id, and its first call looks the address up again. Make the first
// call on a device before any CUDA stream capture begins.
//
// Each call reads the device error flags back and synchronises its stream,
// so a call on a stream that is capturing is refused before it enqueues any
// work (MPM_ERR_ARG), which leaves the caller's capture intact.
//
// The substep itself reuses the library's kernels: P2G (particle_kernels.cuh,
// Eq. 14-15 with the stress of Eq. 7 / 31-33), the grid operation
// (Eq. 16-18) and G2P (Eq. 19-22).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "mpm.h"
#include "runtime_internal.h"

namespace {

constexpr long long kMaxNodes = MPM_NOALLOC_MAX_NODES;

// [0, kMaxNodes): P2G accumulator (m, m v); [kMaxNodes, 2 kMaxNodes): grid velocity.
static __device__ __align__(256) float4 g_noalloc_grid[2 * kMaxNodes];
// [0], [1]: particle offsets of the single instance; [32]: device error flags.
static __device__ __align__(256) int g_noalloc_misc[64];

constexpr int kMaxDevices = 64;
struct Scratch {
    unsigned long long ctx_id = 0;  // context the addresses belong to (0: none yet)
    float4* grid = nullptr;
    int* misc = nullptr;
};
Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// The text of the last failure of this entry point on the calling thread.
thread_local std::string t_last_error;

using GetCtxFn = CUresult (*)(CUcontext*);
using GetCtxIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context (unique within the process),
// through the driver entry points the runtime hands out.
int current_context_id(unsigned long long* id, std::string* why) {
    static GetCtxFn get_ctx = nullptr;
    static GetCtxIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = reinterpret_cast<GetCtxFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetCtxIdFn>(f);
    });
    if (!get_ctx || !get_id) {
        *why = "the driver does not provide cuCtxGetCurrent / cuCtxGetId";
        return MPM_ERR_CUDA;
    }
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, id) != CUDA_SUCCESS) {
        *why = "no current CUDA context";
        return MPM_ERR_CUDA;
    }
    return MPM_OK;
}

int scratch_for_current_device(Scratch* out, std::string* why) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return MPM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *why = "device ordinal out of range";
        return MPM_ERR_ARG;
    }
    // binds the device's primary context to this thread (the runtime creates
    // it here if no call has yet), so that the context id below exists
    if ((e = cudaSetDevice(dev)) != cudaSuccess) {
        *why = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return MPM_ERR_CUDA;
    }
    unsigned long long ctx_id = 0;
    int rc = current_context_id(&ctx_id, why);
    if (rc != MPM_OK) return rc;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    Scratch& s = g_scratch[dev];
    if (s.ctx_id != ctx_id) {
        void* grid = nullptr;
        void* misc = nullptr;
        e = cudaGetSymbolAddress(&grid, g_noalloc_grid);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&misc, g_noalloc_misc);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *why = std::string("cudaGetSymbolAddress (loads the module and its 8 MiB scratch): ") +
                   cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
        }
        s.grid = static_cast<float4*>(grid);
        s.misc = static_cast<int*>(misc);
        s.ctx_id = ctx_id;
    }
    *out = s;
    return MPM_OK;
}

// Clears the accumulator and the error flags left by the previous call and
// writes the instance offsets {0, n}.
__global__ void k_noalloc_setup(float4* __restrict__ acc, long long nodes, int* __restrict__ misc,
                                int n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < nodes; i += (long long)gridDim.x * blockDim.x) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        misc[0] = 0;
        misc[1] = n;
        misc[32] = 0;
    }
}

int report(int code, const std::string& why) {
    t_last_error = "mpm_substep_noalloc: " + why;
    return code;
}

}  // namespace

extern "C" const char* mpm_noalloc_last_error(void) { return t_last_error.c_str(); }

extern "C" int mpm_substep_noalloc(const mpm_config* cfg, int substep, const float* state_in,
                                   const float* phi_bar, const float* mag, const float* field,
                                   float* state_out, void* cuda_stream) {
    t_last_error.clear();
    std::string why;
    int rc = mpm::check_config(cfg, &why);
    if (rc != MPM_OK) return report(rc, why);
    if (cfg->n_instances != 1) return report(MPM_ERR_ARG, "needs exactly one instance");
    if (substep < 0 || substep >= cfg->n_steps) return report(MPM_ERR_ARG, "substep out of [0, n_steps)");
    long long nodes = 1;
    for (int a = 0; a < cfg->dim; ++a) nodes *= cfg->grid_res;
    if (nodes > kMaxNodes)
        return report(MPM_ERR_ARG, "grid_res^dim = " + std::to_string(nodes) + " nodes exceeds the " +
                                       std::to_string(kMaxNodes) + "-node scratch of this entry point");
    const int n = cfg->n_particles[0];
    if (n > 0 && (!state_in || !state_out || !phi_bar || !mag || !field))
        return report(MPM_ERR_ARG, "state_in, state_out, phi_bar, mag and field are required");

    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) {
        cudaGetLastError();
        return report(MPM_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    }
    if (cap != cudaStreamCaptureStatusNone)
        return report(MPM_ERR_ARG, "the stream is capturing; this call synchronises its stream to read "
                                   "back the device status and cannot be captured");

    Scratch sc;
    rc = scratch_for_current_device(&sc, &why);
    if (rc != MPM_OK) return report(rc, why);

    const int d = cfg->dim;
    mpm::Params P{};
    P.res = cfg->grid_res;
    P.bound = cfg->bound;
    P.wall_mode = cfg->wall_mode;
    P.loss_kind = cfg->loss_kind;
    P.simp_q = cfg->simp_q;
    P.n_inst = 1;
    P.n_steps = cfg->n_steps;
    P.n_total = n;
    P.np = n;  // the caller's SoA component stride
    P.nodes = nodes;
    P.dx = (float)(1.0 / cfg->grid_res);
    P.inv_dx = (float)cfg->grid_res;
    P.dt = (float)cfg->dt;
    P.kappa = (float)(4.0 * cfg->grid_res * (double)cfg->grid_res);
    P.p_vol = (float)cfg->p_vol;
    P.rho0 = (float)cfg->rho0;
    P.G = (float)(cfg->E / (2.0 * (1.0 + cfg->nu)));
    P.K = (float)(cfg->E / (3.0 * (1.0 - 2.0 * cfg->nu)));
    P.eps = (float)cfg->simp_eps;
    P.damping = (float)cfg->damping_c;
    P.mu = (float)cfg->floor_mu;
    for (int i = 0; i < 3; ++i) P.gravity[i] = (float)cfg->gravity[i];

    float4* acc = sc.grid;
    float4* V = sc.grid + kMaxNodes;
    int* inst_off = sc.misc;
    int* err = sc.misc + 32;
    k_noalloc_setup<<<(unsigned)((nodes + 255) / 256), 256, 0, st>>>(acc, nodes, sc.misc, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return report(MPM_ERR_CUDA, cudaGetErrorString(e));

    mpm::StepArgs a;
    a.s_in = state_in;
    a.phi = phi_bar;
    a.mag = mag;
    a.field = field;
    a.inst_off = inst_off;
    a.err = err;
    a.acc = acc;
    a.n_p2g = substep;
    if ((e = mpm::launch_forward(d, false, true, false, false, P, a, 128, st)) != cudaSuccess)
        return report(MPM_ERR_CUDA, cudaGetErrorString(e));
    if ((e = mpm::launch_grid(d, P, acc, V, nullptr, false, substep, st)) != cudaSuccess)
        return report(MPM_ERR_CUDA, cudaGetErrorString(e));
    mpm::StepArgs g = a;
    g.acc = nullptr;
    g.s_out = state_out;
    g.V = V;
    g.n_g2p = substep;
    if ((e = mpm::launch_forward(d, true, false, true, false, P, g, 128, st)) != cudaSuccess)
        return report(MPM_ERR_CUDA, cudaGetErrorString(e));

    int flags = 0;
    if ((e = cudaMemcpyAsync(&flags, err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return report(MPM_ERR_CUDA, cudaGetErrorString(e));
    if (flags & mpm::kErrDomain) return report(MPM_ERR_DOMAIN, "a particle stencil left the grid");
    if (flags & mpm::kErrNumeric) return report(MPM_ERR_NUMERIC, "inverted or non-finite deformation gradient");
    return MPM_OK;
}
