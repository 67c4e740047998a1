// Runtime behind the C ABI of include/mpm.h.
//
// One handle owns every device buffer of a batch of simulations (allocated
// once in mpm_create) and drives the kernels of particle_kernels.cuh, kernels_step.cu and
// kernels_sort.cu:
//
//   forward   for each segment of K substeps: sort the particles by cell and
//             reorder the state, save a checkpoint (state, ids, permutation),
//             then per substep: grid operation, fused G2P(n) + P2G(n+1).
//             Between substeps only x and F are stored ("lean" pass).
//   backward  for each segment in reverse: restore its checkpoint, recompute
//             the K substeps storing every state and grid, then per substep in
//             reverse: grid adjoint, fused P2G^T(n) + G2P^T(n-1); the particle
//             adjoint crosses segment boundaries through the saved
//             permutation; design gradients go back to input order.
//
// The paper (arxiv 2503.22767, Section 2.3) differentiates with Taichi's tape;
// the checkpointed recomputation here is what lets contact-rich horizons of
// thousands of substeps fit in HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "mpm.h"
#include "runtime_internal.h"

using mpm::Params;
using mpm::StepArgs;

namespace {

enum KernelClass { kFwdParticle = 0, kAdjParticle = 1, kGrid = 2, kGridAdj = 3, kNumClasses = 4 };

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    double bytes = 0.0;
};

// One sampled launch inside a captured graph: its event pair stays owned by
// the graph and is read after every replay.
struct TimedLaunch {
    int cls;
    cudaEvent_t a, b;
    double bytes;
};

}  // namespace

struct mpm_handle {
    // --- configuration ---
    int dim = 0, res = 0, T = 0, n_inst = 0, K = 0, n_seg = 0, ncomp = 0;
    long long N = 0, np = 0, Nd = 0, nodes = 0, total_nodes = 0;
    std::vector<int> counts, inst_off, design_of, dcount, dbase;
    Params P{};
    int block = 128;
    int timing_stride = 0;  // 0 = off; k = time every k-th launch of a class
    std::string err;

    // --- device buffers ---
    std::vector<void*> allocs;
    long long device_bytes = 0;
    int* d_inst_off = nullptr;
    int* d_dbase = nullptr;
    float* stA = nullptr;
    float* stB = nullptr;
    int* idA = nullptr;
    int* idB = nullptr;
    float* ck_state = nullptr;
    int* ck_id = nullptr;
    int* ck_perm = nullptr;
    float* seg_state = nullptr;
    float4* seg_acc = nullptr;
    float4* seg_V = nullptr;
    float4* acc = nullptr;
    float4* V = nullptr;
    float4* Vbar = nullptr;
    float4* gadj = nullptr;
    float* adj = nullptr;
    float* adj2 = nullptr;
    float* phi_cur = nullptr;
    float* mag_cur = nullptr;
    float* x0_fwd = nullptr;   // forward pass: initial positions in the current order [d][np]
    float* x0_seg = nullptr;   // recomputation: the same per segment set [2][d][np]
    float* gphi_cur = nullptr;
    float* gmag_cur = nullptr;
    float* phi_d = nullptr;
    float* mag_d = nullptr;
    float* field = nullptr;
    float* target = nullptr;
    float* mom = nullptr;
    float* Minst = nullptr;
    float* loss_acc = nullptr;
    float* dloss = nullptr;
    float* gphi_d = nullptr;
    float* gmag_d = nullptr;
    float* gfield_d = nullptr;
    float* st_x0 = nullptr;
    float* st_v0 = nullptr;
    float* st_xout = nullptr;
    float* st_loss = nullptr;
    int* d_err = nullptr;
    int* perm = nullptr;
    mpm::SortBuffers sb;

    float4* acc3 = nullptr;   // fused mode: three rotating P2G accumulators
    float4* Vbar3 = nullptr;  // fused mode: three rotating G2P^T scatter targets
    mpm::Extras* d_ext = nullptr;        // solid boxes (Eq. 18) and the field gradient
    mpm::Extras ext_host{};              // host copy of *d_ext
    float* d_fgrad = nullptr;            // dB/dx per instance and substep
    float* d_gfgrad = nullptr;           // its gradient, filled by the backward pass
    bool backward_done = false;
    float* d_bmotion = nullptr;          // their offsets and velocities per substep

    // --- 3D: grid kernels over the listed node blocks (mpm::ActiveBlocks) ---
    bool blocks = false;      // 3D: the P2G kernels mark and list the node blocks they touch
    bool grid_blocks = true;  // option: the grid kernels walk the lists (else every node)
    long long n_blocks = 0;   // node blocks over all instances
    int grid_ctas = 0;        // persistent CTAs of the list-walking kernels
    long long n_wbox = 0;     // warps of 32 particles
    // lists (flags, list, count, per-warp boxes), each covering one checkpoint
    // segment: 0 and 1 for the forward pass by segment parity, 2 and 3 for the
    // two recomputation sets (4 and up: the resident sets, in res_* below)
    int* blk_flag = nullptr;  // [4][n_blocks]
    int* blk_list = nullptr;  // [4][n_blocks]
    int* blk_count = nullptr; // [4]
    int4* blk_wbox = nullptr; // [4][n_wbox]
    bool seg_dirty = false;   // a backward pass ran over every node: the segment accumulators are not zero

    // --- resident segments (MPM_OPT_RESIDENT_SEGMENTS) ---
    // The forward pass stores the trajectory of the last n_res checkpoint
    // segments into sets of their own (states, accumulators, grid velocities,
    // current-order design and x0, 3D lists 4 .. 4 + n_res - 1), and the
    // backward pass runs their adjoint without recomputing them.
    int n_res = 0;
    std::vector<void*> res_allocs;
    long long res_bytes = 0;
    float* res_state = nullptr;  // [n_res][K + 1][S]
    float4* res_acc = nullptr;   // [n_res][K][G]
    float4* res_V = nullptr;     // [n_res][K][G]
    float* res_phi = nullptr;    // [n_res][np]
    float* res_mag = nullptr;    // [n_res][d][np]
    float* res_x0 = nullptr;     // [n_res][d][np]
    int* res_flag = nullptr;     // [n_res][n_blocks]
    int* res_list = nullptr;     // [n_res][n_blocks]
    int* res_count = nullptr;    // [n_res]
    int4* res_wbox = nullptr;    // [n_res][n_wbox]
    bool res_dirty = false;      // resident accumulators set outside their lists

    // --- persistent passes (MPM_OPT_PERSISTENT) ---
    bool persistent = false;
    long long spin_limit = 1LL << 22;  // polls before a grid-barrier wait gives up
    unsigned* bar = nullptr;           // grid barrier of the persistent kernels

    // --- options ---
    // grid operation folded into the forward particle kernels (off by default:
    // the autotuner keeps the separate grid kernel on all five workloads)
    bool fuse_fwd = false;
    bool fuse_adj = false;  // grid adjoint folded into the adjoint particle kernels
    bool graphs = true;   // replay the forward / backward passes as CUDA graphs
    bool v0_given = false;

    // --- CUDA graphs of the two passes (captured on first use) ---
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux_stream = nullptr;  // recomputation stream of the backward pass
    cudaEvent_t ev_fork = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_adj[2] = {nullptr, nullptr};
    bool two_streams = true;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<TimedLaunch> graph_timing[2];
    bool capturing = false;
    int capture_pass = 0;
    long long graph_launches[2] = {0, 0};  // kernels inside each captured graph
    long long graph_cls[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // per kernel class
    bool ran_graph[2] = {false, false};

    int tune_T = 0;  // > 0 while autotuning: passes stop after this many substeps

    // --- run state ---
    bool forward_done = false;
    float* cur = nullptr;  // final state of the last forward
    int* id_cur = nullptr;

    // --- counters ---
    long long launches = 0;
    std::vector<EventPair> events[kNumClasses];
    size_t ev_used[kNumClasses] = {0, 0, 0, 0};
    long long class_launch[kNumClasses] = {0, 0, 0, 0};
    long long cls_issued[kNumClasses] = {0, 0, 0, 0};  // launches per class since the last reset
    long long timed_launches[kNumClasses] = {0, 0, 0, 0};
    double timed_ms[kNumClasses] = {0, 0, 0, 0};
    double timed_bytes[kNumClasses] = {0, 0, 0, 0};
};

namespace {

#define MPM_CUDA(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return MPM_ERR_CUDA;                                                            \
        }                                                                                   \
    } while (0)

int fail(mpm_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

template <typename T>
int dalloc(mpm_handle* h, T** p, long long count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    size_t bytes = sizeof(T) * (size_t)count;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
    }
    h->allocs.push_back(ptr);
    h->device_bytes += (long long)bytes;
    *p = (T*)ptr;
    return MPM_OK;
}

void drop_graphs(mpm_handle* h) {
    for (int i = 0; i < 2; ++i) {
        if (h->exec[i]) cudaGraphExecDestroy(h->exec[i]);
        h->exec[i] = nullptr;
        for (auto& t : h->graph_timing[i]) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        h->graph_timing[i].clear();
    }
}

// Resident segment sets (MPM_OPT_RESIDENT_SEGMENTS), reserved after creation
// and released on change or destruction.
template <typename T>
int ralloc(mpm_handle* h, T** p, long long count) {
    *p = nullptr;
    size_t bytes = sizeof(T) * (size_t)std::max(1LL, count);
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->err = "cudaMalloc of " + std::to_string(bytes) + " bytes for resident segments failed: " +
                 cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
    }
    h->res_allocs.push_back(ptr);
    h->res_bytes += (long long)bytes;
    h->device_bytes += (long long)bytes;
    *p = (T*)ptr;
    return MPM_OK;
}

// Device bytes of one resident segment set: K + 1 states, K accumulators and
// K grid velocities, the current-order design and x0, and in 3D one
// node-block list.
long long resident_set_bytes(const mpm_handle* h) {
    const long long S = (long long)h->ncomp * h->np, G = h->total_nodes;
    long long b = (long long)sizeof(float) * S * (h->K + 1) + 2LL * (long long)sizeof(float4) * G * h->K +
                  (long long)sizeof(float) * (1 + 2 * h->dim) * h->np;
    if (h->blocks) b += (long long)sizeof(int) * (2 * h->n_blocks + 1) + (long long)sizeof(int4) * h->n_wbox;
    return b;
}

void free_resident(mpm_handle* h) {
    for (void* p : h->res_allocs) cudaFree(p);
    h->res_allocs.clear();
    h->device_bytes -= h->res_bytes;
    h->res_bytes = 0;
    h->n_res = 0;
    h->res_state = h->res_phi = h->res_mag = h->res_x0 = nullptr;
    h->res_acc = h->res_V = nullptr;
    h->res_flag = h->res_list = h->res_count = nullptr;
    h->res_wbox = nullptr;
    h->res_dirty = false;
}

void free_all(mpm_handle* h) {
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
    h->aux_stream = nullptr;
    for (cudaEvent_t* e : {&h->ev_fork, &h->ev_rec[0], &h->ev_rec[1], &h->ev_adj[0], &h->ev_adj[1]}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    free_resident(h);
    for (int c = 0; c < kNumClasses; ++c) {
        for (auto& e : h->events[c]) {
            if (e.a) cudaEventDestroy(e.a);
            if (e.b) cudaEventDestroy(e.b);
        }
        h->events[c].clear();
    }
}

// Reserve r resident segment sets (0 releases them); r is capped at the
// number of segments.  The forward and backward passes change shape, so the
// captured graphs and the last forward are dropped.
int set_resident(mpm_handle* h, int r) {
    r = std::max(0, std::min(r, h->n_seg));
    if (r == h->n_res) return MPM_OK;
    drop_graphs(h);
    h->forward_done = false;
    free_resident(h);
    if (r == 0) return MPM_OK;
    const long long S = (long long)h->ncomp * h->np, G = h->total_nodes;
    int rc;
    if ((rc = ralloc(h, &h->res_state, r * S * (h->K + 1))) || (rc = ralloc(h, &h->res_acc, r * G * h->K)) ||
        (rc = ralloc(h, &h->res_V, r * G * h->K)) || (rc = ralloc(h, &h->res_phi, r * h->np)) ||
        (rc = ralloc(h, &h->res_mag, r * h->dim * h->np)) || (rc = ralloc(h, &h->res_x0, r * h->dim * h->np))) {
        free_resident(h);
        return rc;
    }
    if (h->blocks && ((rc = ralloc(h, &h->res_flag, r * h->n_blocks)) ||
                      (rc = ralloc(h, &h->res_list, r * h->n_blocks)) || (rc = ralloc(h, &h->res_count, r)) ||
                      (rc = ralloc(h, &h->res_wbox, r * h->n_wbox)))) {
        free_resident(h);
        return rc;
    }
    // the sets start as the lists expect them: accumulators, flags and counts zero
    cudaError_t e = cudaMemset(h->res_acc, 0, sizeof(float4) * r * G * h->K);
    if (e == cudaSuccess && h->blocks) e = cudaMemset(h->res_flag, 0, sizeof(int) * r * h->n_blocks);
    if (e == cudaSuccess && h->blocks) e = cudaMemset(h->res_count, 0, sizeof(int) * r);
    if (e == cudaSuccess && h->blocks) e = cudaMemset(h->res_wbox, 0, sizeof(int4) * r * h->n_wbox);
    // the memsets run on the default stream: finish them before any pass on
    // the caller's stream (which may not synchronise with it) uses the sets
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_resident(h);
        return fail(h, MPM_ERR_CUDA, std::string("resident segments: ") + cudaGetErrorString(e));
    }
    h->n_res = r;
    return MPM_OK;
}

// algorithmic bytes of one launch (what the method itself must move; see the
// repository's design notes for the derivation)
enum Variant { kFused = 0, kFusedStore = 1, kFirstP2G = 2, kLastG2PT = 3, kFirstP2GT = 4 };

double particle_bytes(int d, int cls, int variant) {
    const double xf = d + d * d, full = 2 * d + 2 * d * d, design = 1 + d;
    if (cls == kFwdParticle) {
        if (variant == kFirstP2G) return 4.0 * (full + design);             // P2G alone
        return 4.0 * (xf + (variant == kFusedStore ? full : xf) + design);  // G2P(+P2G)
    }
    if (variant == kLastG2PT) return 4.0 * (full + d * d + xf + xf);        // G2P^T alone
    if (variant == kFirstP2GT) return 4.0 * (full + xf + full + 3 * design); // P2G^T alone
    // fused adjoint: state n (full) + state n-1 (x, F) + partial adjoint
    // in and out (x, F) + design + design-gradient read-modify-write
    return 4.0 * (full + xf + 2 * xf + design + 2 * design);
}

// Launch wrapper: counts launches and, when timing is on, brackets every
// timing_stride-th launch of the class with CUDA events.
template <typename F>
int timed(mpm_handle* h, int cls, double bytes, cudaStream_t st, F&& launch) {
    bool time_it = h->timing_stride > 0 && (h->class_launch[cls] % h->timing_stride) == 0;
    h->class_launch[cls]++;
    h->cls_issued[cls]++;
    h->launches++;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (time_it && h->capturing) {
        // event-record nodes of the graph being captured
        MPM_CUDA(h, cudaEventCreate(&ea));
        MPM_CUDA(h, cudaEventCreate(&eb));
        h->graph_timing[h->capture_pass].push_back(TimedLaunch{cls, ea, eb, bytes});
    } else if (time_it) {
        auto& pool = h->events[cls];
        if (h->ev_used[cls] == pool.size()) {
            EventPair e;
            MPM_CUDA(h, cudaEventCreate(&e.a));
            MPM_CUDA(h, cudaEventCreate(&e.b));
            pool.push_back(e);
        }
        EventPair* ev = &pool[h->ev_used[cls]++];
        ev->bytes = bytes;
        ea = ev->a;
        eb = ev->b;
    }
    // inside a capture an event must be recorded "external" to become an
    // event-record node of the graph (a plain record only orders the capture)
    const unsigned rec_flags = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (ea) MPM_CUDA(h, cudaEventRecordWithFlags(ea, st, rec_flags));
    cudaError_t e = launch();
    if (e != cudaSuccess) {
        h->err = std::string("kernel launch failed: ") + cudaGetErrorString(e);
        return MPM_ERR_CUDA;
    }
    if (eb) MPM_CUDA(h, cudaEventRecordWithFlags(eb, st, rec_flags));
    return MPM_OK;
}

// plain launches that are not timed (sort, design gathers, seeds...)
template <typename F>
int counted(mpm_handle* h, int n, F&& launch) {
    h->launches += n;
    cudaError_t e = launch();
    if (e != cudaSuccess) {
        h->err = std::string("launch failed: ") + cudaGetErrorString(e);
        return MPM_ERR_CUDA;
    }
    return MPM_OK;
}

// after a stream sync: fold the sampled launches of a replayed graph
int collect_graph_timing(mpm_handle* h, int pass) {
    for (auto& t : h->graph_timing[pass]) {
        float ms = 0.0f;
        MPM_CUDA(h, cudaEventElapsedTime(&ms, t.a, t.b));
        h->timed_ms[t.cls] += ms;
        h->timed_bytes[t.cls] += t.bytes;
        h->timed_launches[t.cls]++;
    }
    return MPM_OK;
}

// after a stream sync: fold recorded event pairs into the totals
int collect_timing(mpm_handle* h) {
    for (int c = 0; c < kNumClasses; ++c) {
        for (size_t i = 0; i < h->ev_used[c]; ++i) {
            float ms = 0.0f;
            MPM_CUDA(h, cudaEventElapsedTime(&ms, h->events[c][i].a, h->events[c][i].b));
            h->timed_ms[c] += ms;
            h->timed_bytes[c] += h->events[c][i].bytes;
            h->timed_launches[c]++;
        }
        h->ev_used[c] = 0;
    }
    return MPM_OK;
}

int check_device_flags(mpm_handle* h, cudaStream_t st) {
    int flags = 0;
    MPM_CUDA(h, cudaMemcpyAsync(&flags, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    int rc = collect_timing(h);
    if (rc != MPM_OK) return rc;
    if (flags & mpm::kErrDomain) return fail(h, MPM_ERR_DOMAIN, "a particle stencil left the grid");
    if (flags & mpm::kErrNumeric)
        return fail(h, MPM_ERR_NUMERIC, "inverted or non-finite deformation gradient");
    if (flags & mpm::kErrTimeout) return fail(h, MPM_ERR_TIMEOUT, "device wait timed out");
    return MPM_OK;
}

int validate(const mpm_config* c, std::string& why) {
    if (!c) { why = "config is NULL"; return MPM_ERR_ARG; }
    if (c->dim != 2 && c->dim != 3) { why = "dim must be 2 or 3"; return MPM_ERR_ARG; }
    if (c->bound < 0 || c->grid_res < 2 * c->bound + 3 || c->grid_res < 4) {
        why = "grid_res must be >= max(4, 2*bound + 3)";
        return MPM_ERR_ARG;
    }
    if (!(c->dt > 0.0) || !std::isfinite(c->dt)) { why = "dt must be > 0"; return MPM_ERR_ARG; }
    if (c->n_steps < 1) { why = "n_steps must be >= 1"; return MPM_ERR_ARG; }
    if (c->n_instances < 1 || !c->n_particles) { why = "need n_instances >= 1 and n_particles"; return MPM_ERR_ARG; }
    if (c->n_instances > 65535) { why = "at most 65535 instances (one grid row of blocks each)"; return MPM_ERR_ARG; }
    if (!(c->E > 0.0) || !(c->nu >= 0.0 && c->nu < 0.5) || !(c->rho0 > 0.0) || !(c->p_vol > 0.0)) {
        why = "need E > 0, 0 <= nu < 0.5, rho0 > 0, p_vol > 0";
        return MPM_ERR_ARG;
    }
    if (!(c->simp_eps >= 0.0 && c->simp_eps <= 1.0) || c->simp_q < 0 || c->simp_q > 16) {
        why = "need 0 <= simp_eps <= 1 and 0 <= simp_q <= 16";
        return MPM_ERR_ARG;
    }
    if (c->wall_mode != 0 && c->wall_mode != 1) { why = "wall_mode must be 0 or 1"; return MPM_ERR_ARG; }
    if (c->wall_mode == 1 && c->grid_res < 2 * c->bound + 3) { why = "grid too small"; return MPM_ERR_ARG; }
    if (!(c->floor_mu >= 0.0) || !(c->damping_c >= 0.0)) { why = "need floor_mu >= 0, damping_c >= 0"; return MPM_ERR_ARG; }
    if (c->loss_kind != 0 && c->loss_kind != 1) { why = "loss_kind must be 0 or 1"; return MPM_ERR_ARG; }
    if (c->checkpoint_every < 0) { why = "checkpoint_every must be >= 0"; return MPM_ERR_ARG; }
    long long n = 0;
    for (int i = 0; i < c->n_instances; ++i) {
        if (c->n_particles[i] < 0) { why = "negative particle count"; return MPM_ERR_ARG; }
        n += c->n_particles[i];
    }
    if (n > (1LL << 30)) { why = "too many particles"; return MPM_ERR_ARG; }
    if (mpm::sort_key_space(c->dim, c->grid_res, c->n_instances) >= (1LL << 31)) {
        why = "grid_res^dim * n_instances too large for 32-bit cell keys";
        return MPM_ERR_ARG;
    }
    int nd = c->design_of_instance ? c->n_designs : c->n_instances;
    if (nd < 1 || nd > c->n_instances) { why = "n_designs must be in [1, n_instances]"; return MPM_ERR_ARG; }
    if (c->design_of_instance) {
        std::vector<int> cnt(nd, -1);
        for (int i = 0; i < c->n_instances; ++i) {
            int dz = c->design_of_instance[i];
            if (dz < 0 || dz >= nd) { why = "design_of_instance out of range"; return MPM_ERR_ARG; }
            if (cnt[dz] >= 0 && cnt[dz] != c->n_particles[i]) {
                why = "instances sharing a design must have equal particle counts";
                return MPM_ERR_ARG;
            }
            cnt[dz] = c->n_particles[i];
        }
        for (int dz = 0; dz < nd; ++dz)
            if (cnt[dz] < 0) { why = "every design must be used by an instance"; return MPM_ERR_ARG; }
    }
    return MPM_OK;
}

int create_impl(const mpm_config* c, mpm_handle* h) {
    h->dim = c->dim;
    h->res = c->grid_res;
    h->T = c->n_steps;
    h->n_inst = c->n_instances;
    h->K = (c->checkpoint_every <= 0 || c->checkpoint_every > h->T) ? h->T : c->checkpoint_every;
    h->n_seg = (h->T + h->K - 1) / h->K;
    h->ncomp = 2 * h->dim + 2 * h->dim * h->dim;
    h->counts.assign(c->n_particles, c->n_particles + h->n_inst);
    h->inst_off.assign(h->n_inst + 1, 0);
    for (int i = 0; i < h->n_inst; ++i) h->inst_off[i + 1] = h->inst_off[i] + h->counts[i];
    h->N = h->inst_off[h->n_inst];
    h->np = std::max<long long>(32, (h->N + 31) / 32 * 32);
    int nd = c->design_of_instance ? c->n_designs : h->n_inst;
    h->design_of.resize(h->n_inst);
    for (int i = 0; i < h->n_inst; ++i) h->design_of[i] = c->design_of_instance ? c->design_of_instance[i] : i;
    h->dcount.assign(nd, 0);
    for (int i = 0; i < h->n_inst; ++i) h->dcount[h->design_of[i]] = h->counts[i];
    std::vector<int> doff(nd + 1, 0);
    for (int z = 0; z < nd; ++z) doff[z + 1] = doff[z] + h->dcount[z];
    h->Nd = doff[nd];
    h->dbase.resize(h->n_inst);
    for (int i = 0; i < h->n_inst; ++i) h->dbase[i] = doff[h->design_of[i]];
    h->nodes = 1;
    for (int a = 0; a < h->dim; ++a) h->nodes *= h->res;
    h->total_nodes = h->nodes * h->n_inst;

    Params& P = h->P;
    P.res = h->res;
    P.bound = c->bound;
    P.wall_mode = c->wall_mode;
    P.loss_kind = c->loss_kind;
    P.simp_q = c->simp_q;
    P.n_inst = h->n_inst;
    P.n_steps = h->T;
    P.n_total = (int)h->N;
    P.np = h->np;
    P.nodes = h->nodes;
    P.dx = (float)(1.0 / h->res);
    P.inv_dx = (float)h->res;
    P.dt = (float)c->dt;
    P.kappa = (float)(4.0 * h->res * (double)h->res);
    P.p_vol = (float)c->p_vol;
    P.rho0 = (float)c->rho0;
    P.G = (float)(c->E / (2.0 * (1.0 + c->nu)));
    P.K = (float)(c->E / (3.0 * (1.0 - 2.0 * c->nu)));
    P.eps = (float)c->simp_eps;
    P.damping = (float)c->damping_c;
    P.mu = (float)c->floor_mu;
    for (int i = 0; i < 3; ++i) P.gravity[i] = (float)c->gravity[i];
    P.pdl = 1;
    // defaults as the autotuner picks them on the 2D and 3D workloads: the
    // 80-register adjoint budget in 3D
    P.adj_blocks = h->dim == 3 ? 3 : 2;
    P.agg2 = 0;

    const long long S = (long long)h->ncomp * h->np;
    const int d = h->dim;
    int rc;
#define ALLOC(ptr, n) if ((rc = dalloc(h, &(ptr), (n))) != MPM_OK) return rc
    ALLOC(h->d_inst_off, h->n_inst + 1);
    ALLOC(h->d_dbase, h->n_inst);
    ALLOC(h->stA, S);
    ALLOC(h->stB, S);
    ALLOC(h->idA, h->np);
    ALLOC(h->idB, h->np);
    ALLOC(h->ck_state, S * h->n_seg);
    ALLOC(h->ck_id, h->np * h->n_seg);
    ALLOC(h->ck_perm, h->np * h->n_seg);
    // two sets of segment buffers: recomputation and adjoint overlap
    ALLOC(h->seg_state, 2 * S * (h->K + 1));
    ALLOC(h->seg_acc, 2 * h->total_nodes * h->K);
    ALLOC(h->seg_V, 2 * h->total_nodes * h->K);
    ALLOC(h->acc, h->total_nodes);
    ALLOC(h->V, h->total_nodes);
    ALLOC(h->Vbar, h->total_nodes);
    ALLOC(h->gadj, h->total_nodes);
    ALLOC(h->acc3, 3 * h->total_nodes);
    ALLOC(h->Vbar3, 3 * h->total_nodes);
    ALLOC(h->adj, S);
    ALLOC(h->adj2, S);
    ALLOC(h->phi_cur, 2 * h->np);
    ALLOC(h->mag_cur, 2 * d * h->np);
    ALLOC(h->x0_fwd, d * h->np);
    ALLOC(h->x0_seg, 2 * d * h->np);
    ALLOC(h->gphi_cur, h->np);
    ALLOC(h->gmag_cur, d * h->np);
    ALLOC(h->phi_d, h->Nd);
    ALLOC(h->mag_d, d * h->Nd);
    ALLOC(h->field, (long long)h->n_inst * h->T * d);
    ALLOC(h->target, d * h->N);
    ALLOC(h->mom, (long long)h->T * h->n_inst);
    ALLOC(h->Minst, h->n_inst);
    ALLOC(h->loss_acc, h->n_inst);
    ALLOC(h->dloss, h->n_inst);
    ALLOC(h->gphi_d, h->Nd);
    ALLOC(h->gmag_d, d * h->Nd);
    ALLOC(h->gfield_d, (long long)h->n_inst * h->T * d);
    ALLOC(h->d_ext, 1);
    ALLOC(h->d_fgrad, (long long)h->n_inst * h->T * d * d);
    ALLOC(h->d_gfgrad, (long long)h->n_inst * h->T * d * d);
    ALLOC(h->d_bmotion, (long long)mpm::kMaxBoundaries * h->T * 2 * d);
    ALLOC(h->st_x0, d * h->N);
    ALLOC(h->st_v0, d * h->N);
    ALLOC(h->st_xout, d * h->N);
    ALLOC(h->st_loss, h->n_inst);
    ALLOC(h->d_err, 1);
    ALLOC(h->bar, 2);
    ALLOC(h->perm, h->np);
    h->sb.n_keys = mpm::sort_key_space(d, h->res, h->n_inst);
    h->sb.scan_tmp_len = mpm::sort_scan_tmp_len(h->sb.n_keys);
    ALLOC(h->sb.keys, h->np);
    ALLOC(h->sb.slot, h->np);
    ALLOC(h->sb.counts, h->sb.n_keys);
    ALLOC(h->sb.offsets, h->sb.n_keys);
    ALLOC(h->sb.scan_tmp, h->sb.scan_tmp_len);
    if (d == 3) {
        const long long nb = mpm::blocks_per_axis(h->res);
        h->blocks = true;
        h->n_blocks = nb * nb * nb * h->n_inst;
        int dev = 0, sms = 0;
        MPM_CUDA(h, cudaGetDevice(&dev));
        MPM_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        h->grid_ctas = 4 * std::max(1, sms);
        h->n_wbox = h->np / 32;
        ALLOC(h->blk_flag, 4 * h->n_blocks);
        ALLOC(h->blk_list, 4 * h->n_blocks);
        ALLOC(h->blk_count, 4);
        ALLOC(h->blk_wbox, 4 * h->n_wbox);
    }
#undef ALLOC
    MPM_CUDA(h, cudaMemcpy(h->d_inst_off, h->inst_off.data(), sizeof(int) * (h->n_inst + 1),
                           cudaMemcpyHostToDevice));
    MPM_CUDA(h, cudaMemcpy(h->d_dbase, h->dbase.data(), sizeof(int) * h->n_inst,
                           cudaMemcpyHostToDevice));
    if (h->blocks) {
        // the recomputation finds its accumulators, flags and counts zero:
        // every adjoint segment clears what its recomputation listed
        MPM_CUDA(h, cudaMemset(h->seg_acc, 0, sizeof(float4) * 2 * h->total_nodes * h->K));
        MPM_CUDA(h, cudaMemset(h->blk_flag, 0, sizeof(int) * 4 * h->n_blocks));
        MPM_CUDA(h, cudaMemset(h->blk_count, 0, sizeof(int) * 4));
        MPM_CUDA(h, cudaMemset(h->blk_wbox, 0, sizeof(int4) * 4 * h->n_wbox));
    }
    // padding lanes of the state buffers stay finite
    MPM_CUDA(h, cudaMemset(h->stA, 0, sizeof(float) * S));
    MPM_CUDA(h, cudaMemset(h->stB, 0, sizeof(float) * S));
    MPM_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    MPM_CUDA(h, cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&h->ev_fork, &h->ev_rec[0], &h->ev_rec[1], &h->ev_adj[0], &h->ev_adj[1]})
        MPM_CUDA(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    // the initial memsets ran on the default stream; a caller's non-blocking
    // stream does not wait for it
    MPM_CUDA(h, cudaDeviceSynchronize());
    return MPM_OK;
}

StepArgs base_args(mpm_handle* h) {
    StepArgs a;
    a.x0 = h->x0_fwd;
    a.phi = h->phi_cur;
    a.mag = h->mag_cur;
    a.field = h->field;
    a.inst_off = h->d_inst_off;
    a.err = h->d_err;
    a.Minst = h->Minst;
    a.dloss = h->dloss;
    a.gphi = h->gphi_cur;
    a.gmag = h->gmag_cur;
    a.gfield = h->gfield_d;
    return a;
}

// The persistent passes run when asked for, without solid boxes or a field
// gradient (which they do not carry), and in 3D with the node-block lists.
bool use_persist(const mpm_handle* h) {
    return h->persistent && h->P.ext == nullptr && (h->dim == 2 || (h->blocks && h->grid_blocks));
}

// one persistent launch: the barrier is zeroed first
int persist(mpm_handle* h, mpm::PersistKind kind, int cls, double bytes, mpm::PersistArgs& pa, cudaStream_t st) {
    pa.bar = h->bar;
    pa.spin_limit = h->spin_limit;
    MPM_CUDA(h, cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), st));
    // 256-thread CTAs: the barrier's cost grows with the CTAs that arrive at it
    return timed(h, cls, bytes, st, [&] {
        return mpm::launch_persist(h->dim, kind, h->dim == 3, h->P, pa, 256, 0, st);
    });
}

// node-block list i (3D): 0 and 1 for the forward pass, 2 + b for recomputation set b
mpm::ActiveBlocks block_list(const mpm_handle* h, int i) {
    mpm::ActiveBlocks b;
    if (!h->blocks) return b;
    if (i >= 4) {  // a resident set's list
        const int r = i - 4;
        b.flag = h->res_flag + (long long)r * h->n_blocks;
        b.list = h->res_list + (long long)r * h->n_blocks;
        b.count = h->res_count + r;
        b.wbox = h->res_wbox + (long long)r * h->n_wbox;
        return b;
    }
    b.flag = h->blk_flag + (long long)i * h->n_blocks;
    b.list = h->blk_list + (long long)i * h->n_blocks;
    b.count = h->blk_count + i;
    b.wbox = h->blk_wbox + (long long)i * h->n_wbox;
    return b;
}

// Empties list i: its flags (over the listed blocks), its count and the
// warps' boxes; with acc, also zeroes n_sub accumulators (stride acc_stride)
// over the listed blocks.
int clear_list(mpm_handle* h, int i, float4* acc, long long acc_stride, int n_sub, cudaStream_t st) {
    const mpm::ActiveBlocks b = block_list(h, i);
    h->launches++;
    MPM_CUDA(h, mpm::launch_clear_blocks(h->P, acc, acc_stride, b, std::max(1, n_sub), st));
    MPM_CUDA(h, cudaMemsetAsync(b.count, 0, sizeof(int), st));
    MPM_CUDA(h, cudaMemsetAsync(b.wbox, 0, sizeof(int4) * h->n_wbox, st));
    return MPM_OK;
}

// copy src -> dst (device) unless they are the same buffer
int dcopy(mpm_handle* h, void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (dst == src || bytes == 0) return MPM_OK;
    MPM_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return MPM_OK;
}

struct SegSet {
    float* state;   // [K + 1] states
    float4* acc;    // [K] accumulators
    float4* V;      // [K] grid velocities
    float* phi;     // current-order design of the segment
    float* mag;
    float* x0;      // current-order initial positions of the segment
    int list_id;    // 3D: its node-block list (block_list)
};

SegSet seg_set(mpm_handle* h, int b) {
    const long long S = (long long)h->ncomp * h->np;
    const long long G = h->total_nodes;
    SegSet ss;
    ss.state = h->seg_state + (long long)b * S * (h->K + 1);
    ss.acc = h->seg_acc + (long long)b * G * h->K;
    ss.V = h->seg_V + (long long)b * G * h->K;
    ss.phi = h->phi_cur + (long long)b * h->np;
    ss.mag = h->mag_cur + (long long)b * h->dim * h->np;
    ss.x0 = h->x0_seg + (long long)b * h->dim * h->np;
    ss.list_id = 2 + b;
    return ss;
}

// resident set r (MPM_OPT_RESIDENT_SEGMENTS)
SegSet res_set(mpm_handle* h, int r) {
    const long long S = (long long)h->ncomp * h->np;
    const long long G = h->total_nodes;
    SegSet ss;
    ss.state = h->res_state + (long long)r * S * (h->K + 1);
    ss.acc = h->res_acc + (long long)r * G * h->K;
    ss.V = h->res_V + (long long)r * G * h->K;
    ss.phi = h->res_phi + (long long)r * h->np;
    ss.mag = h->res_mag + (long long)r * h->dim * h->np;
    ss.x0 = h->res_x0 + (long long)r * h->dim * h->np;
    ss.list_id = 4 + r;
    return ss;
}

// Trailing segments of an n_seg-segment pass that run from resident sets:
// none while autotuning (a truncated horizon) or in the persistent form.
int resident_segments(const mpm_handle* h, int n_seg) {
    if (h->tune_T > 0 || use_persist(h)) return 0;
    return std::min(h->n_res, n_seg);
}

int recompute_segment(mpm_handle* h, int seg, int T, const SegSet& ss, cudaStream_t st, float* mom = nullptr);

// --- the forward pass: library-owned buffers only, so it can be captured ---
int forward_pass(mpm_handle* h, cudaStream_t st) {
    const int d = h->dim;
    const Params& P = h->P;
    const long long S = (long long)h->ncomp * h->np;
    const long long G = h->total_nodes;
    const bool persistent = use_persist(h);
    const bool fuse = h->fuse_fwd && !persistent;
    auto acc3 = [&](int i) { return h->acc3 + G * (i % 3); };
    int rc;
    MPM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    MPM_CUDA(h, cudaMemsetAsync(h->mom, 0, sizeof(float) * h->T * h->n_inst, st));
    MPM_CUDA(h, cudaMemsetAsync(h->Minst, 0, sizeof(float) * h->n_inst, st));
    MPM_CUDA(h, cudaMemsetAsync(h->loss_acc, 0, sizeof(float) * h->n_inst, st));
    if (fuse) MPM_CUDA(h, cudaMemsetAsync(h->acc3, 0, sizeof(float4) * 2 * G, st));
    else MPM_CUDA(h, cudaMemsetAsync(h->acc, 0, sizeof(float4) * G, st));
    // 3D with the grid kernel: the P2G kernels list the node blocks they
    // touch, and the grid kernel walks the list.  Segment j uses list j & 1;
    // its first P2G runs in the last kernel of segment j - 1, before the
    // sort, so each list is emptied once the segment after it has begun.
    const bool lists = h->blocks && !fuse && h->grid_blocks;
    auto lean_blk = [&](int substep) { return block_list(h, (substep / h->K) & 1); };
    if (lists) {
        int rc0;
        if ((rc0 = clear_list(h, 0, nullptr, 0, 1, st)) || (rc0 = clear_list(h, 1, nullptr, 0, 1, st))) return rc0;
    }

    float* cur = h->stA;
    float* nxt = h->stB;
    int* id_cur = h->idA;
    int* id_nxt = h->idB;
    const int T = h->tune_T > 0 ? std::min(h->T, h->tune_T) : h->T;
    const int n_seg = (T + h->K - 1) / h->K;
    // the last n_res segments are stored into resident sets as they run; the
    // lean substeps end where the first of them begins
    const int first_res = n_seg - resident_segments(h, n_seg);
    const int lean_end = std::min(T, first_res * h->K);
    if ((rc = counted(h, 1, [&] {
             return mpm::launch_init_state(d, P, h->st_x0, h->st_v0, cur, id_cur, h->x0_fwd, st);
         })))
        return rc;
    for (int seg = 0; seg < n_seg; ++seg) {
        const int s0 = seg * h->K, s1 = std::min(s0 + h->K, T);
        // cell sort and reorder of the full state
        if ((rc = counted(h, 5, [&] {
                 return mpm::launch_sort(d, P, cur, h->np, h->d_inst_off, h->sb, h->perm, h->d_err, st, h->x0_fwd);
             })))
            return rc;
        if ((rc = counted(h, 1, [&] {
                 return mpm::launch_reorder(h->ncomp, P, cur, nxt, h->perm, id_cur, id_nxt, st);
             })))
            return rc;
        std::swap(cur, nxt);
        std::swap(id_cur, id_nxt);
        // a new segment: the list of the last segment is done with, and the
        // warps' boxes of this segment's list describe the old particle order
        if (lists && seg > 0) {
            if ((rc = clear_list(h, (seg - 1) & 1, nullptr, 0, 1, st))) return rc;
            MPM_CUDA(h, cudaMemsetAsync(block_list(h, seg & 1).wbox, 0, sizeof(int4) * h->n_wbox, st));
        }
        if ((rc = counted(h, 1, [&] {
                 return mpm::launch_gather_design(d, P, id_cur, h->d_inst_off, h->d_dbase, h->phi_d,
                                                  h->mag_d, h->Nd, h->phi_cur, h->mag_cur, h->st_x0,
                                                  h->x0_fwd, st);
             })))
            return rc;
        MPM_CUDA(h, cudaMemcpyAsync(h->ck_state + S * seg, cur, sizeof(float) * S,
                                    cudaMemcpyDeviceToDevice, st));
        MPM_CUDA(h, cudaMemcpyAsync(h->ck_id + h->np * seg, id_cur, sizeof(int) * h->np,
                                    cudaMemcpyDeviceToDevice, st));
        MPM_CUDA(h, cudaMemcpyAsync(h->ck_perm + h->np * seg, h->perm, sizeof(int) * h->np,
                                    cudaMemcpyDeviceToDevice, st));
        StepArgs a = base_args(h);
        a.mom = h->mom;
        if (seg == 0 && (rc = counted(h, 1, [&] {
                             return mpm::launch_instance_mass(P, h->phi_cur, h->d_inst_off, h->Minst, st);
                         })))
            return rc;
        if (seg >= first_res) {
            // a resident segment: every state and grid stored, as a
            // recomputation would (with the momentum rows of the loss)
            const SegSet ss = res_set(h, seg - first_res);
            const int Ks = s1 - s0;
            // lists: the set holds nothing from an earlier forward pass
            if (h->blocks && h->grid_blocks && (rc = clear_list(h, ss.list_id, ss.acc, G, Ks, st))) return rc;
            if ((rc = recompute_segment(h, seg, T, ss, st, h->mom))) return rc;
            MPM_CUDA(h, cudaMemcpyAsync(cur, ss.state + S * Ks, sizeof(float) * S, cudaMemcpyDeviceToDevice, st));
            continue;
        }
        if (persistent) {
            // the whole segment in one cooperative launch
            mpm::PersistArgs pa;
            pa.base = a;
            pa.s0 = s0;
            pa.s1 = s1;
            pa.T = T;
            pa.first_p2g = seg == 0;
            pa.st[0] = cur;
            pa.st[1] = nxt;
            pa.acc = h->acc;
            pa.V = h->V;
            if (lists) {
                pa.blk = lean_blk(s0);
                pa.blk_next = lean_blk(s1);
            }
            if ((rc = persist(h, mpm::PersistKind::kLean, kFwdParticle,
                              h->N * (s1 - s0) * particle_bytes(d, kFwdParticle, kFused), pa, st)))
                return rc;
            if ((s1 - s0) & 1) std::swap(cur, nxt);  // the final state is in st[(s1 - s0) & 1]
            continue;
        }
        if (seg == 0) {
            a.s_in = cur;
            a.acc = fuse ? acc3(0) : h->acc;
            a.n_p2g = 0;
            if (lists) a.blk = lean_blk(0);
            if ((rc = timed(h, kFwdParticle, h->N * particle_bytes(d, kFwdParticle, kFirstP2G), st, [&] {
                     return mpm::launch_forward(d, false, true, false, fuse, P, a, h->block, st);
                 })))
                return rc;
        }
        for (int n = s0; n < s1; ++n) {
            if (!fuse && (rc = timed(h, kGrid, 48.0 * G, st, [&] {
                              if (lists)
                                  return mpm::launch_grid_blocks(P, h->acc, h->V, lean_blk(n), true, n, h->grid_ctas, st);
                              return mpm::launch_grid(d, P, h->acc, h->V, nullptr, true, n, st);
                          })))
                return rc;
            const bool p2g = n + 1 < lean_end;  // a resident segment runs its own first P2G
            const bool all = n + 1 == s1;
            a.s_in = cur;
            a.s_out = nxt;
            a.n_g2p = n;
            a.n_p2g = n + 1;
            if (fuse) {
                a.accG = acc3(n);
                a.acc = acc3(n + 1);
                a.zero4 = acc3(n + 2);
                a.zero_n = G;
            } else {
                a.V = h->V;
                a.acc = h->acc;
            }
            if (!p2g) a.acc = nullptr;
            if (lists && p2g) a.blk = lean_blk(n + 1);
            if ((rc = timed(h, kFwdParticle, h->N * particle_bytes(d, kFwdParticle, all ? kFusedStore : kFused), st, [&] {
                     return mpm::launch_forward(d, true, p2g, all, fuse, P, a, h->block, st);
                 })))
                return rc;
            std::swap(cur, nxt);
        }
    }
    if ((rc = counted(h, 2, [&] {
             return mpm::launch_loss(d, P, cur, h->x0_fwd, h->target, id_cur, h->d_inst_off, h->Minst, h->mom,
                                     h->loss_acc, h->st_loss, st);
         })))
        return rc;
    h->cur = cur;
    h->id_cur = id_cur;
    return MPM_OK;
}

// --- the backward pass: from h->dloss to gphi_d / gmag_d / gfield_d ---
//
// Per checkpoint segment, in reverse: recompute the segment from its
// checkpoint (storing every state and grid), then run its adjoint.  The
// recomputation of segment s-1 does not depend on the adjoint of segment s,
// so with two streams they overlap: the segment buffers and the
// current-order design come in two sets, used by segment parity.

// mom: the forward pass's momentum rows (locomotion loss), accumulated by the
// G2P of each substep when the forward pass stores a resident segment; null
// in the backward pass.
int recompute_segment(mpm_handle* h, int seg, int T, const SegSet& ss, cudaStream_t st, float* mom) {
    const int d = h->dim;
    const Params& P = h->P;
    const long long S = (long long)h->ncomp * h->np;
    const long long G = h->total_nodes;
    const bool persistent = use_persist(h);
    const bool fuse_rec = h->fuse_fwd && !persistent;
    const int s0 = seg * h->K, s1 = std::min(s0 + h->K, T), Ks = s1 - s0;
    const int* id_seg = h->ck_id + h->np * seg;
    auto state = [&](int k) { return ss.state + S * k; };
    auto gacc = [&](int k) { return ss.acc + G * k; };
    auto gV = [&](int k) { return ss.V + G * k; };
    int rc;
    MPM_CUDA(h, cudaMemcpyAsync(state(0), h->ck_state + S * seg, sizeof(float) * S,
                                cudaMemcpyDeviceToDevice, st));
    if ((rc = counted(h, 1, [&] {
             return mpm::launch_gather_design(d, P, id_seg, h->d_inst_off, h->d_dbase, h->phi_d,
                                              h->mag_d, h->Nd, ss.phi, ss.mag, h->st_x0, ss.x0, st);
         })))
        return rc;
    // with node-block lists, the accumulators are zero where the last use of
    // this set listed blocks (its adjoint cleared them), and zero elsewhere since
    const bool lists = h->blocks && h->grid_blocks;
    if (!lists)
        MPM_CUDA(h, cudaMemsetAsync(gacc(0), 0, sizeof(float4) * G * ((fuse_rec && Ks >= 2) ? 2 : 1), st));
    StepArgs a = base_args(h);
    a.phi = ss.phi;
    a.mag = ss.mag;
    a.x0 = ss.x0;
    if (persistent) {
        mpm::PersistArgs pa;
        pa.base = a;
        pa.s0 = s0;
        pa.s1 = s1;
        pa.T = T;
        pa.state = ss.state;
        pa.S = S;
        pa.acc = ss.acc;
        pa.V = ss.V;
        pa.G = G;
        if (lists) pa.blk = block_list(h, ss.list_id);
        return persist(h, mpm::PersistKind::kStore, kFwdParticle,
                       h->N * Ks * particle_bytes(d, kFwdParticle, kFusedStore), pa, st);
    }
    a.s_in = state(0);
    a.acc = gacc(0);
    a.n_p2g = s0;
    if (lists) a.blk = block_list(h, ss.list_id);
    if ((rc = timed(h, kFwdParticle, h->N * particle_bytes(d, kFwdParticle, kFirstP2G), st, [&] {
             return mpm::launch_forward(d, false, true, false, fuse_rec, P, a, h->block, st);
         })))
        return rc;
    for (int k = 0; k < Ks; ++k) {
        const int n = s0 + k;
        const bool p2g = k + 1 < Ks;
        float4* next_acc = p2g ? gacc(k + 1) : nullptr;
        if (!fuse_rec && (rc = timed(h, kGrid, 48.0 * G, st, [&] {
                          if (lists)
                              return mpm::launch_grid_blocks(P, gacc(k), gV(k), block_list(h, ss.list_id), false, n,
                                                             h->grid_ctas, st);
                          return mpm::launch_grid(d, P, gacc(k), gV(k), next_acc, false, n, st);
                      })))
            return rc;
        a = base_args(h);
        a.phi = ss.phi;
        a.mag = ss.mag;
        a.x0 = ss.x0;
        a.mom = mom;
        a.s_in = state(k);
        a.s_out = state(k + 1);
        a.acc = next_acc;
        a.n_g2p = n;
        a.n_p2g = n + 1;
        if (p2g && lists) a.blk = block_list(h, ss.list_id);
        if (fuse_rec) {
            a.accG = gacc(k);
            a.zero4 = k + 2 < Ks ? gacc(k + 2) : nullptr;
            a.zero_n = G;
        } else {
            a.V = gV(k);
        }
        if ((rc = timed(h, kFwdParticle, h->N * particle_bytes(d, kFwdParticle, kFusedStore), st, [&] {
                 return mpm::launch_forward(d, true, p2g, true, fuse_rec, P, a, h->block, st);
             })))
            return rc;
    }
    return MPM_OK;
}

// The end of a segment's adjoint: design gradients back to input order, and
// the segment set left as its next recomputation expects it (3D lists: the
// accumulators zero over the listed blocks, flags and counts zero).
int finish_adjoint_segment(mpm_handle* h, const int* id_seg, const SegSet& ss, int Ks, cudaStream_t st) {
    const Params& P = h->P;
    int rc;
    if ((rc = counted(h, 1, [&] {
             return mpm::launch_scatter_design_grad(h->dim, P, id_seg, h->d_inst_off, h->d_dbase, h->gphi_cur,
                                                    h->gmag_cur, h->Nd, h->gphi_d, h->gmag_d, st);
         })))
        return rc;
    if (h->blocks && h->grid_blocks && (rc = clear_list(h, ss.list_id, ss.acc, h->total_nodes, Ks, st)))
        return rc;
    return MPM_OK;
}

int adjoint_segment(mpm_handle* h, int seg, int T, const SegSet& ss, float* adj, float* adj_next,
                    cudaStream_t st) {
    const int d = h->dim;
    const Params& P = h->P;
    const long long S = (long long)h->ncomp * h->np;
    const long long G = h->total_nodes;
    const bool persistent = use_persist(h);
    const bool fuse = h->fuse_adj && !persistent;  // grid adjoint evaluated inside the adjoint kernels
    // G2P^T needs the grid velocity: stored by the grid kernel, or (fused
    // recomputation) recovered from the stored accumulator
    const bool fuse_v = fuse || (h->fuse_fwd && !persistent);
    const int s0 = seg * h->K, s1 = std::min(s0 + h->K, T), Ks = s1 - s0;
    const int* id_seg = h->ck_id + h->np * seg;
    auto state = [&](int k) { return ss.state + S * k; };
    auto gacc = [&](int k) { return ss.acc + G * k; };
    auto gV = [&](int k) { return ss.V + G * k; };
    auto vb3 = [&](int i) { return h->Vbar3 + G * (((i % 3) + 3) % 3); };
    // the grid adjoint of substep n = s0 + k: over the node blocks its P2G listed (3D), or every node
    auto grid_adjoint = [&](int k, int n) {
        if (h->blocks && h->grid_blocks)
            return mpm::launch_grid_adjoint_blocks(P, gacc(k), h->Vbar, h->gadj, block_list(h, ss.list_id), n,
                                                   h->grid_ctas, st);
        return mpm::launch_grid_adjoint(d, P, gacc(k), h->Vbar, h->gadj, n, st);
    };
    auto args = [&]() {
        StepArgs a = base_args(h);
        a.phi = ss.phi;
        a.mag = ss.mag;
        a.x0 = ss.x0;
        a.adj = adj;
        a.mom = h->mom;
        return a;
    };
    int rc;
    MPM_CUDA(h, cudaMemsetAsync(h->gphi_cur, 0, sizeof(float) * h->np, st));
    MPM_CUDA(h, cudaMemsetAsync(h->gmag_cur, 0, sizeof(float) * d * h->np, st));
    // --- adjoint of the state at the segment end ---
    if (s1 == T) {
        if ((rc = counted(h, 1, [&] {
                 return mpm::launch_seed(d, P, state(Ks), ss.x0, h->target, id_seg, h->d_inst_off, ss.phi,
                                         h->Minst, h->mom, h->dloss, adj, h->gphi_cur, st);
             })))
            return rc;
    } else {
        if ((rc = counted(h, 1, [&] {
                 return mpm::launch_unpermute(h->ncomp, P, adj_next, adj, h->ck_perm + h->np * (seg + 1), st);
             })))
            return rc;
    }
    if (persistent) {
        mpm::PersistArgs pa;
        pa.base = args();
        pa.base.Vbar = h->Vbar;
        pa.base.gadj = h->gadj;
        pa.s0 = s0;
        pa.s1 = s1;
        pa.T = T;
        pa.state = ss.state;
        pa.S = S;
        pa.acc = ss.acc;
        pa.V = ss.V;
        pa.G = G;
        if (h->blocks) pa.blk = block_list(h, ss.list_id);
        if ((rc = persist(h, mpm::PersistKind::kAdjoint, kAdjParticle,
                          h->N * Ks * particle_bytes(d, kAdjParticle, kFused), pa, st)))
            return rc;
        return finish_adjoint_segment(h, id_seg, ss, Ks, st);
    }
    // G2P^T of the last substep of the segment
    StepArgs a = args();
    a.s_in = state(Ks);
    a.s_aux = state(Ks - 1);
    a.n_p2g = s1;
    if (fuse) {
        a.Vbar = vb3(s1 - 1);
        a.zero4 = vb3(s1 + 1);
        a.zero_n = G;
    } else {
        a.Vbar = h->Vbar;
    }
    if (fuse_v) a.accG = gacc(Ks - 1);
    else a.V = gV(Ks - 1);
    if ((rc = timed(h, kAdjParticle, h->N * particle_bytes(d, kAdjParticle, kLastG2PT), st, [&] {
             return mpm::launch_adjoint(d, false, true, fuse, fuse_v, P, a, h->block, st);
         })))
        return rc;
    for (int k = Ks - 1; k >= 1; --k) {
        const int n = s0 + k;
        if (!fuse && (rc = timed(h, kGridAdj, 64.0 * G, st, [&] { return grid_adjoint(k, n); })))
            return rc;
        a = args();
        a.s_in = state(k);
        a.s_aux = state(k - 1);
        a.n_p2g = n;
        if (fuse) {
            a.accP = gacc(k);
            a.VbarIn = vb3(n);
            a.Vbar = vb3(n - 1);
            a.zero4 = vb3(n + 1);
            a.zero_n = G;
        } else {
            a.Vbar = h->Vbar;
            a.gadj = h->gadj;
        }
        if (fuse_v) a.accG = gacc(k - 1);
        else a.V = gV(k - 1);
        if ((rc = timed(h, kAdjParticle, h->N * particle_bytes(d, kAdjParticle, kFused), st, [&] {
                 return mpm::launch_adjoint(d, true, true, fuse, fuse_v, P, a, h->block, st);
             })))
            return rc;
    }
    if (!fuse && (rc = timed(h, kGridAdj, 64.0 * G, st, [&] { return grid_adjoint(0, s0); })))
        return rc;
    a = args();
    a.s_in = state(0);
    a.n_p2g = s0;
    if (fuse) {
        a.accP = gacc(0);
        a.VbarIn = vb3(s0);
        a.zero4 = vb3(s0 + 2);
        a.zero_n = G;
    } else {
        a.gadj = h->gadj;
    }
    if ((rc = timed(h, kAdjParticle, h->N * particle_bytes(d, kAdjParticle, kFirstP2GT), st, [&] {
             return mpm::launch_adjoint(d, true, false, fuse, fuse_v, P, a, h->block, st);
         })))
        return rc;
    return finish_adjoint_segment(h, id_seg, ss, Ks, st);
}

int backward_pass(mpm_handle* h, cudaStream_t st) {
    const int d = h->dim;
    const long long G = h->total_nodes;
    int rc;
    MPM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    MPM_CUDA(h, cudaMemsetAsync(h->gphi_d, 0, sizeof(float) * h->Nd, st));
    MPM_CUDA(h, cudaMemsetAsync(h->gmag_d, 0, sizeof(float) * d * h->Nd, st));
    MPM_CUDA(h, cudaMemsetAsync(h->gfield_d, 0, sizeof(float) * h->n_inst * h->T * d, st));
    if (h->ext_host.fgrad)
        MPM_CUDA(h, cudaMemsetAsync(h->d_gfgrad, 0, sizeof(float) * h->n_inst * h->T * d * d, st));
    if (h->fuse_adj && !use_persist(h)) MPM_CUDA(h, cudaMemsetAsync(h->Vbar3, 0, sizeof(float4) * 3 * G, st));
    else MPM_CUDA(h, cudaMemsetAsync(h->Vbar, 0, sizeof(float4) * G, st));
    const int T = h->tune_T > 0 ? std::min(h->T, h->tune_T) : h->T;
    const int n_seg = (T + h->K - 1) / h->K;
    float* adj = h->adj;
    float* adj_next = h->adj2;
    // segments first_res .. n_seg - 1 were stored by the forward pass
    const int first_res = n_seg - resident_segments(h, n_seg);
    // (the persistent kernels each take the whole GPU: one stream)
    if (!h->two_streams || n_seg < 2 || first_res == 0 || use_persist(h)) {
        for (int seg = n_seg - 1; seg >= 0; --seg) {
            const bool resident = seg >= first_res;
            const SegSet ss = resident ? res_set(h, seg - first_res) : seg_set(h, 0);
            if (!resident && (rc = recompute_segment(h, seg, T, ss, st))) return rc;
            if ((rc = adjoint_segment(h, seg, T, ss, adj, adj_next, st))) return rc;
            std::swap(adj, adj_next);
        }
        return MPM_OK;
    }
    // recomputation one segment ahead on the second stream; the last
    // recomputed segment starts at once, beside the resident segments' adjoint
    cudaStream_t aux = h->aux_stream;
    MPM_CUDA(h, cudaEventRecord(h->ev_fork, st));
    MPM_CUDA(h, cudaStreamWaitEvent(aux, h->ev_fork, 0));
    const int last = first_res - 1;
    if ((rc = recompute_segment(h, last, T, seg_set(h, last & 1), aux))) return rc;
    MPM_CUDA(h, cudaEventRecord(h->ev_rec[last & 1], aux));
    for (int seg = n_seg - 1; seg >= 0; --seg) {
        if (seg >= first_res) {
            if ((rc = adjoint_segment(h, seg, T, res_set(h, seg - first_res), adj, adj_next, st))) return rc;
            std::swap(adj, adj_next);
            continue;
        }
        if (seg >= 1) {
            // set (seg-1)&1 was last read by the adjoint of segment seg+1
            if (seg + 1 <= last) MPM_CUDA(h, cudaStreamWaitEvent(aux, h->ev_adj[(seg + 1) & 1], 0));
            if ((rc = recompute_segment(h, seg - 1, T, seg_set(h, (seg - 1) & 1), aux))) return rc;
            MPM_CUDA(h, cudaEventRecord(h->ev_rec[(seg - 1) & 1], aux));
        }
        MPM_CUDA(h, cudaStreamWaitEvent(st, h->ev_rec[seg & 1], 0));
        if ((rc = adjoint_segment(h, seg, T, seg_set(h, seg & 1), adj, adj_next, st))) return rc;
        MPM_CUDA(h, cudaEventRecord(h->ev_adj[seg & 1], st));
        std::swap(adj, adj_next);
    }
    return MPM_OK;
}

// Run pass 0 (forward) or 1 (backward) on `st`: directly, or by replaying
// its CUDA graph (captured on an internal stream on first use).
int run_pass(mpm_handle* h, int pass, cudaStream_t st) {
    auto body = [&](cudaStream_t s) { return pass == 0 ? forward_pass(h, s) : backward_pass(h, s); };
    if (!h->graphs) return body(st);
    if (!h->exec[pass]) {
        long long launches_before = h->launches;
        long long cls_before[kNumClasses];
        for (int c = 0; c < kNumClasses; ++c) cls_before[c] = h->cls_issued[c];
        MPM_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        h->capture_pass = pass;
        int rc = body(h->cap_stream);
        h->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (rc != MPM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return fail(h, MPM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->exec[pass], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->exec[pass] = nullptr;
            return fail(h, MPM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        h->graph_launches[pass] = h->launches - launches_before;
        h->launches = launches_before;
        for (int c = 0; c < kNumClasses; ++c) {
            h->graph_cls[pass][c] = h->cls_issued[c] - cls_before[c];
            h->cls_issued[c] = cls_before[c];
        }
    }
    MPM_CUDA(h, cudaGraphLaunch(h->exec[pass], st));
    h->launches += h->graph_launches[pass];
    for (int c = 0; c < kNumClasses; ++c) h->cls_issued[c] += h->graph_cls[pass][c];
    h->ran_graph[pass] = true;
    return MPM_OK;
}

int finish(mpm_handle* h, int pass, cudaStream_t st) {
    int rc = check_device_flags(h, st);
    // a pass that stopped early (a timed-out barrier) may leave the segment
    // accumulators and lists set: the next backward pass clears them in full
    if (rc != MPM_OK && h->blocks) h->seg_dirty = h->res_dirty = true;
    if (h->ran_graph[pass]) {
        h->ran_graph[pass] = false;
        int r2 = collect_graph_timing(h, pass);
        if (rc == MPM_OK) rc = r2;
    }
    return rc;
}

int forward_impl(mpm_handle* h, const float* x0, const float* v0, const float* phi,
                 const float* mag, const float* field, const float* target, float* x_out,
                 float* loss_out, cudaStream_t st) {
    const int d = h->dim;
    const Params& P = h->P;
    if (!loss_out) return fail(h, MPM_ERR_ARG, "loss_out is NULL");
    if (h->N > 0 && (!x0 || !phi || !mag)) return fail(h, MPM_ERR_ARG, "x0, phi_bar and mag are required");
    if (!field) return fail(h, MPM_ERR_ARG, "field is required");
    if (h->N > 0 && P.loss_kind == 0 && !target) return fail(h, MPM_ERR_ARG, "target is required for loss_kind 0");
    h->forward_done = false;
    h->backward_done = false;
    int rc;
    // stage the inputs into library-owned buffers (the passes read only those)
    if ((rc = dcopy(h, h->st_x0, x0, sizeof(float) * d * h->N, st))) return rc;
    if (v0) {
        if ((rc = dcopy(h, h->st_v0, v0, sizeof(float) * d * h->N, st))) return rc;
    } else {
        MPM_CUDA(h, cudaMemsetAsync(h->st_v0, 0, sizeof(float) * d * h->N, st));
    }
    if ((rc = dcopy(h, h->phi_d, phi, sizeof(float) * h->Nd, st))) return rc;
    if ((rc = dcopy(h, h->mag_d, mag, sizeof(float) * d * h->Nd, st))) return rc;
    if ((rc = dcopy(h, h->field, field, sizeof(float) * h->n_inst * h->T * d, st))) return rc;
    if (target && (rc = dcopy(h, h->target, target, sizeof(float) * d * h->N, st))) return rc;
    if (h->n_res > 0 && h->blocks && h->grid_blocks && h->res_dirty) {
        // a pass over every node left the resident accumulators set; the lists expect them zero
        const long long r = h->n_res;
        MPM_CUDA(h, cudaMemsetAsync(h->res_acc, 0, sizeof(float4) * r * h->total_nodes * h->K, st));
        MPM_CUDA(h, cudaMemsetAsync(h->res_flag, 0, sizeof(int) * r * h->n_blocks, st));
        MPM_CUDA(h, cudaMemsetAsync(h->res_count, 0, sizeof(int) * r, st));
        MPM_CUDA(h, cudaMemsetAsync(h->res_wbox, 0, sizeof(int4) * r * h->n_wbox, st));
        h->res_dirty = false;
    }
    if ((rc = run_pass(h, 0, st))) return rc;
    if (h->n_res > 0 && h->blocks && !h->grid_blocks) h->res_dirty = true;
    if ((rc = dcopy(h, loss_out, h->st_loss, sizeof(float) * h->n_inst, st))) return rc;
    if (x_out) {
        h->launches++;
        MPM_CUDA(h, mpm::launch_to_input_order(d, P, h->cur, 0, h->id_cur, x_out, st, 0, h->x0_fwd));
    }
    rc = finish(h, 0, st);
    if (rc != MPM_OK) return rc;
    h->forward_done = true;
    return MPM_OK;
}

int backward_impl(mpm_handle* h, const float* dloss, float* g_phi, float* g_mag, float* g_field,
                  cudaStream_t st) {
    if (!h->forward_done) return fail(h, MPM_ERR_STATE, "mpm_backward needs a successful mpm_forward first");
    if (!dloss) return fail(h, MPM_ERR_ARG, "dloss is NULL");
    const int d = h->dim;
    int rc;
    if ((rc = dcopy(h, h->dloss, dloss, sizeof(float) * h->n_inst, st))) return rc;
    if (h->blocks && h->grid_blocks && h->seg_dirty) {
        // the last backward pass ran over every node and left the segment
        // accumulators set; the lists expect them zero
        MPM_CUDA(h, cudaMemsetAsync(h->seg_acc, 0, sizeof(float4) * 2 * h->total_nodes * h->K, st));
        MPM_CUDA(h, cudaMemsetAsync(h->blk_flag + 2 * h->n_blocks, 0, sizeof(int) * 2 * h->n_blocks, st));
        MPM_CUDA(h, cudaMemsetAsync(h->blk_count + 2, 0, sizeof(int) * 2, st));
        MPM_CUDA(h, cudaMemsetAsync(h->blk_wbox + 2 * h->n_wbox, 0, sizeof(int4) * 2 * h->n_wbox, st));
        h->seg_dirty = false;
    }
    if ((rc = run_pass(h, 1, st))) return rc;
    if (h->blocks && !h->grid_blocks) h->seg_dirty = h->res_dirty = true;
    if (g_phi && (rc = dcopy(h, g_phi, h->gphi_d, sizeof(float) * h->Nd, st))) return rc;
    if (g_mag && (rc = dcopy(h, g_mag, h->gmag_d, sizeof(float) * d * h->Nd, st))) return rc;
    if (g_field && (rc = dcopy(h, g_field, h->gfield_d, sizeof(float) * h->n_inst * h->T * d, st)))
        return rc;
    int rc2 = finish(h, 1, st);
    if (rc2 == MPM_OK) h->backward_done = true;
    return rc2;
}

// ---------------------------------------------------------------------------
// autotuner: time candidate launch configurations, keep the fastest
// ---------------------------------------------------------------------------
struct TuneChoice {
    int block, fuse, adj, agg;  // agg: MPM_OPT_SCATTER_2D (2D)
    double ms;
};

std::string tune_signature(const mpm_handle* h) {
    // problem shape the choice depends on; particle counts bucketed by powers of 2
    long long nb = 1;
    while (nb < h->N) nb <<= 1;
    return "d" + std::to_string(h->dim) + "_res" + std::to_string(h->res) + "_n" +
           std::to_string(nb) + "_inst" + std::to_string(h->n_inst) + "_K" + std::to_string(h->K);
}

// cache file: one JSON object, one entry per line
bool cache_lookup(const char* path, const std::string& sig, TuneChoice* out) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    const std::string key = "\"" + sig + "\": ";
    while (std::fgets(line, sizeof line, f)) {
        const char* p = std::strstr(line, key.c_str());
        if (!p) continue;
        TuneChoice c{};
        if (std::sscanf(p + key.size(),
                        "{\"block\": %d, \"fuse\": %d, \"adj\": %d, \"agg\": %d, \"ms\": %lf}",
                        &c.block, &c.fuse, &c.adj, &c.agg, &c.ms) == 5 &&
            c.adj >= 2 && c.adj <= 4 && (c.agg == 0 || c.agg == 1)) {
            *out = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& sig, const TuneChoice& c) {
    if (!path) return;
    std::vector<std::string> lines;
    if (FILE* f = std::fopen(path, "r")) {
        char line[512];
        const std::string key = "\"" + sig + "\": ";
        while (std::fgets(line, sizeof line, f)) {
            std::string l(line);
            if (l.find("\": {\"block\"") == std::string::npos || l.find(key) != std::string::npos) continue;
            while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
            lines.push_back(l);
        }
        std::fclose(f);
    }
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "  \"%s\": {\"block\": %d, \"fuse\": %d, \"adj\": %d, \"agg\": %d, \"ms\": %.4f}",
                  sig.c_str(), c.block, c.fuse, c.adj, c.agg, c.ms);
    lines.push_back(buf);
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    for (size_t i = 0; i < lines.size(); ++i) std::fprintf(f, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

void apply_choice(mpm_handle* h, const TuneChoice& c) {
    drop_graphs(h);
    h->block = c.block;
    h->fuse_fwd = (c.fuse & 1) != 0;
    h->fuse_adj = (c.fuse & 2) != 0;
    h->P.adj_blocks = c.adj;
    h->P.agg2 = c.agg;
}

int autotune_impl(mpm_handle* h, const char* cache_path, int sample_substeps, cudaStream_t st,
                  TuneChoice* best_out) {
    if (!h->forward_done) return fail(h, MPM_ERR_STATE, "mpm_autotune needs a successful mpm_forward first");
    const std::string sig = tune_signature(h);
    TuneChoice best{};
    if (cache_lookup(cache_path, sig, &best)) {
        apply_choice(h, best);
        *best_out = best;
        return MPM_OK;
    }
    const int sample = sample_substeps > 0 ? sample_substeps : 2 * h->K;
    const bool saved_graphs = h->graphs;
    const int saved_timing = h->timing_stride;
    h->timing_stride = 0;
    cudaEvent_t e0, e1;
    MPM_CUDA(h, cudaEventCreate(&e0));
    MPM_CUDA(h, cudaEventCreate(&e1));
    best.ms = 1e30;
    int rc = MPM_OK;
    for (int block : {64, 128, 256}) {
        for (int fuse : {0, 1}) {
            // register budgets: 2 and 3 blocks per SM, and 4 in 2D; in 2D
            // also the P2G scatter with and without aggregation
            const int n_adj = h->dim == 2 ? 3 : 2;
            for (int cand = 0; cand < n_adj * (h->dim == 2 ? 2 : 1); ++cand) {
                const int adj = 2 + cand % n_adj, agg = cand / n_adj;
                TuneChoice c{block, fuse, adj, agg, 0.0};
                apply_choice(h, c);
                h->tune_T = sample;
                // first run captures the graphs; then time the best of 3
                for (int it = 0; it < 4 && rc == MPM_OK; ++it) {
                    if (it > 0) rc = cudaEventRecord(e0, st) == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
                    if (rc == MPM_OK) rc = run_pass(h, 0, st);
                    if (rc == MPM_OK) rc = run_pass(h, 1, st);
                    if (it > 0 && rc == MPM_OK) rc = cudaEventRecord(e1, st) == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
                    if (rc == MPM_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
                    h->ran_graph[0] = h->ran_graph[1] = false;
                    if (it > 0 && rc == MPM_OK) {
                        float ms = 0.0f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        c.ms = it == 1 ? ms : std::min(c.ms, (double)ms);
                    }
                }
                h->tune_T = 0;
                if (rc != MPM_OK) break;
                if (c.ms < best.ms) best = c;
            }
            if (rc != MPM_OK) break;
        }
        if (rc != MPM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->blocks && !h->grid_blocks) h->seg_dirty = true;
    h->tune_T = 0;
    h->timing_stride = saved_timing;
    h->graphs = saved_graphs;
    if (rc != MPM_OK) {
        drop_graphs(h);
        if (h->err.empty()) h->err = "autotune run failed";
        return rc;
    }
    apply_choice(h, best);
    cache_store(cache_path, sig, best);
    *best_out = best;
    // the tuning runs overwrote the forward state; a new forward is needed
    h->forward_done = false;
    return MPM_OK;
}

}  // namespace

namespace mpm {
int check_config(const mpm_config* cfg, std::string* why) { return validate(cfg, *why); }
}  // namespace mpm

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int mpm_create(const mpm_config* cfg, mpm_handle** out) {
    if (!out) return MPM_ERR_ARG;
    *out = nullptr;
    std::string why;
    int rc = validate(cfg, why);
    if (rc != MPM_OK) {
        std::fprintf(stderr, "mpm_create: %s\n", why.c_str());
        return rc;
    }
    mpm_handle* h = new (std::nothrow) mpm_handle();
    if (!h) return MPM_ERR_OOM;
    try {
        rc = create_impl(cfg, h);
    } catch (...) {
        rc = MPM_ERR_OOM;
    }
    if (rc != MPM_OK) {
        std::fprintf(stderr, "mpm_create: %s\n", h->err.c_str());
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return MPM_OK;
}

int mpm_destroy(mpm_handle* h) {
    if (!h) return MPM_ERR_ARG;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return MPM_OK;
}

const char* mpm_last_error(const mpm_handle* h) { return h ? h->err.c_str() : "null handle"; }

int mpm_forward(mpm_handle* h, const float* x0, const float* v0, const float* phi_bar,
                const float* mag, const float* field, const float* target, float* x_out,
                float* loss_out, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    try {
        return forward_impl(h, x0, v0, phi_bar, mag, field, target, x_out, loss_out,
                            (cudaStream_t)cuda_stream);
    } catch (...) {
        return fail(h, MPM_ERR_CUDA, "unexpected exception in mpm_forward");
    }
}

int mpm_backward(mpm_handle* h, const float* dloss, float* g_phi, float* g_mag, float* g_field,
                 void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    try {
        return backward_impl(h, dloss, g_phi, g_mag, g_field, (cudaStream_t)cuda_stream);
    } catch (...) {
        return fail(h, MPM_ERR_CUDA, "unexpected exception in mpm_backward");
    }
}

int mpm_forward_host(mpm_handle* h, const float* x0, const float* v0, const float* phi_bar,
                     const float* mag, const float* field, const float* target, float* x_out,
                     float* loss_out, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int d = h->dim;
    if (!loss_out || !field || (h->N > 0 && (!x0 || !phi_bar || !mag)))
        return fail(h, MPM_ERR_ARG, "missing input");
    if (h->N > 0 && h->P.loss_kind == 0 && !target) return fail(h, MPM_ERR_ARG, "target is required for loss_kind 0");
    auto h2d = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    MPM_CUDA(h, h2d(h->st_x0, x0, sizeof(float) * d * h->N));
    if (v0) MPM_CUDA(h, h2d(h->st_v0, v0, sizeof(float) * d * h->N));
    MPM_CUDA(h, h2d(h->phi_d, phi_bar, sizeof(float) * h->Nd));
    MPM_CUDA(h, h2d(h->mag_d, mag, sizeof(float) * d * h->Nd));
    MPM_CUDA(h, h2d(h->field, field, sizeof(float) * h->n_inst * h->T * d));
    if (target) MPM_CUDA(h, h2d(h->target, target, sizeof(float) * d * h->N));
    int rc;
    try {
        rc = forward_impl(h, h->st_x0, v0 ? h->st_v0 : nullptr, h->phi_d, h->mag_d, h->field,
                          target ? h->target : nullptr, x_out ? h->st_xout : nullptr, h->st_loss, st);
    } catch (...) {
        return fail(h, MPM_ERR_CUDA, "unexpected exception in mpm_forward_host");
    }
    if (rc != MPM_OK) return rc;
    MPM_CUDA(h, cudaMemcpyAsync(loss_out, h->st_loss, sizeof(float) * h->n_inst, cudaMemcpyDeviceToHost, st));
    if (x_out && h->N > 0)
        MPM_CUDA(h, cudaMemcpyAsync(x_out, h->st_xout, sizeof(float) * d * h->N, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    return MPM_OK;
}

int mpm_backward_host(mpm_handle* h, const float* dloss, float* g_phi, float* g_mag,
                      float* g_field, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (!dloss) return fail(h, MPM_ERR_ARG, "dloss is NULL");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int d = h->dim;
    MPM_CUDA(h, cudaMemcpyAsync(h->dloss, dloss, sizeof(float) * h->n_inst, cudaMemcpyHostToDevice, st));
    int rc;
    try {
        rc = backward_impl(h, h->dloss, nullptr, nullptr, nullptr, st);
    } catch (...) {
        return fail(h, MPM_ERR_CUDA, "unexpected exception in mpm_backward_host");
    }
    if (rc != MPM_OK) return rc;
    if (g_phi && h->Nd)
        MPM_CUDA(h, cudaMemcpyAsync(g_phi, h->gphi_d, sizeof(float) * h->Nd, cudaMemcpyDeviceToHost, st));
    if (g_mag && h->Nd)
        MPM_CUDA(h, cudaMemcpyAsync(g_mag, h->gmag_d, sizeof(float) * d * h->Nd, cudaMemcpyDeviceToHost, st));
    if (g_field)
        MPM_CUDA(h, cudaMemcpyAsync(g_field, h->gfield_d, sizeof(float) * h->n_inst * h->T * d,
                                    cudaMemcpyDeviceToHost, st));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    return MPM_OK;
}

int mpm_read_state(mpm_handle* h, float* x, float* v, float* C, float* F, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (!h->forward_done) return fail(h, MPM_ERR_STATE, "no forward result to read");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int d = h->dim;
    const Params& P = h->P;
    if (x) MPM_CUDA(h, mpm::launch_to_input_order(d, P, h->cur, 0, h->id_cur, x, st, 0, h->x0_fwd));
    if (v) MPM_CUDA(h, mpm::launch_to_input_order(d, P, h->cur, d, h->id_cur, v, st));
    if (C) MPM_CUDA(h, mpm::launch_to_input_order(d * d, P, h->cur, 2 * d, h->id_cur, C, st));
    if (F) MPM_CUDA(h, mpm::launch_to_input_order(d * d, P, h->cur, 2 * d + d * d, h->id_cur, F, st, d));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    return MPM_OK;
}

int mpm_read_state_strain(mpm_handle* h, float* u, float* v, float* C, float* E, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (!h->forward_done) return fail(h, MPM_ERR_STATE, "no forward result to read");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int d = h->dim;
    const Params& P = h->P;
    if (u) MPM_CUDA(h, mpm::launch_to_input_order(d, P, h->cur, 0, h->id_cur, u, st));
    if (v) MPM_CUDA(h, mpm::launch_to_input_order(d, P, h->cur, d, h->id_cur, v, st));
    if (C) MPM_CUDA(h, mpm::launch_to_input_order(d * d, P, h->cur, 2 * d, h->id_cur, C, st));
    if (E) MPM_CUDA(h, mpm::launch_to_input_order(d * d, P, h->cur, 2 * d + d * d, h->id_cur, E, st));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    return MPM_OK;
}

int mpm_sort_particles(mpm_handle* h, const float* x, int* keys, int* perm, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (h->N > 0 && (!x || !keys || !perm)) return fail(h, MPM_ERR_ARG, "x, keys and perm are required");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    MPM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
    MPM_CUDA(h, mpm::launch_sort(h->dim, h->P, x, h->N, h->d_inst_off, h->sb, perm, h->d_err, st));
    if (h->N > 0)
        MPM_CUDA(h, cudaMemcpyAsync(keys, h->sb.keys, sizeof(int) * h->N, cudaMemcpyDeviceToDevice, st));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    return MPM_OK;
}

// Copy the host mirror of the boxes / field gradient to the device and point
// the parameter block at it (or at nothing).  Captured graphs hold the old
// parameter block and are dropped; a backward needs a new forward.
static int upload_extras(mpm_handle* h, cudaStream_t st) {
    MPM_CUDA(h, cudaMemcpyAsync(h->d_ext, &h->ext_host, sizeof(mpm::Extras), cudaMemcpyHostToDevice, st));
    MPM_CUDA(h, cudaStreamSynchronize(st));
    drop_graphs(h);
    h->P.ext = (h->ext_host.n > 0 || h->ext_host.fgrad) ? h->d_ext : nullptr;
    h->forward_done = false;
    h->backward_done = false;
    return MPM_OK;
}

int mpm_set_boundaries(mpm_handle* h, int n, const mpm_boundary* boxes, const float* motion, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (n < 0 || n > MPM_MAX_BOUNDARIES) return fail(h, MPM_ERR_ARG, "n must be in [0, MPM_MAX_BOUNDARIES]");
    if (n > 0 && !boxes) return fail(h, MPM_ERR_ARG, "boxes is NULL");
    mpm::Extras hs = h->ext_host;
    hs.n = n;
    for (int b = 0; b < n; ++b) {
        const mpm_boundary& B = boxes[b];
        if (B.kind < MPM_BOUNDARY_COULOMB || B.kind > MPM_BOUNDARY_ATTACHED)
            return fail(h, MPM_ERR_ARG, "unknown boundary kind");
        if (!(B.mu >= 0.0f) || !std::isfinite(B.mu)) return fail(h, MPM_ERR_ARG, "mu must be finite and >= 0");
        for (int a = 0; a < h->dim; ++a)
            if (!(B.lo[a] <= B.hi[a]) || !std::isfinite(B.lo[a]) || !std::isfinite(B.hi[a]))
                return fail(h, MPM_ERR_ARG, "a box needs finite lo <= hi on every axis");
        hs.box[b].kind = B.kind;
        hs.box[b].mu = B.mu;
        for (int a = 0; a < 3; ++a) {
            hs.box[b].lo[a] = B.lo[a];
            hs.box[b].hi[a] = B.hi[a];
        }
    }
    hs.motion = (n > 0 && motion) ? h->d_bmotion : nullptr;
    for (int b = n; b < mpm::kMaxBoundaries; ++b) hs.box[b] = mpm::Boundary{};
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (hs.motion)
        MPM_CUDA(h, cudaMemcpyAsync(h->d_bmotion, motion, sizeof(float) * (size_t)n * h->T * 2 * h->dim,
                                    cudaMemcpyDeviceToDevice, st));
    h->ext_host = hs;
    return upload_extras(h, st);
}

int mpm_set_field_gradient(mpm_handle* h, const float* grad, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t n = (size_t)h->n_inst * h->T * h->dim * h->dim;
    if (grad) MPM_CUDA(h, cudaMemcpyAsync(h->d_fgrad, grad, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    h->ext_host.fgrad = grad ? h->d_fgrad : nullptr;
    h->ext_host.gfgrad = grad ? h->d_gfgrad : nullptr;
    return upload_extras(h, st);
}

int mpm_field_gradient_grad(mpm_handle* h, float* g_grad, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (!g_grad) return fail(h, MPM_ERR_ARG, "g_grad is NULL");
    if (!h->ext_host.fgrad) return fail(h, MPM_ERR_STATE, "no field gradient is set");
    if (!h->backward_done) return fail(h, MPM_ERR_STATE, "mpm_field_gradient_grad needs a successful mpm_backward");
    const size_t n = (size_t)h->n_inst * h->T * h->dim * h->dim;
    MPM_CUDA(h, cudaMemcpyAsync(g_grad, h->d_gfgrad, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                (cudaStream_t)cuda_stream));
    return MPM_OK;
}

int mpm_set_option(mpm_handle* h, int key, long long value) {
    if (!h) return MPM_ERR_ARG;
    switch (key) {
        case MPM_OPT_TIMING:
            if (value < 0) return fail(h, MPM_ERR_ARG, "timing stride must be >= 0");
            if (h->timing_stride != (int)value) drop_graphs(h);
            h->timing_stride = (int)value;
            for (int c = 0; c < kNumClasses; ++c) h->class_launch[c] = 0;
            return MPM_OK;
        case MPM_OPT_BLOCK:
            if (value < 32 || value > 256 || value % 32) return fail(h, MPM_ERR_ARG, "block must be a multiple of 32 in [32, 256]");
            if (h->block != (int)value) drop_graphs(h);
            h->block = (int)value;
            return MPM_OK;
        case MPM_OPT_FUSE_GRID:
            if (value < 0 || value > 3) return fail(h, MPM_ERR_ARG, "fuse_grid must be in [0, 3]");
            if (h->fuse_fwd != ((value & 1) != 0) || h->fuse_adj != ((value & 2) != 0)) drop_graphs(h);
            h->fuse_fwd = (value & 1) != 0;
            h->fuse_adj = (value & 2) != 0;
            return MPM_OK;
        case MPM_OPT_PERSISTENT:
            if (value != 0 && value != 1) return fail(h, MPM_ERR_ARG, "persistent must be 0 or 1");
            if (h->persistent != (value == 1)) {
                drop_graphs(h);
                // whether the forward pass filled the resident sets may change
                if (h->n_res > 0) h->forward_done = false;
            }
            h->persistent = value == 1;
            return MPM_OK;
        case MPM_OPT_SPIN_LIMIT:
            if (value < 1) return fail(h, MPM_ERR_ARG, "spin limit must be >= 1");
            if (h->spin_limit != value) drop_graphs(h);
            h->spin_limit = value;
            return MPM_OK;
        case MPM_OPT_GRID_BLOCKS:
            if (value != 0 && value != 1) return fail(h, MPM_ERR_ARG, "grid blocks must be 0 or 1");
            if (h->grid_blocks != (value == 1)) {
                drop_graphs(h);
                if (h->n_res > 0) h->forward_done = false;
            }
            h->grid_blocks = value == 1;
            return MPM_OK;
        case MPM_OPT_ADJOINT_BLOCKS:
            if (value < 2 || value > 4) return fail(h, MPM_ERR_ARG, "adjoint blocks must be 2, 3 or 4");
            if (h->P.adj_blocks != (int)value) drop_graphs(h);
            h->P.adj_blocks = (int)value;
            return MPM_OK;
        case MPM_OPT_RESIDENT_SEGMENTS:
            if (value < 0) return fail(h, MPM_ERR_ARG, "resident segments must be >= 0");
            return set_resident(h, (int)std::min<long long>(value, h->n_seg));
        case MPM_OPT_SEGMENT_BYTES:
            return fail(h, MPM_ERR_ARG, "segment bytes is read-only");
        case MPM_OPT_SCATTER_2D:
            if (value != 0 && value != 1) return fail(h, MPM_ERR_ARG, "scatter_2d must be 0 or 1");
            if (h->P.agg2 != (int)value) drop_graphs(h);
            h->P.agg2 = (int)value;
            return MPM_OK;
        case MPM_OPT_PDL:
            if (value != 0 && value != 1) return fail(h, MPM_ERR_ARG, "pdl must be 0 or 1");
            if (h->P.pdl != (int)value) drop_graphs(h);
            h->P.pdl = (int)value;
            return MPM_OK;
        case MPM_OPT_STREAMS:
            if (value != 1 && value != 2) return fail(h, MPM_ERR_ARG, "streams must be 1 or 2");
            if (h->two_streams != (value == 2)) drop_graphs(h);
            h->two_streams = value == 2;
            return MPM_OK;
        case MPM_OPT_GRAPHS:
            if (value != 0 && value != 1) return fail(h, MPM_ERR_ARG, "graphs must be 0 or 1");
            if (value == 0) drop_graphs(h);
            h->graphs = value == 1;
            return MPM_OK;
        default:
            return fail(h, MPM_ERR_ARG, "unknown option");
    }
}

int mpm_autotune(mpm_handle* h, const char* cache_path, int sample_substeps, void* cuda_stream) {
    if (!h) return MPM_ERR_ARG;
    if (sample_substeps < 0) return fail(h, MPM_ERR_ARG, "sample_substeps must be >= 0");
    try {
        TuneChoice c{};
        return autotune_impl(h, cache_path, sample_substeps, (cudaStream_t)cuda_stream, &c);
    } catch (...) {
        return fail(h, MPM_ERR_CUDA, "unexpected exception in mpm_autotune");
    }
}

int mpm_get_option(const mpm_handle* h, int key, long long* value) {
    if (!h || !value) return MPM_ERR_ARG;
    switch (key) {
        case MPM_OPT_TIMING: *value = h->timing_stride; return MPM_OK;
        case MPM_OPT_BLOCK: *value = h->block; return MPM_OK;
        case MPM_OPT_FUSE_GRID: *value = (h->fuse_fwd ? 1 : 0) | (h->fuse_adj ? 2 : 0); return MPM_OK;
        case MPM_OPT_GRAPHS: *value = h->graphs ? 1 : 0; return MPM_OK;
        case MPM_OPT_STREAMS: *value = h->two_streams ? 2 : 1; return MPM_OK;
        case MPM_OPT_PDL: *value = h->P.pdl; return MPM_OK;
        case MPM_OPT_ADJOINT_BLOCKS: *value = h->P.adj_blocks; return MPM_OK;
        case MPM_OPT_GRID_BLOCKS: *value = h->grid_blocks ? 1 : 0; return MPM_OK;
        case MPM_OPT_PERSISTENT: *value = h->persistent ? 1 : 0; return MPM_OK;
        case MPM_OPT_SPIN_LIMIT: *value = h->spin_limit; return MPM_OK;
        case MPM_OPT_SCATTER_2D: *value = h->P.agg2; return MPM_OK;
        case MPM_OPT_RESIDENT_SEGMENTS: *value = h->n_res; return MPM_OK;
        case MPM_OPT_SEGMENT_BYTES: *value = resident_set_bytes(h); return MPM_OK;
        default: return MPM_ERR_ARG;
    }
}

int mpm_get_stats(const mpm_handle* h, mpm_stats* out) {
    if (!h || !out) return MPM_ERR_ARG;
    out->launches = h->launches;
    for (int c = 0; c < 4; ++c) {
        out->timed_launches[c] = h->timed_launches[c];
        out->timed_ms[c] = h->timed_ms[c];
        out->timed_bytes[c] = h->timed_bytes[c];
        out->class_launches[c] = h->cls_issued[c];
    }
    out->device_bytes = h->device_bytes;
    return MPM_OK;
}

int mpm_reset_stats(mpm_handle* h) {
    if (!h) return MPM_ERR_ARG;
    h->launches = 0;
    for (int c = 0; c < 4; ++c) {
        h->timed_launches[c] = 0;
        h->timed_ms[c] = 0.0;
        h->timed_bytes[c] = 0.0;
        h->class_launch[c] = 0;
        h->cls_issued[c] = 0;
    }
    return MPM_OK;
}

}  // extern "C"
