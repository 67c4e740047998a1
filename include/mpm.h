/*
 * mpm.h -- C ABI of the GB300 differentiable magneto-elastic MPM library.
 *
 * The library advances a batch of independent MLS-MPM simulations of
 * hard-magnetic soft material (arxiv 2503.22767, Section 2) and computes the
 * reverse-mode gradients of a scalar objective with respect to the design
 * variables (Section 2.3, Section 3.1):
 *
 *   per substep n (Section 2.2):
 *     sort      particles by grid cell (a performance ordering; not in the paper)
 *     P2G       grid mass and momentum, Eq. 14-15, with the Piola stress of
 *               Eq. 7 interpolated by SIMP, Eq. 31-33
 *     grid op   Eq. 16-17 (damping, gravity) and Eq. 18 (walls, Coulomb floor)
 *     G2P       Eq. 19-22 (velocity, APIC affine matrix, position, F)
 *   objective   shape MSE (Eq. 38, summed over tasks by Eq. 35) or
 *               locomotion (Eq. 40)
 *
 * Conventions shared by every entry point
 *   - Every array argument is float32, contiguous, structure-of-arrays:
 *     a per-particle vector quantity is [d][N], component-major, with the
 *     particles of all instances concatenated in instance order.
 *   - "device" pointers must be CUDA device memory of the current device;
 *     "host" pointers are ordinary (preferably pinned) host memory.  The
 *     caller owns every buffer it passes; the library never frees them and
 *     keeps no reference after the call returns (inputs that the backward pass
 *     needs are copied into library-owned storage).
 *   - Work is enqueued on `cuda_stream` (a cudaStream_t; NULL = legacy
 *     default stream).  forward/backward synchronise that stream before
 *     returning, because the status includes device-side checks.
 *   - Every function returns an mpm_status; no C++ exception or abort
 *     crosses the ABI.  mpm_last_error() gives a text for the last failure.
 *   - One handle must not be used from two threads at once.
 */
#ifndef MPM_H
#define MPM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_handle mpm_handle;

typedef enum {
    MPM_OK = 0,
    MPM_ERR_ARG = -1,     /* invalid argument or configuration (host check) */
    MPM_ERR_CUDA = -2,    /* a CUDA runtime call failed */
    MPM_ERR_OOM = -3,     /* device allocation failed in mpm_create */
    MPM_ERR_STATE = -4,   /* backward without a preceding successful forward */
    MPM_ERR_NUMERIC = -5, /* J <= 0 or a non-finite value appeared on the device */
    MPM_ERR_DOMAIN = -6,  /* a particle's stencil left the grid */
    MPM_ERR_TIMEOUT = -7  /* a bounded device-side wait gave up */
} mpm_status;

/*
 * Problem description (copied by mpm_create; pointers need only live for the
 * duration of that call).
 *
 *   dim, grid_res     2 or 3; res nodes per axis, dx = 1/res, node i at i*dx.
 *   dt, n_steps       substep size and horizon N.
 *   n_instances, n_particles
 *                     independent simulations (1..65535) and their particle
 *                     counts (host array [n_instances]); each instance has its
 *                     own grid.
 *   n_designs, design_of_instance
 *                     topology phi and magnetisation B~_r are given per design;
 *                     instance i uses design design_of_instance[i] (host array,
 *                     NULL = identity).  Instances sharing a design must have
 *                     equal particle counts; their gradients are summed
 *                     (multi-task sharing, Eq. 35).
 *   E, nu, rho0, p_vol
 *                     Young's modulus, Poisson ratio (G = E/(2(1+nu)),
 *                     K = E/(3(1-2nu))), density and particle volume; the
 *                     particle mass is phi * rho0 * p_vol (Eq. 33).
 *   simp_eps, simp_q  SIMP interpolation (Eq. 31).
 *   damping_c, gravity
 *                     damping rate (1/s) and body acceleration (Eq. 17).
 *   bound, wall_mode, floor_mu
 *                     wall band width in nodes; wall_mode 0 = every wall
 *                     non-slip, 1 = Coulomb friction floor (axis 1, low side,
 *                     Eq. 18 with coefficient floor_mu) and non-slip elsewhere.
 *   loss_kind         0 = mean squared distance of final positions to the
 *                     target (Eq. 38), 1 = -sum_{n=1..N} vbar_x(n) dt with the
 *                     mass-averaged velocity (Eq. 40).
 *   checkpoint_every  K: the backward pass recomputes K-substep segments from
 *                     checkpoints, keeping every substep of the segment it
 *                     works on; 0 = one segment over the whole horizon.  With
 *                     MPM_OPT_RESIDENT_SEGMENTS the forward pass keeps the
 *                     last segments instead.
 */
typedef struct {
    int dim;
    int grid_res;
    double dt;
    int n_steps;
    int n_instances;
    const int* n_particles;
    int n_designs;
    const int* design_of_instance;
    double E, nu, rho0, p_vol;
    double simp_eps;
    int simp_q;
    double damping_c;
    double gravity[3];
    int bound;
    int wall_mode;
    double floor_mu;
    int loss_kind;
    int checkpoint_every;
} mpm_config;

/*
 * Create a handle and allocate, on the current device, every buffer the
 * forward and backward passes need (grid, sort scratch, checkpoints, segment
 * store, saved inputs).  No later call allocates device memory, except
 * mpm_set_option(MPM_OPT_RESIDENT_SEGMENTS), which reserves the resident
 * segment sets.
 * Errors: MPM_ERR_ARG (bad config), MPM_ERR_OOM, MPM_ERR_CUDA.  On error
 * *out is set to NULL and nothing stays allocated.
 */
int mpm_create(const mpm_config* cfg, mpm_handle** out);

/* Release everything the handle owns (synchronises the device first). */
int mpm_destroy(mpm_handle* h);

/* Text of the last error on this handle ("" if none).  Owned by the handle. */
const char* mpm_last_error(const mpm_handle* h);

/*
 * Run the N substeps of every instance from rest (C = 0, F = I) and
 * evaluate the objective (Section 2.2, Eq. 14-22; Eq. 38 or Eq. 40).
 *   x0      device [d][N]      initial positions (N = sum of n_particles)
 *   v0      device [d][N]      initial velocities, or NULL for zero
 *   phi_bar device [Nd]        projected topology variable per particle of
 *                              each design (Nd = sum over designs)
 *   mag     device [d][Nd]     residual flux density B~_r in Tesla (Eq. 26)
 *   field   device [n_instances][n_steps][d]
 *                              applied flux density B_applied in Tesla, held
 *                              constant over substep n (t_n = n dt)
 *   target  device [d][N]      target positions (loss_kind 0; NULL otherwise)
 *   x_out   device [d][N]      final positions in input order, or NULL
 *   loss_out device [n_instances] objective of each instance
 * Errors: MPM_ERR_ARG, MPM_ERR_CUDA, MPM_ERR_NUMERIC (inverted or non-finite
 * deformation), MPM_ERR_DOMAIN (a particle's stencil left the grid; the
 * kernels clamp indices so memory stays in bounds).  The inputs needed by
 * mpm_backward are copied; the caller may reuse its buffers on return.
 */
int mpm_forward(mpm_handle* h, const float* x0, const float* v0, const float* phi_bar,
                const float* mag, const float* field, const float* target, float* x_out,
                float* loss_out, void* cuda_stream);

/*
 * Reverse-mode gradients of sum_i dloss[i] * loss_i for the last successful
 * mpm_forward on this handle, by checkpointed recomputation (Section 2.3).
 *   dloss   device [n_instances] upstream gradient
 *   g_phi   device [Nd]        dL/dphi_bar (overwritten)
 *   g_mag   device [d][Nd]     dL/dB~_r   (overwritten)
 *   g_field device [n_instances][n_steps][d] dL/dB_applied (overwritten)
 * Any output may be NULL to skip it.  Errors: MPM_ERR_STATE (no forward),
 * MPM_ERR_ARG, MPM_ERR_CUDA, MPM_ERR_NUMERIC, MPM_ERR_DOMAIN.
 */
int mpm_backward(mpm_handle* h, const float* dloss, float* g_phi, float* g_mag, float* g_field,
                 void* cuda_stream);

/*
 * Same as mpm_forward / mpm_backward but every array argument is a HOST
 * pointer: the library copies inputs to the device and results back inside
 * the call (cudaMemcpyAsync on cuda_stream into buffers allocated by
 * mpm_create).  Use pinned memory for full copy bandwidth.
 */
int mpm_forward_host(mpm_handle* h, const float* x0, const float* v0, const float* phi_bar,
                     const float* mag, const float* field, const float* target, float* x_out,
                     float* loss_out, void* cuda_stream);
int mpm_backward_host(mpm_handle* h, const float* dloss, float* g_phi, float* g_mag,
                      float* g_field, void* cuda_stream);

/*
 * Final particle state of the last forward, in input order (device
 * pointers, each may be NULL): x, v [d][N]; C, F [d][d][N] (row-major
 * components, component (a,b) at offset (a*d+b)*N).
 */
int mpm_read_state(mpm_handle* h, float* x, float* v, float* C, float* F, void* cuda_stream);

/*
 * The same state in the variables the library integrates (Eq. 21-22 written
 * for them): the displacement u = x - x0 and the strain E = F - I, float32,
 * input order, device pointers (each may be NULL): u, v [d][N]; C, E
 * [d][d][N].  Small displacements and strains keep their full float32
 * precision here, where x and F above are rounded next to x0 and I.
 * Errors: MPM_ERR_STATE (no forward yet), MPM_ERR_CUDA.
 */
int mpm_read_state_strain(mpm_handle* h, float* u, float* v, float* C, float* E, void* cuda_stream);

/*
 * The particle ordering used by the substep, exposed for checking: for
 * device positions x [d][N] (N = sum of n_particles, instances concatenated)
 * writes the cell key of every particle and the stable order by key
 * (perm[new] = old; ties keep input order).  Key definition: per axis
 * base = floor(fl(fl(x * res) - 0.5)) in float32 round-to-nearest, clamped
 * to [0, res-3]; blocks of edge 8 (2D) or 4 (3D) cells; key = instance *
 * (blocks * cells per block) + block index * cells per block + cell index in
 * the block, blocks and cells row-major with the last axis fastest.
 * Not in the paper: it is the locality order of the GPU path.
 *   keys, perm: device int32 [N].
 */
int mpm_sort_particles(mpm_handle* h, const float* x, int* keys, int* perm, void* cuda_stream);

/* Options (mpm_set_option keys). */
enum {
    MPM_OPT_TIMING = 1, /* k > 0: time every k-th launch of each kernel class with CUDA
                           events (on the call's stream); 0 (default): off */
    MPM_OPT_BLOCK = 2,  /* threads per block of the particle kernels: a multiple of 32
                           in [32, 256] (default 128) */
    MPM_OPT_FUSE_GRID = 3, /* bit 0: the forward particle kernels apply the grid operation
                              (Eq. 16-18) per stencil node (one kernel per substep);
                              bit 1: the adjoint particle kernels apply its reverse per
                              stencil node; a clear bit keeps the separate grid kernel.
                              Default 0 (both separate, as the autotuner picks on every
                              workload measured) */
    MPM_OPT_GRAPHS = 4, /* 1 (default): each pass is captured once as a CUDA graph on an
                           internal stream and replayed on cuda_stream; 0: direct launches */
    MPM_OPT_STREAMS = 6, /* 2 (default): the backward pass recomputes checkpoint segment s-1
                            on a second stream while the adjoint of segment s runs (two
                            sets of segment buffers); 1: one stream */
    MPM_OPT_PDL = 7,    /* 1 (default): per-substep kernels use programmatic dependent
                           launch, so a kernel's CTAs are scheduled while its predecessor
                           drains; 0: plain stream order */
    MPM_OPT_ADJOINT_BLOCKS = 8, /* register budget of the fused adjoint particle kernel, as
                           resident 256-thread blocks per SM: 2 (default in 2D, <= 128
                           registers), 3 (default in 3D, <= 80 registers: more warps to hide
                           gather latency, at the cost of spills) or 4 (<= 64 registers; 2D
                           only, 3D takes it as 3) */
    MPM_OPT_GRID_BLOCKS = 10, /* 3D: 1 (default): the P2G kernels list the blocks of 4x4x4
                           nodes their stencils touch, and the grid operation and its
                           reverse run over the listed blocks only; 0: over every node.
                           No effect in 2D. */
    MPM_OPT_PERSISTENT = 11, /* 1: each checkpoint segment of each pass (forward, recomputation,
                           adjoint) runs as one persistent cooperative launch whose CTAs walk
                           the substeps, with grid-wide barriers between the grid and the
                           particle phases, instead of two dependent launches per substep.
                           Runs the grid operation separately (MPM_OPT_FUSE_GRID is ignored)
                           and the backward pass on one stream.  Not with solid boxes or a
                           field gradient, nor in 3D without MPM_OPT_GRID_BLOCKS: those keep
                           the chained launches.  0 (default): chained launches */
    MPM_OPT_SPIN_LIMIT = 12, /* polls (>= 1) a persistent kernel's barrier wait makes before it
                           gives up, sets the timeout flag and returns: the call then fails
                           with MPM_ERR_TIMEOUT and the handle stays usable (default 2^22) */
    MPM_OPT_SCATTER_2D = 13, /* 2D P2G of the fused forward particle kernel (Eq. 14-15): 1: the
                           lanes of a warp that share a base node sum their node values in
                           shared memory and issue one atomic per node (as 3D always does);
                           0 (default): one float4 atomic per particle and node.  Without
                           solid boxes or a field gradient only; no effect in 3D. */
    MPM_OPT_RESIDENT_SEGMENTS = 14, /* r >= 0 (capped at the number of checkpoint segments): the
                           forward pass stores every state and grid of the last r segments, as
                           the recomputation of the checkpointed adjoint would, and the
                           backward pass runs their adjoint without recomputing them.  Setting
                           it reserves r segment sets of device memory (MPM_OPT_SEGMENT_BYTES
                           each; MPM_ERR_OOM if that fails, leaving none) and drops the last
                           forward: call mpm_forward again before mpm_backward.  0 (default)
                           releases them.  Not used by the persistent passes or while
                           autotuning; while any are reserved, changing MPM_OPT_PERSISTENT or
                           MPM_OPT_GRID_BLOCKS also drops the last forward. */
    MPM_OPT_SEGMENT_BYTES = 15 /* read only: device bytes of one resident segment set (K + 1
                           states, K accumulator and K velocity grids, the segment's design
                           and initial positions, and in 3D a node-block list) */
};
/* Errors: MPM_ERR_ARG for an unknown key or a value out of range; MPM_ERR_OOM (resident
   segments). */
int mpm_set_option(mpm_handle* h, int key, long long value);
/* Current value of an option.  Errors: MPM_ERR_ARG. */
int mpm_get_option(const mpm_handle* h, int key, long long* value);

/*
 * Solid boundaries beyond the walls (Eq. 18 in general form): obstacles, and
 * clamps or holders attached to the material, static or moving.  Each box is
 * axis-aligned, given at t = 0 in domain units (lo <= hi on every used axis).
 * A grid node inside a box lies on its nearest face, whose outward normal is
 * n_b.  The box may move: motion gives per box and substep its offset from
 * the t = 0 position and its velocity v_b.  Per kind:
 *   MPM_BOUNDARY_COULOMB   when (v - v_b) . n_b < 0, the normal part of v
 *                          becomes v_b's and the tangential part of v - v_b
 *                          shrinks by mu |(v - v_b) . n_b|, to zero at most;
 *   MPM_BOUNDARY_NONSLIP   when (v - v_b) . n_b < 0, v = v_b (mu -> infinity);
 *   MPM_BOUNDARY_ATTACHED  v = v_b always (material attached to the box).
 * Boxes act after the walls, in the given order.  The reverse mode replays
 * them.  Components they overwrite pass no gradient.
 */
#define MPM_MAX_BOUNDARIES 8
enum { MPM_BOUNDARY_COULOMB = 0, MPM_BOUNDARY_NONSLIP = 1, MPM_BOUNDARY_ATTACHED = 2 };
typedef struct {
    int kind;     /* MPM_BOUNDARY_* */
    float mu;     /* friction coefficient (MPM_BOUNDARY_COULOMB) */
    float lo[3];  /* box corners at t = 0 (entries past dim are ignored) */
    float hi[3];
} mpm_boundary;

/*
 * Replace the solid boxes with boxes[0 .. n) (host array, read during the
 * call).  n = 0 removes them.  motion is a device array [n][n_steps][2][dim]
 * (offset, then v_b, at t_n = n dt), or NULL for static boxes (offset and
 * v_b zero).  It is copied into storage that mpm_create allocated.  The call
 * synchronises cuda_stream.  A following mpm_backward needs a new
 * mpm_forward first.
 * Errors: MPM_ERR_ARG (n outside [0, MPM_MAX_BOUNDARIES], unknown kind,
 * negative or non-finite mu, lo > hi), MPM_ERR_CUDA.
 */
int mpm_set_boundaries(mpm_handle* h, int n, const mpm_boundary* boxes, const float* motion, void* cuda_stream);

/*
 * Non-uniform applied field.  The paper assumes a uniform field and notes that
 * non-uniform fields (e.g. from permanent magnets) fit the same framework
 * (Section 5).  Here the field is linear about the domain centre x_c:
 *   B(x, t_n) = field[inst][n] + G[inst][n] (x - x_c),
 * with G = dB_i/dx_j.  Eq. 7 / 31 then use B at the particle, and the
 * SIMP-scaled energy of Eq. 32 depends on position.  Its negative gradient is
 * a body force on every particle,
 *   f_p = (phi_bar_p^q V_p / mu0) G^T (F_p B~_r,p),
 * added to the particle's momentum in P2G (Eq. 15).  The reverse mode gives
 * dL/dG besides the other gradients.
 *
 * mpm_set_field_gradient copies grad (device, [n_instances][n_steps][dim][dim],
 * row-major per substep) into storage from mpm_create, or removes it (NULL).
 * It synchronises cuda_stream, and a following mpm_backward needs a new
 * mpm_forward.  mpm_substep_noalloc stays uniform.
 * mpm_field_gradient_grad copies dL/dG (same layout) after mpm_backward.
 * Errors: MPM_ERR_ARG, MPM_ERR_STATE (no gradient set, or no backward yet),
 * MPM_ERR_CUDA.
 */
int mpm_set_field_gradient(mpm_handle* h, const float* grad, void* cuda_stream);
int mpm_field_gradient_grad(mpm_handle* h, float* g_grad, void* cuda_stream);

/*
 * Autotuner (not in the paper; a launch-configuration search of this
 * library).  Times forward + backward passes over the first sample_substeps
 * substeps (0 = two checkpoint segments) of the inputs staged by the last
 * mpm_forward, for every combination of block size {64, 128, 256}, grid
 * fusion {0, 1}, adjoint register budget {2, 3, and 4 in 2D} and, in 2D, the
 * P2G scatter {per-lane, aggregated} (MPM_OPT_SCATTER_2D), and keeps the
 * fastest.  With a non-NULL cache_path, results are read from and written to that JSON file,
 * keyed by dim, grid_res, particle count (rounded up to a power of 2),
 * instances and checkpoint interval; a cache hit applies the stored choice
 * without timing.  The tuning runs overwrite the forward result: call
 * mpm_forward again before mpm_backward.  Errors: MPM_ERR_STATE (no forward),
 * MPM_ERR_ARG, MPM_ERR_CUDA.
 */
int mpm_autotune(mpm_handle* h, const char* cache_path, int sample_substeps, void* cuda_stream);

/*
 * Counters since creation or the last reset: kernel launches issued by the
 * library (a replayed graph counts every kernel it holds), the launches of
 * each kernel class, and, with MPM_OPT_TIMING on, the number of timed
 * launches and total milliseconds of each class, plus the algorithmic bytes
 * those launches moved.  Kernel classes (array index): 0 = forward particle
 * kernel (G2P + P2G), 1 = adjoint particle kernel (P2G^T + G2P^T), 2 = grid
 * operation, 3 = grid adjoint.
 */
typedef struct {
    long long launches;
    long long timed_launches[4];
    double timed_ms[4];
    double timed_bytes[4];
    long long device_bytes;
    long long class_launches[4];
} mpm_stats;
int mpm_get_stats(const mpm_handle* h, mpm_stats* out);
int mpm_reset_stats(mpm_handle* h);

/*
 * One substep of ONE instance that allocates no device memory.
 *
 * This entry point has no counterpart in the paper: it is an interface for
 * callers that must not call cudaMalloc.  Examples are a host framework whose
 * pool allocator owns the whole device-memory budget, and a latency-critical
 * loop where an allocation could block or fail.  Instead of a handle it keeps
 * its grid scratch in a fixed array compiled into the library: every GPU on
 * which it is called holds MPM_NOALLOC_MAX_NODES x 2 float4 (8 MiB) of it
 * until the process exits.  The caller passes all inputs and outputs.
 *
 * It runs P2G (Eq. 14-15), the grid operation (Eq. 16-18) and G2P
 * (Eq. 19-22) for substep `substep` of the configuration `cfg`:
 *   cfg        n_instances must be 1; grid_res^dim <= MPM_NOALLOC_MAX_NODES
 *              (512^2 in 2D, 64^3 in 3D); n_steps sizes `field`; loss_kind,
 *              checkpoint_every and the design fields are not used
 *   substep    index into field, 0 <= substep < n_steps
 *   state_in   device [2d + 2d^2][N] float32 SoA: x[d], v[d], C[d][d],
 *              E[d][d] with E = F - I (F = I and C = 0 at rest)
 *   phi_bar    device [N]; mag device [d][N] (B~_r, Tesla)
 *   field      device [n_steps][d] (B_applied, Tesla)
 *   state_out  device [2d + 2d^2][N], same layout; may be state_in itself
 * N = 0 is allowed (nothing moves).  The particles are not cell-sorted
 * here: the results do not depend on their order, but the P2G scatter merges
 * the atomics of particles that share a cell only when they are adjacent, so
 * throughput is best with particles passed in cell order.
 * Blocks until the substep finishes on cuda_stream; because it reads the
 * device status back, a call on a stream that is capturing is refused with
 * MPM_ERR_ARG before any work is enqueued.  Errors: MPM_ERR_ARG (bad config,
 * sizes beyond the scratch maximum, missing pointers, a capturing stream),
 * MPM_ERR_OOM or MPM_ERR_CUDA (the scratch could not be loaded; a CUDA call
 * failed), MPM_ERR_DOMAIN, MPM_ERR_NUMERIC; mpm_noalloc_last_error() gives
 * the reason.
 * The first call on a device (in each CUDA context) loads the library's
 * module there, which reserves the scratch array, and looks up its address
 * with cudaGetSymbolAddress; make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents; each
 * call clears what must start at zero, but calls that overlap on the GPU
 * (other streams, threads or processes on the same device) race on it.
 */
#define MPM_NOALLOC_MAX_NODES 262144
int mpm_substep_noalloc(const mpm_config* cfg, int substep, const float* state_in,
                        const float* phi_bar, const float* mag, const float* field,
                        float* state_out, void* cuda_stream);
/* Text of the last failure of mpm_substep_noalloc on the calling thread ("" if
 * its last call succeeded).  Owned by the library; valid until the thread's
 * next call. */
const char* mpm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MPM_H */
