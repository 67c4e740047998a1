/*
 * C ABI of the design representation and optimiser step of the magneto-elastic
 * co-design loop (arxiv 2503.22767, Sections 3.1-3.2).
 *
 * The maps turn the optimiser's variables into the inputs of mpm_forward:
 *   topology   phi [N] --density filter (Eq. 23-24)--> phi~ --Heaviside
 *              (Eq. 25, sharpness beta)--> phi_bar [N];
 *   material   Br [n_m], zeta [dim][n_m] --Eq. 26-28--> B~_r [dim][N],
 *              B~_r,p = Br_max * Br_m(p) * zeta_m(p) / sqrt(|zeta_m(p)|^2 + delta);
 *   stimulus   Ba, f [n_tasks], eta [n_tasks][dim] --Eq. 29-30--> field
 *              [n_tasks][n_steps][dim], B(t_n) = B_max Ba sin(2 pi fbar t_n)
 *              eta / sqrt(|eta|^2 + delta), fbar = (f_max - f_min) f + f_min,
 *              t_n = n dt.
 * mpm_design_backward is the reverse of all three.  mpm_adam_step is one Adam
 * step (Kingma & Ba, 2015) followed by clipping to the box of Eq. 34c-d.
 *
 * Conventions are those of mpm.h.  Array arguments are caller-owned device
 * pointers, float32, with the component-major layouts given above.  Calls are
 * asynchronous on cuda_stream, and the returned status covers the host-side
 * checks and the launches.  The handle owns only the scratch it allocates in
 * mpm_design_create.  It is not thread-safe; use one handle per stream.
 */
#ifndef MPM_DESIGN_H
#define MPM_DESIGN_H

#include "mpm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_design mpm_design;

typedef struct {
    int dim;              /* 2 or 3 */
    int n_particles;      /* N: particles of the design (Eq. 23-28 act per particle) */
    int n_regions;        /* n_m of Eq. 28; 0 = one region per particle (n_m = N) */
    int n_tasks;          /* stimulus schedules: the tasks of Eq. 35 (>= 1) */
    int n_steps;          /* substeps per schedule */
    double dt;            /* substep length; the field is sampled at t_n = n dt */
    double filter_radius; /* R of Eq. 23-24, in domain units (> 0) */
    double Br_max;        /* upper bound of the residual flux density, Eq. 26 (Tesla) */
    double B_max;         /* upper bound of the applied flux density, Eq. 29 (Tesla) */
    double f_min, f_max;  /* frequency range of Eq. 29 (Hz) */
    double delta;         /* regulariser of Eq. 27 and Eq. 30 (>= 0) */
} mpm_design_config;

/*
 * Build the filter from the initial positions x0 (device, [dim][N], the
 * x_p(0) of Eq. 23).  It bins them into cells no smaller than R and stores
 * the per-particle normalisers sum_p' w_pp'.  region (device, [N] ints in
 * [0, n_regions)) assigns particles to magnetisation regions.  It is NULL
 * when n_regions == 0.  Both arrays are read during this call only.  The
 * call synchronises cuda_stream.
 * Errors: MPM_ERR_ARG (bad config, NULL pointers, a region index out of
 * range), MPM_ERR_OOM, MPM_ERR_CUDA.  *out is NULL on error.
 */
int mpm_design_create(const mpm_design_config* cfg, const float* x0, const int* region, mpm_design** out,
                      void* cuda_stream);
int mpm_design_destroy(mpm_design* h);
/* Text of the handle's last error ("" if none). */
const char* mpm_design_last_error(const mpm_design* h);

/*
 * Forward maps.  Inputs: phi [N], Br [n_m], zeta [dim][n_m], Ba [n_tasks],
 * f [n_tasks], eta [n_tasks][dim].  Outputs: phi_bar [N], mag [dim][N], field
 * [n_tasks][n_steps][dim].  beta > 0 is the Heaviside sharpness.  The
 * handle keeps phi~ and beta for mpm_design_backward.
 * Errors: MPM_ERR_ARG (NULL pointer, beta <= 0), MPM_ERR_CUDA.
 */
int mpm_design_forward(mpm_design* h, float beta, const float* phi, const float* Br, const float* zeta,
                       const float* Ba, const float* f, const float* eta, float* phi_bar, float* mag,
                       float* field, void* cuda_stream);

/*
 * Reverse maps at the inputs of the last mpm_design_forward.  g_phi_bar [N],
 * g_mag [dim][N] and g_field [n_tasks][n_steps][dim] are the gradients that
 * mpm_backward returns.  Outputs are overwritten: g_phi [N], g_Br [n_m],
 * g_zeta [dim][n_m], g_Ba [n_tasks], g_f [n_tasks], g_eta [n_tasks][dim].
 * The region sums use float atomics, so their last bits depend on the
 * order of execution.
 * Errors: MPM_ERR_ARG, MPM_ERR_STATE (no forward yet), MPM_ERR_CUDA.
 */
int mpm_design_backward(mpm_design* h, const float* g_phi_bar, const float* g_mag, const float* g_field,
                        float* g_phi, float* g_Br, float* g_zeta, float* g_Ba, float* g_f, float* g_eta,
                        void* cuda_stream);

/*
 * One Adam step at iteration k >= 1 over n variables (device arrays x, g, m, v,
 * updated in place): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * x -= lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps), then x is clipped to
 * [lo, hi].  The optimiser minimises, so pass the objective's gradient.
 * Errors: MPM_ERR_ARG (n < 0, k < 1, lo > hi, NULL with n > 0), MPM_ERR_CUDA.
 */
int mpm_adam_step(long long n, float* x, const float* g, float* m, float* v, int k, double lr, double beta1,
                  double beta2, double eps, double lo, double hi, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MPM_DESIGN_H */
