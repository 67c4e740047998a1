/*
 * FP64 CPU oracle for the magneto-elastic MLS-MPM substep and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Nothing in the product package links, loads
 * or calls it; only the tests, the package's smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA kernels.
 *
 * Everything is double precision, in the order the paper states the
 * algorithm (arxiv 2503.22767):
 *   - Piola stress of the ideal hard-magnetic neo-Hookean solid: Eq. 7
 *     (energy Eq. 4-6), SIMP interpolation of energy and mass: Eq. 31-33.
 *   - P2G with the quadratic B-spline (MLS-MPM, Section 2.2 step 1): Eq. 14-15.
 *   - Grid operation: Eq. 16-17 (damping, gravity), Eq. 18 (contact).
 *   - G2P: Eq. 19-22.
 *   - Objectives: Eq. 38 (shape MSE) and Eq. 40 (mass-averaged locomotion).
 *   - Reverse mode through all of the above (Section 2.3), hand-derived.
 *
 * Readings where the paper is silent or garbled (each is also listed in the
 * design notes of the repository):
 *   R1  Eq. 15 prints the stress term without dt and with offset x_p - x_i.
 *       We use the standard MLS-MPM form the paper cites: offsets are always
 *       x_i - x_p (node minus particle) and the affine matrix is
 *       A = m_p C_p - dt (4/dx^2) v_p P_p F_p^T.
 *   R2  2D is plane strain: F3 = diag(F, 1), so I1 = |F|^2 + 1, J = det F and
 *       P is the in-plane block of Eq. 7.
 *   R3  Stencil: base = floor(x/dx - 0.5) per axis, 3^d nodes.
 *   R4  Damping c is a rate (1/s): v <- v + dt(-c v + g) after v = mv/m.
 *   R5  Walls: a band of `bound` nodes at each side of each axis.  A node in a
 *       band whose velocity points into the wall is projected; all walls are
 *       non-slip (v = 0) except, in wall mode 1, the low side of axis 1 (the
 *       floor) which applies Coulomb friction, Eq. 18 with v_b = 0.  Bands are
 *       applied axis by axis (axis 0 low, axis 0 high, axis 1 low, ...).
 *   R6  Eq. 18 with zero tangential speed or a negative friction-reduced speed
 *       gives v = 0; its derivative there is taken as 0.
 *   R7  Nodes with m = 0 get v = 0.
 *   R8  The field of substep n is field[n] (t_n = n dt, held for the substep).
 *   R9  Locomotion loss sums the mass-averaged x-velocity after each of the
 *       N substeps (n = 1..N), times dt, with a minus sign.  A body of zero
 *       total mass has zero loss.
 *   R10 Shape MSE is the mean over the instance's particles of |x_p(T) - xbar_p|^2.
 *   R11 Derivatives through floor() are zero (the weights are C1 across cells).
 *   R18 Solid boxes beyond the walls (Eq. 18 in general form): every node
 *       inside an axis-aligned box, faces included, is "on" it with the
 *       outward normal of the nearest face (ties: lowest axis, low face
 *       first); Coulomb and non-slip boxes act when (v - v_b) . n_b < 0,
 *       attached boxes always set v = v_b; boxes act after the walls, in
 *       order; a box's offset and v_b are given per substep.
 *   R19 Non-uniform applied field (the paper assumes a uniform one and notes
 *       that non-uniform fields fit the framework): a linear field about the
 *       domain centre, B(x) = B_a + G (x - x_c).  Eq. 7 / 31 use B at the
 *       particle; the SIMP-scaled energy of Eq. 32 then depends on x, and
 *       its negative x-derivative f = (phi^q V / mu0) G^T (F B~_r) enters the
 *       particle's momentum in P2G.
 *
 * Threads (orc_set_threads; default 1): with OpenMP the particle loops run
 * on several host cores without changing a single result bit.  A gather
 * (G2P, P2G^T) or a per-node loop (grid operation and its reverse) writes
 * nothing another particle or node writes.  A scatter (P2G, G2P^T) splits
 * the node columns along axis 0 into slabs, one per thread: each thread
 * visits the particles in index order and adds only to the nodes of its own
 * slab, so every node receives its terms in the serial order.  Sums over
 * all particles (dL/dB_a, dL/dG, momentum, loss) stay serial loops over
 * per-particle terms.  Hence the threaded oracle equals the serial one bit
 * for bit, which the tests check.
 *
 * Layout: per particle x[3], v[3], C[9], F[9] (row-major 3x3; in 2D only the
 * leading 2 components / 2x2 block are used and the rest stay zero).
 * Instances are independent simulations concatenated in particle order, each
 * with its own res^d grid.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)
#define ORC_ERR_NUMERIC (-5)
#define ORC_ERR_DOMAIN (-6)

static const double MU0 = 4.0e-7 * 3.14159265358979323846; /* vacuum permeability */

typedef struct {
    int dim;       /* 2 or 3 */
    int res;       /* nodes per axis, dx = 1/res, node i sits at i*dx */
    int n_steps;   /* number of substeps N */
    int bound;     /* wall band width in nodes */
    int wall_mode; /* 0: every wall non-slip; 1: Coulomb floor (axis 1 low) */
    int loss_kind; /* 0: shape MSE (Eq. 38); 1: locomotion (Eq. 40) */
    int simp_q;    /* SIMP exponent q_w (Eq. 31) */
    int pad_;
    double dt, E, nu, rho0, p_vol, simp_eps, damping, floor_mu;
    double gravity[3];
    /* Solid boxes of Eq. 18 (reading R18): n_bnd entries of 8 doubles
     * {kind, mu, lo[3], hi[3]} (kind 0 Coulomb, 1 non-slip, 2 attached),
     * and optionally per substep and box the offset and velocity v_b,
     * bmotion[((b * n_steps + n) * 2 + {0, 1}) * 3 + i]. */
    int n_bnd;
    int pad2_;
    const double* bnd;
    const double* bmotion;
    /* Non-uniform applied field (reading R19): B(x, t_n) = B_a[n] + G[n] (x - x_c),
     * x_c the domain centre, G[n] = fgrad[(inst * n_steps + n) * 9 + 3 i + j]
     * = dB_i/dx_j (row-major 3x3, d x d used), or NULL for a uniform field.
     * The reverse writes dL/dG to g_fgrad (same layout) when it is given. */
    const double* fgrad;
    double* g_fgrad;
} orc_params;

/* ------------------------------------------------------------------ */
/* host threads (see the header: results do not depend on them)         */
/* ------------------------------------------------------------------ */

#define ORC_MAX_THREADS 256
static int g_threads = 1;

/* Use n host threads (clamped to [1, 256]; 1 without OpenMP).  Returns the
 * number in effect. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : (n > ORC_MAX_THREADS ? ORC_MAX_THREADS : n);
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* ------------------------------------------------------------------ */
/* small dense helpers (3x3 storage, d x d used)                       */
/* ------------------------------------------------------------------ */

static double det_d(int d, const double* F) {
    if (d == 2) return F[0] * F[4] - F[1] * F[3];
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* H = F^{-T} via the adjugate. */
static void inv_transpose_d(int d, const double* F, double J, double* H) {
    memset(H, 0, 9 * sizeof(double));
    if (d == 2) {
        /* F^{-1} = [F11 -F01; -F10 F00]/J, transpose it */
        H[0] = F[4] / J;
        H[1] = -F[3] / J;
        H[3] = -F[1] / J;
        H[4] = F[0] / J;
        return;
    }
    /* cofactor matrix divided by J is F^{-T} */
    H[0] = (F[4] * F[8] - F[5] * F[7]) / J;
    H[1] = -(F[3] * F[8] - F[5] * F[6]) / J;
    H[2] = (F[3] * F[7] - F[4] * F[6]) / J;
    H[3] = -(F[1] * F[8] - F[2] * F[7]) / J;
    H[4] = (F[0] * F[8] - F[2] * F[6]) / J;
    H[5] = -(F[0] * F[7] - F[1] * F[6]) / J;
    H[6] = (F[1] * F[5] - F[2] * F[4]) / J;
    H[7] = -(F[0] * F[5] - F[2] * F[3]) / J;
    H[8] = (F[0] * F[4] - F[1] * F[3]) / J;
}

static double ddot_d(int d, const double* A, const double* B) {
    double s = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) s += A[a * 3 + b] * B[a * 3 + b];
    return s;
}

static double ipow(double x, int q) {
    double r = 1.0;
    for (int i = 0; i < q; ++i) r *= x;
    return r;
}

static void lame(const orc_params* P, double* G, double* K) {
    *G = P->E / (2.0 * (1.0 + P->nu));
    *K = P->E / (3.0 * (1.0 - 2.0 * P->nu));
}

/* ------------------------------------------------------------------ */
/* constitutive model: Eq. 4-7 with the SIMP interpolation of Eq. 31    */
/* ------------------------------------------------------------------ */

/* Interpolated energy density, Eq. 6 under Eq. 31 (used by the FD pin). */
double orc_energy(int d, double G, double K, const double* F, double phi, int q, double eps,
                  const double* Br, const double* Ba) {
    double J = det_d(d, F);
    double I1 = ddot_d(d, F, F) + (d == 2 ? 1.0 : 0.0);
    double We = 0.5 * G * (pow(J, -2.0 / 3.0) * I1 - 3.0) + 0.5 * K * (J - 1.0) * (J - 1.0);
    double FBr_dot_Ba = 0.0;
    for (int a = 0; a < d; ++a) {
        double FBr = 0.0;
        for (int b = 0; b < d; ++b) FBr += F[a * 3 + b] * Br[b];
        FBr_dot_Ba += FBr * Ba[a];
    }
    double Wm = -FBr_dot_Ba / MU0;
    double s = ipow(phi, q);
    return (eps + (1.0 - eps) * s) * We + s * Wm;
}

/* Piola stress P = dW/dF, Eq. 7 under Eq. 31. Returns J. */
double orc_stress(int d, double G, double K, const double* F, double phi, int q, double eps,
                  const double* Br, const double* Ba, double* Pout) {
    double J = det_d(d, F);
    double H[9];
    inv_transpose_d(d, F, J, H);
    double I1 = ddot_d(d, F, F) + (d == 2 ? 1.0 : 0.0);
    double a = G * pow(J, -2.0 / 3.0);
    double b = K * J * (J - 1.0);
    double s = ipow(phi, q);
    double sE = eps + (1.0 - eps) * s;
    memset(Pout, 0, 9 * sizeof(double));
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double Pe = a * (F[i * 3 + j] - I1 / 3.0 * H[i * 3 + j]) + b * H[i * 3 + j];
            double Pm = -Ba[i] * Br[j] / MU0;
            Pout[i * 3 + j] = sE * Pe + s * Pm;
        }
    return J;
}

/* Reverse of orc_stress: given Pbar, accumulate Fbar, phibar, Brbar, Babar. */
void orc_stress_adjoint(int d, double G, double K, const double* F, double phi, int q, double eps,
                        const double* Br, const double* Ba, const double* Pbar, double* Fbar,
                        double* phibar, double* Brbar, double* Babar) {
    double J = det_d(d, F);
    double H[9];
    inv_transpose_d(d, F, J, H);
    double I1 = ddot_d(d, F, F) + (d == 2 ? 1.0 : 0.0);
    double a = G * pow(J, -2.0 / 3.0);
    double b = K * J * (J - 1.0);
    double s = ipow(phi, q);
    double ds = (q > 0) ? q * ipow(phi, q - 1) : 0.0;
    double sE = eps + (1.0 - eps) * s;

    /* the two stress parts, needed for the phi derivative */
    double Pe[9] = {0}, Pm[9] = {0};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            Pe[i * 3 + j] = a * (F[i * 3 + j] - I1 / 3.0 * H[i * 3 + j]) + b * H[i * 3 + j];
            Pm[i * 3 + j] = -Ba[i] * Br[j] / MU0;
        }
    *phibar += ddot_d(d, Pbar, Pe) * (1.0 - eps) * ds + ddot_d(d, Pbar, Pm) * ds;

    /* magnetic part: P_m = -(1/mu0) Ba (x) Br, scaled by s */
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double pm = s * Pbar[i * 3 + j];
            Babar[i] += -pm * Br[j] / MU0;
            Brbar[j] += -pm * Ba[i] / MU0;
        }

    /* elastic part, scaled by sE:  Fbar += dPe/dF : PbarE
     *   dJ = J H:dF, dI1 = 2 F:dF, dH = -H dF^T H, da = -(2/3) a H:dF,
     *   db = K (2J - 1) J H:dF.                                          */
    double Pb[9] = {0};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Pb[i * 3 + j] = sE * Pbar[i * 3 + j];
    double PbF = ddot_d(d, Pb, F);
    double PbH = ddot_d(d, Pb, H);
    /* HPtH = H Pb^T H */
    double HPtH[9] = {0};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double acc = 0.0;
            for (int k = 0; k < d; ++k)
                for (int l = 0; l < d; ++l) acc += H[i * 3 + k] * Pb[l * 3 + k] * H[l * 3 + j];
            HPtH[i * 3 + j] = acc;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            int ij = i * 3 + j;
            double g = 0.0;
            /* term a F */
            g += PbF * (-2.0 / 3.0 * a) * H[ij] + a * Pb[ij];
            /* term -(a/3) I1 H */
            g += -(1.0 / 3.0) * (I1 * PbH * (-2.0 / 3.0 * a) * H[ij] + 2.0 * a * PbH * F[ij] -
                                 a * I1 * HPtH[ij]);
            /* term b H */
            g += PbH * K * (2.0 * J - 1.0) * J * H[ij] - b * HPtH[ij];
            Fbar[ij] += g;
        }
}

/* ------------------------------------------------------------------ */
/* quadratic B-spline, Section 2.2 step 1 (reading R3)                  */
/* ------------------------------------------------------------------ */

/* 1D weights at fractional offset r in [0.5, 1.5) and their r-derivatives. */
void orc_bspline(double r, double* w, double* dw) {
    w[0] = 0.5 * (1.5 - r) * (1.5 - r);
    w[1] = 0.75 - (r - 1.0) * (r - 1.0);
    w[2] = 0.5 * (r - 0.5) * (r - 0.5);
    dw[0] = -(1.5 - r);
    dw[1] = -2.0 * (r - 1.0);
    dw[2] = r - 0.5;
}

typedef struct {
    int base[3];
    double r[3];      /* x/dx - base */
    double w[3][3];   /* [axis][offset] */
    double dw[3][3];  /* d w / d(x/dx) */
} stencil_t;

static int make_stencil(const orc_params* P, const double* xp, stencil_t* S) {
    double inv_dx = (double)P->res;
    for (int a = 0; a < 3; ++a) {
        S->base[a] = 0;
        S->r[a] = 0.0;
        S->w[a][0] = 1.0; S->w[a][1] = 0.0; S->w[a][2] = 0.0;
        S->dw[a][0] = S->dw[a][1] = S->dw[a][2] = 0.0;
    }
    int ok = 1;
    for (int a = 0; a < P->dim; ++a) {
        double fx = xp[a] * inv_dx;
        if (!(fx == fx)) return 0;
        int b = (int)floor(fx - 0.5);
        if (b < 0 || b > P->res - 3) ok = 0;
        S->base[a] = b;
        S->r[a] = fx - b;
        orc_bspline(S->r[a], S->w[a], S->dw[a]);
    }
    return ok;
}

static int n_offsets(int d) { return d == 2 ? 9 : 27; }

/* offset index -> (o0,o1,o2); weight, weight gradient (d/dx) and node index */
static void stencil_node(const orc_params* P, const stencil_t* S, int k, int* node, double* w,
                         double* gw, double* dpos) {
    int d = P->dim, res = P->res;
    int o[3];
    if (d == 2) { o[0] = k / 3; o[1] = k % 3; o[2] = 0; }
    else { o[0] = k / 9; o[1] = (k / 3) % 3; o[2] = k % 3; }
    double dx = 1.0 / res, inv_dx = (double)res;
    double ww = 1.0;
    for (int a = 0; a < d; ++a) ww *= S->w[a][o[a]];
    *w = ww;
    for (int c = 0; c < 3; ++c) {
        gw[c] = 0.0;
        dpos[c] = 0.0;
    }
    for (int c = 0; c < d; ++c) {
        double g = S->dw[c][o[c]] * inv_dx;
        for (int a = 0; a < d; ++a)
            if (a != c) g *= S->w[a][o[a]];
        gw[c] = g;
        dpos[c] = ((double)o[c] - S->r[c]) * dx; /* x_i - x_p */
    }
    int idx = 0;
    for (int a = 0; a < d; ++a) idx = idx * res + (S->base[a] + o[a]);
    *node = idx;
}

static long grid_size(const orc_params* P) {
    long g = 1;
    for (int a = 0; a < P->dim; ++a) g *= P->res;
    return g;
}

/* ------------------------------------------------------------------ */
/* forward substep pieces                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double* x;
    double* v;
    double* C;
    double* F;
} state_t;

static double particle_mass(const orc_params* P, double phi) { return phi * P->rho0 * P->p_vol; } /* Eq. 33 */

/* Field at a particle (R19): B_a + G (x - x_c), or B_a when Gn is NULL. */
static void field_at(int d, const double* Ba, const double* Gn, const double* x, double* B) {
    for (int i = 0; i < 3; ++i) B[i] = Ba[i];
    if (!Gn) return;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) B[i] += Gn[3 * i + j] * (x[j] - 0.5);
}

/* Body force of a non-uniform field (R19): minus the position derivative of
 * the SIMP-scaled magnetic energy of Eq. 31-32,
 *   f = (phi^q V / mu0) G^T (F B~_r). */
static void magnetic_force(const orc_params* P, const double* Gn, const double* F, const double* Br,
                           double phi, double* f) {
    int d = P->dim;
    for (int i = 0; i < 3; ++i) f[i] = 0.0;
    if (!Gn) return;
    double c = ipow(phi, P->simp_q) * P->p_vol / MU0;
    double FB[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) FB[i] += F[3 * i + k] * Br[k];
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) f[j] += c * Gn[3 * i + j] * FB[i];
}

/* Axis-0 offset of stencil entry k (the order of stencil_node). */
static int offset0(int d, int k) { return d == 2 ? k / 3 : k / 9; }

/* Split the node columns [0, res) along axis 0 into T slabs of about equal
 * scatter work (a particle with base column b adds to columns b .. b+2);
 * slab t is [lo[t], lo[t+1]).  b0[p] is the base column of particle p. */
static void make_slabs(const orc_params* P, const int* b0, int p0, int p1, int T, int* lo) {
    int res = P->res;
    double* work = (double*)calloc((size_t)res + 1, sizeof(double));
    double total = 0.0;
    if (work) {
        for (int p = p0; p < p1; ++p)
            for (int o = 0; o < 3; ++o) work[b0[p] + o] += 1.0;
        for (int c = 0; c < res; ++c) total += work[c];
    }
    lo[0] = 0;
    double acc = 0.0;
    int t = 1;
    for (int c = 0; c < res && t < T; ++c) {
        acc += work ? work[c] : 0.0;
        while (t < T && acc >= total * t / T) lo[t++] = c + 1;
    }
    while (t < T) lo[t++] = res;
    lo[T] = res;
    free(work);
}

/* Base column (axis 0) and stencil check of particles [p0, p1): returns 1
 * when every stencil lies inside the grid. */
static int base_columns(const orc_params* P, int p0, int p1, const double* x, int* b0) {
    int ok = 1;
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(&& : ok)
    for (int p = p0; p < p1; ++p) {
        stencil_t S;
        int good = make_stencil(P, x + 3 * p, &S);
        ok = ok && good;
        b0[p] = good ? S.base[0] : 0;
    }
    return ok;
}

/* P2G (Eq. 14-15 with reading R1) of particle p into the nodes whose axis-0
 * index lies in [c_lo, c_hi).  Returns 0 when J <= 0. */
static int p2g_particle(const orc_params* P, int p, const state_t* s, const double* phi,
                        const double* mag, const double* Ba, const double* Gn, double* gm,
                        double* gmv, int c_lo, int c_hi) {
    int d = P->dim;
    double G, K;
    lame(P, &G, &K);
    double dx = 1.0 / P->res;
    double kappa = 4.0 / (dx * dx);
    stencil_t S;
    make_stencil(P, s->x + 3 * p, &S);
    double Pst[9], Bp[3], fp[3];
    field_at(d, Ba, Gn, s->x + 3 * p, Bp);
    double J = orc_stress(d, G, K, s->F + 9 * p, phi[p], P->simp_q, P->simp_eps, mag + 3 * p, Bp, Pst);
    double mp = particle_mass(P, phi[p]);
    const double* F = s->F + 9 * p;
    magnetic_force(P, Gn, F, mag + 3 * p, phi[p], fp);
    const double* C = s->C + 9 * p;
    double A[9] = {0};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double PFt = 0.0;
            for (int k = 0; k < d; ++k) PFt += Pst[i * 3 + k] * F[j * 3 + k];
            A[i * 3 + j] = mp * C[i * 3 + j] - P->dt * kappa * P->p_vol * PFt;
        }
    for (int k = 0; k < n_offsets(d); ++k) {
        int c0 = S.base[0] + offset0(d, k);
        if (c0 < c_lo || c0 >= c_hi) continue;
        int node;
        double w, gw[3], dpos[3];
        stencil_node(P, &S, k, &node, &w, gw, dpos);
        gm[node] += w * mp;
        for (int i = 0; i < d; ++i) {
            double Ad = 0.0;
            for (int j = 0; j < d; ++j) Ad += A[i * 3 + j] * dpos[j];
            gmv[3 * node + i] += w * (mp * s->v[3 * p + i] + P->dt * fp[i] + Ad);
        }
    }
    return J > 0.0;
}

/* P2G (Eq. 14-15 with reading R1) for the particles [p0, p1) into one grid;
 * Gn is the field gradient of this instance and substep, or NULL.  Each
 * thread scatters into its own slab of node columns (see the header). */
static int p2g(const orc_params* P, int p0, int p1, const state_t* s, const double* phi,
               const double* mag, const double* Ba, const double* Gn, double* gm, double* gmv) {
    if (p1 <= p0) return ORC_OK;
    int* b0 = (int*)malloc(sizeof(int) * (size_t)p1);
    if (!b0) return ORC_ERR_OOM;
    if (!base_columns(P, p0, p1, s->x, b0)) {
        free(b0);
        return ORC_ERR_DOMAIN;
    }
    int T = g_threads;
    int lo[ORC_MAX_THREADS + 1];
    make_slabs(P, b0, p0, p1, T, lo);
    int good = 1;
#pragma omp parallel num_threads(T) reduction(&& : good)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        for (int p = p0; p < p1; ++p) {
            if (b0[p] + 2 < lo[t] || b0[p] >= lo[t + 1]) continue;
            good = p2g_particle(P, p, s, phi, mag, Ba, Gn, gm, gmv, lo[t], lo[t + 1]) && good;
        }
    }
    free(b0);
    return good ? ORC_OK : ORC_ERR_NUMERIC;
}

/* Boundary projection trace of one node (readings R5/R6/R18). */
#define ORC_MAX_OPS (6 + 8)
typedef struct {
    int n_ops;
    int kind[ORC_MAX_OPS];     /* 1 = velocity set (non-slip / attached), 2 = Coulomb */
    int axis[ORC_MAX_OPS];
    double sgn[ORC_MAX_OPS];   /* outward normal of the solid: sgn * e_axis */
    double mu[ORC_MAX_OPS];
    double vin[ORC_MAX_OPS][3]; /* velocity relative to the boundary before the op */
} bc_trace;

static void node_index_coords(const orc_params* P, long idx, int* c) {
    c[0] = c[1] = c[2] = 0;
    for (int a = P->dim - 1; a >= 0; --a) {
        c[a] = (int)(idx % P->res);
        idx /= P->res;
    }
}

/* Coulomb projection of Eq. 18 on velocity v relative to a boundary moving
 * at vb, with outward normal sgn * e_a, when the relative velocity points
 * into the solid (vn < 0): the normal part becomes vb's, the tangential
 * part shrinks by mu |vn| (to zero at most). */
static void coulomb(int d, int a, double sgn, double mu, const double* vb, double* v) {
    double vr[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) vr[i] = v[i] - vb[i];
    double vn = sgn * vr[a];
    double t2 = 0.0;
    for (int i = 0; i < d; ++i)
        if (i != a) t2 += vr[i] * vr[i];
    double u = sqrt(t2);
    double sp = u + mu * vn;
    double f = (u > 0.0 && sp > 0.0) ? sp / u : 0.0;
    for (int i = 0; i < d; ++i) v[i] = vb[i] + (i == a ? 0.0 : vr[i] * f);
}

/* Boundary conditions on velocity v (in place) at substep `step`, recording
 * what fired: the walls (R5), then every solid box in order (R18). */
static void apply_bc(const orc_params* P, const int* c, double* v, bc_trace* tr, int step) {
    int d = P->dim;
    tr->n_ops = 0;
    for (int a = 0; a < d; ++a) {
        for (int side = 0; side < 2; ++side) {
            int in_band = side == 0 ? (c[a] < P->bound) : (c[a] >= P->res - P->bound);
            if (!in_band) continue;
            double vn = side == 0 ? v[a] : -v[a]; /* v . n with n the inward wall normal */
            if (!(vn < 0.0)) continue;
            int op = tr->n_ops++;
            tr->axis[op] = a;
            tr->sgn[op] = side == 0 ? 1.0 : -1.0;
            tr->mu[op] = P->floor_mu;
            for (int i = 0; i < 3; ++i) tr->vin[op][i] = v[i];
            if (P->wall_mode == 1 && a == 1 && side == 0) {
                /* Coulomb floor, Eq. 18 with v_b = 0, normal +e_1 */
                static const double zero[3] = {0, 0, 0};
                tr->kind[op] = 2;
                coulomb(d, a, 1.0, P->floor_mu, zero, v);
            } else {
                tr->kind[op] = 1; /* non-slip, the mu -> infinity limit */
                for (int i = 0; i < d; ++i) v[i] = 0.0;
            }
        }
    }
    /* solid boxes: a node inside the (moved) box lies on its nearest face */
    double dx = 1.0 / P->res;
    for (int b = 0; b < P->n_bnd; ++b) {
        const double* B = P->bnd + 8 * b;
        int kind = (int)B[0];
        double off[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
        if (P->bmotion) {
            const double* m = P->bmotion + ((size_t)b * P->n_steps + step) * 6;
            for (int i = 0; i < 3; ++i) {
                off[i] = m[i];
                vb[i] = m[3 + i];
            }
        }
        int inside = 1, axis = 0;
        double sgn = -1.0, best = 1e300;
        for (int a = 0; a < d; ++a) {
            double x = c[a] * dx, lo = B[2 + a] + off[a], hi = B[5 + a] + off[a];
            if (x < lo || x > hi) inside = 0;
            if (x - lo < best) { best = x - lo; axis = a; sgn = -1.0; }
            if (hi - x < best) { best = hi - x; axis = a; sgn = 1.0; }
        }
        if (!inside) continue;
        double vn = sgn * (v[axis] - vb[axis]);
        if (kind != 2 && !(vn < 0.0)) continue; /* separating: free */
        int op = tr->n_ops++;
        tr->axis[op] = axis;
        tr->sgn[op] = sgn;
        tr->mu[op] = B[1];
        for (int i = 0; i < 3; ++i) tr->vin[op][i] = v[i] - vb[i];
        if (kind == 0) {
            tr->kind[op] = 2;
            coulomb(d, axis, sgn, B[1], vb, v);
        } else { /* non-slip obstacle when moving into it; attached always */
            tr->kind[op] = 1;
            for (int i = 0; i < d; ++i) v[i] = vb[i];
        }
    }
}

/* Grid operation, Eq. 16-18, on every node of one grid at substep `step`. */
static void grid_update(const orc_params* P, const double* gm, const double* gmv, double* gv, int step) {
    long G = grid_size(P);
    int d = P->dim;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (long n = 0; n < G; ++n) {
        for (int i = 0; i < 3; ++i) gv[3 * n + i] = 0.0;
        if (!(gm[n] > 0.0)) continue; /* reading R7 */
        double v[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i) {
            v[i] = gmv[3 * n + i] / gm[n];
            v[i] = v[i] + P->dt * (-P->damping * v[i] + P->gravity[i]);
        }
        int c[3];
        node_index_coords(P, n, c);
        bc_trace tr;
        apply_bc(P, c, v, &tr, step);
        for (int i = 0; i < d; ++i) gv[3 * n + i] = v[i];
    }
}

/* G2P, Eq. 19-22, for particles [p0, p1): s_in -> s_out. */
static int g2p(const orc_params* P, int p0, int p1, const state_t* si, const double* gv, state_t* so) {
    int d = P->dim;
    double dx = 1.0 / P->res;
    double kappa = 4.0 / (dx * dx);
    int inside = 1, positive = 1;
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(&& : inside, positive)
    for (int p = p0; p < p1; ++p) {
        stencil_t S;
        if (!make_stencil(P, si->x + 3 * p, &S)) {
            inside = 0;
            continue;
        }
        double vp[3] = {0, 0, 0}, Cp[9] = {0};
        for (int k = 0; k < n_offsets(d); ++k) {
            int node;
            double w, gw[3], dpos[3];
            stencil_node(P, &S, k, &node, &w, gw, dpos);
            for (int i = 0; i < d; ++i) {
                vp[i] += w * gv[3 * node + i];
                for (int j = 0; j < d; ++j) Cp[i * 3 + j] += kappa * w * gv[3 * node + i] * dpos[j];
            }
        }
        const double* F = si->F + 9 * p;
        double Fn[9] = {0};
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double acc = F[i * 3 + j];
                for (int k = 0; k < d; ++k) acc += P->dt * Cp[i * 3 + k] * F[k * 3 + j];
                Fn[i * 3 + j] = acc;
            }
        for (int i = 0; i < 3; ++i) {
            so->x[3 * p + i] = si->x[3 * p + i] + (i < d ? P->dt * vp[i] : 0.0);
            so->v[3 * p + i] = vp[i];
        }
        memcpy(so->C + 9 * p, Cp, sizeof Cp);
        memcpy(so->F + 9 * p, Fn, sizeof Fn);
        if (!(det_d(d, Fn) > 0.0)) positive = 0;
    }
    if (!inside) return ORC_ERR_DOMAIN;
    return positive ? ORC_OK : ORC_ERR_NUMERIC;
}

/* ------------------------------------------------------------------ */
/* whole-horizon driver                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_params* P;
    int n_inst;
    const int* counts;
    int* offs;    /* [n_inst + 1] */
    int N;
    long G;
    double* gm;   /* [G] scratch (one instance at a time) */
    double* gmv;  /* [3G] */
    double* gv;   /* [3G] */
} sim_t;

static int sim_init(sim_t* S, const orc_params* P, int n_inst, const int* counts) {
    if (!P || !counts || n_inst <= 0 || (P->dim != 2 && P->dim != 3) || P->res < 2 * P->bound + 3 ||
        P->n_steps < 0 || P->n_bnd < 0 || P->n_bnd > 8 || (P->n_bnd > 0 && !P->bnd))
        return ORC_ERR_ARG;
    S->P = P;
    S->n_inst = n_inst;
    S->counts = counts;
    S->offs = (int*)malloc(sizeof(int) * (n_inst + 1));
    if (!S->offs) return ORC_ERR_OOM;
    S->offs[0] = 0;
    for (int i = 0; i < n_inst; ++i) {
        if (counts[i] < 0) return ORC_ERR_ARG;
        S->offs[i + 1] = S->offs[i] + counts[i];
    }
    S->N = S->offs[n_inst];
    S->G = grid_size(P);
    S->gm = (double*)calloc(S->G, sizeof(double));
    S->gmv = (double*)calloc(3 * S->G, sizeof(double));
    S->gv = (double*)calloc(3 * S->G, sizeof(double));
    if (!S->gm || !S->gmv || !S->gv) return ORC_ERR_OOM;
    return ORC_OK;
}

static void sim_free(sim_t* S) {
    free(S->offs);
    free(S->gm);
    free(S->gmv);
    free(S->gv);
}

static int state_alloc(state_t* s, int N) {
    s->x = (double*)calloc((size_t)3 * N + 1, sizeof(double));
    s->v = (double*)calloc((size_t)3 * N + 1, sizeof(double));
    s->C = (double*)calloc((size_t)9 * N + 1, sizeof(double));
    s->F = (double*)calloc((size_t)9 * N + 1, sizeof(double));
    return (s->x && s->v && s->C && s->F) ? ORC_OK : ORC_ERR_OOM;
}

static void state_free(state_t* s) {
    free(s->x);
    free(s->v);
    free(s->C);
    free(s->F);
}

static void state_copy(state_t* dst, const state_t* src, int N) {
    memcpy(dst->x, src->x, sizeof(double) * 3 * N);
    memcpy(dst->v, src->v, sizeof(double) * 3 * N);
    memcpy(dst->C, src->C, sizeof(double) * 9 * N);
    memcpy(dst->F, src->F, sizeof(double) * 9 * N);
}

static void state_zero(state_t* s, int N) {
    memset(s->x, 0, sizeof(double) * 3 * N);
    memset(s->v, 0, sizeof(double) * 3 * N);
    memset(s->C, 0, sizeof(double) * 9 * N);
    memset(s->F, 0, sizeof(double) * 9 * N);
}

static void initial_state(const sim_t* S, const double* x0, const double* v0, state_t* s) {
    int d = S->P->dim;
    state_zero(s, S->N);
    for (int p = 0; p < S->N; ++p) {
        for (int i = 0; i < d; ++i) {
            s->x[3 * p + i] = x0[3 * p + i];
            s->v[3 * p + i] = v0 ? v0[3 * p + i] : 0.0;
        }
        for (int i = 0; i < d; ++i) s->F[9 * p + 4 * i] = 1.0;
    }
}

/* one substep n for every instance: s_in -> s_out */
static int substep(sim_t* S, int n, const state_t* si, const double* phi, const double* mag,
                   const double* field, state_t* so) {
    const orc_params* P = S->P;
    int worst = ORC_OK;
    for (int inst = 0; inst < S->n_inst; ++inst) {
        int p0 = S->offs[inst], p1 = S->offs[inst + 1];
        const double* Ba = field + ((size_t)inst * P->n_steps + n) * 3;
        memset(S->gm, 0, sizeof(double) * S->G);
        memset(S->gmv, 0, sizeof(double) * 3 * S->G);
        const double* Gn = P->fgrad ? P->fgrad + ((size_t)inst * P->n_steps + n) * 9 : NULL;
        int st = p2g(P, p0, p1, si, phi, mag, Ba, Gn, S->gm, S->gmv);
        if (st == ORC_ERR_DOMAIN) return st;
        if (st != ORC_OK) worst = st;
        grid_update(P, S->gm, S->gmv, S->gv, n);
        st = g2p(P, p0, p1, si, S->gv, so);
        if (st == ORC_ERR_DOMAIN) return st;
        if (st != ORC_OK) worst = st;
    }
    return worst;
}

/* total mass of each instance (Eq. 33 summed) */
static void instance_mass(const sim_t* S, const double* phi, double* M) {
    for (int inst = 0; inst < S->n_inst; ++inst) {
        double m = 0.0;
        for (int p = S->offs[inst]; p < S->offs[inst + 1]; ++p) m += particle_mass(S->P, phi[p]);
        M[inst] = m;
    }
}

/* sum_p m_p v_{p,0} per instance (numerator of the Eq. 40 average) */
static void instance_momentum_x(const sim_t* S, const state_t* s, const double* phi, double* out) {
    for (int inst = 0; inst < S->n_inst; ++inst) {
        double acc = 0.0;
        for (int p = S->offs[inst]; p < S->offs[inst + 1]; ++p)
            acc += particle_mass(S->P, phi[p]) * s->v[3 * p + 0];
        out[inst] = acc;
    }
}

/*
 * Forward over the whole horizon.
 *   x0, v0, target: [N][3]; C0, F0: [N][9] (NULL: 0 and I); phi: [N]; mag: [N][3] (B~_r, Tesla);
 *   field: [n_inst][n_steps][3] (B_applied, Tesla).  v0/target may be NULL.
 *   Outputs: final state (any may be NULL), loss[n_inst], and optionally
 *   traj_x [(n_steps+1)][N][3] and mom_x [n_steps][n_inst] (sum m v_x after step n+1).
 */
int orc_forward_ex(const orc_params* P, int n_inst, const int* counts, const double* x0,
                   const double* v0, const double* C0, const double* F0, const double* phi,
                   const double* mag, const double* field, const double* target, double* x_out,
                   double* v_out, double* C_out, double* F_out, double* loss, double* traj_x,
                   double* mom_x) {
    sim_t S;
    int st = sim_init(&S, P, n_inst, counts);
    if (st != ORC_OK) return st;
    int N = S.N, d = P->dim;
    state_t a, b;
    if (state_alloc(&a, N) != ORC_OK || state_alloc(&b, N) != ORC_OK) return ORC_ERR_OOM;
    initial_state(&S, x0, v0, &a);
    if (C0) memcpy(a.C, C0, sizeof(double) * 9 * N);
    if (F0) memcpy(a.F, F0, sizeof(double) * 9 * N);
    double* M = (double*)calloc(n_inst, sizeof(double));
    double* mx = (double*)calloc(n_inst, sizeof(double));
    double* lsum = (double*)calloc(n_inst, sizeof(double));
    instance_mass(&S, phi, M);
    if (traj_x) memcpy(traj_x, a.x, sizeof(double) * 3 * N);
    int worst = ORC_OK;
    for (int n = 0; n < P->n_steps; ++n) {
        st = substep(&S, n, &a, phi, mag, field, &b);
        if (st == ORC_ERR_DOMAIN) { worst = st; break; }
        if (st != ORC_OK) worst = st;
        state_t t = a; a = b; b = t;
        if (traj_x) memcpy(traj_x + (size_t)(n + 1) * 3 * N, a.x, sizeof(double) * 3 * N);
        instance_momentum_x(&S, &a, phi, mx);
        for (int i = 0; i < n_inst; ++i) {
            if (mom_x) mom_x[(size_t)n * n_inst + i] = mx[i];
            if (M[i] > 0.0) lsum[i] += mx[i] / M[i];
        }
    }
    for (int i = 0; i < n_inst; ++i) {
        if (!loss) break;
        if (P->loss_kind == 1) {
            loss[i] = -P->dt * lsum[i];
        } else {
            double acc = 0.0;
            int p0 = S.offs[i], p1 = S.offs[i + 1];
            for (int p = p0; p < p1; ++p)
                for (int c = 0; c < d; ++c) {
                    double e = a.x[3 * p + c] - (target ? target[3 * p + c] : 0.0);
                    acc += e * e;
                }
            loss[i] = (p1 > p0) ? acc / (p1 - p0) : 0.0;
        }
    }
    if (x_out) memcpy(x_out, a.x, sizeof(double) * 3 * N);
    if (v_out) memcpy(v_out, a.v, sizeof(double) * 3 * N);
    if (C_out) memcpy(C_out, a.C, sizeof(double) * 9 * N);
    if (F_out) memcpy(F_out, a.F, sizeof(double) * 9 * N);
    free(M); free(mx); free(lsum);
    state_free(&a); state_free(&b);
    sim_free(&S);
    return worst;
}

/* Forward from rest: C0 = 0, F0 = I (the method's initial state). */
int orc_forward(const orc_params* P, int n_inst, const int* counts, const double* x0,
                const double* v0, const double* phi, const double* mag, const double* field,
                const double* target, double* x_out, double* v_out, double* C_out, double* F_out,
                double* loss, double* traj_x, double* mom_x) {
    return orc_forward_ex(P, n_inst, counts, x0, v0, NULL, NULL, phi, mag, field, target, x_out,
                          v_out, C_out, F_out, loss, traj_x, mom_x);
}

/*
 * One P2G + grid operation on given particle states (used by the
 * conservation and torque pins).  Grids are [n_inst][G], [n_inst][G][3].
 * Ba: [n_inst][3].
 */
int orc_p2g_grid(const orc_params* P, int n_inst, const int* counts, const double* x,
                 const double* v, const double* C, const double* F, const double* phi,
                 const double* mag, const double* Ba, double* gm_out, double* gmv_out,
                 double* gv_out) {
    sim_t S;
    int st = sim_init(&S, P, n_inst, counts);
    if (st != ORC_OK) return st;
    state_t s = {(double*)x, (double*)v, (double*)C, (double*)F};
    int worst = ORC_OK;
    for (int inst = 0; inst < n_inst; ++inst) {
        double* gm = gm_out + (size_t)inst * S.G;
        double* gmv = gmv_out + (size_t)inst * 3 * S.G;
        double* gv = gv_out + (size_t)inst * 3 * S.G;
        memset(gm, 0, sizeof(double) * S.G);
        memset(gmv, 0, sizeof(double) * 3 * S.G);
        const double* Gn = P->fgrad ? P->fgrad + (size_t)inst * P->n_steps * 9 : NULL;
        st = p2g(P, S.offs[inst], S.offs[inst + 1], &s, phi, mag, Ba + 3 * inst, Gn, gm, gmv);
        if (st == ORC_ERR_DOMAIN) { sim_free(&S); return st; }
        if (st != ORC_OK) worst = st;
        grid_update(P, gm, gmv, gv, 0);
    }
    sim_free(&S);
    return worst;
}

/* ------------------------------------------------------------------ */
/* reverse mode (Section 2.3), hand-derived                             */
/* ------------------------------------------------------------------ */

/* Reverse of the grid operation on one node: Vbar -> (mbar, mvbar). */
static void grid_update_adjoint_node(const orc_params* P, long n, double m, const double* mv,
                                     const double* Vbar, double* mbar, double* mvbar, int step) {
    int d = P->dim;
    *mbar = 0.0;
    for (int i = 0; i < 3; ++i) mvbar[i] = 0.0;
    if (!(m > 0.0)) return;
    double v0[3] = {0, 0, 0}, v1[3] = {0, 0, 0};
    double keep = 1.0 - P->dt * P->damping;
    for (int i = 0; i < d; ++i) {
        v0[i] = mv[i] / m;
        v1[i] = v0[i] + P->dt * (-P->damping * v0[i] + P->gravity[i]);
    }
    int c[3];
    node_index_coords(P, n, c);
    bc_trace tr;
    double v2[3] = {v1[0], v1[1], v1[2]};
    apply_bc(P, c, v2, &tr, step);
    double vb[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) vb[i] = Vbar[i];
    for (int op = tr.n_ops - 1; op >= 0; --op) {
        if (tr.kind[op] == 1) { /* output independent of the input */
            for (int i = 0; i < 3; ++i) vb[i] = 0.0;
            continue;
        }
        /* Coulomb on the relative velocity r (the boundary velocity is a
         * constant): out_t = r_t (1 + mu vn / u), out_n = 0, vn = sgn r_a,
         * u = |r_t|, when u > 0 and u + mu vn > 0 */
        int a = tr.axis[op];
        double sg = tr.sgn[op], mu = tr.mu[op];
        const double* vin = tr.vin[op];
        double vn = sg * vin[a];
        double u2 = 0.0;
        for (int i = 0; i < d; ++i)
            if (i != a) u2 += vin[i] * vin[i];
        double u = sqrt(u2);
        double sp = u + mu * vn;
        double out[3] = {0, 0, 0};
        if (u > 0.0 && sp > 0.0) {
            double tdot = 0.0; /* vbar_out . r_t */
            for (int i = 0; i < d; ++i)
                if (i != a) tdot += vb[i] * vin[i];
            double f = 1.0 + mu * vn / u;
            for (int i = 0; i < d; ++i) {
                if (i == a) continue;
                out[i] = vb[i] * f - mu * vn * vin[i] * tdot / (u * u * u);
            }
            out[a] = sg * mu * tdot / u;
        }
        for (int i = 0; i < 3; ++i) vb[i] = out[i];
    }
    /* v1 = keep * v0 + dt g ; v0 = mv / m */
    for (int i = 0; i < d; ++i) {
        double v0b = keep * vb[i];
        mvbar[i] = v0b / m;
        *mbar += -v0b * v0[i] / m;
    }
}

typedef struct {
    double* x;  /* [3N] */
    double* v;  /* [3N] */
    double* C;  /* [9N] */
    double* F;  /* [9N] */
} adj_t;

/* Reverse of G2P (Eq. 19-22) for particle p: consumes the adjoint ab of
 * the state after the substep, writes the particle's partial adjoint into an
 * (when `owner`) and adds its terms to Vbar at the nodes whose axis-0 index
 * lies in [c_lo, c_hi). */
static void g2p_adjoint_particle(const orc_params* P, int p, const state_t* sn, const double* gv,
                                 const adj_t* ab, adj_t* an, double* Vbar, int c_lo, int c_hi,
                                 int owner) {
    int d = P->dim;
    double dx = 1.0 / P->res;
    double kappa = 4.0 / (dx * dx);
    stencil_t Sp;
    make_stencil(P, sn->x + 3 * p, &Sp);
    /* recompute v', C' */
    double vp[3] = {0, 0, 0}, Cp[9] = {0};
    for (int k = 0; k < n_offsets(d); ++k) {
        int node;
        double w, gw[3], dpos[3];
        stencil_node(P, &Sp, k, &node, &w, gw, dpos);
        for (int i = 0; i < d; ++i) {
            vp[i] += w * gv[3 * node + i];
            for (int j = 0; j < d; ++j) Cp[i * 3 + j] += kappa * w * gv[3 * node + i] * dpos[j];
        }
    }
    const double* F = sn->F + 9 * p;
    const double* xb1 = ab->x + 3 * p;
    const double* vb1 = ab->v + 3 * p;
    const double* Cb1 = ab->C + 9 * p;
    const double* Fb1 = ab->F + 9 * p;
    /* x' = x + dt v' ; F' = (I + dt C') F */
    double vtot[3] = {0, 0, 0}, Ctot[9] = {0};
    for (int i = 0; i < d; ++i) vtot[i] = vb1[i] + P->dt * xb1[i];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double acc = 0.0; /* (Fbar' F^T)_ij */
            for (int k = 0; k < d; ++k) acc += Fb1[i * 3 + k] * F[j * 3 + k];
            Ctot[i * 3 + j] = Cb1[i * 3 + j] + P->dt * acc;
        }
    double xbn[3] = {0, 0, 0}, Fbn[9] = {0};
    for (int i = 0; i < d; ++i) xbn[i] = xb1[i];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            /* ((I + dt C')^T Fbar')_ij */
            double acc = Fb1[i * 3 + j];
            for (int k = 0; k < d; ++k) acc += P->dt * Cp[k * 3 + i] * Fb1[k * 3 + j];
            Fbn[i * 3 + j] = acc;
        }
    for (int k = 0; k < n_offsets(d); ++k) {
        int node;
        double w, gw[3], dpos[3];
        stencil_node(P, &Sp, k, &node, &w, gw, dpos);
        const double* V = gv + 3 * node;
        double Vdotv = 0.0, VCd = 0.0;
        for (int i = 0; i < d; ++i) {
            Vdotv += V[i] * vtot[i];
            for (int j = 0; j < d; ++j) VCd += V[i] * Ctot[i * 3 + j] * dpos[j];
        }
        for (int c = 0; c < d; ++c) {
            double CtV = 0.0;
            for (int i = 0; i < d; ++i) CtV += Ctot[i * 3 + c] * V[i];
            xbn[c] += gw[c] * (Vdotv + kappa * VCd) - kappa * w * CtV;
        }
        int c0 = Sp.base[0] + offset0(d, k);
        if (c0 < c_lo || c0 >= c_hi) continue;
        for (int i = 0; i < d; ++i) {
            double Cd = 0.0;
            for (int j = 0; j < d; ++j) Cd += Ctot[i * 3 + j] * dpos[j];
            Vbar[3 * node + i] += w * (vtot[i] + kappa * Cd);
        }
    }
    if (!owner) return;
    for (int i = 0; i < 3; ++i) an->x[3 * p + i] = xbn[i];
    for (int i = 0; i < 9; ++i) an->F[9 * p + i] = Fbn[i];
    for (int i = 0; i < 3; ++i) an->v[3 * p + i] = 0.0;
    for (int i = 0; i < 9; ++i) an->C[9 * p + i] = 0.0;
}

/*
 * Reverse of substep n for all instances.
 *   sn: state at the start of substep n; ab: adjoint of the state after it
 *   (consumed); an: adjoint of sn (overwritten).  Accumulates design grads.
 */
static int substep_adjoint(sim_t* S, int n, const state_t* sn, const double* phi,
                           const double* mag, const double* field, const adj_t* ab, adj_t* an,
                           double* g_phi, double* g_mag, double* g_field) {
    const orc_params* P = S->P;
    int d = P->dim;
    double G, K;
    lame(P, &G, &K);
    double dx = 1.0 / P->res;
    double kappa = 4.0 / (dx * dx);
    long Gn = S->G;
    double* Vbar = (double*)calloc(3 * Gn, sizeof(double));
    double* mbar = (double*)calloc(Gn, sizeof(double));
    double* mvbar = (double*)calloc(3 * Gn, sizeof(double));
    if (!Vbar || !mbar || !mvbar) return ORC_ERR_OOM;
    for (int inst = 0; inst < S->n_inst; ++inst) {
        int p0 = S->offs[inst], p1 = S->offs[inst + 1];
        const double* Ba = field + ((size_t)inst * P->n_steps + n) * 3;
        double* gBa = g_field + ((size_t)inst * P->n_steps + n) * 3;
        /* recompute the forward grid of this substep */
        memset(S->gm, 0, sizeof(double) * Gn);
        memset(S->gmv, 0, sizeof(double) * 3 * Gn);
        const double* Gf = P->fgrad ? P->fgrad + ((size_t)inst * P->n_steps + n) * 9 : NULL;
        double* gGf = (P->fgrad && P->g_fgrad) ? P->g_fgrad + ((size_t)inst * P->n_steps + n) * 9 : NULL;
        int st = p2g(P, p0, p1, sn, phi, mag, Ba, Gf, S->gm, S->gmv);
        if (st == ORC_ERR_DOMAIN) { free(Vbar); free(mbar); free(mvbar); return st; }
        grid_update(P, S->gm, S->gmv, S->gv, n);
        memset(Vbar, 0, sizeof(double) * 3 * Gn);

        /* --- reverse of G2P (Eq. 19-22) --- */
        {
            int* b0 = (int*)malloc(sizeof(int) * (size_t)(p1 > 0 ? p1 : 1));
            if (!b0) { free(Vbar); free(mbar); free(mvbar); return ORC_ERR_OOM; }
            base_columns(P, p0, p1, sn->x, b0);
            int T = g_threads;
            int lo[ORC_MAX_THREADS + 1];
            make_slabs(P, b0, p0, p1, T, lo);
#pragma omp parallel num_threads(T)
            {
                int t = 0;
#ifdef _OPENMP
                t = omp_get_thread_num();
#endif
                for (int p = p0; p < p1; ++p) {
                    if (b0[p] + 2 < lo[t] || b0[p] >= lo[t + 1]) continue;
                    /* the thread whose slab holds the base column writes the
                     * particle's own adjoint; every thread adds to its nodes */
                    int owner = b0[p] >= lo[t] && b0[p] < lo[t + 1];
                    g2p_adjoint_particle(P, p, sn, S->gv, ab, an, Vbar, lo[t], lo[t + 1], owner);
                }
            }
            free(b0);
        }

        /* --- reverse of the grid operation (Eq. 16-18) --- */
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (long nd = 0; nd < Gn; ++nd)
            grid_update_adjoint_node(P, nd, S->gm[nd], S->gmv + 3 * nd, Vbar + 3 * nd, mbar + nd,
                                     mvbar + 3 * nd, n);

        /* --- reverse of P2G (Eq. 14-15, stress Eq. 7, SIMP Eq. 31-33) ---
         * per-particle terms of dL/dB_a and dL/dG are kept and summed in
         * particle order after the loop */
        size_t np_ = (size_t)(p1 - p0);
        double* tBa = (double*)calloc(3 * np_ + 1, sizeof(double));
        double* tG = gGf ? (double*)calloc(18 * np_ + 1, sizeof(double)) : NULL;
        if (!tBa || (gGf && !tG)) { free(tBa); free(tG); free(Vbar); free(mbar); free(mvbar); return ORC_ERR_OOM; }
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int p = p0; p < p1; ++p) {
            stencil_t Sp;
            make_stencil(P, sn->x + 3 * p, &Sp);
            const double* F = sn->F + 9 * p;
            const double* C = sn->C + 9 * p;
            const double* v = sn->v + 3 * p;
            double Pst[9], Bp[3], fp[3];
            field_at(d, Ba, Gf, sn->x + 3 * p, Bp);
            orc_stress(d, G, K, F, phi[p], P->simp_q, P->simp_eps, mag + 3 * p, Bp, Pst);
            double mp = particle_mass(P, phi[p]);
            magnetic_force(P, Gf, F, mag + 3 * p, phi[p], fp);
            double A[9] = {0};
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    double PFt = 0.0;
                    for (int k = 0; k < d; ++k) PFt += Pst[i * 3 + k] * F[j * 3 + k];
                    A[i * 3 + j] = mp * C[i * 3 + j] - P->dt * kappa * P->p_vol * PFt;
                }
            double mpbar = 0.0, Abar[9] = {0}, fbar[3] = {0, 0, 0};
            double* xbn = an->x + 3 * p;
            double* vbn = an->v + 3 * p;
            for (int k = 0; k < n_offsets(d); ++k) {
                int node;
                double w, gw[3], dpos[3];
                stencil_node(P, &Sp, k, &node, &w, gw, dpos);
                const double* mvb = mvbar + 3 * node;
                double mb = mbar[node];
                /* contribution value: w * (mb * mp + mvb . (mp v + dt f + A dpos)) */
                double inner = mb * mp;
                for (int i = 0; i < d; ++i) {
                    inner += mvb[i] * P->dt * fp[i];
                    fbar[i] += w * P->dt * mvb[i];
                }
                double vcd = 0.0;
                for (int i = 0; i < d; ++i) {
                    double Ad = 0.0, Cd = 0.0;
                    for (int j = 0; j < d; ++j) {
                        Ad += A[i * 3 + j] * dpos[j];
                        Cd += C[i * 3 + j] * dpos[j];
                    }
                    inner += mvb[i] * (mp * v[i] + Ad);
                    vcd += mvb[i] * (v[i] + Cd);
                }
                mpbar += w * (mb + vcd);
                for (int i = 0; i < d; ++i) {
                    vbn[i] += w * mp * mvb[i];
                    for (int j = 0; j < d; ++j) Abar[i * 3 + j] += w * mvb[i] * dpos[j];
                }
                for (int c = 0; c < d; ++c) {
                    double Atm = 0.0; /* (A^T mvb)_c */
                    for (int i = 0; i < d; ++i) Atm += A[i * 3 + c] * mvb[i];
                    xbn[c] += gw[c] * inner - w * Atm;
                }
            }
            /* A = mp C - dt kappa vol P F^T */
            double* Cbn = an->C + 9 * p;
            double* Fbn = an->F + 9 * p;
            double Mb[9] = {0}, Pbar[9] = {0};
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    Cbn[i * 3 + j] += mp * Abar[i * 3 + j];
                    Mb[i * 3 + j] = -P->dt * kappa * P->p_vol * Abar[i * 3 + j];
                }
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    double pb = 0.0, fb = 0.0;
                    for (int k = 0; k < d; ++k) {
                        pb += Mb[i * 3 + k] * F[k * 3 + j];   /* (Mb F)_ij */
                        fb += Mb[k * 3 + i] * Pst[k * 3 + j]; /* (Mb^T P)_ij */
                    }
                    Pbar[i * 3 + j] = pb;
                    Fbn[i * 3 + j] += fb;
                }
            double phib = 0.0, Bpb[3] = {0, 0, 0};
            orc_stress_adjoint(d, G, K, F, phi[p], P->simp_q, P->simp_eps, mag + 3 * p, Bp, Pbar, Fbn,
                               &phib, g_mag + 3 * p, Bpb);
            /* B_p = B_a + G (x_p - x_c): dL/dB_a, dL/dG and the x_p term */
            double* tBap = tBa + 3 * (size_t)(p - p0);
            double* tGp = tG ? tG + 18 * (size_t)(p - p0) : NULL;
            for (int i = 0; i < d; ++i) tBap[i] = Bpb[i];
            if (Gf) {
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j) {
                        if (tGp) tGp[3 * i + j] = Bpb[i] * (sn->x[3 * p + j] - 0.5);
                        xbn[j] += Gf[3 * i + j] * Bpb[i];
                    }
                /* f = c G^T (F B~_r), c = phi^q V / mu0 */
                const double* Br = mag + 3 * p;
                double c = ipow(phi[p], P->simp_q) * P->p_vol / MU0;
                double FB[3] = {0, 0, 0}, Gfb[3] = {0, 0, 0}, fraw = 0.0;
                for (int i = 0; i < d; ++i)
                    for (int k = 0; k < d; ++k) FB[i] += F[3 * i + k] * Br[k];
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j) Gfb[i] += Gf[3 * i + j] * fbar[j]; /* G fbar */
                for (int i = 0; i < d; ++i) {
                    fraw += Gfb[i] * FB[i]; /* fbar . G^T F B~_r */
                    for (int k = 0; k < d; ++k) {
                        Fbn[3 * i + k] += c * Gfb[i] * Br[k];
                        g_mag[3 * p + k] += c * Gfb[i] * F[3 * i + k];
                    }
                    if (tGp)
                        for (int j = 0; j < d; ++j) tGp[9 + 3 * i + j] = c * FB[i] * fbar[j];
                }
                double dsdphi = P->simp_q > 0 ? P->simp_q * ipow(phi[p], P->simp_q - 1) : 0.0;
                phib += dsdphi * P->p_vol / MU0 * fraw;
            }
            g_phi[p] += phib + mpbar * P->rho0 * P->p_vol;
        }
        for (int p = p0; p < p1; ++p) {
            const double* tBap = tBa + 3 * (size_t)(p - p0);
            for (int i = 0; i < d; ++i) gBa[i] += tBap[i];
            if (Gf && gGf) {
                const double* tGp = tG + 18 * (size_t)(p - p0);
                for (int e = 0; e < 9; ++e) gGf[e] += tGp[e];
                for (int e = 0; e < 9; ++e) gGf[e] += tGp[9 + e];
            }
        }
        free(tBa);
        free(tG);
    }
    free(Vbar);
    free(mbar);
    free(mvbar);
    return ORC_OK;
}

/* loss seed on the state after substep n (n in 1..N), added into a. */
static void loss_seed(const sim_t* S, int n, const state_t* s, const double* phi, const double* target,
                      const double* dloss, const double* M, adj_t* a, double* g_phi) {
    const orc_params* P = S->P;
    int d = P->dim;
    for (int inst = 0; inst < S->n_inst; ++inst) {
        int p0 = S->offs[inst], p1 = S->offs[inst + 1];
        if (P->loss_kind == 1) {
            if (!(M[inst] > 0.0)) continue;
            double mx = 0.0;
            for (int p = p0; p < p1; ++p) mx += particle_mass(P, phi[p]) * s->v[3 * p];
            double vbar = mx / M[inst];
            for (int p = p0; p < p1; ++p) {
                double mp = particle_mass(P, phi[p]);
                a->v[3 * p] += -P->dt * mp / M[inst] * dloss[inst];
                /* dL/dm_p through both the numerator and M (Eq. 40) */
                g_phi[p] += -P->dt * (s->v[3 * p] - vbar) / M[inst] * dloss[inst] * P->rho0 * P->p_vol;
            }
        } else if (n == P->n_steps && p1 > p0) {
            for (int p = p0; p < p1; ++p)
                for (int c = 0; c < d; ++c) {
                    double e = s->x[3 * p + c] - (target ? target[3 * p + c] : 0.0);
                    a->x[3 * p + c] += 2.0 * e / (p1 - p0) * dloss[inst];
                }
        }
    }
}

/*
 * Gradients of sum_i dloss[i] * loss_i with respect to phi [N], mag [N][3],
 * field [n_inst][n_steps][3], and (if non-NULL) x0, v0 [N][3].
 * Recomputes the forward with a checkpoint every ckpt_every substeps
 * (deterministic, so it reproduces the forward bit for bit).
 */
int orc_backward(const orc_params* P, int n_inst, const int* counts, const double* x0,
                 const double* v0, const double* phi, const double* mag, const double* field,
                 const double* target, const double* dloss, int ckpt_every, double* g_phi,
                 double* g_mag, double* g_field, double* g_x0, double* g_v0) {
    sim_t S;
    int st = sim_init(&S, P, n_inst, counts);
    if (st != ORC_OK) return st;
    int N = S.N, T = P->n_steps;
    if (ckpt_every <= 0) ckpt_every = T > 0 ? T : 1;
    int n_ck = (T + ckpt_every - 1) / ckpt_every + 1;
    state_t* ck = (state_t*)calloc(n_ck, sizeof(state_t));
    state_t* seg = (state_t*)calloc(ckpt_every + 1, sizeof(state_t));
    for (int i = 0; i < n_ck; ++i)
        if (state_alloc(&ck[i], N) != ORC_OK) return ORC_ERR_OOM;
    for (int i = 0; i <= ckpt_every; ++i)
        if (state_alloc(&seg[i], N) != ORC_OK) return ORC_ERR_OOM;
    memset(g_phi, 0, sizeof(double) * N);
    memset(g_mag, 0, sizeof(double) * 3 * N);
    memset(g_field, 0, sizeof(double) * 3 * (size_t)n_inst * T);
    double* M = (double*)calloc(n_inst, sizeof(double));
    instance_mass(&S, phi, M);

    /* forward, keeping a checkpoint at every multiple of ckpt_every */
    state_t cur, nxt;
    state_alloc(&cur, N);
    state_alloc(&nxt, N);
    initial_state(&S, x0, v0, &cur);
    state_copy(&ck[0], &cur, N);
    int worst = ORC_OK;
    for (int n = 0; n < T; ++n) {
        st = substep(&S, n, &cur, phi, mag, field, &nxt);
        if (st == ORC_ERR_DOMAIN) { worst = st; goto done; }
        if (st != ORC_OK) worst = st;
        state_t t = cur; cur = nxt; nxt = t;
        if ((n + 1) % ckpt_every == 0) state_copy(&ck[(n + 1) / ckpt_every], &cur, N);
    }

    {
        adj_t ab, an;
        state_t tmpa, tmpb;
        state_alloc(&tmpa, N);
        state_alloc(&tmpb, N);
        ab.x = tmpa.x; ab.v = tmpa.v; ab.C = tmpa.C; ab.F = tmpa.F;
        an.x = tmpb.x; an.v = tmpb.v; an.C = tmpb.C; an.F = tmpb.F;
        state_zero(&tmpa, N);
        /* seed at the final state */
        if (T > 0) loss_seed(&S, T, &cur, phi, target, dloss, M, &ab, g_phi);
        for (int s0 = ((T - 1) / ckpt_every) * ckpt_every; T > 0 && s0 >= 0; s0 -= ckpt_every) {
            int s1 = s0 + ckpt_every < T ? s0 + ckpt_every : T;
            /* recompute the segment, storing every state */
            state_copy(&seg[0], &ck[s0 / ckpt_every], N);
            for (int n = s0; n < s1; ++n) substep(&S, n, &seg[n - s0], phi, mag, field, &seg[n - s0 + 1]);
            for (int n = s1 - 1; n >= s0; --n) {
                st = substep_adjoint(&S, n, &seg[n - s0], phi, mag, field, &ab, &an, g_phi, g_mag, g_field);
                if (st != ORC_OK) { worst = st; break; }
                if (n >= 1) loss_seed(&S, n, &seg[n - s0], phi, target, dloss, M, &an, g_phi);
                adj_t t = ab; ab = an; an = t;
            }
            if (st != ORC_OK && st != ORC_ERR_NUMERIC) break;
        }
        if (g_x0) memcpy(g_x0, ab.x, sizeof(double) * 3 * N);
        if (g_v0) memcpy(g_v0, ab.v, sizeof(double) * 3 * N);
        state_free(&tmpa);
        state_free(&tmpb);
    }
done:
    for (int i = 0; i < n_ck; ++i) state_free(&ck[i]);
    for (int i = 0; i <= ckpt_every; ++i) state_free(&seg[i]);
    free(ck);
    free(seg);
    free(M);
    state_free(&cur);
    state_free(&nxt);
    sim_free(&S);
    return worst;
}

/* ------------------------------------------------------------------ */
/* cell keys and the stable sort (the ordering definition)              */
/* ------------------------------------------------------------------ */

/*
 * Cell key of every particle, computed in FP32 exactly as defined for the
 * sort: base_a = floor(x_a * res - 0.5) in float arithmetic (one rounded
 * multiply, one rounded subtract), clamped to [0, res - 3];
 * key = inst * nb^d * bs^d + block-major linear index with block edge bs
 * (nb = ceil(res / bs) blocks per axis; blocks and cells inside a block are
 * both row-major with the last axis fastest).
 *   xf: float positions [d][N] (SoA).  Output keys [N] (int32).
 */
void orc_cell_keys(int d, int res, int bs, int n_inst, const int* counts, const float* xf, int N,
                   int* keys) {
    int nb = (res + bs - 1) / bs;
    long per_block = 1, n_blocks = 1;
    for (int a = 0; a < d; ++a) {
        per_block *= bs;
        n_blocks *= nb;
    }
    long per_inst = per_block * n_blocks;
    int inst = 0, end = counts[0];
    volatile float fres = (float)res;
    for (int p = 0; p < N; ++p) {
        while (p >= end && inst + 1 < n_inst) end += counts[++inst];
        long blk = 0, cel = 0;
        for (int a = 0; a < d; ++a) {
            volatile float prod = xf[(size_t)a * N + p] * fres; /* rounded to float */
            volatile float t = prod - 0.5f;                      /* rounded to float */
            int b = (int)floorf(t);
            if (b < 0) b = 0;
            if (b > res - 3) b = res - 3;
            blk = blk * nb + b / bs;
            cel = cel * bs + b % bs;
        }
        keys[p] = (int)(inst * per_inst + blk * per_block + cel);
    }
}

typedef struct { int key, id; } kid_t;

static int cmp_kid(const void* a, const void* b) {
    const kid_t* x = (const kid_t*)a;
    const kid_t* y = (const kid_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

/* Stable order by key (ties by original index): perm[new] = old. */
int orc_sort_perm(const int* keys, int N, int* perm) {
    kid_t* a = (kid_t*)malloc(sizeof(kid_t) * (N > 0 ? N : 1));
    if (!a) return ORC_ERR_OOM;
    for (int i = 0; i < N; ++i) {
        a[i].key = keys[i];
        a[i].id = i;
    }
    qsort(a, N, sizeof(kid_t), cmp_kid);
    for (int i = 0; i < N; ++i) perm[i] = a[i].id;
    free(a);
    return ORC_OK;
}
