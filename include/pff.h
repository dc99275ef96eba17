/*
 * pff.h -- C ABI of libpff, a GB300 (sm_103a) implementation of the staggered
 * per-load-step solve of quasi-static phase-field fracture of
 * W. B. Andrews and L. Pastewka, "Crack-path selection in phase-field models
 * for brittle fracture", arXiv:2203.16467.
 *
 * One problem = one periodic 2-D pixel grid (nx columns along x, ny rows along
 * y, pixel size dx) with a heterogeneous Young's modulus E(x), a uniform
 * Poisson ratio, a phase field phi (the paper's crack field) and a strain
 * eps = eps_bar + eps* (Sec. 3.1.1: the strain, not the displacement, is the
 * unknown).  A load step is one pass of the while-loop of Algorithm 4
 * (near-equilibrium evolution, Sec. 3.2.3):
 *   mechanics (Fourier-Galerkin Newton-CG, Sec. 3.1.1)
 *   -> rescale of eps when -F_phi exceeds its bound (Algorithm 4 lines 4-10)
 *   -> phase field (BCCG, Algorithm 1, Sec. 3.1.2)
 *   -> stiffness C-bar and strain increment (Algorithm 4 lines 12-14).
 *
 * Conventions shared by every entry point:
 *   - Fields are row-major with y the slow index: value (y, x) at y*nx + x.
 *   - Tensor fields (strain, stress) are 3 planes of nx*ny values in the order
 *     xx, yy, xy (tensor shear component, not engineering shear).
 *   - Host arrays are FP64 regardless of the problem's storage precision and
 *     are owned by the caller; the library copies in/out and keeps no pointer.
 *   - on_device != 0 means the pointer is a CUDA device pointer on the
 *     problem's device (FP64, same layout); the copy runs on the problem's stream.
 *   - The library owns all device memory of a problem; it is freed by
 *     pff_destroy_problem.  Device pointers returned by pff_get_device_ptr
 *     stay valid until then.
 *   - Every function returns PFF_OK (0) or a negative PFF_ERR_* code; no
 *     exception crosses the ABI.  pff_last_error(h) returns a message owned
 *     by the handle (valid until the next call on it).  A handle is not
 *     thread-safe; different handles may be used from different threads.
 *   - PFF_ERR_CUDA covers CUDA runtime errors, including a kernel launch that
 *     the runtime rejects (reported by the call that issued it, at its next
 *     synchronisation point, never as a non-converging solve).
 *   - Grid sizes: nx and ny are powers of two from 16 to 2048.
 *   - The library needs an sm_103a GPU; there is no CPU fallback.
 */
#ifndef PFF_H
#define PFF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PFF_OK = 0,
    PFF_ERR_INVALID_ARG = -1,
    PFF_ERR_OOM = -2,
    PFF_ERR_NOT_CONVERGED = -3,
    PFF_ERR_BARRIER_TIMEOUT = -4,
    PFF_ERR_CUDA = -5,
    PFF_ERR_STATE = -6
};

/* Storage / arithmetic precision of a problem. */
enum {
    PFF_FP64 = 0,   /* all fields and arithmetic in FP64 */
    PFF_MIXED = 1   /* fields and pointwise/FFT arithmetic in FP32.  Dot products
                       and norms: each product formed exactly (FMA split), each
                       thread's sum a compensated float pair, the pairs of a
                       block summed in double-float arithmetic (about 44
                       significant bits), block totals and the cross-block sum
                       in FP64.  Solver scalars, the driving-force field, its
                       maximum, x* and gamma in FP64.  Phase-field bound
                       decisions (the sign of the residual at the bound): in FP64
                       from the FP32 stored operands wherever the FP32 sign could
                       differ from it. */
};

/* Local fracture energy f(phi) (Eq. fracturelocal): AT1 f = phi, c_w = 8/3;
 * AT2 f = phi^2, c_w = 2 (the form whose optimal profile is Eq. AT2_analytical). */
enum { PFF_AT1 = 1, PFF_AT2 = 2 };

/* Energy split (Sec. 2.1, Eqs. isotropic_en, strain_spectral_en, vol_dev_en).
 * SPECTRAL_STRESSFREE and SPECTRAL_VOLDEV are the non-variational pairings of
 * Sec. 4.2: the strain-spectral crack driving force with the isotropic
 * (stress-free crack) or the volumetric-deviatoric contact model.  VOLDEV
 * reads Eq. vol_dev_en with the sums over the two in-plane components and the
 * 1/3 of the 3-D deviator (the form of the values quoted in Sec. 4.2.1). */
enum { PFF_ISOTROPIC = 0, PFF_SPECTRAL = 1, PFF_SPECTRAL_STRESSFREE = 2, PFF_VOLDEV = 3, PFF_SPECTRAL_VOLDEV = 4 };

/* Irreversibility (Eq. constraint_field): within the crack set phi >= 0.9, or
 * in the whole domain ("damage"). */
enum { PFF_CRACK_SET = 0, PFF_DAMAGE = 1 };

/* Field selectors for pff_get_fields / pff_get_device_ptr. */
enum {
    PFF_FIELD_STRAIN = 0,         /* eps = eps_bar + eps*, 3 planes */
    PFF_FIELD_EPS_STAR = 1,       /* eps*, 3 planes */
    PFF_FIELD_STRESS = 2,         /* sigma(eps, phi) of the contact model, 3 planes */
    PFF_FIELD_PHI = 3,            /* phi */
    PFF_FIELD_PSI_PLUS = 4,       /* psi_0^+(eps) of the crack-driving-force model */
    PFF_FIELD_DRIVING_FORCE = 5,  /* -F_phi(phi, eps) */
    PFF_FIELD_MODULUS = 6,        /* E */
    PFF_FIELD_ACTIVE = 7,         /* 1.0 where the last BCCG iterate had v = v_con and r > 0, else 0.0 */
    PFF_FIELD_UPDATE = 8          /* v = phi_new - phi_old of the last phase-field solve */
};

/* Model and solver parameters (Sec. 3.3).  pff_default_params fills the
 * paper's values: nu 0.2, G_c 1, ell 1, dx 1, tolerances 1e-6,
 * (dphi)_min 1e-3, (-F_phi)_max 0.7 G_c/ell, (-h' psi_0^+)_thresh 1 G_c/ell,
 * eta/dt = 2^-16 G_c/ell ((dt)_max = 2^16 eta/(G_c/ell)), C_broken <= 0 meaning
 * 0.01 * mean(E). */
typedef struct pff_params {
    double nu;                 /* Poisson ratio (plane strain Lame constants) */
    double Gc;                 /* critical energy release rate */
    double ell;                /* crack width parameter */
    double dx;                 /* pixel size */
    double mech_tol;           /* Newton stop: ||P sigma||_2 <= mech_tol * ||C_0 : eps_bar||_2 */
    double mech_cg_rtol;       /* inner CG relative tolerance of nonlinear (spectral-stress) Newton steps */
    int mech_max_newton;
    int mech_max_cg;
    double pf_tol;             /* BCCG stop: ||r||_2 <= max(pf_tol ||r^0||_2, pf_atol) */
    double pf_atol;
    int pf_max_iter;
    double eta_over_dt;        /* eta / dt of the backward-Euler phase-field step; < 0: default */
    double F_max;              /* (-F_phi)_max; < 0: default */
    double thresh;             /* (-h' psi_0^+)_thresh; < 0: default */
    double dphi_min;           /* (dphi)_min, with ||dphi||_1 = (dx/ell)^2 sum |dphi| */
    double C_broken;           /* termination stiffness; <= 0: 0.01 * mean(E) */
    double crack_set_threshold;/* 0.9 in Eq. constraint_field */
    double d_eps_bar[3];       /* strain increment (xx, yy, xy) */
    int compute_energies;      /* fill F_e and F_f in step reports (one extra scalar FFT pair per step) */
    int evolution;             /* PFF_NEAR_EQUILIBRIUM (Algorithm 4), PFF_ALTERNATING_MIN (Algorithm 2)
                                  or PFF_TIME_DEPENDENT (Algorithm 3) */
    double tol_am;             /* Tol_AM of Algorithm 2 (||dphi||_1 of an inner iteration) */
    int am_max_inner;          /* cap on the inner iterations of one increment */
    double dt_min, dt_max;     /* (dt)_min, (dt)_max of Algorithm 3 in units of eta/(G_c/ell) */
    double dphi_max;           /* (dphi)_max of Algorithm 3 */
    int pf_precondition;       /* 0 (default): BCCG exactly as Algorithm 1.  1: the same projected CG
                                  with the Fourier-space preconditioner (a_mean + 2 c ell^2 |2 pi q|^2)^-1
                                  applied to the residual masked to the free set (Polak-Ribiere beta
                                  in the preconditioned inner product): the same bound-constrained
                                  solution in 2-6x fewer iterations, one more FFT pair per
                                  iteration.  No counterpart in the paper. */
} pff_params;

/* Evolution methods (Sec. 3.2): one pff_step_load step is one pass of the
 * while-loop of Algorithm 4, one strain increment (outer iteration s) of
 * Algorithm 2, or one time step n of Algorithm 3. */
enum { PFF_NEAR_EQUILIBRIUM = 0, PFF_ALTERNATING_MIN = 1, PFF_TIME_DEPENDENT = 2 };

/* Per-load-step report.  eps_bar is the macroscopic strain the step ended
 * with before the increment (after any rescale); sig_bar is the mean stress
 * sigma(eps_n, phi_{n+1}) (Algorithm 4 line 12). */
typedef struct pff_step_report {
    double eps_bar[3];
    double sig_bar[3];
    double C_bar;
    double gamma;              /* rescale factor (1.0 when no rescale) */
    double dphi_L1;
    double F_e;                /* elastic energy sum psi dA of the contact model */
    double F_f;                /* fracture energy of Eq. Ff */
    double mF_max;             /* max of -F_phi before the rescale */
    double D_max;              /* max of -h' psi_0^+ before the rescale */
    double mech_res;           /* final ||P sigma||_2 */
    double pf_res;             /* final ||r||_2 of BCCG */
    int rescaled;
    int incremented;
    int newton_iters;
    int mech_cg_iters;
    int bccg_iters;
    int n_active;
    int istar;                 /* linear index of argmax -F_phi */
    int broken;                /* C_bar < C_broken */
    int status;                /* PFF_OK or PFF_ERR_NOT_CONVERGED */
    int bccg_clamp_iters;      /* BCCG iterations in which the projection onto v >= v_con changed v */
    double dt;                 /* time-dependent method: the time step for the next step (units of eta/(G_c/ell)) */
    int inner_iters;           /* alternating minimisation: inner iterations; time-dependent: phase-field tries */
    int bccg_full_iters;       /* BCCG iterations that evaluated J v explicitly (the others used
                                  r_new = r + alpha J p, exact when the projection changed nothing) */
} pff_step_report;

typedef struct pff_problem pff_problem;
typedef struct pff_batch pff_batch;

/* Fill *p with the paper's default parameters (Sec. 3.3). */
int pff_default_params(pff_params* p);

/* Create a problem of nx x ny pixels on the current CUDA device.
 * precision: PFF_FP64 or PFF_MIXED.  cuda_stream: a cudaStream_t (may be NULL
 * for the legacy default stream) on which every kernel and copy of this
 * problem is issued.  Initial state: E = 1, phi = 0, eps = 0, default params,
 * model AT1 / SPECTRAL / CRACK_SET.  PFF_ERR_OOM if device memory runs out. */
int pff_create_problem(int nx, int ny, int precision, void* cuda_stream, pff_problem** out);
int pff_destroy_problem(pff_problem* h);
const char* pff_last_error(pff_problem* h);
/* Grid size and precision of a problem. */
int pff_problem_info(pff_problem* h, int* nx, int* ny, int* precision);
/* Device bytes held by a problem of this size and precision (for admission). */
size_t pff_problem_bytes(int nx, int ny, int precision);

int pff_set_params(pff_problem* h, const pff_params* p);
int pff_get_params(pff_problem* h, pff_params* p);
/* fracture: PFF_AT1|PFF_AT2; split: PFF_ISOTROPIC|PFF_SPECTRAL|PFF_SPECTRAL_STRESSFREE;
 * irreversibility: PFF_CRACK_SET|PFF_DAMAGE (Sec. 2.1, Eq. constraint_field). */
int pff_set_model(pff_problem* h, int fracture, int split, int irreversibility);
/* Young's modulus field E(x) >= 0 with a positive mean, nx*ny values (zeros
 * appear in the crack of pff_init_crack with PFF_IC_MODULUS).  A field that is
 * negative or not finite anywhere returns PFF_ERR_INVALID_ARG and leaves the
 * stored field unchanged.  Host arrays of FP32 problems are copied as they are
 * into a device staging buffer of nx*ny doubles (part of the problem, counted
 * by pff_problem_bytes) and converted there; page-locked host memory makes the
 * copy a single DMA.  Returns after the copy: the caller may reuse its buffer. */
int pff_set_modulus_field(pff_problem* h, const double* E, int on_device);
/* Phase field, nx*ny values in [0, 1] (initial condition; default 0). */
int pff_set_phase_field(pff_problem* h, const double* phi, int on_device);

/* ---- Initial conditions (Sec. 4.1.1, Eq. init_crack; Sec. 4.2.2) ----
 * Horizontal crack centred at (xc, yc) (lengths in the unit of dx; grid point
 * (i, j) at (i dx, j dx)): phi_init = (1 - |r|/(2 ell))^2 where |r| <= 2 ell,
 * else 0, with ell the problem's parameter and
 *   PFF_CRACK_EDGE:    r = (max(x - length/2, 0), y), x, y from the centre, x in
 *                      [-Lx/2, Lx/2): the equation as printed, a notch from the
 *                      periodic cut to a rounded tip (the periodic
 *                      single-edge-notched specimen of Sec. 3.3);
 *   PFF_CRACK_SEGMENT: r = (max(|x| - length/2, 0), y), two rounded tips;
 *                      length 0 is the small void of Sec. 4.1.1.
 * target PFF_IC_PHASE_FIELD sets phi = phi_init; PFF_IC_MODULUS sets the crack
 * in E, E = h(phi_init) E0 = (1 - phi_init)^2 E0 (replacing the modulus field).
 * Computed on the device in FP64 on the problem's stream; synchronises it.
 * PFF_ERR_INVALID_ARG for an unknown target or shape, length < 0, E0 <= 0. */
enum { PFF_CRACK_SEGMENT = 0, PFF_CRACK_EDGE = 1 };
enum { PFF_IC_PHASE_FIELD = 0, PFF_IC_MODULUS = 1 };
int pff_init_crack(pff_problem* h, int target, int shape, double xc, double yc, double length, double E0);

/* ---- Microstructure generators (Sec. 3.3) ----
 * E = E0 xi from nx*ny standard-normal samples xi (drawn by the caller: host or
 * device FP64, row-major), low-pass filtered in Fourier space to the modes with
 * 0 < |q| <= 2 pi / L_cut (decided as kx^2 (Ly L_cut)^2 + ky^2 (Lx L_cut)^2 <=
 * (Lx Ly)^2), then
 *   PFF_MICRO_RANDOM:    xi_r = xi std_target / STD(xi) + 1 (population
 *                        standard deviation), values below 1 mapped to
 *                        1 - d D / (d^10 + D^10)^(1/10), d = 1 - xi_r,
 *                        D = 1 - xi_min (Eq. sigmoid);
 *   PFF_MICRO_TWO_PHASE: xi_p = sgn(xi), ac_iters iterations of Eq. ACsmooth
 *                        (explicit Allen-Cahn step, periodic 5-point Laplacian in
 *                        pixel units), xi_p := a xi_p + 1.
 * The result replaces the problem's modulus field.  All steps run on the
 * device in FP64 (the filter through the library's FFT passes) on the
 * problem's stream; temporary device scratch (about 4 nx ny doubles) is
 * allocated and freed inside the call, which synchronises the stream.
 * pff_default_micro_params fills the paper's values: L_cut 6 (in units of
 * ell = 1), std_target 0.3, xi_min 0.01, a 0.875, ac_iters 21, E0 1. */
enum { PFF_MICRO_RANDOM = 0, PFF_MICRO_TWO_PHASE = 1 };
typedef struct pff_micro_params {
    int kind;                  /* PFF_MICRO_RANDOM or PFF_MICRO_TWO_PHASE */
    double L_cut;              /* cutoff wavelength (unit of dx), > 0 */
    double std_target;         /* random: target standard deviation STD_t */
    double xi_min;             /* random: lower bound of the sigmoid floor, < 1 */
    double a;                  /* two-phase: xi_p := a xi_p + 1, 0 < a < 1 */
    int ac_iters;              /* two-phase: Allen-Cahn iterations, >= 0 */
    double E0;                 /* E = E0 xi, > 0 */
} pff_micro_params;
int pff_default_micro_params(pff_micro_params* mp);
int pff_generate_modulus(pff_problem* h, const pff_micro_params* mp, const double* noise, int noise_on_device);
/* Strain state: eps_star (3 planes, may be NULL for zero) and eps_bar[3] (host). */
int pff_set_strain(pff_problem* h, const double* eps_star, const double eps_bar[3], int on_device);
/* Reset the near-equilibrium Flag of Algorithm 4 (set once the trigger is met). */
int pff_set_flag(pff_problem* h, int flag);

/* Run n_steps steps of the problem's evolution method (by default load steps,
 * i.e. Algorithm 4 iterations); out (n_steps entries, may be NULL) receives a
 * report per step.  Stops early, returning the number of
 * steps done through *steps_done (may be NULL), once C_bar < C_broken.
 * Returns PFF_ERR_NOT_CONVERGED if a sub-solver hit its iteration cap (the
 * state is kept). */
int pff_step_load(pff_problem* h, int n_steps, pff_step_report* out, int* steps_done);

/* Single sub-problems on the current state (for parity checks of one solve):
 * the mechanics Newton-CG solve at the current eps_bar and phi (Sec. 3.1.1);
 * and the phase-field BCCG solve with the current strain and phi_con(phi)
 * (Sec. 3.1.2, Algorithm 1), which replaces phi by phi + v. */
int pff_solve_mechanics(pff_problem* h, pff_step_report* out);
int pff_solve_phase_field(pff_problem* h, pff_step_report* out);

/* Copy a field out (FP64, host; FP32 problems convert on the device, through
 * the staging buffer above).  Tensor fields fill 3*nx*ny values.  Returns when
 * host_out holds the values. */
int pff_get_fields(pff_problem* h, int which, double* host_out);
/* Device view of a stored field: *p receives the device pointer, *dtype 0 for
 * FP64 / 1 for FP32; tensor fields are 3 contiguous planes.  Only fields that
 * are stored (EPS_STAR, PHI, MODULUS) are available. */
int pff_get_device_ptr(pff_problem* h, int which, void** p, int* dtype);

/* Operator entry points on one problem's grid (single rows of the path):
 * pff_apply_projection: out = F^-1 Gamma F in, the compatibility projection of
 *   Sec. 3.1.1 applied to a 3-plane tensor field (Nyquist modes of Gamma are 0).
 * pff_apply_laplacian: out = nabla^2_N in (Sec. 3.1.2).
 * pff_constitutive: for strain eps (3 planes) and phi, returns the stress
 *   (3 planes), psi_0^+ (1 plane) and, if p3 != NULL, the tangent C:p (3 planes)
 *   of the problem's model (Sec. 2.1, Sec. 3.1.1); any output may be NULL.
 * All arrays are FP64 host arrays; the arithmetic runs in the problem's precision. */
int pff_apply_projection(pff_problem* h, const double* in3, double* out3);
int pff_apply_laplacian(pff_problem* h, const double* in, double* out);
int pff_constitutive(pff_problem* h, const double* eps3, const double* phi, const double* p3,
                     double* sig3, double* psi, double* tang3);

/* Kernel variants (no counterpart in the paper); both variants of a kind compute
 * the same method, only the summation order of their reductions differs
 * (results agree to the rounding of the storage precision, not bitwise).
 *   PFF_VARIANT_COLUMN_SHAPE: the 512-point FP32 column pass with ncomp (1 or 3)
 *     components (grid_n = 512): variant 0 = four spectrum columns per
 *     256-thread block (default), 1 = two columns per 128-thread block (twice the
 *     blocks: more SMs busy when a launch carries one simulation).
 *   PFF_VARIANT_BCCG_PASSES (grid_n, ncomp ignored): variant 0 = Algorithm 1 in
 *     three operator passes per iteration (the step length alpha from the column
 *     pass by Parseval, the iterate fused into the J p pass; default), 1 = four
 *     passes (alpha from p.Jp summed in real space, the iterate in its own
 *     elementwise kernel; what the preconditioned option always uses).
 * Takes effect at the next launch; captured CUDA graphs are re-captured.
 * Synchronises the device.  Unsupported arguments: PFF_ERR_INVALID_ARG. */
enum { PFF_VARIANT_COLUMN_SHAPE = 2, PFF_VARIANT_BCCG_PASSES = 3 };
int pff_set_kernel_variant(int kind, int grid_n, int ncomp, int variant);
int pff_get_kernel_variant(int kind, int grid_n, int ncomp, int* variant);

/* Autotuner of the kernel variants on ordinary load steps of a batch: the eight
 * combinations (one-component column shape, three-component column shape, BCCG
 * passes) = (c & 1, (c >> 1) & 1, (c >> 2) & 1), c = 0..7, run in steps_each
 * rounds; in each round every combination runs two load steps in the batch's own
 * launch configuration (the first after the change is not timed: graphs are
 * re-captured), odd rounds in reverse order, so that all combinations are
 * measured on the same stretch of the simulations; scored by pixel-iterations per
 * second of host wall time (steps_each >= 2 recommended).  The
 * best combination stays set and is returned in chosen[3]; scores[8] (optional)
 * receives the eight scores.  reports / steps_done as pff_batch_autotune (per
 * slot, 16 steps_each entries).  The steps advance the batch's simulations. */
int pff_batch_autotune_kernels(pff_batch* b, int steps_each, int* chosen, double* scores, pff_step_report* reports,
                               int* steps_done);

/* Batching: several problems (any sizes, precisions, models) advanced
 * together.  pff_batch_admit fails with PFF_ERR_OOM if the problem's device
 * bytes do not fit the remaining budget or PFF_ERR_STATE if all slots are
 * taken.  pff_batch_step runs n_steps load steps of every admitted, not yet
 * broken problem; problems of equal size and precision share every kernel
 * launch.  reports: max_slots * n_steps entries, slot-major (may be NULL);
 * steps_done: max_slots entries (may be NULL).  Batches advance near-equilibrium
 * problems only (admission rejects other evolution methods). */
int pff_create_batch(int max_slots, size_t hbm_budget, void* cuda_stream, pff_batch** out);
int pff_destroy_batch(pff_batch* b);
int pff_batch_admit(pff_batch* b, pff_problem* h, int* slot);
int pff_batch_release(pff_batch* b, int slot);
int pff_batch_step(pff_batch* b, int n_steps, pff_step_report* reports, int* steps_done);
/* Launch grouping of a batch: problems of one shape are split into groups of at
 * most max_problems_per_group (0, the default: one group per shape).  Each group
 * shares every kernel launch and advances in lock step; different groups run
 * on their own streams and host threads and overlap on the device. */
int pff_batch_set_group_size(pff_batch* b, int max_problems_per_group);
/* Picks the launch grouping of a batch by measurement: for each of the
 * n_candidates group sizes (as for pff_batch_set_group_size) it runs one
 * untimed load step (regrouping recaptures the graphs) and steps_each timed load
 * steps of every admitted simulation, scores the candidate by pixels x (mechanics
 * CG + Newton + BCCG iterations) per second of wall time, and keeps the fastest
 * (*chosen, may be NULL).  The n_candidates x (steps_each + 1) steps are
 * ordinary load steps of the simulations (the grouping does not change any
 * simulation's arithmetic); reports: max_slots x n_candidates x (steps_each + 1)
 * entries, slot-major, filled up to steps_done[slot] (both may be NULL).
 * Returns PFF_ERR_NOT_CONVERGED like pff_batch_step.  No counterpart in the
 * paper (a tuning aid of this library). */
int pff_batch_autotune(pff_batch* b, const int* group_sizes, int n_candidates, int steps_each, int* chosen,
                       pff_step_report* reports, int* steps_done);

/* Collocation Laplacian without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- for
 * example a framework that has already reserved all device memory for its own
 * pool, or a latency-critical loop that cannot afford the device-wide
 * synchronisation an allocation may cause.
 *   out_dev = nabla^2_N in_dev on an nx x ny periodic grid of spacing dx, both
 *   FP64 device arrays of nx*ny values (row-major, y slow), owned by the caller.
 * Scratch (one half spectrum, about 2.2 MB), twiddle table and kernel
 * descriptor are static device arrays that every GPU loading the library holds
 * until the process exits.  The first call on a device sets them up (with that
 * device current): make that first call before any stream capture.  Calls
 * share the arrays, so calls whose kernels overlap on the GPU (different
 * streams, or different host threads) race; serialise them.  Nothing in the
 * scratch needs to start at zero.  Sizes other than powers of two from 16 to
 * PFF_NOALLOC_MAX_N are rejected with PFF_ERR_INVALID_ARG before any launch;
 * *err_msg (optional) then points to a static message.  Kernels run on
 * cuda_stream (may be NULL); the call does not synchronise. */
#define PFF_NOALLOC_MAX_N 512
int pff_apply_laplacian_noalloc(int nx, int ny, double dx, const double* in_dev, double* out_dev,
                                void* cuda_stream, const char** err_msg);
/* The same in FP32 (the storage precision of PFF_MIXED problems): in_dev and
 * out_dev are caller-owned FP32 device fields of nx*ny values; its own static
 * scratch (about 1.1 MB), with the same sharing rule and errors as above. */
int pff_apply_laplacian_noalloc_f32(int nx, int ny, double dx, const float* in_dev, float* out_dev,
                                    void* cuda_stream, const char** err_msg);

/* Library-wide counters: kernel launches issued since load (for benchmarks). */
unsigned long long pff_kernel_launches(void);

/* Replay the fixed per-iteration launch sequences of the CG and BCCG loops
 * from captured CUDA graphs (default on = 1: plain graphs, in which the
 * explicit J v - b chain of a BCCG iteration that does not need it launches and
 * returns at once).  on = 2 puts that chain in a conditional graph node that a
 * one-thread kernel opens only in iterations that need it (measured slower on
 * GB300 than the returning kernels); 0 launches every kernel directly.  Results do not depend on the
 * setting.  Graphs are used only on problems or batches created with a
 * non-NULL stream and while kernel timing is off.  Synchronises the device. */
int pff_set_graphs(int on);

/* Launch the FP32 FFT-pass and elementwise kernels with programmatic stream
 * serialization (default on): each kernel's blocks may be scheduled while its
 * predecessor on the stream is still running and wait on the device for its
 * completion before touching any field, which hides the launch latency between
 * the short kernels of one solver iteration.  Applies to direct launches only
 * (graph replays keep plain edges, which measured faster).  Results do not
 * depend on the setting.  Off while kernel timing is on.  Synchronises the
 * device.  No counterpart in the paper (an execution detail of this library). */
int pff_set_pdl(int on);

/* Solve the phase-field sub-problem of a single FP32 512 x 512 problem (a
 * problem, or a batch group of one) in one persistent cooperative launch
 * (default off): the BCCG iterations of Algorithm 1 run without kernel
 * boundaries, their phases separated by grid barriers that carry the
 * reductions.  Measured slower than the per-phase kernels on GB300 (94.6 vs
 * 39.4 us per iteration of one simulation when the launch takes an eighth of
 * the device, as it must for eight simulations to run side by side), because a
 * phase then runs several row items one after another per block.  The
 * summation order of the dot products differs from the per-phase kernels (both
 * are deterministic).  Barrier waits are bounded (about two seconds); a
 * timeout ends the solve with PFF_ERR_BARRIER_TIMEOUT.  When the device cannot
 * host the launch the per-phase kernels run instead.  Synchronises the device.
 * No counterpart in the paper. */
int pff_set_persistent(int on);

/* Mechanics sub-problem of FP32 512 x 512 problems in one launch per solve
 * (default off): one thread-block cluster of 16 CTAs per problem keeps the
 * three-component half spectrum in distributed shared memory, so the column
 * FFTs and the projection Gamma (Sec. 3.1.1) never move the spectrum through
 * HBM, and the Newton rounds and CG iterations (Eqs. mech_newton,
 * elasticity_newton_linear) run inside the launch with FP64 cluster
 * reductions.  The CG step lengths use p.Ap = p.(C_m:p) and r.Ap = r.(C_m:p),
 * exact for iterates in the range of the projection, and q.q from the
 * projected modes (Parseval); the stopping tests are those of the per-kernel
 * path.  Measured slower than the per-kernel path on GB300 (164 vs 53 us per
 * CG iteration of one problem): the spectrum fills the shared memory of each
 * SM, which then hosts one 8-warp CTA whose row steps are latency-bound, and
 * the spectrum that the per-kernel path moves mostly stays in L2.  on = 0
 * (default) selects the per-kernel path (three kernels per CG iteration) for
 * every problem.  Problems of other sizes or FP64 problems always use the
 * per-kernel path, as does a device that cannot host a 16-CTA cluster of
 * about 210 KB of shared memory per CTA.  Synchronises the device.  No
 * counterpart in the paper. */
int pff_set_cluster_mechanics(int on);

/* Wait limit of every grid barrier of the persistent solve, in SM clock cycles
 * (cycles > 0; 0 restores the default of 4e9 cycles, about two seconds at the
 * maximum clock).  A block that is not released within the limit sets the
 * problem's abort flag and returns; the other blocks return at their next
 * barrier, the solve ends with PFF_ERR_BARRIER_TIMEOUT, the phase field is left
 * unchanged and the handle stays usable.  A short limit (one cycle) makes the
 * first barrier time out, which tests use to exercise that path.  Takes effect
 * at the next launch.  Negative values: PFF_ERR_INVALID_ARG.  No counterpart in
 * the paper. */
int pff_set_barrier_spin_limit(long long cycles);

/* Kernel timing for benchmarks.  When enabled, every launch of the library is
 * bracketed by CUDA events on its own stream; pff_timing_read returns the
 * summed device time (ms) and the launch count of one kernel class since the
 * last reset.  family: 0 row-forward (FFT along x with a fused prologue),
 * 1 row-inverse (inverse FFT along x with a fused epilogue), 2 column pass,
 * 3 elementwise; op: the step within the family, in load-step order
 * (row-forward: 0 Newton residual, 1 mechanics CG, 2 phi, 3 BCCG direction,
 * 4 BCCG iterate; row-inverse: 0 Newton, 1 CG, 2 Laplacian, 3 energy,
 * 4 BCCG direction, 5 BCCG residual; column: 0 Newton, 1 CG, 3 driving force,
 * 4 BCCG; elementwise: 0 fold, 1 BCCG start, 2 post-step, 3 driving-force
 * maximum).  Enabling, resetting and reading synchronize the device. */
int pff_timing_enable(int on);
int pff_timing_reset(void);
int pff_timing_read(int family, int op, double* total_ms, unsigned long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* PFF_H */
