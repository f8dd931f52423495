/*
 * fftg: FFT-Galerkin Newton-CG solver for periodic small-strain J2
 * micromechanics on one GB300 GPU (sm_103a).
 *
 * The method is that of Zeman, de Geus, Vondrejc, Peerlings and Geers,
 * "A finite element perspective on non-linear FFT-based micromechanical
 * simulations" (arXiv:1601.05970). A periodic cell of N^3 voxels (N odd,
 * a product of 3s and 5s, 3 <= N <= 243) with a two- or more-phase
 * microstructure is loaded by a macroscopic strain E; the library solves the
 * nodal equilibrium G sigma(E + eps*) = 0 (Eq. nodal_equilibrium_equations)
 * for the compatible fluctuation eps* by the incremental Newton-CG scheme of
 * Algorithm 1, with the J2 elasto-plastic law of Section 4.2 (linear
 * isotropic hardening), and returns the homogenised stress (Eq. trapz: the
 * nodal mean of sigma). The finite-strain extension (deformation gradient,
 * first Piola-Kirchhoff stress) is declared in fftg_fs.h.
 *
 * Conventions shared by every entry point:
 *  - A symmetric tensor is 6 doubles in the order (11, 22, 33, 23, 13, 12),
 *    tensor (not engineering, not Mandel) components.
 *  - A field is [6][N][N][N] (component slowest, then x1, x2, x3 fastest);
 *    a scalar field is [N][N][N].
 *  - Return value: FFTG_OK (0) or a negative FFTG_E* code. On any error the
 *    committed state (E, eps*, plastic history) is left as it was.
 *  - The caller owns every host array; the library copies what it needs.
 *    A handle owns (or borrows, see fftg_options.workspace) its device
 *    memory. One handle is used from one host thread at a time.
 *  - Device pointers (the fftg_op_* calls) are plain CUDA device addresses
 *    on the handle's device, in the handle's stream order.
 */
#ifndef FFTG_H
#define FFTG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define FFTG_OK               0
#define FFTG_EINVAL          -1  /* bad argument: even N, N not 3^a 5^b, phase id, tolerance <= 0 */
#define FFTG_ENOMEM          -2  /* device allocation failed or workspace too small */
#define FFTG_ENOCONV_NEWTON  -3  /* Newton reached max_newton without meeting tol_newton */
#define FFTG_ENOCONV_CG      -4  /* a CG solve reached max_cg without meeting its tolerance */
#define FFTG_ENAN            -5  /* a residual or norm became NaN or Inf */
#define FFTG_ECUDA           -6  /* a CUDA call failed */
#define FFTG_ESTATE          -7  /* call out of order (e.g. tangent before any step) */

/* ---------------------------------------------------------------- precision */
#define FFTG_SOLVER_CG 0          /* conjugate gradients (Section 2.5) */
#define FFTG_SOLVER_RICHARDSON 1  /* basic scheme (Section 3.2), comparison only */

#define FFTG_FP64   0  /* every step in FP64 */
#define FFTG_MIXED  1  /* FP32 inner CG (FFT, projection, tangent contraction);
                          FP64 return mapping, Newton test and homogenised
                          stress, and a residual G sigma from FP64 data with
                          double-float FFTs (FFTG_DD): Newton acts as
                          iterative refinement */
#define FFTG_DD     2  /* fftg_op_project only: FP64 buffers, FFTs in
                          double-float arithmetic (pairs of FP32 numbers,
                          about 48 significant bits), as in the residual of
                          the FFTG_MIXED path */

/* ---------------------------------------------------------------- fields */
#define FFTG_FIELD_STRAIN  0  /* total strain E + eps*, [6][N^3] */
#define FFTG_FIELD_STRESS  1  /* stress at the committed state, [6][N^3] */
#define FFTG_FIELD_EPBAR   2  /* accumulated plastic strain, [N^3] */
#define FFTG_FIELD_EPS_P   3  /* plastic strain tensor, [6][N^3] */
#define FFTG_FIELD_TANGENT 4  /* compact consistent tangent of the last stress
                                 update (Section 4.2), [7][N^3]: K', 2G_eff,
                                 w11, w22, w23, w13, w12, with C = |K'| I(x)I +
                                 2G_eff I_d - sign(K') w(x)w and w33 =
                                 -(w11 + w22); converted to FP64 from the inner
                                 precision it is stored in (FP32 in
                                 FFTG_MIXED). FFTG_ESTATE before any update */

typedef struct fftg_handle fftg_handle;

/* Constitutive models of Section 4 (fftg_phase.model). */
#define FFTG_MODEL_J2 0          /* J2 elasto-plasticity, Section 4.2 */
#define FFTG_MODEL_NLELASTIC 1   /* non-linear elasticity, Section 4.1 */
#define FFTG_MODEL_VISCO 2       /* visco-plasticity, Section 4.3 */

/* One material phase.
 * FFTG_MODEL_J2 (Section 4.2): C_e = K I(x)I + 2G I_d, yield function
 *   Phi = sigma_eq - (sigma_y + H epbar^n). n = 1 is linear hardening, whose
 *   return is in closed form; for other n the scalar return equation is
 *   solved for dgamma by a Newton iteration kept inside a bracket. A phase
 *   with sigma_y >= 1e300 is linear elastic. Uses K, G, sigma_y, H, n.
 * FFTG_MODEL_NLELASTIC (Section 4.1): sigma = K tr(eps) I +
 *   sigma_y (eps_eq / eps0)^n N, N = 2/3 eps_d / eps_eq; no history. Uses
 *   K, sigma_y (the reference stress sigma_0), eps0, n.
 * FFTG_MODEL_VISCO (Section 4.3): the elasticity of Section 4.2 with
 *   Norton's rule gamma_dot = (eps0 / t0) (sigma_eq / sigma_y)^(1/n),
 *   integrated by backward Euler over the time step fftg_options.dt of each
 *   increment. Uses K, G, sigma_y (the reference stress), eps0, t0, n.
 * Parameters a model does not use are ignored. */
typedef struct {
    double K;        /* bulk modulus, > 0 */
    double G;        /* shear modulus, > 0 (J2, VISCO) */
    double sigma_y;  /* J2: initial yield stress sigma_0; NLELASTIC, VISCO:
                        reference stress sigma_0; > 0 */
    double H;        /* J2: hardening modulus, >= 0 */
    double n;        /* J2: hardening exponent; NLELASTIC: exponent; VISCO:
                        strain-rate sensitivity; > 0 */
    double eps0;     /* NLELASTIC, VISCO: reference strain eps_0, > 0 */
    double t0;       /* VISCO: reference time t_0, > 0 */
    int    model;    /* FFTG_MODEL_* (0 = J2) */
} fftg_phase;

typedef struct {
    int    precision;       /* FFTG_FP64 or FFTG_MIXED (default FFTG_MIXED) */
    int    max_newton;      /* Newton iteration cap per increment (default 50) */
    int    max_cg;          /* CG iteration cap per solve (default 2000) */
    double cg_inner_floor;  /* FFTG_MIXED: the FP32 CG tolerance is
                               max(tol_cg, cg_inner_floor) (default 1e-5) */
    int    fixed_cg;        /* > 0: every CG solve runs exactly this many
                               iterations (parity mode); 0 = off */
    int    fixed_newton;    /* > 0: every increment runs exactly this many
                               Newton iterations (parity mode); 0 = off */
    void*  stream;          /* cudaStream_t the handle works in; NULL = the
                               legacy default stream */
    void*  workspace;       /* optional device memory of at least
                               fftg_workspace_size() bytes, 256-byte aligned,
                               owned by the caller and kept alive until
                               fftg_destroy; NULL = the library allocates */
    size_t workspace_bytes;
    int    nrhs_tangent;    /* right-hand sides held for fftg_tangent: 0 (no
                               tangent), or 6 (default 6) */
    int    cg_graph;        /* 1 (default): run each CG solve as one CUDA graph
                               whose conditional WHILE node loops on the device
                               (no host round trip per iteration); 0: enqueue
                               iterations in chunks from the host. Profiling
                               (fftg_profile_enable) uses the chunked path. */
    double dt;              /* time step of each increment, for rate-dependent
                               phases (FFTG_MODEL_VISCO), > 0 (default 1) */
    int    solver;          /* linear solver of each Newton iteration (and of
                               fftg_tangent): FFTG_SOLVER_CG (default), or
                               FFTG_SOLVER_RICHARDSON, the basic scheme of
                               Section 3.2 as a comparison: Richardson's
                               iteration with the reference medium
                               C_ref = (lambda_min + lambda_max)/2 I_s updated
                               at every Newton iteration from the extreme
                               eigenvalues of the local tangents. It needs
                               positive definite tangents (else FFTG_ENAN) and
                               takes O(lambda_max/lambda_min) iterations where
                               CG takes O(sqrt(lambda_max/lambda_min)). */
} fftg_options;

/* Per-increment diagnostics of the last fftg_step (Algorithm 1). */
#define FFTG_MAX_NEWTON_LOG 64
typedef struct {
    int    status;                              /* return code of the step */
    int    newton_iters;                        /* linear solves performed */
    int    cg_iters;                            /* sum over the solves */
    int    cg_per_newton[FFTG_MAX_NEWTON_LOG];
    double newton_norm[FFTG_MAX_NEWTON_LOG];    /* ||d eps*|| / ||E||_field, Algorithm 1 Newton test */
    double residual[FFTG_MAX_NEWTON_LOG];       /* ||G sigma|| / ||sigma|| (Table 3 analogue) */
    double cg_relres[FFTG_MAX_NEWTON_LOG];      /* final recursive ||r||/||r0|| of each solve */
    int    cg_status[FFTG_MAX_NEWTON_LOG];      /* how each solve ended: 1 converged, 2 max_cg
                                                   reached, 4 stagnated (FFTG_MIXED inner solve:
                                                   no progress for 25 iterations, or a
                                                   non-positive <p, Ap> from rounding) */
} fftg_stats;

/* Fill *opt with the defaults listed above. */
void fftg_default_options(fftg_options* opt);

/* Library version string. */
const char* fftg_version(void);

/* Device bytes a handle of this size needs (workspace for fftg_options). */
int fftg_workspace_size(int N, const fftg_options* opt, size_t* bytes);

/* Create a cell: validates N (odd 3^a 5^b, Section 2.3: odd grids give a
 * conforming trigonometric space with no Nyquist mode), copies the phase
 * map (uint8 [N][N][N], x1 slowest, values < nphase) and the nphase
 * materials to the device, and zeroes E, eps* and the plastic history
 * (Algorithm 1, initial conditions). */
int fftg_create(fftg_handle** h, int N, const uint8_t* phase, int nphase,
                const fftg_phase* mats, const fftg_options* opt);

/* One load increment (Algorithm 1, one pass of the increment loop) of a
 * single-cell handle (FFTG_EINVAL for a batch):
 * E <- E + dE, Newton iterations on G sigma(E + eps*) = 0 starting from the
 * previous eps* (Alg. 1 "initial guess for the next increment"), each
 * solving G C d eps* = -G sigma (Eq. linear_system) by CG to the relative
 * residual tol_cg (the CG test of Algorithm 1), until
 * ||d eps*|| / ||E||_field <= tol_newton (its Newton test). Then the stress at the converged strain is homogenised into
 * sigma_out[6] and the plastic history is committed.
 * newton_iters / cg_iters may be NULL. On error nothing is committed. */
int fftg_step(fftg_handle* h, const double dE[6], double tol_newton,
              double tol_cg, double sigma_out[6], int* newton_iters,
              int* cg_iters);

/* Diagnostics of the last increment of the selected cell. */
int fftg_last_stats(fftg_handle* h, fftg_stats* out);

/* ---------------------------------------------------------------- batches
 * A handle may hold ncells cells of the same grid (own microstructure, own
 * state, own Newton and CG iteration). Every kernel launch of the path then
 * covers all of them; a cell that has converged skips the work of later
 * launches. The single-cell calls (fftg_step excepted) act on the cell
 * chosen by fftg_select_cell (default 0). Not in the paper: the batching
 * is how many RVE problems (FE^2 Gauss points) share the GPU.
 * phase is [ncells][N][N][N]. */
int fftg_workspace_size_batch(int N, int ncells, const fftg_options* opt, size_t* bytes);
int fftg_create_batch(fftg_handle** h, int N, int ncells, const uint8_t* phase, int nphase,
                      const fftg_phase* mats, const fftg_options* opt);
int fftg_batch_size(const fftg_handle* h);
int fftg_select_cell(fftg_handle* h, int cell);
/* One load increment for every cell: dE [ncells][6]; outputs
 * sigma_out [ncells][6], newton_iters / cg_iters [ncells] (may be NULL),
 * status [ncells] (0 or FFTG_E*; a failed cell is not committed, the others
 * are). Returns 0 or the first cell's error. */
int fftg_batch_step(fftg_handle* h, const double* dE, double tol_newton, double tol_cg,
                    double* sigma_out, int* newton_iters, int* cg_iters, int* status);

/* 6x6 macroscopic algorithmic tangent dSigma/dE at the last converged
 * increment (not in the paper; the quantity an FE^2 macro solver needs).
 * Column j perturbs tensor component j (a shear perturbs (i,j) and (j,i)
 * together by 1): the six right-hand sides -G(C : E_j) are solved in one
 * batched CG with the consistent tangent C of the converged state, and
 * C_out[i*6 + j] = mean(C : (E_j + d eps_j))_i. Row-major. */
int fftg_tangent(fftg_handle* h, double tol_cg, double C_out[36], int* cg_iters);

/* Checkpoint/restore of the committed state: E[6], eps*[6][V], eps_p[6][V],
 * epbar[V] as FP64, in that order (fftg_state_bytes() bytes). */
size_t fftg_state_bytes(const fftg_handle* h);
int fftg_get_state(fftg_handle* h, void* host_buf, size_t bytes);
int fftg_set_state(fftg_handle* h, const void* host_buf, size_t bytes);

/* Reset the committed state of the selected cell to the undeformed one:
 * E = 0, eps* = 0, no plastic history (the microstructure is kept), as if
 * the cell had just been created; the next fftg_step starts the load path
 * again. Keeps the handle's cached CUDA graphs. */
int fftg_reset_state(fftg_handle* h);

/* Copy a committed field to host memory (FFTG_FIELD_*; FP64), or the
 * tangent of the last stress update (FFTG_FIELD_TANGENT). */
int fftg_get_field(fftg_handle* h, int which, double* host_out);

void fftg_destroy(fftg_handle* h);

/* ---------------------------------------------------------------- operators
 * The steps of the path on caller device buffers, for callers that drive
 * their own iteration and for parity tests. All run in the handle's stream
 * and return after enqueueing, except where a host output is written (then
 * the stream is synchronised). `precision` selects FP64 (double buffers) or
 * FP32 (float buffers) for the FFT-side operators. */

/* out = G tau (Eq. discrete_projection) for a real field tau [6][N^3]:
 * forward DFT, Ghat of Appendix A Eq. (FT_projection) at every frequency
 * (Ghat(0) = 0), inverse DFT. tau and out may alias. precision: FFTG_FP64
 * (double buffers), FFTG_MIXED (float buffers) or FFTG_DD (double buffers,
 * double-float FFTs). */
int fftg_op_project(fftg_handle* h, int precision, const void* tau_dev, void* out_dev);

/* Evaluate the constitutive law at E_trial + eps where E_trial = E + dE
 * (dE may be NULL) and eps [6][N^3] FP64 is a device field (NULL = the
 * committed eps*), against the committed history: writes sigma [6][N^3]
 * FP64 (may be NULL) and keeps the consistent tangent (Section 4.2) for
 * fftg_op_matvec. */
int fftg_op_constitutive(fftg_handle* h, const double dE[6], const double* eps_dev,
                         double* sigma_dev);

/* q = G (C : p) with the tangent of the last fftg_op_constitutive (or of
 * the last converged increment), p and q [6][N^3] in `precision`; writes
 * <p, q> (Frobenius, summed over voxels) to *pq when pq is not NULL. */
int fftg_op_matvec(fftg_handle* h, int precision, const void* p_dev, void* q_dev,
                   double* pq);

/* ---------------------------------------------------------------- groups
 * One increment of every cell of several batch handles (cells of several
 * grid sizes) as ONE CUDA graph launch: per handle a branch of the graph
 * runs Algorithm 1's Newton loop and each Newton iteration's CG loop as
 * device-side WHILE loops (conditional graph nodes), with the Newton test
 * taken per cell on the device, then commits the converged cells; the
 * branches of different handles run concurrently. The results are those of
 * fftg_batch_step on each handle (the same kernels in the same order). The
 * graph is built at the first step and again when the tolerances change;
 * it holds the handles' buffers, so the handles must outlive the group and
 * not be used on their own streams while a group step runs (the call
 * synchronises them first). Handles must use the CG solver (not the basic
 * scheme). Not in the paper: it serves the FE^2 setting of Section 1, where
 * many RVEs of different sizes take one increment per macroscopic step. */
typedef struct fftg_group fftg_group;
int fftg_group_create(fftg_group** g, fftg_handle* const* handles, int n);
/* dE, run, sigma_out, newton_iters, cg_iters, status: the cells of all
 * handles in group order ([sum of batch sizes][6] or [sum of batch sizes]);
 * run may be NULL (every cell runs); newton_iters and cg_iters may be NULL.
 * Returns the first failing cell's status (others are still reported). */
int fftg_group_step(fftg_group* g, const double* dE, const int* run, double tol_newton, double tol_cg,
                    double* sigma_out, int* newton_iters, int* cg_iters, int* status);
/* Kernel launches the group's graphs made (counted from the iterations). */
long long fftg_group_launch_count(const fftg_group* g);
void fftg_group_destroy(fftg_group* g);

/* ---------------------------------------------------------------- serving
 * Continuous batching of RVE increments (not in the paper; the FE^2 use of
 * Section 1: a macro solver issues one strain increment per Gauss point).
 * A server holds `slots` cells of one grid size (choose slots from the HBM
 * budget: fftg_workspace_size_batch(N, slots) bytes), one stream and one
 * worker thread. fftg_server_submit queues (request, session, dE); a new
 * session must pass its microstructure (N^3 bytes, copied) and starts from
 * the zero state. The worker admits queued requests into free cells between
 * Newton iterations, so new work joins the batch already on the GPU; when
 * every cell is taken it evicts the least recently used idle session to
 * host memory (its committed state) and restores it on its next request.
 * Requests of one session run in submission order. A cell's result does
 * not depend on what shares its launches. */
typedef struct fftg_server fftg_server;
typedef struct {
    long long request_id;
    long long session_id;
    int       status;         /* 0 or FFTG_E*; a failed increment is not committed */
    int       newton_iters;
    int       cg_iters;
    double    sigma[6];       /* homogenised stress after the increment */
    double    t_submit;       /* seconds on fftg_server_clock() */
    double    t_start;        /* admitted into a cell */
    double    t_done;
} fftg_result;

double fftg_server_clock(void);
int fftg_server_start(fftg_server** s, int N, int slots, int nphase, const fftg_phase* mats,
                      const fftg_options* opt, double tol_newton, double tol_cg);
int fftg_server_submit(fftg_server* s, long long request_id, long long session_id,
                       const uint8_t* phase, const double dE[6]);
/* Completed requests (up to max) into out; waits up to wait_s seconds when
 * none is ready. Returns the worker's error code (0 while healthy). */
int fftg_server_poll(fftg_server* s, fftg_result* out, int max, int* n, double wait_s);
int fftg_server_info(fftg_server* s, long long* completed, long long* evictions,
                     long long* restores, int* max_concurrent, double* mean_batch);
/* Drops every request not yet admitted into a cell (queued ones); requests
 * in flight complete and are reported as usual. Dropped requests produce no
 * result. `cancelled` (may be NULL) receives their number. */
int fftg_server_cancel_pending(fftg_server* s, long long* cancelled);
/* Drains the queue, stops the worker and frees everything. */
int fftg_server_stop(fftg_server* s);

/* ---------------------------------------------------------------- no allocation
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory. A host code that has reserved all of its
 * device memory up front (an FE^2 macro solver with its own pool, calling
 * the material law from inside its assembly loop) cannot have the library
 * call cudaMalloc: the call fails while the pool holds the memory, or it
 * stalls the whole device. This call needs no handle and no workspace.
 *
 * It evaluates the material update of the phases' models at E + eps
 * against the history (eps_p, epbar); rate-dependent phases
 * (FFTG_MODEL_VISCO, which need a time step) are not accepted here
 * (FFTG_EINVAL). Every phase id in phase_dev must be < nphase: the call
 * checks this on the device and returns FFTG_EINVAL otherwise, with the
 * outputs unspecified (voxels with such ids get NaN). It writes
 * sigma [6][N^3] (and, where the pointers are not
 * NULL, the updated history and the compact tangent [7][N^3] in FP32
 * (FFTG_MIXED) or FP64 (FFTG_FP64): per voxel K', 2G_eff, w11, w22, w23,
 * w13, w12 with C = |K'| I(x)I + 2G_eff I_d - sign(K') w(x)w, where w33 =
 * -(w11 + w22); K' < 0 marks a positive N(x)N coefficient, possible for
 * exponents n > 1), and returns the homogenised stress
 * mean(sigma) in sigma_mean[6] (host). Every field is a caller device buffer
 * in the unpadded layout [6][N^3] ([N^3] for epbar and phase).
 *
 * Its scratch (block partial sums, the reduction ticket, the material table,
 * the phase-id flag) is one fixed array of about 250 KB compiled into the library, held by every
 * GPU that loads it until the process exits. Limits: N <= 243, nphase <= 256;
 * larger values return FFTG_EINVAL. The first call on a device looks up the
 * array's device address (once per device, with that device current): make
 * that first call before any stream capture. All calls share the array and
 * it keeps the last call's contents, so calls that overlap on the GPU (two
 * streams, or two host threads) race: serialise them. The call synchronises
 * `stream` (NULL = legacy default stream) to return sigma_mean. */
int fftg_constitutive_noalloc(int N, const double E[6], const double* eps_dev,
                              const double* eps_p_dev, const double* epbar_dev,
                              const uint8_t* phase_dev, int nphase, const fftg_phase* mats,
                              int tangent_precision, void* tangent_dev, double* sigma_dev,
                              double* eps_p_new_dev, double* epbar_new_dev,
                              double sigma_mean[6], void* stream);

/* ---------------------------------------------------------------- profiling
 * Per-kernel timing of a handle's own launches with CUDA events recorded in
 * its stream around every launch (off by default; a few microseconds per
 * launch when on). Kernel kinds are numbered 0 .. fftg_profile_kinds()-1. */
int fftg_profile_kinds(void);
const char* fftg_profile_name(int kind);
int fftg_profile_enable(fftg_handle* h, int on);
int fftg_profile_reset(fftg_handle* h);
/* Synchronises the stream; total device milliseconds and launches of `kind`
 * since the last reset (or since profiling was enabled). */
int fftg_profile_read(fftg_handle* h, int kind, double* total_ms, long long* launches);
/* Kernels this handle has launched since creation (always counted). */
long long fftg_launch_count(const fftg_handle* h);

/* ---------------------------------------------------------------- schedules
 * The FP32 passes of the mixed CG iteration run one of FFTG_SCHED_VARIANTS
 * schedules per grid size and pass: the radix split of the pencil transform
 * (the default split or the other one, e.g. 27 x 9 or 9 x 27 at N = 243)
 * and the tile (rows per block of P1/P5, columns per block of P2-P4; for
 * P3 also the default tile with stage B, Ghat and the inverse stage B in one
 * phase).
 * Every schedule computes the same transforms (results agree to FP32
 * rounding). The choice is process-wide per grid size and applies to
 * launches enqueued afterwards; a handle's CUDA graphs keep the kernels they
 * captured, so set or tune schedules before creating the handles that should
 * use them. Not part of the paper's method. */
#define FFTG_SCHED_P1 0        /* x3 transform + C : p (CG)            */
#define FFTG_SCHED_P2 1        /* x2 transform                          */
#define FFTG_SCHED_P3 2        /* x1 transform + Ghat + inverse          */
#define FFTG_SCHED_P4 3        /* inverse x2 transform                  */
#define FFTG_SCHED_P5 4        /* inverse x3 transform + r update (CG)  */
#define FFTG_SCHED_KINDS 5
#define FFTG_SCHED_VARIANTS 4
#define FFTG_TUNE_CACHE 1      /* read and write the schedule cache file */
#define FFTG_TUNE_FORCE 2      /* time again even when the cache has the grid */
/* Select schedule `variant` (0 = default) of pass `kind` at grid N. */
int fftg_schedule_set(int N, int kind, int variant);
/* The variant in use, or FFTG_EINVAL. */
int fftg_schedule_get(int N, int kind);
/* shape[5]: radix split n1, n2; rows per block; columns per block; blocks
 * per field of the launch. */
int fftg_schedule_describe(int N, int kind, int variant, int shape[5]);
/* Times every variant of every kind at grid N on one field of scratch
 * device memory (cudaMalloc'd for the call, about 170 B per voxel) in
 * `stream` (synchronised), and selects the fastest of each kind (a variant
 * replaces the default only when at least 2 % faster). ms (may be NULL):
 * [FFTG_SCHED_KINDS][FFTG_SCHED_VARIANTS] median milliseconds, -1 when the
 * cache supplied the choice; chosen[FFTG_SCHED_KINDS]. With FFTG_TUNE_CACHE
 * the choices are read from / appended to the cache file
 * $FFTG_SCHEDULE_CACHE (default $XDG_CACHE_HOME/fftg/schedules.txt, else
 * ~/.cache/fftg/schedules.txt), keyed by device name, grid size and library
 * build, and a grid found there is not timed again (unless FFTG_TUNE_FORCE).
 * Thread-safe against itself; not against solves running meanwhile. */
int fftg_autotune(int N, int flags, void* stream, double* ms, int* chosen);

/* Fused multiply-add throughput of the current device in TFLOP/s (2 flops
 * per FMA), FP64 (precision FFTG_FP64) or FP32 (FFTG_MIXED): one launch of
 * 8 blocks per SM whose threads each run 8 independent chains of `iters`
 * FMAs, timed with CUDA events in `stream` (NULL = legacy default stream;
 * the call synchronises it). The roofline denominator of ALU-bound passes;
 * the paper has no counterpart. FFTG_EINVAL for iters < 8 or another
 * precision. */
int fftg_probe_fma_rate(int precision, int iters, void* stream, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* FFTG_H */
