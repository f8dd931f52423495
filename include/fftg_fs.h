/*
 * fftg finite strain: the FFT-Galerkin Newton-CG scheme of arXiv:1601.05970
 * carried over to finite strain, the extension its Section 6 names as the
 * next step, on one GB300 GPU (sm_103a).
 *
 * The small-strain method (Algorithm 1, Eq. linear_system) is kept and the
 * strain is replaced by the deformation gradient:
 *  - unknown F = Fbar + F*, F* a compatible fluctuation (the gradient of a
 *    periodic displacement) with zero mean, Fbar the prescribed macroscopic
 *    deformation gradient;
 *  - equilibrium G P(F) = 0 with the first Piola-Kirchhoff stress P, where
 *    G projects onto gradient fields: in Fourier space row i of a tensor
 *    field is projected onto xi, Ghat_ijlm = delta_il xi_j xi_m / |xi|^2
 *    (Ghat(0) = 0);
 *  - Newton iterations G K(F) : dF* = -G P(F), K = dP/dF, each solved by CG
 *    with the Frobenius product sum_ij A_ij B_ij (F is not symmetric), until
 *    ||dF*|| / (sqrt(N^3) ||Fbar - I||_F) <= tol_newton;
 *  - material: St. Venant-Kirchhoff per phase (the paper gives no finite-
 *    strain law), E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E, P = F S.
 *
 * Conventions (as in fftg.h where not stated):
 *  - A 3x3 tensor is 9 doubles, row major: component 3i + j is A_ij.
 *  - A tensor field is [9][N][N][N] (component slowest, then x1, x2, x3).
 *  - Grids: N odd, a product of 3s and 5s, 3 <= N <= 243 (the grid sizes of
 *    fftg.h).
 *  - Precision as in fftg.h: FFTG_MIXED runs the CG in FP32 and the
 *    residual G P from FP64 stresses with double-float FFTs.
 *  - Return values are FFTG_OK or FFTG_E*; on error the committed state
 *    (Fbar, F*) is unchanged. The caller owns host arrays; the handle owns
 *    its device memory; one host thread uses a handle at a time.
 */
#ifndef FFTG_FS_H
#define FFTG_FS_H

#include "fftg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftg_fs_handle fftg_fs_handle;

/* One hyperelastic phase: St. Venant-Kirchhoff with Lame constants
 * lambda >= 0 and mu > 0. */
typedef struct {
    double lambda;
    double mu;
} fftg_svk_phase;

#define FFTG_FS_FIELD_DEFGRAD 0  /* F = Fbar + F* at the committed state, [9][N^3] */
#define FFTG_FS_FIELD_STRESS  1  /* P at the committed state, [9][N^3] */

/* Create a cell. phase: uint8 [N][N][N], values < nphase (<= 256); mats:
 * nphase phases. Options used: precision (FFTG_FP64, or FFTG_MIXED: FP32
 * inner CG; FP64 stress, Newton test and mean P; the residual from the FP64
 * stress with double-float FFTs, as in fftg.h),
 * max_newton, max_cg, cg_inner_floor, fixed_cg, fixed_newton, stream,
 * cg_graph. A workspace, solver != FFTG_SOLVER_CG or an invalid value of
 * the others gives FFTG_EINVAL; the rest are ignored. NULL opt: defaults.
 * Starts from Fbar = I, F* = 0. */
int fftg_fs_create(fftg_fs_handle** h, int N, const uint8_t* phase, int nphase,
                   const fftg_svk_phase* mats, const fftg_options* opt);

/* One load increment: Fbar <- Fbar + dF (row major), Newton from the
 * previous F* as described above, each linear solve by CG to tol_cg
 * (relative residual). Writes the homogenised first Piola-Kirchhoff stress
 * (the voxel mean of P) to P_out[9] and commits. newton_iters / cg_iters may
 * be NULL. FFTG_ENOCONV_NEWTON, FFTG_ENAN (NaN or a CG breakdown, e.g. a
 * tangent that is not positive definite) leave the state unchanged. */
int fftg_fs_step(fftg_fs_handle* h, const double dF[9], double tol_newton, double tol_cg,
                 double P_out[9], int* newton_iters, int* cg_iters);

/* 9x9 macroscopic tangent dPbar/dFbar at the committed state (not in the
 * paper; what an FE^2 macro solver needs): C_out[9*(3i+j) + (3k+l)] =
 * dPbar_ij / dFbar_kl. For each unit tensor E_kl, CG solves the linearised
 * equilibrium G K x = -G (K : E_kl) to tol_cg (with the handle's precision
 * and inner floor), and the column is the voxel mean of K : (E_kl + x).
 * cg_iters (may be NULL) gets the CG iterations of the nine solves. */
int fftg_fs_tangent(fftg_fs_handle* h, double tol_cg, double C_out[81], int* cg_iters);

/* Diagnostics of the last increment (fields as in fftg.h; newton_norm is
 * the finite-strain Newton test above, residual ||G P|| / ||P||). */
int fftg_fs_last_stats(fftg_fs_handle* h, fftg_stats* out);

/* Checkpoint/restore of the committed state: Fbar[9] then F*[9][N^3], FP64
 * (fftg_fs_state_bytes() bytes). set_state rejects a wrong size or a
 * non-finite entry (FFTG_EINVAL) and then leaves the state unchanged. */
size_t fftg_fs_state_bytes(const fftg_fs_handle* h);
int fftg_fs_get_state(fftg_fs_handle* h, void* host_buf, size_t bytes);
int fftg_fs_set_state(fftg_fs_handle* h, const void* host_buf, size_t bytes);

/* Copy a committed field (FFTG_FS_FIELD_*) to host memory, FP64 [9][N^3]. */
int fftg_fs_get_field(fftg_fs_handle* h, int which, double* host_out);

/* out = G A for a device field A [9][N^3] (FP64 for FFTG_FP64 and FFTG_DD,
 * FP32 for FFTG_MIXED, which needs a mixed handle): forward DFT, Ghat above
 * at every frequency, inverse DFT; FFTG_DD runs the FFTs in double-float
 * arithmetic, as the mixed path's residual does. A and out may alias.
 * Enqueued on the handle's stream. */
int fftg_fs_op_project(fftg_fs_handle* h, int precision, const void* A_dev, void* out_dev);

/* q = G (K : p) with K = dP/dF at the committed F (St. Venant-Kirchhoff's
 * tangent), p and q device fields [9][N^3] in `precision`; <p, q> to *pq
 * when pq is not NULL (then the stream is synchronised). */
int fftg_fs_op_matvec(fftg_fs_handle* h, int precision, const void* p_dev, void* q_dev, double* pq);

/* Per-kernel device time of the handle's launches (CUDA events around each
 * launch, off by default). Kinds 0 .. fftg_fs_profile_kinds()-1. */
int fftg_fs_profile_kinds(void);
const char* fftg_fs_profile_name(int kind);
int fftg_fs_profile_enable(fftg_fs_handle* h, int on);
int fftg_fs_profile_read(fftg_fs_handle* h, int kind, double* total_ms, long long* launches);

/* Kernels this handle has launched since creation. */
long long fftg_fs_launch_count(const fftg_fs_handle* h);

/* Device bytes a handle of grid N holds (one allocation). */
int fftg_fs_workspace_size(int N, const fftg_options* opt, size_t* bytes);

void fftg_fs_destroy(fftg_fs_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* FFTG_FS_H */
