/*
 * stokes_dcamg.h - C ABI of the GB300 solve phase of the defect-correction
 * monolithic AMG preconditioner for Stokes (Voronin, MacLachlan, Olson,
 * Tuminaro, arXiv 2306.06795).
 *
 * The library solves K0 x = b, the saddle-point system of Eq. saddle
 * (Sec. 2) for Taylor-Hood P2/P1 or Scott-Vogelius P2/P1disc, with restarted
 * flexible GMRES (Sec. 4) right-preconditioned by the defect-correction
 * cycle of Eq. TG-operator-full (Sec. 3.1): relaxation on K0, a residual
 * taken with K0 and weighted by eta (Eq. eta), transfer to the P1isoP2/P1
 * operator K1 (Eq. interp), one Galerkin V-cycle (Eq. TG-operator) of the
 * Alg. 1 hierarchy K1, K2, ... with an exact coarsest solve, prolongation
 * and relaxation on K0.  Relaxation is additive Vanka (Sec. 3.3.1,
 * Eq. vanka) with block-factorised patch solves (Eqs. vanka_fact1/2), or
 * DLSC (Sec. 3.3.2, Alg. 2) on any level.
 *
 * Conventions
 *  - Every function returns STOKES_OK (0), a positive status
 *    (STOKES_NOT_CONVERGED) or a negative error code; stokes_last_error()
 *    gives a one-line message for the last error of the calling thread.
 *  - Host arrays passed to stokes_setup are read during the call and
 *    copied; the caller keeps ownership and may free them afterwards.
 *  - Vectors passed to stokes_vcycle, stokes_fgmres_solve and
 *    stokes_level_op are caller-owned DEVICE pointers of FP64 values,
 *    holding all instances of a batched handle concatenated in instance
 *    order.  stokes_fgmres_solve_host takes HOST pointers instead.
 *  - Work is queued on the CUDA stream given to stokes_setup (the handle's
 *    own stream when NULL).  stokes_vcycle and stokes_level_op are
 *    asynchronous; the solve functions synchronise before returning.
 *  - The handle owns all device memory it allocates; stokes_destroy frees
 *    it.  A handle is not thread-safe: one host thread at a time.
 *  - Nothing here falls back to the CPU: without a usable CUDA device the
 *    calls fail with STOKES_ERR_CUDA.
 */
#ifndef STOKES_DCAMG_H
#define STOKES_DCAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  STOKES_OK = 0,
  STOKES_NOT_CONVERGED = 1,        /* maxit reached; info is filled */
  STOKES_ERR_INVALID_ARG = -1,     /* bad size, index, order or parameter */
  STOKES_ERR_CUDA = -2,            /* a CUDA runtime call failed */
  STOKES_ERR_OOM = -3,             /* device allocation failed */
  STOKES_ERR_SINGULAR_PATCH = -4,  /* a patch block or Schur complement is singular */
  STOKES_ERR_NAN = -5,             /* a non-finite residual appeared */
  STOKES_ERR_STATE = -6            /* call out of order (e.g. cycle before factorisation) */
};

enum { STOKES_TH = 0, STOKES_SV = 1 };                       /* K0 element pair */
enum { STOKES_DC_ALL = 0, STOKES_DC_SKIP1 = 1, STOKES_DC_SKIP0 = 2 };  /* Sec. 4 schedules */
/* Relaxation per level.  VANKA: nu damped additive Vanka sweeps
 * x += omega M^-1 (b - K x) (Eq. vanka).  DLSC: dlsc_sweeps Chebyshev LSC-DGS
 * sweeps of Alg. 2 per relaxation call (Mu = diag(Mu_diag) on level 0, I on
 * levels >= 1; omega unused).  VANKA_KRYLOV: the Krylov-wrapped relaxation of
 * Sec. 3.3.1, nu steps of flexible GMRES on K e = b - K x, each
 * right-preconditioned by one undamped Vanka sweep, then x += Z y with y
 * the least-squares minimiser (nu <= 4; omega unused). */
enum { STOKES_RELAX_VANKA = 0, STOKES_RELAX_DLSC = 1, STOKES_RELAX_VANKA_KRYLOV = 2 };
enum { STOKES_FP32 = 0, STOKES_FP64 = 1 };                   /* cycle precision */
/* Preconditioner of the FGMRES solve (and of stokes_vcycle): the DC cycle,
 * or the block-triangular comparison preconditioner BTP of Sec. 4. */
enum { STOKES_PRECOND_DC = 0, STOKES_PRECOND_BTP = 1 };

/* A sparse matrix in CSR form, host memory, FP64 values.  Column indices
 * must be sorted ascending and unique within each row. */
typedef struct {
  int32_t nrows, ncols;
  int64_t nnz;
  const int64_t* rowptr; /* [nrows + 1] */
  const int32_t* col;    /* [nnz] */
  const double* val;     /* [nnz] */
} stokes_csr;

/* Vanka patches of one level (Sec. 3.3.1).  Patch i holds the level DoFs
 * dof[ptr[i] .. ptr[i+1]): the velocity DoFs of component 0 ascending, then
 * those of component 1 (and 2), then its pressure seed DoF(s) ascending.
 * nvel[i*dim + c] is the number of velocity DoFs of component c and
 * npres[i] the number of seeds (1 for Taylor-Hood and P1isoP2 levels, 3 for
 * the Scott-Vogelius cell patches). */
typedef struct {
  int32_t npatch;
  const int64_t* ptr;   /* [npatch + 1] */
  const int32_t* dof;   /* [ptr[npatch]] */
  const int32_t* nvel;  /* [npatch * dim] */
  const int32_t* npres; /* [npatch] */
} stokes_patches;

/* Data of the block-triangular preconditioner BTP (Sec. 4), built by the
 * host setup step: with [r_u, r_p] = r it returns
 *   du = Q_A^-1 r_u,   dp = Q_B^-1 (B du - r_p),
 * Q_A^-1 one SA V-cycle on the vector Laplacian A (levels A[l], prolongators
 * PA[l] mapping level l+1 to l, Galerkin coarse operators, btp_steps
 * Krylov-wrapped Jacobi steps before and after the coarse correction, exact
 * coarsest solve), Q_B^-1 the same kind of V-cycle on M (M[0] = M_p / nu,
 * Taylor-Hood) or the exact inverse Minv (Scott-Vogelius, block diagonal).
 * Dirichlet velocity rows return r_u. */
typedef struct {
  int32_t nlevels_a;              /* >= 1 */
  const stokes_csr* A;            /* [nlevels_a]: A[0] = velocity block of K0 */
  const stokes_csr* PA;           /* [nlevels_a - 1] */
  const stokes_csr* B;            /* pressure rows x velocity columns of K0 */
  int32_t nlevels_m;              /* levels of the M hierarchy, 0 when Minv is given */
  const stokes_csr* M;            /* [nlevels_m] */
  const stokes_csr* PM;           /* [nlevels_m - 1] */
  const stokes_csr* Minv;         /* exact inverse of M_p / nu, or NULL */
} stokes_btp;

/* One Stokes problem and its solver hierarchy, built by a host setup step.
 * Level 0 is K0 (high order), level 1 the P1isoP2/P1 operator K1, levels
 * >= 2 the Galerkin operators K_{l+1} = P_l^T K_l P_l of Alg. 1.  On every
 * level the DoFs are ordered velocity component 0, component 1[, 2], then
 * pressure; field_off[l*(dim+2) + c] is the first DoF of field c on level l
 * and field_off[l*(dim+2) + dim + 1] the level size. */
typedef struct {
  int32_t dim;                    /* 2 or 3 */
  int32_t disc;                   /* STOKES_TH or STOKES_SV */
  int32_t nlevels;                /* >= 2 */
  const int64_t* field_off;       /* [nlevels * (dim + 2)] */
  const stokes_csr* K;            /* [nlevels] */
  const stokes_csr* P;            /* [nlevels - 1]: P[l] maps level l+1 to l;
                                     P[0] is P0 of Eq. interp (identity for TH) */
  const stokes_patches* patches;  /* [nlevels - 1]: levels 0 .. nlevels-2 */
  const double* coarse_null;      /* [size of level nlevels-1]: null vector of the
                                     coarsest operator (zero velocity, pressure
                                     near-null); used to border its exact solve */
  const uint8_t* dirichlet;       /* [size of level 0]: 1 on Dirichlet identity rows */
  /* Scott-Vogelius pressure restriction R0^p = Mcg^-1 Pi^T M_dg (Sec. 3.1) */
  const stokes_csr* R0p;          /* Pi^T M_dg, n_cg x n_dg, or NULL for TH */
  const stokes_csr* Mcg;          /* P1 mass matrix of the K1 pressure, or NULL */
  double mcg_lo, mcg_hi;          /* interval holding the eigenvalues of diag(Mcg)^-1 Mcg */
  /* DLSC (Sec. 3.3.2): largest-eigenvalue estimates per level, may be NULL.
   * A level's Chebyshev interval is one per handle: the instances of a
   * handle that relax a level with DLSC must give the same lambda_A and
   * lambda_S for it (stokes_setup rejects others). */
  const double* lambda_A;         /* [nlevels] of the velocity block A */
  const double* lambda_S;         /* [nlevels] of B Mu^-1 B^T */
  /* BTP (Sec. 4), used when stokes_params.preconditioner is
   * STOKES_PRECOND_BTP (single-instance handles); may be NULL otherwise */
  const stokes_btp* btp;
  /* DLSC on level 0 (Sec. 3.3.2: on the P2 grid Mu is the diagonal of the
   * velocity mass matrix; the P1isoP2 levels use Mu = I): the diagonal,
   * [velocity DoFs of level 0], all entries > 0.  Needed only when level 0
   * relaxes with DLSC (lambda_S[0] is then the estimate for B Mu^-1 B^T);
   * may be NULL otherwise. */
  const double* Mu_diag;
} stokes_problem;

/* Parameters of the defect-correction cycle (Table param_ref). */
typedef struct {
  int32_t schedule;          /* STOKES_DC_ALL, _SKIP1 or _SKIP0 */
  int32_t nu1, nu2;          /* pre- and post-relaxation sweeps per level */
  double eta_u, eta_p;       /* residual weights of Eq. eta on level 0 */
  const double* omega;       /* [nlevels-1] Vanka damping per relaxed level */
  const int32_t* relax;      /* [nlevels-1] STOKES_RELAX_*, NULL = Vanka everywhere */
  int32_t cheb_deg[3];       /* DLSC Chebyshev degrees: momentum, continuity, pressure correction */
  int32_t dlsc_sweeps;       /* DLSC sweeps per relaxation call */
  int32_t mcg_deg;           /* Chebyshev-Jacobi degree of the SV mass-matrix solve */
  int32_t precision;         /* STOKES_FP32 or STOKES_FP64 cycle */
  int32_t preconditioner;    /* STOKES_PRECOND_DC or STOKES_PRECOND_BTP */
  int32_t btp_steps;         /* BTP: Krylov-wrapped Jacobi steps per relaxation (1..4) */
  int32_t factor_tcgen05;    /* FP32 factorisation of patch blocks with three 32 x 32 tile rows
                                (3D vertex patches): 0 = trailing products on mma.sync (default,
                                faster at these sizes), 1 = on tcgen05 with TMEM accumulators */
} stokes_params;

typedef struct {
  int32_t iters;             /* FGMRES iterations (preconditioner applications) */
  int32_t status;            /* STOKES_OK or STOKES_NOT_CONVERGED */
  double true_relres;        /* ||b - K0 x|| / ||b|| recomputed in FP64 at exit */
} stokes_solve_info;

typedef struct stokes_handle stokes_handle;

/* Build the device-side solver for ninstances independent problems (one
 * for a single solve; several are stacked block-diagonally and solved
 * together, each with its own FGMRES scalars).  Copies every CSR to the
 * device (FP64, plus FP32 copies for an FP32 cycle), forms R_l = P_l^T,
 * the Vanka transpose maps and the bordered inverse of each coarsest
 * operator (FP64 LU with partial pivoting on the host).  Validates index
 * ranges, ordering and sizes (STOKES_ERR_INVALID_ARG).  cuda_stream is a
 * cudaStream_t or NULL.  On success *out receives the handle. */
int stokes_setup(const stokes_problem* const* probs, int32_t ninstances,
                 const stokes_params* params, void* cuda_stream, stokes_handle** out);

/* Factorise every Vanka patch on the device in the cycle precision
 * (Eqs. vanka_fact1/2): per patch the inverse of the velocity block of each
 * component (one block when the components' blocks are identical), U =
 * A^-1 B^T and S^-1 with S = -B A^-1 B^T.  *nsingular (may be NULL)
 * receives the number of patches with a pivot below 1e-12 relative;
 * returns STOKES_ERR_SINGULAR_PATCH when it is nonzero. */
int stokes_factor_patches(stokes_handle* h, int64_t* nsingular);

/* z = M_dc^-1 r: one defect-correction cycle (Eq. TG-operator-full,
 * gamma = 1) from a zero initial guess, over all instances.  r_dev and
 * z_dev are device FP64 vectors of the level-0 size; they must not alias.
 * The cycle runs as a captured CUDA graph. */
int stokes_vcycle(stokes_handle* h, const double* r_dev, double* z_dev);

/* Solve K0 x = b by restarted FGMRES(restart), right-preconditioned by the
 * DC cycle, per instance, until ||b - K0 x|| <= rtol ||b|| (true residual,
 * FP64) or maxit iterations.  x_dev holds the initial guess on entry and
 * the solution on exit.  info[ninstances] (may be NULL) receives per
 * instance the iterations, status and true relative residual.  Returns
 * STOKES_NOT_CONVERGED when any instance missed rtol, STOKES_ERR_INVALID_ARG
 * for restart outside 1..1024, maxit < 0 or rtol <= 0. */
int stokes_fgmres_solve(stokes_handle* h, const double* b_dev, double* x_dev,
                        double rtol, int32_t restart, int32_t maxit,
                        stokes_solve_info* info);

/* Same solve with HOST vectors: copies b and x0 to the device, solves and
 * copies x back, all inside the call. */
int stokes_fgmres_solve_host(stokes_handle* h, const double* b_host, double* x_host,
                             double rtol, int32_t restart, int32_t maxit,
                             stokes_solve_info* info);

/* Autotuner of the Vanka apply (the paper has no counterpart: a tiling
 * choice of this implementation).  For every level and patch bin, times the
 * bulk-copy apply for patches per tile in {t/2, t, 2t} around the setup's
 * choice t and a 2- or 3-stage shared-memory ring, `reps` launches each
 * (CUDA events on the handle's stream), and keeps the fastest.  Results do
 * not change (the per-patch arithmetic is independent of the tiling);
 * CUDA graphs captured before are dropped and recaptured on next use.
 * Requires stokes_factor_patches.  stokes_autotune_report returns the
 * choices as JSON, owned by the handle. */
int stokes_autotune(stokes_handle* h, int32_t reps);
const char* stokes_autotune_report(const stokes_handle* h);

/* Device-side Galerkin product of the AMG setup (Alg. 1): C = P^T K P in
 * FP64 on the GPU (a setup step; the solve path does not call it).  K
 * (n x n) and P (n x nc) are host CSRs as in stokes_setup; C receives
 * nc x nc host arrays with sorted columns, allocated by the library and
 * released with stokes_csr_free.  Deterministic: every entry sums its
 * partial products in a fixed order.  Runs on cuda_stream (NULL: the
 * default stream) and returns after the copy back.  STOKES_ERR_INVALID_ARG
 * when an output row has more than 4096 partial products. */
int stokes_galerkin(const stokes_csr* K, const stokes_csr* P, void* cuda_stream, stokes_csr* C);
void stokes_csr_free(stokes_csr* C);

/* Further device steps of the smoothed-aggregation setup of Alg. 1 (setup
 * steps; the solve path does not call them).  Host arrays in; outputs are
 * host arrays allocated by the library (stokes_csr_free,
 * stokes_patch_lists_free).  All run on cuda_stream (NULL: the default
 * stream), return after the copy back, and are deterministic.
 *
 * stokes_sa_strength: strength-of-connection pattern S of a square A (Sec.
 *   3.2): off-diagonal j is strong for row i when |a_ij| > theta
 *   sqrt(|a_ii| |a_jj|), theta >= 0; values 1, columns sorted.
 * stokes_sa_tentative: tentative prolongator of aggregates agg[n] (-1 for
 *   a node outside every aggregate, otherwise 0 .. naggregates-1, every
 *   aggregate non-empty) with near-null vector B[n]: T (n x naggregates)
 *   holds B_i / ||B on the aggregate||_2 in column agg_i; Bc[naggregates]
 *   (caller-allocated) receives the norms, so that T Bc = B on aggregated
 *   rows.  Norms sum the squares in node order.
 * stokes_sa_smooth: Jacobi-smoothed prolongator P = T - omega D^-1 A T
 *   (D the diagonal of A; rows without a nonzero off-diagonal entry get
 *   D^-1 = 0), each entry t - omega (d_i^-1 (A T)_ij), exact zeros dropped.
 *   omega is the caller's (4/3 over the spectral radius of D^-1 A in the
 *   host setup).  STOKES_ERR_INVALID_ARG when a row of A T has more than
 *   4096 partial products.
 * stokes_vanka_patches: Vanka patch lists of a Galerkin level (Sec. 3.3.1)
 *   of K with field offsets field_off[dim + 2] (velocity components of
 *   equal size, then pressure): patch s holds every velocity node j linked
 *   to pressure DoF s by max over components |b_sj| > rel_tol times the
 *   largest of the row, with all dim components (nodes ascending), then
 *   the seed; layout as stokes_patches, one seed per patch.
 *   STOKES_ERR_INVALID_ARG when a pressure row has more than 4096
 *   velocity entries. */
typedef struct {
  int32_t npatch;
  int64_t* ptr;   /* [npatch + 1] */
  int32_t* dof;   /* [ptr[npatch]] */
  int32_t* nvel;  /* [npatch * dim] */
  int32_t* npres; /* [npatch] */
} stokes_patch_lists;
int stokes_sa_strength(const stokes_csr* A, double theta, void* cuda_stream, stokes_csr* S);
int stokes_sa_tentative(int32_t n, const int32_t* agg, int32_t naggregates, const double* B, void* cuda_stream,
                        stokes_csr* T, double* Bc);
int stokes_sa_smooth(const stokes_csr* A, const stokes_csr* T, double omega, void* cuda_stream, stokes_csr* P);
int stokes_vanka_patches(const stokes_csr* K, const int64_t* field_off, int32_t dim, double rel_tol, void* cuda_stream,
                         stokes_patch_lists* out);
void stokes_patch_lists_free(stokes_patch_lists* p);

/* Single steps of the cycle on one level, for testing and measurement.
 * All vectors are device FP64 of the sizes stated; the operation runs in
 * the cycle precision unless its name says FP64.
 *   STOKES_OP_SPMV      y = K_l x                     (x, y: level l)
 *   STOKES_OP_SPMV_F64  y = K_l x in FP64             (x, y: level l)
 *   STOKES_OP_RESIDUAL  y = b - K_l x                 (level l)
 *   STOKES_OP_RESTRICT  y = R_l x  (l >= 1: P_l^T; l = 0: R0 of Eq. interp)
 *                                                     (x: level l, y: level l+1)
 *   STOKES_OP_PROLONG   y = P_l x                     (x: level l+1, y: level l)
 *   STOKES_OP_VANKA     y = M_l^-1 x, Eq. vanka (sum of weighted patch solves)
 *   STOKES_OP_RELAX     y = x + omega_l M_l^-1 (b - K_l x), one sweep
 *                       (one DLSC sweep when level l relaxes with DLSC; one
 *                       Krylov-wrapped relaxation of max(nu1, nu2) steps
 *                       when it relaxes with STOKES_RELAX_VANKA_KRYLOV)
 *   STOKES_OP_COARSE    y = exact bordered solve with the coarsest K (l = nlevels-1)
 */
enum {
  STOKES_OP_SPMV = 0, STOKES_OP_SPMV_F64 = 1, STOKES_OP_RESIDUAL = 2,
  STOKES_OP_RESTRICT = 3, STOKES_OP_PROLONG = 4, STOKES_OP_VANKA = 5,
  STOKES_OP_RELAX = 6, STOKES_OP_COARSE = 7
};
int stokes_level_op(stokes_handle* h, int32_t op, int32_t level,
                    const double* x_dev, const double* b_dev, double* y_dev);

/* Sizes: number of levels (the deepest instance) and the concatenated size
 * of level l over all instances present on it. */
int stokes_num_levels(const stokes_handle* h);
int64_t stokes_level_size(const stokes_handle* h, int32_t level);

/* Algorithmic bytes that one DC cycle must move through HBM in the handle's
 * precision (matrix values and indices, patch factors and index lists,
 * vectors read and written), and the bytes of the patch factors of one
 * Vanka sweep of level l; both derived from the stored sizes. */
double stokes_cycle_bytes(const stokes_handle* h);
double stokes_sweep_factor_bytes(const stokes_handle* h, int32_t level);

/* Measurement support.
 * stokes_time_kernel runs one hot kernel of level l alone `reps` times on
 * the handle's stream; before each launch it overwrites a 256 MiB buffer
 * (untimed) so that no launch finds its data in L2, brackets the launch
 * with CUDA events and returns the mean duration in ms and the algorithmic
 * bytes of one launch (the same count stokes_cycle_bytes uses).  The first
 * call allocates the flush buffer.
 *   STOKES_KERNEL_VANKA_APPLY  gather + block-factorised patch solves of level l
 *   STOKES_KERNEL_SCATTER      weighted scatter of level l
 *   STOKES_KERNEL_SPMV         residual SpMV of level l in the cycle precision
 *   STOKES_KERNEL_DC_RESIDUAL  the FP64 K0 residual of the DC step (l = 0)
 * stokes_kernel_launches returns the number of kernels the handle has
 * launched so far (graph replays count every kernel node). */
enum { STOKES_KERNEL_VANKA_APPLY = 0, STOKES_KERNEL_SCATTER = 1, STOKES_KERNEL_SPMV = 2,
       STOKES_KERNEL_DC_RESIDUAL = 3 };
int stokes_time_kernel(stokes_handle* h, int32_t which, int32_t level, int32_t reps,
                       double* avg_ms, double* bytes);
int64_t stokes_kernel_launches(const stokes_handle* h);

/* y = M_l^-1 x on level l (the sum of weighted Vanka patch solves, the
 * same result as stokes_level_op with STOKES_OP_VANKA) without allocating
 * any device memory during the call.  It is meant for callers that cannot
 * call cudaMalloc while they run (a fixed device-memory budget, or a
 * context in which allocation is not permitted); they create and factorise
 * the handle beforehand and pass the input and output vectors (device FP64,
 * the level-l size).  The paper has no counterpart: this is an
 * implementation service.  Its scratch (the cycle-precision copy of x, the
 * patch-major solutions and the result before conversion) is one fixed
 * 32 MiB device array inside the library, held by every GPU that loads the
 * library until the process exits; a level needing more returns
 * STOKES_ERR_INVALID_ARG with the sizes in stokes_last_error().  Every call
 * shares that array and overwrites it completely before reading it, so no
 * part must start at zero; calls that overlap on the GPU (from several
 * threads or streams) race on it.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The work is queued on the handle's stream;
 * before returning, the call waits for it and reads the level's bulk-copy
 * error flag: a pipeline wait that ran out (the patch solutions are then
 * incomplete) returns STOKES_ERR_CUDA, and y must not be used. */
int stokes_vanka_noalloc(stokes_handle* h, int32_t level, const double* x_dev, double* y_dev);

/* Test support for the error path (the paper has no counterpart): sets the
 * device error flag of level l's bulk-copy Vanka apply as a bounded wait
 * that ran out would, without running any kernel.  Every later call that
 * checks the flags (stokes_level_op, stokes_fgmres_solve,
 * stokes_vanka_noalloc) then returns STOKES_ERR_CUDA.  The flag is never
 * cleared: use a handle made for the test.  Synchronises the handle's
 * stream.  STOKES_ERR_INVALID_ARG for a level without patches. */
int stokes_inject_pipeline_error(stokes_handle* h, int32_t level);

/* Release all device memory of the handle (NULL is allowed). */
void stokes_destroy(stokes_handle* h);

const char* stokes_status_string(int status);
const char* stokes_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_DCAMG_H */
