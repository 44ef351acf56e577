/*
 * msrsb.h -- C ABI of a GB300 (sm_103a) implementation of the enhanced
 * multiscale restriction-smoothed basis (MsRSB) two-level preconditioner of
 * Bosma, Klevtsov, Moyner and Castelletto, arXiv 1912.06934.
 *
 * Problem statement (Sec. 2, Eq. 1-3): solve A u = f with a Krylov method
 * preconditioned by a prolongation P built by restricted smoothing (Alg. 1),
 * the Galerkin coarse operator A_c = P^T A P and a fine-scale smoother
 * (Alg. 2-4).
 *
 * Conventions shared by every entry point
 *  - Array arguments are DEVICE pointers unless the name ends in _h (host).
 *    The caller allocates and owns them; no call frees or keeps them, except
 *    msrsb_setup, which keeps a non-owning reference to A (see there).
 *  - Integer index arrays are int32; fine rows n < 2^24 (the smoothing kernel
 *    packs an 8-bit support mask beside each column index).
 *  - The fine operator A is FP64 CSR (bdim = 1) or FP64 3x3 block CSR
 *    (bdim = 3, blocks row-major, dof = 3*node + component) with sorted
 *    column indices and the diagonal present in every row.
 *  - Grids are Cartesian, x fastest: flat = x + nx*(y + ny*z); coarse ids use
 *    the same ordering over the coarse grid.
 *  - The prolongation pattern is an ELL array p_ids[n][W], W = 2^dim, entries
 *    -1 where unused. Slot s of every row only ever holds coarse nodes of
 *    colour s, colour(J) = sum_d (J_d mod 2) 2^d: coarse nodes whose supports
 *    overlap differ in colour, so a node sits in the same slot in every row.
 *    P values are p_val[comp][n][W] in the precision given by msrsb_prec.
 *  - Work is stream-ordered on the cudaStream_t passed in. Calls that return
 *    host values (arguments ending in _h) synchronise that stream first.
 *  - Every call returns msrsb_status; on anything but MSRSB_OK,
 *    msrsb_last_error() gives a message (per host thread). Outputs are then
 *    unspecified, except for MSRSB_ENOCONV (see msrsb_solve). Nothing ever
 *    traps or aborts the process.
 */
#ifndef MSRSB_H
#define MSRSB_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSRSB_OK = 0,
    MSRSB_EINVAL = 1,      /* bad argument (null pointer, unsupported option) */
    MSRSB_ESHAPE = 2,      /* inconsistent sizes */
    MSRSB_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    MSRSB_ENOMEM = 4,      /* device allocation failed */
    MSRSB_EBREAKDOWN = 5,  /* zero pivot (coarse inverse, ILU(0), block diagonal) or Krylov breakdown */
    MSRSB_ENOCONV = 6,     /* Krylov iteration limit reached before the tolerance */
    MSRSB_ETIMEOUT = 7,    /* a bounded device-side wait expired */
    MSRSB_ENAN = 8         /* non-finite value in a residual */
} msrsb_status;

typedef enum { MSRSB_F64 = 0, MSRSB_F32 = 1 } msrsb_prec;
typedef enum {
    MSRSB_SMOOTH_NONE = 0,
    MSRSB_SMOOTH_ILU0 = 1,
    MSRSB_SMOOTH_GS = 2,
    MSRSB_SMOOTH_L1JAC = 3,
    MSRSB_SMOOTH_IC0 = 4
} msrsb_smoother;
typedef enum { MSRSB_GMRES = 0, MSRSB_PCG = 1, MSRSB_RICHARDSON = 2 } msrsb_krylov;
typedef enum { MSRSB_RESTRICT_GALERKIN = 0, MSRSB_RESTRICT_FV = 1 } msrsb_restriction;
typedef enum { MSRSB_ORDER_LINES = 0, MSRSB_ORDER_PARITY = 1 } msrsb_ordering;

/* Sparse FP64 fine operator, device arrays (rowptr[nrows+1], colidx[nnz],
 * val[nnz * bdim * bdim]). nrows and nnz count block rows / blocks. */
typedef struct {
    int32_t nrows, nnz, bdim;
    const int32_t *rowptr, *colidx;
    const double *val;
} msrsb_mat;

/* Cartesian fine grid and uniform coarse partition (Sec. 2.1).
 * dim 2 or 3; (nx, ny, nz) fine points (cells for centering 0, nodes for
 * centering 1; nz = 1 in 2D); (hx, hy, hz) coarse block edge in cells or
 * elements; ncomp 1 (pressure) or 3 (displacement, with bdim = 3). */
typedef struct {
    int32_t dim, nx, ny, nz, hx, hy, hz, centering, ncomp;
} msrsb_grid;

/* Alg. 1 controls: omega (Eq. 6, the paper uses 2/3); e_it is checked when
 * k mod n_it == 0 (k = 0, 1, ... counts passes); the loop stops when
 * e_it <= tol or after max_iter passes. */
typedef struct {
    double omega, tol;
    int32_t n_it, max_iter;
} msrsb_basis_opts;

typedef struct {
    msrsb_basis_opts basis;
    int32_t smoother;  /* msrsb_smoother: post-smoother for GMRES/Richardson;
                          MSRSB_SMOOTH_GS = forward pre + backward post
                          (symmetric, for PCG); MSRSB_SMOOTH_L1JAC = l1-Jacobi
                          sweeps z += D_l1^-1 (v - A z), d_i = sum_j |a_ij| over
                          the scalar row (Sec. 4: "2 sweeps of l1-Jacobi"),
                          scalar or 3x3 block operators; MSRSB_SMOOTH_IC0 =
                          incomplete Cholesky IC(0) (Sec. 4.1, 4.3), the same
                          M = L U before and after the coarse stage: for 3x3
                          blocks the incomplete factorisation on A's block
                          pattern in the node colour order (equal to the
                          pointwise one in that order, since the pattern is
                          made of whole blocks); for scalar operators ILU(0),
                          which is IC(0) for a symmetric A. ILU0, GS and IC0
                          sweep whole colours (or line blocks) at once: A's
                          (block) pattern must lie within each point's
                          3^dim neighbourhood on the grid, with at most 32
                          entries a row, else set-up returns MSRSB_EINVAL */
    int32_t pre, post; /* enable the pre / post stage of Alg. 4; for
                          MSRSB_SMOOTH_L1JAC the number of sweeps of each */
    int32_t krylov;    /* msrsb_krylov */
    int32_t restart;   /* GMRES restart length (<= 512) */
    int32_t prec;      /* msrsb_prec: F64 = all FP64; F32 = basis, P and smoother
                          in FP32 with FP32 accumulation, Krylov vectors and
                          the coarse operator in FP64 */
    int32_t no_coarse; /* 1: leave out the multiscale stage (Alg. 3) of the
                          apply, the smoothing-only baseline of Sec. 3.2 and
                          Sec. 4; 0 (default): the two-stage operator */
    int32_t restriction; /* msrsb_restriction (Sec. 2, Alg. 2): GALERKIN (default),
                          R = P^T; FV, the Petrov-Galerkin choice of the
                          multiscale finite-volume method: R_Ji = 1 for the
                          fine points i of primal block J (every component),
                          so A_c = R A P sums the fine equations over each
                          block and the coarse correction conserves mass
                          block by block. A_c is then not symmetric: not
                          with MSRSB_PCG */
    int32_t ordering;    /* msrsb_ordering: elimination order of the scalar
                          ILU(0) smoother. LINES (default): blocks of whole
                          x-lines, 2 lines high in y (and 2 deep in z), the
                          blocks coloured by the parity of their y (z) index
                          (2 colours in 2D, 4 in 3D), natural order inside a
                          block; grids with nx <= 256 and patterns whose rows
                          hold at most 32 entries coupling at most one point
                          along x and two along y and z (others use PARITY).
                          PARITY: points coloured by coordinate parity (4 / 8
                          colours), natural order inside a colour. The paper
                          eliminates in the natural order; both are parallel
                          orders, LINES the closer one */
} msrsb_opts;

typedef struct msrsb_handle msrsb_handle;

typedef struct {
    int32_t n, bdim, nc, W;           /* fine rows, block size, coarse nodes, ELL width */
    int32_t basis_iters;              /* passes of Alg. 1 performed */
    double basis_e_it;                /* last e_it evaluated */
    int32_t n_zero_diag;              /* rows with D_hat_ii = 0 (update skipped) */
    int32_t ncolours;                 /* colour classes of the smoother */
    double phase_ms[7];               /* set-up phases on the set-up stream, device time (only while
                                         msrsb_profile(1) is on, else 0): partition, filter + basis,
                                         Galerkin, coarse inverse, workspaces, wait for the smoother
                                         set-up (run on a side stream beside the Galerkin product and
                                         the coarse factorisation); then the smoother set-up's own span
                                         on the side stream */
} msrsb_info;

/* Sizes implied by a grid: fine points n, coarse nodes nc, ELL width W.
 * Host only; no device work. */
msrsb_status msrsb_partition_size(const msrsb_grid *g, int32_t *n_h, int32_t *nc_h, int32_t *W_h);

/* Primal partition, coarse nodes and support pattern (Sec. 2.1, Fig. 1).
 * part[n]: primal block of each fine point; cnode[nc]: fine index of each
 * coarse node (cell-centred: lower-middle cell of the block; vertex-centred:
 * nodes 0, H, 2H, ...); p_ids[n][W]: coarse nodes whose support holds the
 * point, in colour slots (support of J = open interval between J's
 * neighbouring coarse nodes per axis, tensor product); skel[n] = 1 where the
 * point lies on a coarse-node line of any axis. Integer results only. */
msrsb_status msrsb_partition(const msrsb_grid *g, int32_t *part, int32_t *cnode, int32_t *p_ids,
                             uint8_t *skel, cudaStream_t stream);

/* M-matrix filter (Eq. 8 and Eq. 4; Alg. 1 first steps):
 * A_hat_ij = min(A_ij, 0) off the diagonal, A_hat_ii = -sum_{j != i} A_hat_ij.
 * bdim = 1: ahat_val[nnz] in A's pattern, comp must be 0.
 * bdim = 3: separate-displacement-component block (Eq. 20, Remark 2) of
 * component comp in {0,1,2} (the (comp, comp) entry of every block), filtered;
 * ahat_val[nnz] in the block pattern.
 * n_zero_diag_h (nullable) receives the number of rows whose filtered
 * diagonal is 0 (Alg. 1 then leaves those rows unchanged). */
msrsb_status msrsb_filter(const msrsb_mat *A, int32_t comp, double *ahat_val, int32_t *n_zero_diag_h,
                          cudaStream_t stream);

/* Restricted smoothing of one scalar basis family (Eq. 6, Alg. 1).
 * Ahat: filtered scalar operator (bdim 1). p_ids/skel as from
 * msrsb_partition, W in {4, 8}. p_val[n][W] in precision prec: on entry the
 * initial basis (e.g. the block indicator, or a previous P as warm start,
 * Alg. 2), on return the smoothed, row-normalised P. Each pass forms
 * dP = -omega D_hat^-1 A_hat P on P's pattern only, adds it, divides every
 * row by its sum, and on check passes takes e_it = max |dP| over non-skeleton
 * rows. iters_h, e_it_h (nullable): passes done and last e_it. */
msrsb_status msrsb_build_basis(const msrsb_mat *Ahat, const int32_t *p_ids, const uint8_t *skel, int32_t W,
                               const msrsb_basis_opts *opts, int32_t prec, void *p_val, int32_t *iters_h,
                               double *e_it_h, cudaStream_t stream);

/* Allocation-free variant of msrsb_build_basis (no counterpart in the
 * paper). For callers that cannot allocate device memory: code running under
 * an external memory manager that already owns the GPU's memory (a serving
 * framework's caching allocator, a memory-capped container), or host loops
 * that must not take the allocator's locks and implicit synchronisation.
 * Same arguments and results as msrsb_build_basis (the filtered operator is
 * read in CSR form directly; the row normalisation divides where
 * msrsb_build_basis multiplies by a reciprocal, so results agree to rounding);
 * the scratch it needs lives in one static device array of 10 MiB + 33,288
 * bytes that every GPU loading the library holds until the process exits.
 * Limits: n * W <= 1,048,576, n <= 262,144 and max_iter <= 4096; larger
 * inputs return MSRSB_ESHAPE and do nothing.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture. All calls on a device share the array and each call resets the
 * parts that must start at zero: calls that overlap on the GPU (different
 * streams or host threads at the same time) race and give wrong results.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
msrsb_status msrsb_build_basis_noalloc(const msrsb_mat *Ahat, const int32_t *p_ids, const uint8_t *skel,
                                       int32_t W, const msrsb_basis_opts *opts, int32_t prec, void *p_val,
                                       int32_t *iters_h, double *e_it_h, cudaStream_t stream);

/* Galerkin coarse operator A_c = P^T A P (Eq. 3, Alg. 2) with the
 * unfiltered A, as a block CSR matrix. g is the grid P was built on
 * (msrsb_partition); p_ids[n][W] in colour slots. For bdim = 3, P is block
 * diagonal per component (Sec. 4): p_val holds 3 families [3][n][W].
 * A_c has nc block rows of bdim x bdim blocks (coarse dof = bdim*J +
 * component); row J stores the coarse nodes at most one coarse step from J on
 * every axis (its 3^dim stencil), columns ascending: ac_rowptr[nc+1],
 * ac_colidx[nnzb], ac_val[nnzb][bdim][bdim] (row-major blocks), device
 * arrays owned by the caller. *nnzb_h (host, required) receives the number
 * of blocks, prod_d (3 nb_d - 2) for nb_d coarse nodes along axis d. With
 * ac_val == NULL the call only sets *nnzb_h (no device work), so a caller can
 * size the arrays first. Deterministic (fixed summation order). */
msrsb_status msrsb_coarse_op(const msrsb_mat *A, const msrsb_grid *g, const int32_t *p_ids, const void *p_val,
                             int32_t prec, int32_t *ac_rowptr, int32_t *ac_colidx, double *ac_val,
                             int32_t *nnzb_h, cudaStream_t stream);

/* Alg. 2 set-up of the whole preconditioner: partition, filter, Alg. 1, A_c,
 * the FP64 coarse solver M_c^-1 = A_c^-1 and the smoother (multicolour
 * ILU(0), multicolour block Gauss-Seidel, or l1-Jacobi). The coarse solver is
 * an exact block LU of A_c over the planes of the coarse grid along its last
 * axis (z in 3D, y in 2D): the dense inverse of each plane's Schur
 * complement, by Gauss-Jordan elimination with partial pivoting inside the
 * plane. A plane holds nb_x * nb_y * bdim (3D) or nb_x * bdim (2D) coarse
 * unknowns; beyond about 640 of them (one thread-block cluster's shared
 * memory) the dense inverse of the whole A_c is used instead, which needs
 * nc * bdim <= 8192, else MSRSB_ESHAPE. A zero pivot gives MSRSB_EBREAKDOWN.
 * p_init (nullable, device, layout of p_val) is a warm-start basis; NULL
 * starts from the block indicator. The handle keeps a non-owning reference
 * to A's arrays, which must stay alive and unchanged until msrsb_destroy; it
 * owns everything else it allocates (stream-ordered allocations on `stream`).
 * *out receives the handle. */
msrsb_status msrsb_setup(const msrsb_mat *A, const msrsb_grid *g, const msrsb_opts *opts, const void *p_init,
                         msrsb_handle **out, cudaStream_t stream);

/* Alg. 4 (with Alg. 3 inside) from z = 0: optional pre-smoothing, coarse
 * correction with the residual, optional post-smoothing. v, z: FP64[n*bdim]. */
msrsb_status msrsb_apply(msrsb_handle *h, const double *v, double *z, cudaStream_t stream);

/* Krylov solve of A x = b preconditioned by Alg. 4: right-preconditioned
 * GMRES (restarted; Arnoldi by classical Gram-Schmidt with the
 * reorthogonalisation delayed one step) or PCG, until
 * ||b - A x||_2 <= rtol ||b||_2 or maxit iterations. x: in initial guess, out solution (FP64). iters_h, relres_h
 * receive the iteration count and the final true relative residual; hist_h
 * (nullable, host, maxit+1 doubles) the relative residual estimate per
 * iteration. Returns MSRSB_ENOCONV, with x holding the last iterate, when
 * maxit is reached first. */
msrsb_status msrsb_solve(msrsb_handle *h, const double *b, double *x, double rtol, int32_t maxit,
                         int32_t *iters_h, double *relres_h, double *hist_h, cudaStream_t stream);

/* msrsb_solve for nrhs right-hand sides of the handle's operator: B, X
 * FP64 [nrhs][n*bdim] (right-hand side r at B + r*n*bdim; X: in initial
 * guesses, out solutions); iters_h, relres_h host [nrhs]. In the
 * configuration of the flow cases (scalar operator, GMRES, coarse stage, one
 * ILU(0) post-sweep in the line-block order on grids of nx <= 128, no
 * pre-smoother) up to 8 right-hand sides run in lockstep: every step applies
 * the preconditioner and A to all of them with kernels that read A, P, the
 * coarse inverse and the ILU(0) factors once for all; each right-hand side
 * performs exactly the operations of its own msrsb_solve, so its iterations
 * and solution are the same. Otherwise the right-hand sides are solved one
 * after another. Synchronises `stream`. Returns the first failure
 * (MSRSB_ENOCONV and others as msrsb_solve); the right-hand sides before it
 * are solved. */
msrsb_status msrsb_solve_multi(msrsb_handle *h, int32_t nrhs, const double *B, double *X, double rtol, int32_t maxit,
                               int32_t *iters_h, double *relres_h, cudaStream_t stream);

/* y = A x for a fine operator (FP64 CSR or 3x3 block CSR, device arrays;
 * x, y FP64 [nrows * bdim], not aliased). Stream-ordered. */
msrsb_status msrsb_spmv(const msrsb_mat *A, const double *x, double *y, cudaStream_t stream);

/* Copies of the set-up results, for checks: p_ids[n][W], p_val[comp][n][W]
 * (handle precision), Ac_dense[nC][nC] (A_c expanded to a dense row-major
 * matrix, nC = nc * bdim); any pointer may be NULL. */
msrsb_status msrsb_get_setup(msrsb_handle *h, int32_t *p_ids, void *p_val, double *Ac_dense, cudaStream_t stream);
msrsb_status msrsb_get_info(const msrsb_handle *h, msrsb_info *info_h);

/* Releases everything the handle owns (after synchronising its stream). */
msrsb_status msrsb_destroy(msrsb_handle *h);

/* End-to-end call with HOST buffers: copies A and b to the device, runs
 * msrsb_setup and msrsb_solve, copies x back, frees its device memory.
 * A_h arrays and b_h, x_h are host pointers (pinned memory recommended). */
msrsb_status msrsb_solve_host(const msrsb_mat *A_h, const msrsb_grid *g, const msrsb_opts *opts, const double *b_h,
                              double *x_h, double rtol, int32_t maxit, int32_t *iters_h, double *relres_h,
                              cudaStream_t stream);

/* Ensembles (the paper solves one problem at a time; this is the Alg. 2
 * set-up followed by solves with Alg. 4, applied to many independent
 * problems, e.g. permeability realisations of different grid sizes, each with
 * several right-hand sides). One problem: its operator (device arrays, as for
 * msrsb_setup), grid, nrhs right-hand sides b (device, FP64, nrhs*n*bdim,
 * right-hand side r at offset r*n*bdim) and solutions x (device, same layout;
 * in: initial guesses, out: solutions), and host arrays iters_h[nrhs],
 * relres_h[nrhs] for the per-solve results. */
typedef struct {
    const msrsb_mat *A;
    const msrsb_grid *g;
    const double *b;
    double *x;
    int32_t nrhs;
    int32_t *iters_h;
    double *relres_h;
    msrsb_status status; /* out: this problem's status (MSRSB_OK, or its first error) */
} msrsb_problem;

/* Runs msrsb_setup, nrhs x msrsb_solve and msrsb_destroy for every problem,
 * `concurrency` problems at a time (1..64), each on a stream of its own from
 * a pool of host threads; the set-ups and solves of different problems
 * overlap on the GPU. Every problem's results are those its own
 * setup/solve/destroy sequence gives (the kernels are deterministic).
 * Returns MSRSB_OK when every problem succeeded, else the status of the
 * lowest-numbered failed problem (each problem's own status is in
 * probs[i].status). Blocks until all problems are done. */
msrsb_status msrsb_solve_ensemble(int32_t nprob, msrsb_problem *probs, const msrsb_opts *opts, double rtol,
                                  int32_t maxit, int32_t concurrency);

/* Adjoint support (the paper has no adjoint; an objective J(x) of the
 * solution of A x = b has dJ/db = lambda and dJ/dA_ij = -lambda_i x_j with
 * A^T lambda = dJ/dx).
 * msrsb_transpose_values: for a structurally symmetric A (columns ascending
 * in every row), writes the values of A^T in A's own pattern into val_t
 * (device, same length as A->val, must not alias it): val_t at entry (i, j)
 * is A(j, i), 3x3 blocks transposed. A's rowptr/colidx with val_t form A^T,
 * on which msrsb_setup builds the MsRSB preconditioner of the adjoint system.
 * Returns MSRSB_ESHAPE when an entry has no mirror entry. Synchronises the
 * stream. */
msrsb_status msrsb_transpose_values(const msrsb_mat *A, double *val_t, cudaStream_t stream);

/* grad (device, same layout as A->val) = alpha * lambda x^T restricted to A's
 * pattern: entry (i, j) gets alpha * lam[i] * x[j] (blocks: row l of block
 * row i, column m of block column j). With alpha = -1 this is dJ/dA. */
msrsb_status msrsb_pattern_outer(const msrsb_mat *A, double alpha, const double *lam, const double *x, double *grad,
                                 cudaStream_t stream);

/* MPFA-O Darcy operator of a 3D grid of unit cells and its adjoint
 * derivative (the paper has no adjoint; this differentiates the forward model
 * that the preconditioner serves). Cell tensors K_c = exp(theta_c) K_hat_c,
 * K_hat [n][9] row-major 3x3, theta [n], cells x fastest; MPFA-O with the
 * continuity points at the half-face midpoints (the O-method on unit cells),
 * no-flow outer faces, bottom-hole-pressure wells at the cells
 * well_cells_h[w] (host) with pressures well_pw_h[w]: A_ii += WI_i,
 * b_i = WI_i p_w, WI_i the MPFA-O diagonal A_ii. g must be 3D, cell-centred,
 * ncomp 1.
 * msrsb_mpfa_assemble: val (device, nnz) in the caller's CSR pattern
 * rowptr/colidx, which must be each cell's in-grid 3x3x3 neighbours in
 * ascending order; b (device, n). Interaction regions are solved in FP64,
 * rows gathered in a fixed order (deterministic). Synchronises the stream.
 * msrsb_mpfa_gradient: grad (device, n) = -lambda^T (dA/dtheta_c) p +
 * lambda^T (db/dtheta_c) for every cell c, i.e. dJ/dtheta when A p = b and
 * A^T lambda = dJ/dp (lambda, p device vectors). Per interaction region the
 * local system C u = D p and its adjoint C^T mu = G^T w are solved (w the
 * differences of lambda across the half-faces) and each cell's share is
 * gathered in a fixed order. */
msrsb_status msrsb_mpfa_assemble(const msrsb_grid *g, const double *K_hat, const double *theta, int32_t nwells,
                                 const int32_t *well_cells_h, const double *well_pw_h, const int32_t *rowptr,
                                 const int32_t *colidx, double *val, double *b, cudaStream_t stream);
msrsb_status msrsb_mpfa_gradient(const msrsb_grid *g, const double *K_hat, const double *theta, int32_t nwells,
                                 const int32_t *well_cells_h, const double *well_pw_h, const double *lam,
                                 const double *p, double *grad, cudaStream_t stream);

/* Launch-shape autotuner (no counterpart in the paper; the paper's method is
 * unchanged by it). The restricted-smoothing pass of Eq. 6 / Alg. 1 has
 * several launch shapes that give bit-identical results: 1 or 2 lanes per
 * fine row (32 or 16 rows per warp; a lane gathers W/lanes of P's colour
 * slots), 256 or 128 threads per CTA, and 0, 2 or 3 of the row's operator
 * entries loaded ahead of the current entry's gather, with registers left
 * free or capped at the one-lane kernel's occupancy. Variants 0..5 are
 * (lanes, threads, ahead, capped) = (1,256,0,0) (1,128,0,0) (2,256,0,0)
 * (1,256,2,0) (1,256,2,1) (1,256,3,1). With MSRSB_TUNE_AUTO (the default)
 * the first Alg. 1 loop of a new size class runs each shape in turn for a
 * warm pass (leaving the caches as that shape leaves them) and two passes
 * timed together by one pair of CUDA events on the loop's stream, so that the
 * second overlaps the first's tail as in the loop (a pair never starts on a
 * check pass: one more warm pass instead); one host synchronisation at the
 * end; it then uses the shape with the fastest timed pair for its remaining
 * passes and for every later loop of the same class in the process. A class is
 * (kernel, device, value size, W, ceil(log2 n), ceil(log2 of the operator's
 * stored entries per row)); loops with max_iter < 27 use variant 0 without
 * tuning, and a loop that converges during its trial passes stores nothing.
 * The table is process-wide and guarded for concurrent host threads.
 * msrsb_tune_mode(m): m = MSRSB_TUNE_AUTO, or 0..5 to force that variant for
 * every loop (no timing, no table update); EINVAL otherwise.
 * msrsb_tune_reset(): empties the table. msrsb_tune_table(out, cap, count_h):
 * writes min(cap, entries) entries to host array out (nullable when cap = 0)
 * and the number of entries to *count_h. Host bookkeeping only. */
#define MSRSB_TUNE_AUTO (-1)
typedef enum { MSRSB_TUNE_SMOOTH = 0 } msrsb_tune_kernel;
typedef struct {
    int32_t kernel;      /* msrsb_tune_kernel */
    int32_t device;      /* CUDA device ordinal */
    int32_t value_bytes; /* 4 (FP32 basis) or 8 (FP64 basis) */
    int32_t W;           /* colour slots per row (4 or 8) */
    int32_t n_log2;      /* ceil(log2 n) */
    int32_t width_log2;  /* ceil(log2 (stored entries / n)) */
    int32_t variant;     /* the chosen shape */
    int32_t lanes;       /* its lanes per row */
    int32_t threads;     /* its threads per CTA */
    int32_t ahead;       /* its operator entries loaded ahead */
    int32_t capped;      /* its registers capped for occupancy */
    int32_t n_variants;  /* shapes timed */
    float us[8];         /* each shape's timed pair, microseconds per pass */
} msrsb_tune_entry;
msrsb_status msrsb_tune_mode(int32_t mode);
msrsb_status msrsb_tune_reset(void);
msrsb_status msrsb_tune_table(msrsb_tune_entry *out, int32_t cap, int32_t *count_h);

/* Measurement support (no counterpart in the paper). msrsb_profile(1)
 * resets the counters and brackets every Alg. 1 loop (the restricted-smoothing
 * passes of one basis family) with one pair of CUDA events on its stream, so
 * that the passes keep their programmatic overlap; msrsb_profile(0) resets and
 * stops the event timing. msrsb_profile_read returns the number of kernel
 * launches the library made since the last reset (every kernel of csrc/, not
 * counting CUB's sort/scan kernels), the number of smoothing launches that did
 * work (launches that left at once after convergence are excluded) and the
 * summed device time (ms) of the loops they ran in. Host bookkeeping only. */
msrsb_status msrsb_profile(int32_t enable);
msrsb_status msrsb_profile_read(int64_t *launches_h, int64_t *smooth_launches_h, double *smooth_ms_h);

/* Arithmetic-rate probe (measurement support, no counterpart in the paper):
 * launches blocks_per_sm (1..64) CTAs of 256 threads per SM, every thread
 * running 8 independent chains of 2048 fused multiply-adds in precision prec
 * (MSRSB_F64 or MSRSB_F32), and returns the best rate of 5 event-timed
 * launches in fma_per_s_h (FMAs per second, host) and that launch's time in
 * ms_h. The roofline denominator for kernels bound by the FP64 or FP32 pipe.
 * Synchronises `stream`. */
msrsb_status msrsb_fma_rate(int32_t prec, int32_t blocks_per_sm, double *fma_per_s_h, double *ms_h,
                            cudaStream_t stream);

/* Self-test of the bounded device-side wait (no counterpart in the paper).
 * The coarse inverse's CTAs wait on a publication counter with a wall-time and
 * poll limit, after which the waiting CTA records a time-out status and
 * releases the others. This launches one thread waiting on a counter that
 * nothing raises, with a limit of limit_ms (0 < limit_ms <= 1000), and
 * synchronises `stream`. Returns MSRSB_ETIMEOUT when the wait gave up and
 * reported it as designed (the expected outcome; the context stays usable),
 * MSRSB_EINVAL for a bad limit or any other outcome. */
msrsb_status msrsb_wait_selftest(double limit_ms, cudaStream_t stream);

/* Message for the last non-OK status returned on this host thread. */
const char *msrsb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MSRSB_H */
