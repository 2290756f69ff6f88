/*
 * pbfb -- nonlinear Poisson-Boltzmann FEM-BEM Newton solver for one GPU.
 *
 * C ABI of libpbfb.so.  The method is the self-adjusting FEM-BEM coupling of
 * Guerrero-Montero, Bosy and Cooper (arXiv 2511.21713): the three-region
 * model of Eq. pbe_vp, the Newton-Raphson iteration of Eqs. NR_main /
 * Ec_NL_NR / Norma_Newton-Raphson with the cubic Taylor nonlinearity in the
 * first iteration (Sec. 3.2, scheme T3-HS), the optimal relaxation factor of
 * Eq. fd=0 found by Newton's method (Appendix A), the L_e skip rule and the
 * adjustable GMRES tolerance (Appendix B), and the solvation energy of
 * Eqs. Esolv / Potential_in_Omega_m.
 *
 * Discretisation solved (the three-region FEM-BEM system, reduced potential
 * u = e phi / kB T, lengths in Angstrom):
 *
 *   [ A + J(u)           eps_m R_m' M_m    -eps_s R_s' M_s ] [u    ]   [ 0            ]
 *   [ (M_m/2 + K_L) R_m  -V_L               0              ] [lam_m] = [ <u_coul,psi> ]
 *   [ (M_s/2 - K_Y) R_s   0                 V_Y            ] [lam_s]   [ 0            ]
 *
 * P1 elements everywhere; the volume unknown u lives on every vertex of the
 * tetrahedral shell Omega_i (including the vertices of Gamma_m and Gamma_s),
 * lam_m on the vertices of Gamma_m and lam_s on the vertices of Gamma_s, each
 * surface vertex list sorted by ascending shell vertex id.
 *
 * Conventions for every call:
 *   - return value: PBFB_OK (0) or an error code below; pbfb_last_error()
 *     then returns a message (thread-local, owned by the library, valid until
 *     the next call on the same thread).
 *   - input arrays are copied; the caller keeps ownership.
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *     global memory on the device that was current when the mesh was made.
 *   - all GPU work of a mesh is ordered on the stream given at creation
 *     (0 = the legacy default stream); calls return after that work is done
 *     unless stated otherwise.
 *   - there is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns PBFB_ERR_CUDA.
 *   - a mesh handle may be used by one thread at a time.
 */
#ifndef PBFB_H
#define PBFB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PBFB_OK = 0,
  PBFB_ERR_INVALID = 1,        /* bad argument or mesh */
  PBFB_ERR_CUDA = 2,           /* CUDA runtime error or no device */
  PBFB_ERR_GMRES_NOCONV = 3,   /* GMRES hit max_gmres above its tolerance */
  PBFB_ERR_NEWTON_NOCONV = 4,  /* Newton hit max_newton */
  PBFB_ERR_OMEGA = 5,          /* no relaxation factor reduced ||d|| */
  PBFB_ERR_NONFINITE = 6,      /* NaN / Inf in a residual, update or energy */
  PBFB_ERR_OOM = 7,            /* device allocation failed */
  PBFB_ERR_STATE = 8,          /* call out of order (e.g. solve before charges) */
  PBFB_ERR_TIMEOUT = 9         /* a bounded wait ended without a result (pbfb_server_poll) */
};

/* Precisions.  PBFB_FP64: everything float64.  PBFB_MIXED: GMRES operator far
 * field in float32, Newton-residual far field in float-float (pairs of float32
 * values, about 48 significant bits, on the float32 pipes), all other steps
 * float64.  PBFB_FLOAT2 (pbfb_set_params / step calls only): far field in
 * float-float. */
enum { PBFB_FP64 = 0, PBFB_MIXED = 1, PBFB_FLOAT2 = 2 };
/* Nonlinearity F of the load N(u) = eps_s kappa^2 int F(u_h) v: u, the Taylor
 * polynomials of sinh of degree 3, 5, 7, or sinh (Sec. 3.2 schemes). */
enum { PBFB_LINEAR = 0, PBFB_T3 = 1, PBFB_HS = 2, PBFB_T5 = 3, PBFB_T7 = 4 };
enum { PBFB_NEWTON = 0, PBFB_PICARD = 1 };
enum { PBFB_GAMMA_M = 0, PBFB_GAMMA_S = 1 };
enum { PBFB_PRECOND_JACOBI = 0, PBFB_PRECOND_BLOCK = 1, PBFB_PRECOND_BLOCK_DENSE = 2 };

typedef struct pbfb_mesh pbfb_mesh;

/* Newton options; the defaults (pbfb_default_opts) are the paper's best
 * Newton configuration (Appendix B: L_e = 0.35, Tol_omega = 0.1,
 * Tol_GR0 = 1e-3, Tol_GR = 1e-6, Tol_NL = 1e-3; omega_0 = 2 for the T3
 * iteration and 1 afterwards, Sec. 3.3), with the block preconditioner with
 * dense single-layer inverses on the surface rows (30 inner iterations on the
 * FEM block; the paper does not state its preconditioner).
 * In the PBFB_MIXED precision the GMRES operator (and the omega-search
 * direction p = -Acal(0) Delta, whose f_d root is needed only to Tol_omega)
 * evaluates the far field in float32, while the Newton residual
 * d = b - Acal(0) Phi - N(Phi) uses the float-float far field (float64-level
 * accuracy at a fraction of GB300's float64 cost); PBFB_FP64 uses float64
 * everywhere. */
typedef struct pbfb_newton_opts {
  int precision;        /* PBFB_FP64, or PBFB_MIXED: BEM far field in float32 */
  double tol_nl;        /* stop when e_k = omega ||Delta||_2 < tol_nl */
  double tol_gmres;     /* final relative GMRES tolerance Tol_GR */
  double tol_gmres0;    /* initial tolerance Tol_GR0 (linear part, early steps) */
  double tol_omega;     /* |f_d(omega)| < tol_omega ends the omega search */
  double L_e;           /* reuse the previous omega once e_k < L_e (0 = never) */
  double omega0_first;  /* start of the omega search in the first iteration */
  double omega0_rest;   /* start afterwards */
  double omega_max;     /* admissible omega in (0, omega_max], finite */
  int max_newton;
  int max_gmres;        /* GMRES iterations per linear solve */
  int restart;          /* GMRES restart length (<= 400) */
  int max_omega_iters;
  int n_taylor;         /* iterations 0..n_taylor-1 use taylor[k], later ones sinh (0..4);
                           default 1 with taylor[0] = PBFB_T3 (the paper's T3-HS) */
  int taylor[4];        /* PBFB_T3 / PBFB_T5 / PBFB_T7 (e.g. T3-T5-T7-T7-HS) */
  int method;           /* PBFB_NEWTON (Sec. 2.4.2) or PBFB_PICARD (Sec. 2.4.1: the same
                           increment with J = 0 in the linear operator; omega by the direct
                           secant of Appendix A, Eq. SEC_FD, and the R_e reuse rule) */
  double R_e;           /* Picard: recompute omega only when e_{k-1}/e_k < R_e (0: always) */
  int omega_warm_start; /* Newton, first iteration: start the omega search from three
                           bisection steps of f_d on [2, 3] followed by secant steps until
                           |d omega| < 0.05 (Sec. 3.5); 0 = start from omega0_first */
  int omega_search;     /* 1: automatic omega; 0: constant omega0_first / omega0_rest */
  int precond;          /* PBFB_PRECOND_JACOBI: diagonal of the coupled operator;
                           PBFB_PRECOND_BLOCK: flexible GMRES with a block-triangular
                           preconditioner: the diagonal on the surface rows, then
                           inner_iters Jacobi-PCG iterations on the FEM block A + J for
                           the FEM right-hand side minus its coupling to those rows;
                           PBFB_PRECOND_BLOCK_DENSE (default): the same FEM block, and on
                           the surface rows the inverses of the dense float32 single-layer
                           matrices (-V_L on Gamma_m, V_Y on Gamma_s; see
                           pbfb_single_layer_dense), which keep the GMRES iteration count
                           flat under mesh refinement.  A surface of more than 40960
                           vertices keeps the diagonal.  The inverse of V_L is built once
                           per mesh, that of V_Y once per kappa: about 2 (n/128*128)^3
                           float32 flops and 4 (n/128*128)^2 bytes of device memory per
                           surface of n vertices (n rounded up to a multiple of 128). */
  int inner_iters;      /* PCG iterations per block-preconditioner application (1..500) */
  double accept_ratio;  /* a relaxation factor is accepted when ||d(omega)||^2 < accept_ratio
                           ||d(0)||^2, in [0, 1]; 1 (default) is the paper's global convergence
                           condition ||d(omega)|| < ||d(0)|| (Sec. 2.5.2), smaller values ask for
                           a sufficient decrease, and 0 makes every search fail (PBFB_ERR_OMEGA),
                           which tests use to force that path */
  double residual_update; /* PBFB_MIXED only; 0 (default) evaluates the Newton residual's far field
                           in float-float at every step.  tau > 0: a step may instead update it by
                           linearity, b - Acal(0) Phi_{k+1} = (b - Acal(0) Phi_k) + omega_k p_k
                           with p_k = -Acal(0) Delta_k from the float32 operator, while the sum of
                           the updates omega ||Delta|| since the last float-float evaluation stays
                           below tau ||Phi_{k+1}||; the updates' rounding is that of the float32
                           far field applied to the increments, not to Phi */
  int residual_far;       /* PBFB_MIXED only: far field of the Newton residual b - Acal(0) Phi
                           where it is evaluated in full.  PBFB_FLOAT2 (default): float-float
                           direct sum; PBFB_MIXED: the GMRES operator's float32 far field (direct
                           or treecode as tuned, about 1e-6 of the largest entry), the rounding
                           the residual updates above already carry.  Any other value:
                           PBFB_ERR_INVALID */
} pbfb_newton_opts;

#define PBFB_MAX_TRACE 64

/* Result of one solve; energies in kcal/mol (Eq. Esolv). */
typedef struct pbfb_result {
  double dG_total, dG_LC, dG_NC, dG_Omega_i;
  int status;
  int newton_iters;
  int linear_gmres_iters;
  int omega_fallbacks;                 /* omega searches that needed the scan */
  int gmres_iters[PBFB_MAX_TRACE];
  double omega[PBFB_MAX_TRACE];
  double e[PBFB_MAX_TRACE];            /* e_{k+1} = omega ||Delta||_2; a step whose residual d is
                                          exactly zero (no charges) stops with omega = e = 0 */
  int omega_evals[PBFB_MAX_TRACE];     /* batched residual evaluations per step */
  double ms_linear, ms_newton, ms_energy;
  int residual_updates;                /* Newton steps whose residual was updated by linearity
                                          (pbfb_newton_opts.residual_update) */
} pbfb_result;

/* Fills *opts with the defaults above. */
void pbfb_default_opts(pbfb_newton_opts* opts);

/* Creates a mesh on the current CUDA device.
 *   xyz      host, n_v x 3 float64 vertex coordinates of the shell Omega_i.
 *   tets     host, n_t x 4 int32 vertex ids (any orientation, nonzero volume).
 *   gm_tris  host, n_gm x 3 int32 ids of the Gamma_m faces, oriented with the
 *            normal pointing into Omega_i (out of the solute).
 *   gs_tris  host, n_gs x 3 int32 ids of the Gamma_s faces, oriented with the
 *            normal pointing out of Omega_i (into the far field).
 *   stream   cudaStream_t as an integer (0 = default stream).
 * The two surfaces must be closed and disjoint, and together be exactly the
 * boundary faces of the tets (PBFB_ERR_INVALID otherwise).  Builds the CSR
 * pattern and element-to-slot maps of the FEM rows, the surface quadrature
 * data, and the Laplace near-field correction of Gamma_m (Sauter-Schwab
 * quadrature for touching triangle pairs, subdivided quadrature for close
 * ones).  *out is owned by the caller until pbfb_mesh_destroy. */
int pbfb_mesh_create(const double* xyz, int32_t n_v, const int32_t* tets, int64_t n_t,
                     const int32_t* gm_tris, int32_t n_gm, const int32_t* gs_tris, int32_t n_gs,
                     uintptr_t stream, pbfb_mesh** out);

/* Creates a mesh of Omega_m and Omega_i together: the paper's own formulation (Sec. 2.2,
 * Eq. fembem_matrix), with FEM over both regions (eps_m in Omega_m, eps_s and the ions in
 * Omega_i), the charges as point loads 4 pi l_B sum_k z_k v_i(x_k) of the P1 hat functions,
 * and the Yukawa BEM on Gamma_s.
 *   tet_region  host, n_t int32: 0 for a tet of Omega_m, 1 for one of Omega_i.
 *   gm_tris     the faces between Omega_m and Omega_i tets (every one of them, each once),
 *               oriented with the normal into Omega_i.
 *   gs_tris     the boundary faces of the tets (all of them), normal out of Omega_i.
 * Other arguments as pbfb_mesh_create.  The unknowns keep the layout [u; lam_m; lam_s]: during
 * the solve the lam_m rows are the identity (lam_m = 0, no coupling); a converged solve then
 * fills lam_m from the Gamma_m boundary integral equation of Sec. 2.3.1 (pbfb_gamma_m_flux) and
 * takes the energy as for a shell mesh (Eq. Esolv, Eq. Potential_in_Omega_m), Delta G_Omega_i
 * over the Omega_i tets.  pbfb_charges_set then requires every charge to lie in an Omega_m tet
 * (barycentric coordinates >= -1e-12; PBFB_ERR_INVALID otherwise).  pbfb_solve_batch takes such
 * meshes like any other; the request server builds them from requests with tet_region set. */
int pbfb_mesh_create_full(const double* xyz, int32_t n_v, const int32_t* tets, int64_t n_t,
                          const int32_t* tet_region, const int32_t* gm_tris, int32_t n_gm,
                          const int32_t* gs_tris, int32_t n_gs, uintptr_t stream, pbfb_mesh** out);

/* Flux lam_m on Gamma_m from the trace of u (Sec. 2.3.1, the Gamma_m limit of
 * Eq. Potential_in_Omega_m): solves V_L lam = (M_m/2 + K_L) u|Gamma_m
 * - c (l_B/eps_m) <u_coul, psi>, c = coulomb (0 or 1), by preconditioned CG on V_L (dense
 * float32 V_L^-1 as preconditioner up to 40960 vertices, else its diagonal; far field in float64
 * for FP64, float-float otherwise) to a relative residual of 1e-13.  x_dev: device, n float64
 * (only the u part is read); lam_dev: device, n_m float64 (may point into x_dev's lam_m part).
 * Needs pbfb_set_params, and pbfb_charges_set when coulomb = 1 (PBFB_ERR_STATE).  On a shell
 * mesh it reproduces a solution's own lam_m (the same Gamma_m row).  PBFB_ERR_GMRES_NOCONV if
 * CG stalls. */
int pbfb_gamma_m_flux(pbfb_mesh* mesh, const double* x_dev, int coulomb, double* lam_dev);

/* sizes[0..7] = n_v, n_t, n_m, n_s, n = n_v + n_m + n_s, nnz of the FEM rows,
 * nnz of the Gamma_m and Gamma_s BEM-row sparse parts.  sizes: host. */
int pbfb_mesh_sizes(const pbfb_mesh* mesh, int64_t* sizes);

/* Shell vertex ids of the vertices of surface `which` (PBFB_GAMMA_M/S), in
 * the order of the lam_m / lam_s unknowns.  out: host, n_m or n_s int32. */
int pbfb_surface_vertices(const pbfb_mesh* mesh, int which, int32_t* out);

/* Sets the point charges (host, n_q x 3 positions in Angstrom, n_q charges in
 * units of e) and computes <sum_k z_k / |x - x_k|, psi_i> on Gamma_m
 * (the Coulomb data of Sec. 2.3.1).  Charges must be finite; n_q >= 1.  On a
 * shell mesh every charge must lie strictly inside Gamma_m (in Omega_m, as the
 * three-region model of Sec. 2.1 places them), checked on the host by the
 * winding number of pbfb_check_charges before any GPU work; PBFB_ERR_INVALID
 * otherwise, the mesh keeping its previous charges. */
int pbfb_charges_set(pbfb_mesh* mesh, const double* xyz, const double* z, int32_t n_q);

/* Host-only input check (no GPU needed): the generalised winding number
 * w(x) = (1/4 pi) sum over Gamma_m's triangles of their signed solid angles at
 * each charge (1 inside, 0 outside, 1/2 on the surface, for the orientation of
 * pbfb_mesh_create: normal out of the solute).  xyz: host, n_v x 3 float64;
 * gm_tris: host, n_gm x 3 int32; q_xyz: host, n_q x 3 float64; winding_out:
 * host, n_q float64 or NULL.  Returns PBFB_ERR_INVALID (with the first
 * offending charge in pbfb_last_error) unless every w > 3/4, or for a bad
 * argument (vertex id out of range, non-finite position). */
int pbfb_check_charges(const double* xyz, int32_t n_v, const int32_t* gm_tris, int32_t n_gm,
                       const double* q_xyz, int32_t n_q, double* winding_out);

/* Full solve (Sec. 2.4): linear part, Newton with the omega search, energy.
 * eps_in = eps_m, eps_out = eps_s (> 0), kappa >= 0 in 1/Angstrom, T > 0 K.
 * opts: NULL for the defaults.  u_out (n_v), lam_m_out (n_m), lam_s_out (n_s):
 * host buffers for Phi_T = Phi_L + Phi_NL, or NULL to skip.  res: host, may
 * be NULL.  Returns the solve status (also in res->status). */
int pbfb_solve(pbfb_mesh* mesh, double eps_in, double eps_out, double kappa, double T,
               const pbfb_newton_opts* opts, double* u_out, double* lam_m_out,
               double* lam_s_out, pbfb_result* res);

/* As pbfb_solve, with x_out a device buffer of n float64 receiving
 * [u; lam_m; lam_s] (or NULL). */
int pbfb_solve_device(pbfb_mesh* mesh, double eps_in, double eps_out, double kappa, double T,
                      const pbfb_newton_opts* opts, double* x_out_dev, pbfb_result* res);

/* Releases every resource of the mesh (NULL is accepted). */
int pbfb_mesh_destroy(pbfb_mesh* mesh);

/* Message of the last error on this thread ("" if none). */
const char* pbfb_last_error(void);

/* ---- Step-level entry points (device pointers), for verification and timing. */

/* Sets eps_in, eps_out, kappa, T and the precision used by the calls below;
 * builds the Yukawa near-field correction of Gamma_s for this kappa (cached
 * until kappa changes).  The Jacobian block is reset to J = 0. */
int pbfb_set_params(pbfb_mesh* mesh, double eps_in, double eps_out, double kappa, double T,
                    int precision);

/* Step a1 (Eqs. Vector_c, NR_main): for u (device, n_v) and scheme
 * PBFB_LINEAR / PBFB_T3 / PBFB_HS, stores J(u) = eps_s kappa^2 int F'(u_h) v_i v_j
 * in the operator's FEM block and, if N_out is not NULL, writes
 * N(u)_i = eps_s kappa^2 int F(u_h) v_i (device, n_v). */
int pbfb_assemble(pbfb_mesh* mesh, int scheme, const double* u_dev, double* N_out_dev);

/* Resets the Jacobian block to J = 0 (the operator Acal of Eq. general_nonlinear). */
int pbfb_clear_jacobian(pbfb_mesh* mesh);

/* Steps a2-a4: y = Acal(J) x for the current J (device, n each). */
int pbfb_apply(pbfb_mesh* mesh, const double* x_dev, double* y_dev);

/* One boundary operator alone on surface `which`: op 0 = V (single layer),
 * op 1 = K (double layer), Laplace on Gamma_m and Yukawa on Gamma_s, applied
 * to the P1 coefficients x (device, n_m or n_s); y (device) same length. */
int pbfb_bem_apply(pbfb_mesh* mesh, int which, int op, const double* x_dev, double* y_dev);

/* pbfb_bem_apply without device allocation (the paper has no counterpart).
 * For callers that may not allocate GPU memory while they run -- for example
 * a host that has handed all device memory to its own pool, or a request
 * loop that must not call cudaMalloc/cudaFree (which synchronise the device)
 * between requests.  Computes V x or K x on surface `which` as
 * pbfb_bem_apply does with the float32 far field (whatever precision
 * pbfb_set_params chose) plus the float64 near-field correction: the same
 * split kernel, targets per thread and split rule, with at most 8 source
 * splits (results equal to float64 rounding), except that a mesh tuned to the
 * mutual-pair kernel (pbfb_tuning.nbody_packed = 2) runs the packed split
 * kernel instead (equal to float32 rounding), and a mesh whose float32 far
 * field runs the treecode (pbfb_tuning.treecode) the direct sum (equal to the
 * treecode's approximation, about 1e-6 of the largest entry).  Its
 * working memory is one fixed library-wide device array of 6 MiB (float32
 * source records and float64 partial sums), present on every device that
 * loads the library until the process exits; the call allocates nothing.
 * Limit: 65,536 quadrature points (10,922 triangles) on the surface; larger
 * surfaces return PBFB_ERR_INVALID.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (other streams or threads) race and corrupt each other's
 * results.  x, y: device, n_m or n_s float64, distinct. */
int pbfb_bem_apply_noalloc(pbfb_mesh* mesh, int which, int op, const double* x_dev, double* y_dev);

/* Dense single-layer matrix of one surface (which: PBFB_GAMMA_M, Laplace; or
 * PBFB_GAMMA_S, Yukawa with the kappa of pbfb_set_params) in float32, or its
 * inverse (inverse = 1).  The matrix is the Galerkin V_ij of Eq. KV (Sec. 2.2)
 * assembled from the pieces of pbfb_bem_apply's op 0 (6 x 6-point rule over
 * all point pairs plus the exact-minus-regular corrections of touching and
 * near pairs), then symmetrised (V + V^T) / 2; the inverse is taken by the
 * sweep operator in float32 (the paper has no counterpart: this is the
 * surface block of the PBFB_PRECOND_BLOCK_DENSE preconditioner).
 * out_dev: device float32, n_m or n_s rows of row stride ld_out >= that
 * count, caller-owned.  Errors: INVALID for a bad argument or a surface of
 * more than 40960 vertices, STATE before pbfb_set_params, NONFINITE when a
 * pivot of the sweep is not positive (V not positive definite in float32).
 * Allocates the matrix (4 ld^2 bytes, ld = n rounded up to 128, kept with
 * the mesh) and a build scratch of at most 256 MiB, released before the call
 * returns; with inverse = 0 the preconditioner's stored inverse is rebuilt at
 * its next use. */
int pbfb_single_layer_dense(pbfb_mesh* mesh, int which, int inverse, float* out_dev, int32_t ld_out);

/* FEM rows in CSR over the full unknown vector: rowptr (n_v + 1), col and val
 * (nnz) copied to host buffers (val = A + J and the coupling masses). */
int pbfb_fem_rows(const pbfb_mesh* mesh, int32_t* rowptr, int32_t* col, double* val);

/* Step a5: GMRES (restarted, x0 = 0, right preconditioned, CGS2) on
 * Acal(J) x = b; stops when ||b - Acal x|| <= tol ||b||.  b, x: device (n).
 * precond: PBFB_PRECOND_JACOBI, PBFB_PRECOND_BLOCK or PBFB_PRECOND_BLOCK_DENSE
 * (flexible GMRES with inner_iters PCG iterations on the FEM block; the last
 * with the dense single-layer inverses on the surface rows).  iters and relres: host
 * outputs (may be NULL). */
int pbfb_gmres(pbfb_mesh* mesh, const double* b_dev, double* x_dev, double tol, int restart,
               int maxit, int precond, int inner_iters, int* iters, double* relres);

/* Step a7, batched over n_omega relaxation factors (host array omegas):
 * with w = u + omega du (device, n_v each), c = b - Acal(0) Phi and
 * p = -Acal(0) Delta (device, n each), writes for every omega 8 scalars to
 * dots (host, n_omega x 8):
 *   (p+r').r, (p+r').p, (p+r').r', r.r'', p.r'', r.r, p.r, p.p
 * where r = c - [N(w);0;0], r' = -[J(w) du;0;0], r'' = -[N''(w)[du,du];0;0]
 * (Eq. ab_pic and Appendix A).  These give f_d, f_d' and ||d(omega)||^2. */
int pbfb_omega_eval(pbfb_mesh* mesh, int scheme, const double* u_dev, const double* du_dev,
                    const double* c_dev, const double* p_dev, const double* omegas,
                    int n_omega, double* dots);

/* Step a9: energies (kcal/mol) of x_L and x_NL (device, n each) into
 * out[0..3] = Total, LC, NC, dG_Omega_i (host) (Eq. Esolv).  The reaction potential takes
 * lam_m from the vectors as given: on a mesh of Omega_m and Omega_i fill it first with
 * pbfb_gamma_m_flux (coulomb = 1 for x_L, 0 for x_NL), as a solve does. */
int pbfb_energy(pbfb_mesh* mesh, const double* xL_dev, const double* xNL_dev, double* out);

/* Launch-shape knobs of the float32 far field (an autotuner sets them):
 * targets per thread (1, 2, 4 or 8), target blocks per SM used to choose the
 * number of source splits (1..64), and packed = 1 for the variant that
 * evaluates two targets per f32x2 instruction (needs 2 or more targets per
 * thread).  0 restores the built-in heuristic.  The unpacked shapes change
 * results only in float64 rounding; the packed variant rounds the same float32
 * operations (no fused reassociation differences beyond FMA contraction).
 * Bit 1 of packed (packed = 2 or 3) selects the one-target-per-thread
 * float-float far field instead of the built-in choice (they agree to
 * float-float rounding). */
int pbfb_set_tuning(pbfb_mesh* mesh, int nbody_targets_per_thread, int nbody_blocks_per_sm,
                    int nbody_packed);

/* Launch shapes of the far-field and SpMV kernels.  Zero in a field means the
 * built-in choice.  Shapes change the order of floating-point sums only
 * (results agree to rounding), never the discrete operator. */
typedef struct pbfb_tuning {
  int32_t nbody_targets_per_thread;  /* float32 far field: 1, 2, 4 or 8 */
  int32_t nbody_blocks_per_sm;       /* float32 far field source splits: 1..64 */
  int32_t nbody_packed;              /* 1: f32x2 kernel (needs 2+ targets per thread);
                                        2: mutual pairs, each point pair evaluated once for
                                        both directions (4 targets per thread; blocks_per_sm
                                        counts one-warp blocks) */
  int32_t ff_blocks_per_sm;          /* float-float far field source splits: 1..64 */
  int32_t ff_kernel;                 /* float-float far field: 1 one target per thread,
                                        2 two per thread (float2), 3 mutual pairs, 4 mutual
                                        pairs with two targets per thread (float2) */
  int32_t spmv_lanes;                /* lanes per row of the operator's SpMV: 4, 8, 16 */
  int32_t spmv_block;                /* threads per block of that SpMV: 128, 256, 512 */
  int32_t pcg_blocks_per_sm;         /* blocks per SM of the cooperative inner PCG: 1..32
                                        (0: as many as fit) */
  int32_t pcg_lanes;                 /* lanes per row of its sparse product: 2, 4 or 8 (CSR), or
                                        1: one lane per row over a sliced-ELL copy of the block
                                        (slices of 32 rows, coalesced column-by-column storage) */
  int32_t treecode;                  /* float32 far field (GMRES operator): 1 the direct sum over
                                        all point pairs, 2 the treecode (two targets per thread; 3:
                                        the same with four targets per thread) (a binary tree over the
                                        quadrature points, leaves of 256; a cluster with
                                        r_leaf + r_cluster < 0.6 times the centre distance is
                                        replaced by 7^3 barycentric Lagrange proxies; the
                                        hierarchical far field the paper takes for large surfaces,
                                        Sec. 3); 0 built-in: the treecode for surfaces of 65,536
                                        quadrature points or more.  The treecode approximates the
                                        float32 operator (about 1e-6 of the largest entry); the
                                        Newton residual's far field follows
                                        pbfb_newton_opts.residual_far. */
  int32_t pcg_precision;             /* arithmetic of the cooperative inner PCG (CSR forms):
                                        1 float64, 2 float32 (float32 matrix and vectors, float64
                                        block and grid sums; meshes of at most 480 FEM rows per SM
                                        run the pipelined form with each row and its vectors held
                                        in registers, one grid barrier per step, for
                                        pcg_lanes 2, 4 or 8 alike); 0 built-in: float32 in the PBFB_MIXED
                                        precision, float64 otherwise.  The sliced-ELL form
                                        (pcg_lanes 1) is float64 only. */
} pbfb_tuning;

/* Current launch shapes of a mesh (zeros where the built-in choice applies). */
int pbfb_get_tuning(const pbfb_mesh* mesh, pbfb_tuning* out);

/* Sets all launch shapes at once (e.g. a cached autotuner result); INVALID if
 * a field is outside the ranges above. */
int pbfb_apply_tuning(pbfb_mesh* mesh, const pbfb_tuning* t);

/* Autotuner (the paper has no counterpart: launch shapes are a property of
 * this implementation).  Times, with CUDA events on the mesh's stream, every
 * candidate shape of the float32 far field (targets per thread 1/2/4, packed
 * or not, 8/16/32 blocks per SM of source splits; or mutual pairs with
 * 16/32/64 one-warp blocks per SM) and of the float-float far
 * field (4/8/16 blocks per SM; one or two targets per thread, or mutual
 * pairs evaluated once for both directions) on both
 * surfaces of this mesh at the current parameters, and of the operator's
 * SpMV (4/8/16 lanes per row x 128/256/512 threads) and of the cooperative
 * inner PCG of the block preconditioner (1/2/4/8 blocks per SM or all that
 * fit, 2, 4 or 8 lanes per row; 20 iterations at the current Jacobian), each
 * over reps
 * repetitions after one untimed run, and applies the fastest.  best (host,
 * may be NULL) receives the chosen shapes; ms (host, 3 doubles, may be NULL)
 * the best time per repetition of the three kernels.  Needs pbfb_set_params
 * (STATE otherwise); reps in 1..20.  Allocates two work vectors of n
 * doubles for the duration of the call (and the block preconditioner's
 * workspace, kept for later solves).  ms: 4 doubles (float32 far field,
 * float-float far field, SpMV, inner PCG). */
int pbfb_autotune(pbfb_mesh* mesh, int reps, pbfb_tuning* best, double* ms);

/* Per-kernel-class timing (CUDA events around each launch of the class) and
 * launch counters.  enable != 0 turns event timing on (it adds a little host
 * overhead per launch).  stats (host, 20 doubles):
 *   [0] launches of all kernels since the last reset,
 *   [1] float32 BEM far-field (N-body) launches, [2] their total ms, [3] their
 *       pair interactions, [4] FEM SpMV launches, [5] their ms,
 *   [6] element (assembly + omega) launches, [7] their ms,
 *   [8] float32 far-field flops (18 per Laplace pair, 24 per Yukawa pair),
 *   [9] float64 far-field launches, [10] their ms, [11] their pairs,
 *   [12] float-float far-field launches, [13] their ms, [14] their pairs,
 *   [15] ms spent building dense single-layer matrices and inverses,
 *   [16..19] host ms of pbfb_mesh_create: validation, surfaces (pair classes and
 *       correction patterns), operator pattern and gather lists, and the device
 *       set-up (geometry, stiffness, Laplace corrections) until synchronised.
 * reset != 0 zeroes the counters after reading (not the
 * set-up times). */
int pbfb_profile(pbfb_mesh* mesh, int enable, int reset, double* stats);

/* ---- Serving and batching (the paper has no counterpart; the solves are the same). */

typedef struct pbfb_server pbfb_server;

/* One solve request.  All arrays are host memory with the layouts of
 * pbfb_mesh_create / pbfb_charges_set; they are copied by pbfb_server_submit.
 * opts: NULL for the defaults. */
typedef struct pbfb_request {
  int64_t id;
  const double* xyz;
  int32_t n_v;
  const int32_t* tets;
  int64_t n_t;
  const int32_t* gm_tris;
  int32_t n_gm;
  const int32_t* gs_tris;
  int32_t n_gs;
  const double* q_xyz;
  const double* q_z;
  int32_t n_q;
  double eps_in, eps_out, kappa, T;
  const pbfb_newton_opts* opts;
  const int32_t* tet_region;  /* NULL: a shell mesh (as pbfb_mesh_create); else n_t entries, the
                                 mesh of Omega_m and Omega_i (as pbfb_mesh_create_full) */
} pbfb_request;

/* Completed request: status and result of the solve; times in ms on the host's
 * steady clock (submit, start of the solve's set-up, completion). */
typedef struct pbfb_response {
  int64_t id;
  int status;
  pbfb_result result;
  double t_submit_ms, t_start_ms, t_done_ms;
  char error[256];
} pbfb_response;

/* Starts a request server on `device`: max_inflight worker threads (1..64),
 * each with its own CUDA stream, admit queued requests in arrival order while
 * the sum of their estimated device memory stays within hbm_budget_bytes (a
 * request alone is always admitted), and run mesh creation, charges and the
 * full solve; requests that arrive while others run start as memory frees and
 * their work overlaps on the GPU.  Up to cached_meshes (0..1024) meshes stay
 * resident after their request (counted in the budget; idle ones are evicted,
 * least recently used first, when a new request needs the memory): a request
 * whose geometry equals a resident mesh's (coordinates, tets and surfaces
 * compared exactly) reuses it, skipping mesh creation, the Laplace near-field
 * corrections and dense inverse, and, at the same kappa, the Yukawa ones.
 * Each request is solved with deterministic kernels on buffers no other
 * request uses meanwhile: its result is identical to solving it alone. */
int pbfb_server_create(int device, uint64_t hbm_budget_bytes, int max_inflight, int cached_meshes,
                       pbfb_server** out);

/* Queues a request (copies its arrays; returns at once).  PBFB_ERR_OOM if its
 * estimated memory exceeds the whole budget. */
int pbfb_server_submit(pbfb_server* server, const pbfb_request* request);

/* Moves up to `max` completed responses to out (host), waiting up to
 * timeout_us microseconds for the first one; *n_out = how many.  With
 * timeout_us > 0 and no response by then: *n_out = 0 and PBFB_ERR_TIMEOUT
 * (the server is unaffected); timeout_us = 0 returns at once, PBFB_OK with
 * *n_out = 0 when nothing is ready. */
int pbfb_server_poll(pbfb_server* server, pbfb_response* out, int max, int timeout_us, int* n_out);

/* stats (host, 8 doubles): submitted, completed, queued, bytes in use
 * (running requests and resident meshes), peak bytes in use, budget,
 * requests served on a resident mesh, resident meshes. */
int pbfb_server_stats(pbfb_server* server, double* stats);

/* Finishes the requests already admitted, drops the queued ones, frees all. */
int pbfb_server_destroy(pbfb_server* server);

/* Parameters of one instance of pbfb_solve_batch (opts: NULL = defaults). */
typedef struct pbfb_batch_params {
  double eps_in, eps_out, kappa, T;
  const pbfb_newton_opts* opts;
} pbfb_batch_params;

/* Solves n meshes (charges already set) with up to max_concurrent host threads;
 * meshes created on different streams run concurrently on the GPU.  results:
 * host, n entries.  Returns the first failing instance's status. */
int pbfb_solve_batch(pbfb_mesh* const* meshes, const pbfb_batch_params* params, int n, int max_concurrent,
                     pbfb_result* results);

#ifdef __cplusplus
}
#endif
#endif /* PBFB_H */
