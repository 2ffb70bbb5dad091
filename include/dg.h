/*
 * dg.h - C ABI of the GB300 library for the high-order LDG discretisation of the thermosphere
 * model of Vila-Perez, Nguyen & Peraire (arXiv 2306.01085).
 *
 * The operations follow the semi-discrete form of Sec. 3.1 (Eq. DGformulation with the LDG trace
 * and flux of Eq. LDG2) for the nondimensional system of Eq. fluxSWNondimensional, and the
 * matrix-free Newton-GMRES solution of the DIRK stages of Sec. 3.1-3.2.
 *
 * Conventions (all calls):
 *   - Every pointer named u, q, r, v, jv, x, y is a DEVICE pointer owned by the caller, on the
 *     device that was current when the mesh was created. The library never frees them.
 *   - Layouts (row-major, contiguous, FP64 unless stated):
 *       u, r, v, jv  [n_elem][5][n_p]        variables (varrho, sqrt(rho) v_x, v_y, v_z, sqrt(rho) T)
 *       q            [n_elem][3][5][n_p]     q[e][d][c][i] ~ d u_c / d x_d (LDG gradient)
 *       x            [n_elem][3][n_p]        node coordinates (nondimensional)
 *     n_p = (p+1)^3 nodes per element: tensor GLL nodes, node i = a + (p+1) b + (p+1)^2 c with a
 *     along the first reference coordinate. Values are nodal coefficients of the Lagrange basis.
 *   - Element numbering: box e = i + nx (j + ny k); shell e = k + nz (i + nx (j + nx P)) for panel
 *     P (cube faces centred on +x, +y, -x, -y, +z, -z), angular cell (i, j) and radial layer k.
 *   - stream is a cudaStream_t (NULL: the legacy default stream). Calls are stream-ordered and
 *     asynchronous unless stated; the host reads back only what a call documents.
 *   - Every call returns DG_OK (0) or a negative status; dg_last_error() gives a thread-local
 *     message. No exception crosses the ABI.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK        0
#define DG_EINVAL   -1   /* bad argument (null pointer, unsupported size, p out of range) */
#define DG_ECUDA    -2   /* a CUDA call failed; the message names it */
#define DG_ENOMEM   -3   /* device allocation failed */
#define DG_ENOTCONV -4   /* Newton or GMRES did not reach its tolerance within its limits */
#define DG_ENAN     -5   /* a NaN or Inf appeared in a norm the solver checks */

#define DG_KIND_BOX    0 /* [0,lx]x[0,ly]x[0,lz], periodic in x and y */
#define DG_KIND_SHELL  1 /* cubed-sphere shell between r_inner and r_outer */

#define DG_BC_PERIODIC 0 /* box z ends only: periodic in z */
#define DG_BC_WALL     1 /* no-slip isothermal wall (Sec. 2.5): u_hat = (varrho,0,0,0,e^{varrho/2} T_wall) */
#define DG_BC_OUTFLOW  2 /* adiabatic, zero viscous normal stress: u_hat = u, F_hat.n = F_inv(u).n */

#define DG_JV_EXACT 0    /* exact directional derivative (forward-mode tangent of every step) */
#define DG_JV_FD    1    /* one-sided difference (r(u + eps v) - r(u)) / eps (Sec. 3.2) */

/* Problem description. Physics fields are the nondimensional numbers of Sec. 2.4. */
typedef struct dg_mesh_desc {
    int32_t kind;          /* DG_KIND_* */
    int32_t p;             /* polynomial degree k, 1 <= p <= 4 */
    int32_t nx, ny, nz;    /* box: elements per direction; shell: nx = panel cells per side, nz = layers */
    int32_t bc_lo, bc_hi;  /* DG_BC_* of the lower (z = 0 / inner) and upper (z = lz / outer) boundary */
    double lx, ly, lz;     /* box lengths */
    double r_inner, r_outer, h_first; /* shell radii, first-layer height (<= 0: uniform layers) */
    double gamma;          /* ratio of specific heats */
    double grashof;        /* Gr; viscous coefficient 1/sqrt(gamma Gr) */
    double prandtl;        /* Pr; conduction coefficient sqrt(gamma/Gr)/Pr */
    double mass;           /* m* (c_v* = 1/m*) */
    double visc_exp;       /* mu* = kappa* = T*^visc_exp (0: constant) */
    double lambda0;        /* sigma_c = lambda0 I (global Lax-Friedrichs, Eq. LDG2) */
    double t_wall;         /* wall temperature T* */
    int32_t gravity_kind;  /* 0: constant g* = gvec; 1: g* = -(g_r0/|r|)^2 r/|r| */
    int32_t euv;           /* DG_EUV_GAUSS: sub-solar Gaussian heating; DG_EUV_EUVAC: EUVAC / Chapman */
    double gvec[3];
    double g_r0;
    double omega[3];       /* rotation vector omega* */
    double froude;         /* Fr */
    double euv_amp;        /* peak heating Q* (nondimensional) */
    double euv_sigma;      /* zenith-angle standard deviation [rad] */
    double euv_r_peak;     /* radius of the peak */
    double euv_width;      /* vertical half width at half maximum */
    double euv_omega_t;    /* sub-solar rotation angle per unit nondimensional time */
    /* DG_EUV_EUVAC (Sec. 2.2): q_euv = eps n sum_j phi_j I0_j exp(-tau_j) h c/lambda_j for the single
     * constituent (atomic oxygen) with the flux, cross sections and Chapman optical depths described
     * at DG_EUV_EUVAC; q* = q H0 / (rho0 c_v0 T0 a0) enters the energy source as q* e^{-varrho/2}/c_v */
    double euv_day;        /* day of the year N_d (solar declination) */
    double euv_f107;       /* daily F10.7 index */
    double euv_f107a;      /* its 81-day mean */
    double euv_eff;        /* heating efficiency epsilon */
    double euv_dsun;       /* Sun distance [astronomical units] */
    double ref_T0;         /* reference temperature [K] */
    double ref_rho0;       /* reference density [kg/m^3] */
    double ref_m;          /* reference molecular mass [kg] (m = ref_m * mass) */
    double ref_g0;         /* gravity at the radius g_r0 [m/s^2] */
    /* Variable composition (Sec. 2.1.1-2.1.2), comp = 1: the mass fractions of N2, O2, He are
     * chi_s = sum_{j<2} comp_a[2s+j] exp(comp_b[2s+j] |r|) (|r| nondimensional), chi_O = 1 - the others;
     * m* = [sum_s chi_s/m_s*]^-1 and c_v* = 1/m* vary in space, the energy source gains
     * -(1/c_v)(sqrt(rho) T v - c_kappa kappa/(sqrt(rho) c_v) grad T).grad c_v, the transport follows
     * mu* = sqrt(T* m*) + eddy_nu rho*, kappa* = (sum_s x_s alpha_s/alpha_O) T*^0.69 + eddy_alpha rho* / m*
     * (x_s number fractions, alpha_N2 = alpha_O2 = 3.6e-4, alpha_O = alpha_He = 5.6e-4; visc_exp and
     * mass are not used), and EUVAC heating absorbs on all four species. */
    int32_t comp;
    int32_t reserved_comp; /* zero */
    double comp_a[6];      /* [species N2, O2, He][term] */
    double comp_b[6];
    double eddy_nu;        /* nu_eddy / nu_0 */
    double eddy_alpha;     /* alpha_eddy / alpha_0 */
} dg_mesh_desc;

/*
 * Heating models (dg_mesh_desc.euv):
 * DG_EUV_GAUSS: Q* = euv_amp exp(-chi^2/(2 sigma^2)) exp(-ln 2 ((|r| - r_peak)/w)^2), cos chi = r.s/|r|,
 *   s = (cos wt, -sin wt, 0).
 * DG_EUV_EUVAC: I0_j = F_j max{0.8, 1 + A_j ((F10.7 + F10.7_81)/2 - 80)} / d^2 over the 37 bands of
 *   the paper's appendix table (band centres or lines for lambda_j); tau_j = n phi_j H Ch with
 *   H = k_B T/(m g), r~ = |r|/H, y = sqrt(r~/2)|cos chi| and the Smith & Smith Chapman factor
 *   Ch = sqrt(pi r~/2) erfcx(y) (cos chi > 0), sqrt(pi r~/2)(2 exp(r~(1 - sin chi)) - erfcx(y))
 *   (cos chi <= 0 and sin chi > R0/|r|), no heating in the Earth's shadow; the Sun direction in the
 *   rotating frame is s = (-cos(delta) cos(wt), cos(delta) sin(wt), sin(delta)) with the declination
 *   delta = asin(sin(-23.44 deg) cos(2 pi/365.24 (N_d + 9) + 2 (0.0167) sin(2 pi/365.24 (N_d - 3)))).
 */
#define DG_EUV_GAUSS 1
#define DG_EUV_EUVAC 2

typedef struct dg_mesh dg_mesh;

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* dg_last_error(void);

/*
 * Build the mesh, its face connectivity, and the isoparametric geometry at the quadrature points
 * (Sec. 3.1: k-th degree curved elements; (p+1)^3 Gauss points per element, (p+1)^2 per face).
 * nodes: optional HOST array [n_elem][3][n_p] of GLL node coordinates in the numbering above (the
 * mesh as input data, read during the call only); NULL generates them from desc (Sec. 3.3 cubed
 * sphere with geometric radial growth from h_first, or the box). Faces are matched from the node
 * coordinates (corner nodes, periodic in x and y for boxes, and z when bc_lo is periodic); faces
 * left unmatched take bc_lo (box z = 0 / inner sphere) or bc_hi. Allocates all library storage on
 * the current device and synchronises it. *out receives an opaque handle to release with
 * dg_mesh_destroy. Errors: DG_EINVAL (p outside 1..4, non-positive sizes, inconsistent
 * boundaries, faces that do not match), DG_ENOMEM, DG_ECUDA.
 */
int dg_mesh_create(const dg_mesh_desc* desc, const double* nodes, dg_mesh** out);

/* Release every library allocation of the mesh (synchronises the device). NULL is ignored. */
void dg_mesh_destroy(dg_mesh* mesh);

/* Sizes: elements, nodes per element, unknowns (5 n_elem n_p). Any output pointer may be NULL. */
int dg_mesh_sizes(const dg_mesh* mesh, int64_t* n_elem, int32_t* n_p, int64_t* n_dof);

/* Copy the node coordinates x [n_elem][3][n_p] into a caller device buffer (stream-ordered). */
int dg_mesh_nodes(const dg_mesh* mesh, double* x, void* stream);

/*
 * How the FP64 evaluations (dg_gradient, dg_residual, dg_jvp with DG_JV_EXACT, the FP64 solver
 * paths) form the Gauss values and face traces of u from its nodal values (Sec. 3.1: the nodes ->
 * quadrature points map B x B x B and the extrapolation to the faces):
 *   DG_INTERP_FP64: sum-factorised 1D passes in FP64 arithmetic on the CUDA cores;
 *   DG_INTERP_TC:   one dense contraction per element on the tensor cores (tcgen05, FP16 operands
 *                   with FP32 accumulation), FP64-accurate by error-free slicing: both operands
 *                   rounded to 53 bits relative to their row / column maximum and split into seven
 *                   digits (exact in FP16); digit products of level <= 7 accumulated exactly in
 *                   FP32; the error is about 1e-15 of each variable's largest nodal value in its
 *                   element (FP64 passes: about 2e-16). Slower than DG_INTERP_FP64 on GB300.
 * The mode applies to later calls on this mesh (not stream-ordered: set it between evaluations).
 * Errors: DG_EINVAL for an unknown mode.
 */
#define DG_INTERP_FP64 0
#define DG_INTERP_TC   1
int dg_mesh_set_interp(dg_mesh* mesh, int32_t mode);

/*
 * LDG gradient, Eq. DGformulation (first equation): q solves (q, p) = -(u, div p) + <u_hat, p.n>
 * for every p in Q_h, with u_hat = (u + u^-)/2 on interior faces and the boundary traces of
 * DG_BC_*. Output q is nodal, layout [n_elem][3][5][n_p]. u and q must not overlap.
 */
int dg_gradient(dg_mesh* mesh, const double* u, double* q, void* stream);

/*
 * Residual, Eq. DGformulation (second equation), tested against every nodal basis function:
 *   r = (F(u,q), grad w) - <F_hat.n, w> + (s(u,q), w),   F_hat.n of Eq. LDG2,
 * i.e. r = M du/dt. q: nodal gradient from dg_gradient, or NULL to compute it internally from u.
 * t is the nondimensional time (used by the heating source). r must not overlap u or q.
 */
int dg_residual(dg_mesh* mesh, const double* u, const double* q, double t, double* r, void* stream);

/*
 * Jacobian-vector product of the residual, J v = d r(u + s v)/ds at s = 0 (Sec. 3.2), where q is
 * recomputed from u (the LDG gradient is part of r).
 *   mode DG_JV_EXACT: forward-mode tangent of every step; r_out (may be NULL) receives r(u) from
 *                     the same pass.
 *   mode DG_JV_FD:    (r(u + eps v) - r(u)) / eps. eps <= 0 selects
 *                     eps = sqrt(2^-52) (1 + ||u||_2) / ||v||_2 (Knoll & Keyes 2004), which reads
 *                     two norms back to the host (synchronises the stream). r_out may be NULL.
 * jv must not overlap u, v or r_out.
 */
int dg_jvp(dg_mesh* mesh, const double* u, const double* v, double t, int32_t mode, double eps,
           double* jv, double* r_out, void* stream);

/*
 * FP32 variants of dg_residual (q from u) and of the exact dg_jvp: the same discrete operators
 * with every intermediate (Gauss values, traces, gradient, fluxes, geometry) stored and computed in
 * FP32, including exp(varrho/2) = sqrt(rho) (varrho is rounded to FP32 on load, which already bounds
 * its relative error near 7e-7 at the top of the shells). Inputs and outputs are FP64 as above. The first call allocates the FP32 workspace and FP32 copies of the
 * geometry (synchronises the device once). Used as the inner Jv of the mixed-precision GMRES.
 */
int dg_residual_f32(dg_mesh* mesh, const double* u, double t, double* r, void* stream);
int dg_jvp_f32(dg_mesh* mesh, const double* u, const double* v, double t, double* jv, double* r_out, void* stream);

/*
 * Precision study of the basis contractions (interpolation to Gauss points, face extrapolation,
 * weak derivatives, lifting, projection back to the nodes) on top of the FP32 variant:
 *   DG_CM_FP32   FP32 operands (same as dg_residual_f32 / dg_jvp_f32)
 *   DG_CM_BF16   operands rounded to bfloat16, products exact, FP32 accumulation
 *   DG_CM_FP16   operands rounded to binary16, products exact, FP32 accumulation
 *   DG_CM_BF16X3 each operand split into bf16 hi + lo, three products (hi hi + hi lo + lo hi)
 *   DG_CM_FP16X3 the same with binary16 parts
 * The arithmetic of each contraction is that of a tensor-core MMA with FP32 accumulation; the
 * pointwise fluxes stay FP32. Computes r (v == NULL) or the fused r and exact
 * J v (r may then be NULL). FP64 inputs and outputs.
 */
#define DG_CM_FP32   0
#define DG_CM_BF16   1
#define DG_CM_FP16   2
#define DG_CM_BF16X3 3
#define DG_CM_FP16X3 4
int dg_eval_precision(dg_mesh* mesh, int32_t mode, const double* u, const double* v, double t, double* r,
                      double* jv, void* stream);

/* Mass matrix product (M v)_i = sum_j (phi_i, phi_j) v_j per element and variable (Sec. 3.1). */
int dg_mass_apply(dg_mesh* mesh, const double* v, double* mv, void* stream);
/* Inverse mass matrix product M^{-1} v, element by element: with (p+1)^3 Gauss points the nodal
 * mass matrix factors as B^T W B (B the square GLL-to-Gauss interpolation, W = w |J|), so
 * M^{-1} = B^{-1} W^{-1} B^{-T} (three 1D passes each way). v and mv may alias. */
int dg_mass_inverse_apply(dg_mesh* mesh, const double* v, double* mv, void* stream);

/*
 * The residual of dg_residual (q computed from u) for callers that must not have the library
 * allocate device memory during the call: applications whose own caching allocator has reserved
 * the device's memory, or loops that cannot absorb the device synchronisation that cudaMalloc and
 * cudaFree may cause. The paper has no counterpart; this is a deployment variant.
 * The call allocates nothing: its scratch is one 16 MiB FP64 array in the library's device image
 * (a file-scope __device__ array that every GPU loading the library holds until process exit).
 * A mesh needs n_elem (20 n_p + 150 (p+1)^2) doubles of it, so at most 1,109 elements at p = 2,
 * 569 at p = 3 and 335 at p = 4; larger meshes are rejected with DG_EINVAL and a message giving
 * both sizes. The array becomes resident on a device when the first mesh is created there:
 * dg_mesh_create looks up its device address (cudaGetSymbolAddress, with that device current,
 * which also loads the module holding it) and keeps it in the mesh, so this call does no set-up of
 * its own. All calls share the one array and every call
 * overwrites what it reads before reading it, so nothing needs clearing between calls; calls that
 * overlap on the GPU (other streams, other threads) race on the array and must be serialised by
 * the caller. The mesh itself (geometry, connectivity) is allocated by dg_mesh_create as usual.
 */
int dg_residual_static(dg_mesh* mesh, const double* u, double t, double* r, void* stream);

/* ----------------------------------------------------------------------------------------------
 * Implicit time step (Sec. 3.1-3.2): DIRK stages solved by Newton-GMRES
 * -------------------------------------------------------------------------------------------- */
#define DG_PC_NONE 0         /* no preconditioner */
#define DG_PC_BJ   1         /* exact element diagonal blocks of J_G, FP32 inverses (block-Jacobi) */
#define DG_PC_MLP  2         /* learned diagonal + low-rank inverse per element */
#define DG_PC_RB   3         /* reduced basis of the last Newton updates over the mass matrix (Sec. 3.2) */
#define DG_PC_RB_BJ 4        /* reduced basis over block-Jacobi */
#define DG_PC_BJ16 5         /* block-Jacobi with the FP32 inverses stored as FP16, power-of-two scale per column */

#define DG_REFRESH_STEP   0  /* build the preconditioner once per step, at u_n */
#define DG_REFRESH_STAGE  1  /* rebuild at the start of every stage */
#define DG_REFRESH_NEWTON 2  /* rebuild at every Newton iteration */
#define DG_REFRESH_LAGGED 3  /* build at u_n of one step and reuse it for the next refresh_every - 1
                                steps (a lagged preconditioner: the operator changes little over a
                                step); rebuilt sooner when the kind, the precision, dt a_11 or the
                                mesh's solver storage changes, and after a failed step */

#define DG_PREC_F64 0
#define DG_PREC_F32 1

#define DG_STATS_HIST 64

typedef struct dg_solver_opts {
    int32_t stages;          /* DIRK stages: 1 (backward Euler), 2 (DIRK(2,2)), 3 (DIRK(3,3)) */
    int32_t gmres_restart;   /* Krylov basis size before restart, 1..63 (30) */
    int32_t max_restarts;    /* GMRES cycles per Newton system before DG_ENOTCONV (10) */
    int32_t max_newton;      /* Newton iterations per stage before DG_ENOTCONV (20) */
    int32_t precond;         /* DG_PC_* */
    int32_t precond_refresh; /* DG_REFRESH_* */
    int32_t jv_mode;         /* DG_JV_EXACT or DG_JV_FD for the GMRES operator */
    int32_t jv_prec;         /* DG_PREC_F64, or DG_PREC_F32 (mixed): FP32 inner Jv, block assembly and
                                Gram-Schmidt arithmetic; the Krylov basis is stored in FP32 when
                                gmres_restart <= 31 and gmres_rtol >= 1e-6 (FP64 otherwise) */
    double newton_rtol;      /* stop when ||G||_2 <= newton_rtol ||G(U^0)||_2 (1e-8) */
    double gmres_rtol;       /* each Newton system to ||b - J x|| <= gmres_rtol ||b|| (1e-3) */
    double abs_floor;        /* or when ||G||_2 <= abs_floor ||M U||_2 (1e-14) */
    int32_t rb_size;         /* DG_PC_RB*: Newton updates kept in the reduced basis, 1..16 (8) */
    int32_t flags;           /* DG_OPT_* bits (0) */
    int32_t refresh_every;   /* DG_REFRESH_LAGGED: steps served by one preconditioner build, >= 1 (3) */
    int32_t reserved;        /* zero */
} dg_solver_opts;

/* dg_solver_opts.flags: recompute the state's Gauss values, traces and LDG gradient in every
 * operator application and every block-assembly sweep, instead of once per Krylov solve and once
 * per assembly (same results; for checking). */
#define DG_OPT_RECOMPUTE_VALUE 1

typedef struct dg_step_stats {
    int32_t status;                 /* the call's return code */
    int32_t newton_iters[3];        /* Newton iterations per stage */
    int32_t gmres_iters[3];         /* GMRES iterations per stage (all Newton systems) */
    int32_t n_hist;                 /* entries of res_hist */
    double res_hist[DG_STATS_HIST]; /* ||G||_2 at every Newton iterate, stage after stage */
    double wall_ms;                 /* host wall time of the call */
    double precond_ms;              /* of which building preconditioners */
} dg_step_stats;

/* Defaults: 3 stages, GMRES(30), 10 cycles, 20 Newton iterations, no preconditioner, exact Jv,
 * Newton 1e-8 relative, GMRES 1e-3 relative, floor 1e-14, reduced basis of 8 updates. */
void dg_solver_opts_default(dg_solver_opts* opts);

/* The DIRK tableau the step uses, derived from the order conditions: a [stages][stages] row-major,
 * c [stages]. */
int dg_dirk_tableau(int32_t stages, double* a, double* c);

/*
 * One DIRK step u_n -> u_{n+1} in place on u (device, [n_elem][5][n_p]) for M du/dt = r(u), Sec.
 * 3.1: stage i solves G(U) = M (U - u_n) - dt sum_{j<i} a_ij r(U_j) - dt a_ii r(U) = 0 by Newton's
 * method (Eq. NewtonSolve) from the previous stage value; every Newton system J_G dU = -G,
 * J_G = M - dt a_ii J_r, is solved by right-preconditioned restarted GMRES with FP64 Arnoldi
 * (classical Gram-Schmidt applied twice) and FP64 least squares. Synchronises the stream (the host
 * reads norms and Hessenberg columns). stats may be NULL. Errors: DG_ENOTCONV (Newton or GMRES
 * limits), DG_ENAN (non-finite norm or a zero block pivot), DG_EINVAL, DG_ENOMEM, DG_ECUDA. On an
 * error u is left unchanged; the caller may retry with a smaller dt.
 */
int dg_implicit_step(dg_mesh* mesh, double* u, double t, double dt, const dg_solver_opts* opts,
                     dg_step_stats* stats, void* stream);

/*
 * Build a preconditioner of J_G = M - dt_aii J_r(u) at state u and time t (DG_PC_MLP: network
 * inference for every element; see dg_mlp_init).
 * DG_PC_BJ: the exact diagonal block of every element (including the path through the
 * neighbours' LDG gradients) is computed column by column by block-diagonal tangent sweeps and
 * inverted in place in FP32 by Gauss-Jordan elimination with partial pivoting (one CTA per block in
 * shared memory when it fits; otherwise blocked by panels of 16 to 32 columns in global memory,
 * each panel's transform applied to the other columns as one product of that rank), so that applying the
 * preconditioner is one coalesced dense product per element. Synchronises the stream.
 * DG_ENAN on a zero pivot.
 * DG_PC_BJ16: as DG_PC_BJ, then every column j of an inverse is divided by the power of two c_j
 * just above its largest magnitude and rounded to FP16 (relative error 2^-11 per entry down to
 * 2^-14 c_j); the apply streams half the bytes of DG_PC_BJ and sums in FP32. Extra storage:
 * n_elem (5 n_p) ceil8(5 n_p) halves and n_elem 5 n_p floats.
 * The blocks are exact when no two faces of an element border the same neighbour (every shell;
 * boxes with at least 3 elements along each periodic direction); otherwise the gradient lifted
 * from one shared face into the other is left out and the block is an approximation.
 */
int dg_precond_setup(dg_mesh* mesh, int32_t kind, const double* u, double t, double dt_aii, void* stream);

/* y = P^{-1} x with the preconditioner last built (x, y FP64 [n_elem][5][n_p]; may alias). */
int dg_precond_apply(dg_mesh* mesh, int32_t kind, const double* x, double* y, void* stream);

/*
 * Reduced-basis preconditioner and initial guess (Sec. 3.2). The RB space W is the span of the last
 * rb_size Newton updates, kept by dg_implicit_step as a rolling window over Newton iterations,
 * stages and steps (it survives between calls until dg_rb_reset). At every Newton iteration the
 * window is orthonormalised (classical Gram-Schmidt twice, updates within 1e-10 of the span of the
 * others dropped), Z = J_G W is formed with the step's Jv mode and precision, and GMRES is
 * right-preconditioned with the inverse of
 *     J~ = P0 + (Z - P0 W) W^T,
 * which equals J_G on the RB space and the base P0 on its orthogonal complement: P0 = M (the
 * element mass matrix, DG_PC_RB, nothing assembled) or the block-Jacobi blocks (DG_PC_RB_BJ, built
 * as DG_PC_BJ is, per precond_refresh). Applied by the Woodbury identity,
 *     J~^{-1} x = P0^{-1} x - (P0^{-1} Z - W) (W^T P0^{-1} Z)^{-1} W^T P0^{-1} x,
 * i.e. one base solve, rb_size dot products and axpys. GMRES starts from the RB least-squares
 * guess x0 = W a, a = argmin ||b - Z a||_2, when it reduces the residual. With an empty window
 * J~ = P0 and x0 = 0.
 */

/* Replace the window by the r vectors w ([r][n_elem][5][n_p], device, r <= 16) and build the RB
 * preconditioner of J_G = M - dt_aii J_r(u) at (u, t) with exact FP64 Jv; base DG_PC_RB or
 * DG_PC_RB_BJ (which also builds the block-Jacobi blocks at u). dg_precond_apply with the same
 * kind then applies J~^{-1}. Synchronises the stream. */
int dg_rb_load(dg_mesh* mesh, const double* w, int32_t r, const double* u, double t, double dt_aii, int32_t base,
               void* stream);
/* x0 = W a, a = argmin ||b - Z a||_2 with the RB preconditioner last built (x0 = 0 when the space
 * is empty or the guess does not reduce ||b||). Synchronises the stream. */
int dg_rb_initial_guess(dg_mesh* mesh, const double* b, double* x0, void* stream);
/* Empty the window (the next implicit step starts without a reduced basis). */
int dg_rb_reset(dg_mesh* mesh);

/* Assemble the exact diagonal blocks of J_G = M - dt_aii J_r(u) (the ones DG_PC_BJ factors) into a
 * caller device buffer out, FP32 [n_elem][5 n_p][5 n_p], each block column-major (out[e][j][i] =
 * row i, column j; rows and columns in the element's [var][node] order). Stream-ordered. */
int dg_block_assemble(dg_mesh* mesh, const double* u, double t, double dt_aii, float* out, void* stream);

/* ----------------------------------------------------------------------------------------------
 * Learned element preconditioner (DG_PC_MLP; the paper has none, Sec. 3.2 uses a reduced basis).
 * Per element, features x (nodal varrho - mean, v, T/mean(T) - 1, mean(varrho)/10, log mean(T),
 * log(dt a_ii), log of the three element extents; 5 n_p + 6 values) go through a two-hidden-layer
 * SiLU network to D = 1 + o[:n], U, V (n x rank, row-major), n = 5 n_p, and the preconditioner is
 * P = S^{-1/2} (diag(D) + U V^T) S^{-1/2} with S the diagonal of the element mass matrix. Training
 * minimises mean || S^{-1/2} B S^{-1/2} (diag(D) + U V^T) - I ||_F^2 / n (P as a right inverse, as
 * GMRES applies it) over harvested exact blocks B of J_G with Adam; forward, backward and optimiser
 * run in the library's own FP32 kernels.
 * Supported for p <= 3.
 * -------------------------------------------------------------------------------------------- */
/* Create the network (weights from SplitMix64 with seed) and room for max_samples samples. */
int dg_mlp_init(dg_mesh* mesh, int32_t hidden, int32_t rank, int64_t max_samples, uint64_t seed);
/* Sizes: parameters, inputs, outputs, harvested samples (any pointer may be NULL). */
int dg_mlp_sizes(dg_mesh* mesh, int64_t* n_params, int32_t* n_in, int32_t* n_out, int64_t* n_samples);
/* Copy the FP32 parameters (W1 [hidden][n_in], b1, W2 [hidden][hidden], b2, W3 [n_out][hidden], b3)
 * to out and/or replace them from in (device buffers; either may be NULL). */
int dg_mlp_params(dg_mesh* mesh, float* out, const float* in, void* stream);
/* Features [n_elem][n_in] and mass diagonals [n_elem][n_p] of state u (device outputs, may be NULL). */
int dg_mlp_features(dg_mesh* mesh, const double* u, double dt_aii, float* feat, float* sdiag, void* stream);
/* Assemble the exact blocks of J_G at (u, t, dt_aii) and append every stride-th element's
 * (features, scaled block) to the training set (until full). Synchronises the stream. */
int dg_mlp_harvest(dg_mesh* mesh, const double* u, double t, double dt_aii, int32_t stride, int64_t* n_samples,
                   void* stream);
/* Loss and parameter gradient of nb samples given on the device (X [nb][n_in], scaled blocks
 * [nb][n][n] row-major); grad (device, n_params floats) may be NULL. Synchronises the stream. */
int dg_mlp_loss_grad(dg_mesh* mesh, const float* X, const float* Bs, int32_t nb, double* loss, float* grad,
                     void* stream);
/* Adam over the harvested set, mini-batches of `batch`, `epochs` passes; mean loss of the first
 * and the last pass. */
int dg_mlp_train(dg_mesh* mesh, int32_t epochs, int32_t batch, double lr, double* loss_first, double* loss_last,
                 void* stream);

/*
 * Tracing. dg_profile_start makes every kernel the library launches for this mesh record a pair
 * of CUDA events on the stream it runs on (capacity = most launches recorded; launches beyond it
 * are counted, not timed). dg_profile_stop synchronises those events, accumulates the device time
 * per kernel kind into ms[kind] and the launches into count[kind] for kind < n_kinds (either
 * array may be NULL), returns the total number of launches through *total (may be NULL), and
 * switches tracing off. dg_kernel_name(kind) names a kind ("" past the last one).
 */
int dg_profile_start(dg_mesh* mesh, int32_t capacity);
int dg_profile_stop(dg_mesh* mesh, int32_t n_kinds, double* ms, int32_t* count, int64_t* total);
const char* dg_kernel_name(int32_t kind);

/* ----------------------------------------------------------------------------------------------
 * Radial 1D ensemble (Sec. 4.3: the radial one-dimensional model, run for parametric studies).
 * The paper does not print the 1D equations; the library takes the spherically symmetric restriction
 * of the 3D problem: fields of r only, radial velocity, u = (varrho, sqrt(rho) v_r, sqrt(rho) T); the
 * LDG weak form of Eq. DGformulation with trial and test functions restricted to symmetric fields and
 * the measure r^2 dr, so that the gradient of the radial velocity has a tangential part v/r and the
 * momentum residual gains the tangential stress 2 F_tt / r; Eq. fluxSWNondimensional without the
 * rotating-frame terms (not spherically symmetric); radial gravity; mu* = T*^visc_exp and
 * kappa* = alpha0 T*^visc_exp (the conductivity factor of Sec. 4.3); EUVAC heating (DG_EUV_EUVAC,
 * oxygen absorber) above the column's site with the column's efficiency epsilon; wall / outflow
 * boundaries and the numerical flux of Eq. LDG2; (p+1)-point Gauss quadrature including the r^2.
 * All columns share one radial mesh and the physics numbers; each has its own
 * (epsilon, alpha0, latitude, longitude).
 * Layout of u, r, v, jv (device, FP64): [3][n_elem][p+1][n_col] with the column index fastest
 * (consecutive columns adjacent, so one thread per column reads coalesced), nodal GLL values.
 * -------------------------------------------------------------------------------------------- */
typedef struct dg_radial_desc {
    int32_t p;            /* degree, 1..4 */
    int32_t n_elem;       /* radial elements (shared by every column) */
    int32_t n_col;        /* columns of the ensemble */
    int32_t euv;          /* 0 (no heating) or DG_EUV_EUVAC */
    int32_t bc_lo, bc_hi; /* DG_BC_WALL or DG_BC_OUTFLOW at the inner / outer radius */
    double r_inner, r_outer, h_first;  /* radii and first-layer height (<= 0: uniform layers) */
    double gamma, grashof, prandtl, mass, visc_exp, lambda0, t_wall;   /* as in dg_mesh_desc */
    double g_r0;          /* g* = -(g_r0/r)^2 r_hat; also the Earth radius of the shadow test */
    double euv_omega_t, euv_day, euv_f107, euv_f107a, euv_dsun;        /* as in dg_mesh_desc */
    double ref_T0, ref_rho0, ref_m, ref_g0;
} dg_radial_desc;

typedef struct dg_radial dg_radial;

typedef struct dg_radial_stats {
    int32_t status;            /* the call's return code */
    int32_t newton_iters[3];   /* Newton iterations per stage (the most any column needed) */
    double max_ratio;          /* largest ||G||_2 / ||G(U^0)||_2 over columns at the end of the last stage */
    double wall_ms;            /* host wall time of the call */
} dg_radial_stats;

/* Build the ensemble on the current device. node_r: optional HOST array [n_elem][p+1] of the node
 * radii (NULL: geometric layers from desc); params: HOST array [n_col][4] = (epsilon, alpha0,
 * latitude, longitude [rad]), read during the call. Allocates the library storage (synchronises).
 * Errors: DG_EINVAL (sizes, p, boundaries, non-positive radii or alpha0, more than 6000 unknowns
 * 3 (p+1) n_elem per column: the banded solve keeps a column's right-hand side in shared memory),
 * DG_ENOMEM, DG_ECUDA. */
int dg_radial_create(const dg_radial_desc* desc, const double* node_r, const double* params, dg_radial** out);
void dg_radial_destroy(dg_radial* rad);

/* Residual r = (F_r, w')_{r^2} + (S, w)_{r^2} - [r^2 F_hat w] of every column at time t (FP64,
 * stream-ordered). r must not overlap u. */
int dg_radial_residual(dg_radial* rad, const double* u, double t, double* r, void* stream);

/* Exact Jacobian-vector product J v of every column (forward-mode tangent, FP64); r_out (may be
 * NULL) receives r(u) from the same pass. jv must not overlap u, v or r_out. */
int dg_radial_jvp(dg_radial* rad, const double* u, const double* v, double t, double* jv, double* r_out,
                  void* stream);

/* One DIRK step (stages 1, 2 = DIRK(2,2), 3 = DIRK(3,3); the tableaux of dg_dirk_tableau) of
 * M du/dt = r(u) for every column, in place on u. Each stage solves G(U) = 0 by a Newton iteration
 * on the FP64 residual whose linear systems use the column's exact stage Jacobian
 * J_G = M - dt a_ii J_r at the stage's first iterate, assembled in FP32 by colored tangent probing
 * and factored by FP32 banded LU with partial pivoting (one thread per column); every column
 * iterates until max over columns of ||G||_2 / ||G(U^0)||_2 <= newton_rtol or
 * ||G||_2 <= 1e-14 ||M U||_2. Synchronises the stream (the host reads the largest ratio after every
 * iteration). stats may be NULL. Errors: DG_ENOTCONV after max_newton iterations of a stage,
 * DG_ENAN (non-finite norm or zero pivot), DG_EINVAL, DG_ENOMEM, DG_ECUDA; on an error u is left
 * unchanged. */
int dg_radial_step(dg_radial* rad, double* u, double t, double dt, int32_t stages, double newton_rtol,
                   int32_t max_newton, dg_radial_stats* stats, void* stream);

/* Sizes: columns, nodes per column (n_elem (p+1)), unknowns (3 n_col n_node). */
int dg_radial_sizes(const dg_radial* rad, int64_t* n_col, int32_t* n_node, int64_t* n_dof);

/* Tracing of the radial kernels, as dg_profile_start / dg_profile_stop for a mesh. */
int dg_radial_profile_start(dg_radial* rad, int32_t capacity);
int dg_radial_profile_stop(dg_radial* rad, int32_t n_kinds, double* ms, int32_t* count, int64_t* total);
const char* dg_radial_kernel_name(int32_t kind);

/*
 * FP64 throughput probe (the ceiling of the FP64 path, which is FP64-pipe bound on this part):
 * a fused multiply-add loop over 8 independent chains per thread on every SM, timed with CUDA
 * events on the legacy stream; *tflops receives the achieved FP64 TFLOP/s (2 flops per FMA).
 */
int dg_probe_fp64(double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
