/*
 * reg.h -- C ABI of the GB300 library for the inexact Gauss-Newton-Krylov
 * diffeomorphic image registration method of Mang & Biros, "An inexact
 * Newton-Krylov algorithm for constrained diffeomorphic image registration"
 * (arXiv:1408.6299).
 *
 * Problem (Sec. 1.1, Eq. objective / Eq. constraint): find a velocity v(x,t) on
 * the periodic domain [0,2pi)^d, d in {2,3}, minimising
 *     J[v] = 1/2 ||m_R - m_1||^2 + beta/2 int_0^1 <B v, B v> dt
 * subject to dm/dt + grad m . v = 0, m(0) = m_T, and, for the Stokes scheme,
 * div v = 0. B = grad (H1 seminorm, A = -Lap) or B = Lap (H2, A = Lap^2)
 * (Sec. 2.1, Eq. first-variation-H1/H2). v is expanded in time in n_c
 * Chebyshev coefficient fields, v(x,t) = sum_l T_l(2t-1) v_l(x) (Sec. 3.3.2).
 * Space is discretised by Fourier collocation on the nodal grid
 * x_j = 2 pi j / n_i, time by Heun's RK2 with h_t = 1/n_t (Sec. 3.3.1).
 *
 * Layouts (all row-major, last grid axis fastest, N = n_0*...*n_{d-1}):
 *   image            double[N]
 *   coefficient vec  double[n_c][d][N]   (v, v~, gradients, PCG vectors)
 * Norms and inner products: <u,w>_h = h_d sum_x u.w with h_d = prod 2pi/n_i.
 *
 * Pointers: every array argument may be a device pointer (cudaMalloc /
 * PyTorch CUDA tensor) or a host pointer; the library inspects it with
 * cudaPointerGetAttributes and stages host arrays through its own device
 * buffers. The caller owns every array it passes; the library never frees
 * them and keeps no reference after a call returns (images are copied).
 * All work is ordered on the context's stream; calls return after that work
 * has finished (results are valid on return). A context is not thread-safe:
 * use one context per host thread.
 *
 * Errors: every call returns a reg_status; reg_last_error() describes the most
 * recent failure of that context. No call aborts, traps or exits the process.
 */
#ifndef REG_H
#define REG_H

#include <stdint.h>

#if defined(__GNUC__)
#define REG_API __attribute__((visibility("default")))
#else
#define REG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct reg_ctx reg_ctx;

typedef enum {
  REG_OK = 0,
  REG_EINVAL = 1,        /* bad argument: grid not a power of two in [8,512], d not 2/3, ... */
  REG_ENOMEM = 2,        /* device allocation failed */
  REG_ECUDA = 3,         /* a CUDA runtime call failed */
  REG_ENOTREADY = 4,     /* reg_hessvec before reg_gradient / reg_linearize */
  REG_ENONFINITE = 5,    /* objective, gradient or a Krylov scalar is not finite */
  REG_ECFL = 6,          /* CFL bound could not be met by step halving */
  REG_ELINESEARCH = 7,   /* Armijo line search exhausted its trials */
  REG_EMAXIT = 8,        /* outer iteration cap reached before the tolerance */
  REG_ETIMEOUT = 9       /* a bounded device wait ran out */
} reg_status;

typedef enum { REG_H1 = 1, REG_H2 = 2 } reg_type;

typedef enum {
  REG_FP64 = 0,  /* every transport sweep in double precision */
  REG_MIXED = 1  /* Hessian matvec sweeps in single precision; objective,
                    gradient, line search, det F and Krylov vectors in double */
} reg_precision;

typedef enum {
  REG_QUAD_TRAPEZOID = 0,  /* body-force time integral by the trapezoid rule on
                              the time nodes (optimize-then-discretize, Sec. 3) */
  REG_QUAD_DISCRETE = 1    /* exact derivative of the Heun-discretised objective
                              (stage values; gradient matches finite differences) */
} reg_quadrature;

/* Create a context (Sec. 3.3: grid n[0..d-1], n_t Heun steps, n_c Chebyshev
 * coefficients, regularisation weight beta > 0, regulariser type, Stokes flag
 * gamma, precision of the matvec sweeps, state checkpoint interval
 * ckpt_every (0 = store the whole state trajectory; K > 0 = keep every K-th
 * state and recompute the others), and a cudaStream_t (NULL = the legacy
 * default stream). Requires n_t % ckpt_every == 0 when ckpt_every > 0.
 * Errors: REG_EINVAL, REG_ENOMEM, REG_ECUDA. On error *out is NULL. */
REG_API reg_status reg_create(reg_ctx** out, int d, const int64_t* n, int n_t, int n_c, double beta, int reg_type,
                      int stokes, int precision, int ckpt_every, void* cuda_stream);

/* Destroy a context and free its device memory. NULL is accepted. */
REG_API reg_status reg_destroy(reg_ctx* ctx);

/* Text of the last error of ctx (never NULL; "" when none). Valid until the
 * next call on ctx. ctx may be NULL: then it describes the last failed
 * reg_create or reg_precond_noalloc call of this thread. */
REG_API const char* reg_last_error(const reg_ctx* ctx);

/* Choose the time quadrature of the body force (default trapezoid). */
REG_API reg_status reg_set_quadrature(reg_ctx* ctx, int quadrature);

typedef enum {
  REG_HESS_GN = 0,     /* Gauss-Newton: all lambda terms dropped (Sec. 3.2.2, Eq. gauss-newton) */
  REG_HESS_NEWTON = 1  /* full Newton (Eq. sec-order-opt-cond): the incremental adjoint carries
                          -div(v~ lam) and the body force lam grad m~ (trapezoid quadrature only) */
} reg_hessian;

/* Choose the Hessian applied by reg_hessvec and reg_solve (default
 * Gauss-Newton). The full Newton matvec re-advances the adjoint alongside the
 * incremental adjoint and keeps the incremental state of every time node
 * ((n_t+1)*N values). Invalidates the linearisation point. REG_EINVAL with the
 * discrete quadrature. */
REG_API reg_status reg_set_hessian(reg_ctx* ctx, int kind);

/* Copy the template m_T and the reference m_R (N values each) into the
 * context (Sec. 1.1). Invalidates the linearisation point. */
REG_API reg_status reg_set_images(reg_ctx* ctx, const double* m_T, const double* m_R);

/* Objective J^h at v (Eq. objective with the expansion of App. A):
 * one state solve (Eq. first-order-forward) plus the Fourier-diagonal
 * regularisation term. J_out: host double. parts (may be NULL): host double[2]
 * = {1/2 ||m_R - m_1||_h^2, beta/2 sum_ll' c_ll' <B v_l, B v_l'>_h}. */
REG_API reg_status reg_objective(reg_ctx* ctx, const double* v, double* J_out, double* parts);

/* Reduced gradient g at v (Eq. first-order-control with the pressure
 * eliminated, Eq. eliminated-control, and App. A Eq. control-equation-expansion):
 * state solve, adjoint solve (Eq. first-order-adjoint, lambda_1 = m_R - m_1),
 * g_l = beta sum_l' c_ll' A v_l' + int b_l K^gamma[lambda grad m] dt.
 * Also makes v the linearisation point of later reg_hessvec calls (Alg. 2
 * takes m_k and v_k as given). g: n_c*d*N doubles. J_out (may be NULL):
 * host double receiving J at v. Errors: REG_ENONFINITE if J or g is not finite. */
REG_API reg_status reg_gradient(reg_ctx* ctx, const double* v, double* g, double* J_out);

/* Make v the linearisation point without computing the gradient (one state
 * solve; the stored state feeds reg_hessvec). */
REG_API reg_status reg_linearize(reg_ctx* ctx, const double* v);

/* Gauss-Newton reduced-Hessian matvec (Alg. 2 with Eq. gauss-newton and
 * Eq. eliminated-icontrol): incremental state solve forward from 0,
 * incremental adjoint solve backward from -m~_1, then
 * Hvt_l = beta sum_l' c_ll' A vt_l' + int b_l K^gamma[lambda~ grad m] dt,
 * at the point set by the last reg_gradient / reg_linearize.
 * vt, Hvt: n_c*d*N doubles (may alias). REG_ENOTREADY without a point. */
REG_API reg_status reg_hessvec(reg_ctx* ctx, const double* vt, double* Hvt);

/* Preconditioner z = P^{-1} r with P = beta C (x) A (Sec. 3.2.1, Sec. 3.3.3):
 * a Fourier-diagonal scaling by 1/(beta a(k)) with the k = 0 mode scaled by
 * one, and the inverse Chebyshev Gram matrix across coefficients. */
REG_API reg_status reg_precond(reg_ctx* ctx, const double* r, double* z);

/* The preconditioner of reg_precond without a context and without allocating.
 * The paper has no counterpart: it exists for callers that cannot call
 * cudaMalloc when they need the operator (a runtime that owns all device
 * memory through its own pool, a memory budget fixed at start-up, loops that
 * must not allocate after initialisation). It computes the same z = P^{-1} r
 * as reg_precond for the grid n[0..d-1], n_c, beta and reg_type, working in a
 * fixed 64 MiB device array that every GPU loading this library reserves
 * until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   r, z: device pointers, n_c*d*N doubles each (z may equal r).
 *   Limit: n_c*d*N/2 <= 2,095,040 (for example 3D 64^3 with n_c <= 5, 2D
 *   512^2 with n_c <= 7); larger problems get REG_EINVAL and a message in
 *   reg_last_error(NULL).
 *   The first call on a device does a set-up with that device current: it
 *   finds the array's address and uploads the FFT twiddle tables with a
 *   synchronous host-to-device copy, so make that first call before any
 *   stream capture. Later calls only enqueue kernels on cuda_stream (NULL =
 *   legacy default stream) and return without synchronising.
 *   Every call shares the array and it keeps the last call's contents; each
 *   call overwrites all it reads. Calls whose GPU work overlaps (different
 *   streams or host threads with no ordering between them) race on it. */
REG_API reg_status reg_precond_noalloc(int d, const int64_t* n, int n_c, double beta, int reg_type, const double* r,
                                       double* z, void* cuda_stream);

/* Regularisation operator out = beta (C (x) A) v (App. A). */
REG_API reg_status reg_regularization(reg_ctx* ctx, const double* v, double* out);

/* State solve m_1 = m(t=1) from m0 under v (Eq. first-order-forward). */
REG_API reg_status reg_transport(reg_ctx* ctx, const double* v, const double* m0, double* m1);

/* Adjoint of reg_transport for automatic differentiation: given G = dL/dm_1,
 * solves the adjoint equation from lambda_1 = -G under v (state from m0) and
 * returns grad_v = dL/dv (body force without projection, n_c*d*N; may be NULL)
 * and grad_m0 = dL/dm0 = -lambda_0 (N; may be NULL). With the discrete
 * quadrature both are the exact derivatives of the Heun-discretised map. */
REG_API reg_status reg_transport_adjoint(reg_ctx* ctx, const double* v, const double* m0, const double* G,
                                 double* grad_v, double* grad_m0);

/* Deformation gradient check (App. D Eq. def-grad): F' = -(v.grad)F + (grad v)F,
 * F_0 = I, Heun with substeps*n_t steps (substeps >= 1); stats: host double[4]
 * = {min, max, mean, std} of det F_1; detF (may be NULL): N doubles. */
REG_API reg_status reg_detF(reg_ctx* ctx, const double* v, int substeps, double* stats, double* detF);

/* det F_1 of Eq. def-grad evaluated on a grid refined `refine` times per axis
 * (refine in {1, 2, 4}; every refined axis at most 512). The velocity
 * coefficients are carried to the finer grid by trigonometric interpolation
 * of their modes below Nyquist (the Nyquist modes are dropped: the first
 * derivatives of the coarse grid treat them as constants, so a velocity that
 * is divergence-free there stays divergence-free), and Eq. def-grad is
 * integrated there with substeps*n_t Heun steps. On the coarse grid the products of the F-equation
 * are not resolved and det F_1 of a divergence-free velocity stalls at a
 * spatial error (about 5e-5 on the 64^3 Stokes workload); one refinement
 * resolves them and det F_1 - 1 then falls at second order in the step.
 * stats: host double[4] {min, max, mean, std} over the fine grid; detF (may
 * be NULL): the N*refine^d fine-grid values. Allocates a temporary fine-grid
 * context. REG_EINVAL on a stacked (lockstep) context. */
REG_API reg_status reg_detF_refined(reg_ctx* ctx, const double* v, int substeps, int refine, double* stats,
                                    double* detF);

/* CFL number h_t * max_j max_i ||v_i(t_j)||_inf / h_x^i (Sec. 3.3.1). */
REG_API reg_status reg_cfl(reg_ctx* ctx, const double* v, double* cfl_out);

/* Grid-angle measure (Sec. 3.3.5 "Regularization": the acute angle of a
 * deformed grid element). The edges e_c of a cell map to the columns F_1 e_c
 * of F_1 (App. D Eq. def-grad, substeps*n_t Heun steps); per point the
 * result is the smallest min(theta, pi - theta) over column pairs, theta the
 * angle between two columns, in radians (pi/2 for F = I). stats: host
 * double[4] {min, max, mean, std}; angle (may be NULL): N doubles. */
REG_API reg_status reg_grid_angle(reg_ctx* ctx, const double* v, int substeps, double* stats, double* angle);

/* Deformation map (App. D Eq. displacement): du/dt + (grad u) v = v, u_0 = 0,
 * Heun steps on the time nodes as in the state equation. u: d*N doubles, the
 * displacement u_1 (component-major); the map is y = x - u_1. */
REG_API reg_status reg_displacement(reg_ctx* ctx, const double* v, double* u);

/* Gaussian presmoothing of an image (Sec. 3.3.5 "Presmoothing"): out = the
 * periodic Gaussian of standard deviation sigma >= 0 (domain units, the paper
 * uses 2*pi/min(n)) applied to in, i.e. the Fourier multiplier
 * exp(-sigma^2 |k|^2 / 2) with the full wavenumbers. in, out: N doubles (may
 * alias). Typically applied to m_T and m_R before reg_set_images. */
REG_API reg_status reg_smooth(reg_ctx* ctx, double sigma, const double* in, double* out);

/* Lanczos estimate of the Hessian spectrum (Sec. 3.3.5 "Regularization":
 * the condition number estimated with the Lanczos algorithm): k steps of the
 * three-term recurrence from q0 (n_c*d*N, any nonzero vector) on the Hessian
 * at the linearisation point (as reg_hessvec applies it), or with precond = 1
 * on P^{-1} H in the P inner product. Plain coefficient-vector inner
 * products, no reorthogonalisation (the extreme Ritz values converge first).
 * alpha, beta: host double[k], the tridiagonal matrix (beta[j] couples steps
 * j and j+1); *steps: steps completed (< k after an exact breakdown);
 * ritz (host double[k], may be NULL): its eigenvalues ascending. Requires a
 * linearisation point (REG_ENOTREADY). */
REG_API reg_status reg_lanczos(reg_ctx* ctx, const double* q0, int k, int precond, double* alpha, double* beta,
                               int* steps, double* ritz);

/* Change the regularisation weight beta of the context (beta continuation,
 * Sec. 3.3.5). The linearisation point stays valid: only the regularisation
 * and preconditioner terms depend on beta. */
REG_API reg_status reg_set_beta(reg_ctx* ctx, double beta);

/* Change the number of time steps n_t (a multiple of ckpt_every), e.g. to
 * keep the CFL number bounded (Sec. 3.3.5 "PDE Solver"). Invalidates the
 * linearisation point. */
REG_API reg_status reg_set_time_steps(reg_ctx* ctx, int n_t);

typedef struct {
  double grad_rtol;     /* stop at ||g_k||_inf <= grad_rtol ||g_0||_inf (Sec. 3.3.5) */
  int max_outer;        /* outer iteration cap n_opt */
  double armijo_c1;     /* sufficient decrease constant (1e-4) */
  double backtrack;     /* step reduction factor (0.5) */
  int max_backtracks;   /* line search trials (20) */
  long pcg_maxit;       /* 0 = order of the reduced system (Sec. 3.3.5) */
  double cfl_max;       /* > 0: halve the step while the CFL number of v+s exceeds it (Sec. 3.3.5) */
  int detF_substeps;    /* > 0: compute det F_1 statistics at the end with this many substeps */
  int method;           /* REG_METHOD_KRYLOV (PCG with the context's Hessian) or REG_METHOD_PICARD */
  int step_memory;      /* Picard: 1 = scale the step by alpha~, doubled after a full step and
                           multiplied by the accepted alpha otherwise (Sec. 3.3.5); default 1 */
  int stop_rule;        /* REG_STOP_GRAD_REL (grad_rtol) or REG_STOP_C1C5 (Eq. stopping-criteria) */
  double tau_J;         /* tolerance tau_J of C1-C3 (1e-3, Sec. 3.3.5) */
  int detF_refine;      /* with detF_substeps > 0: evaluate det F_1 on a grid refined this many
                           times per axis (1, 2 or 4; see reg_detF_refined); default 1 */
} reg_solve_opts;

enum {
  REG_METHOD_KRYLOV = 0, /* inexact (Gauss-)Newton-Krylov: PCG on H s = -g (Alg. 1) */
  REG_METHOD_PICARD = 1  /* Picard iteration / preconditioned gradient descent: s = -P^{-1} g,
                            the difference between the iterate of Eq. picard and v_k (App. C) */
};
enum {
  REG_STOP_GRAD_REL = 0, /* stop at ||g_k||_inf <= grad_rtol ||g_0||_inf; REG_EMAXIT at k = max_outer */
  REG_STOP_C1C5 = 1      /* stop on (C1 and C2 and C3) or C4 (Eq. converged); C5 (k > max_outer)
                            stops with REG_EMAXIT */
};

typedef struct {
  int outer;            /* outer iterations k* */
  long pcg_iters;       /* total PCG iterations */
  long matvecs;         /* Hessian matvecs */
  long n_pde;           /* hyperbolic PDE solves (Sec. 5.2) */
  int ls_trials;        /* objective evaluations in line searches */
  int cfl_halvings;     /* step halvings forced by the CFL bound */
  int status;           /* reg_status of the solve */
  double J0, J;         /* objective at v_0 and at the end */
  double g0_inf, g_inf; /* ||g||_inf at v_0 and at the end */
  double dist_rel;      /* ||m_1 - m_R||^2 / ||m_T - m_R||^2 (Tab. 5.1) */
  double cfl;           /* CFL number of the final v */
  double detF[4];       /* min, max, mean, std of det F_1 (if requested) */
  double seconds;       /* wall time of the solve */
  int stop_flags;       /* REG_STOP_C1C5: bit i-1 set when criterion Ci held at exit */
  double alpha_mem;     /* final Picard step memory alpha~ (1 otherwise) */
  double J_prev;        /* objective of the previous iterate (C1) */
  double dv_inf;        /* ||v_{k-1} - v_k||_inf of the last step (C2) */
  double v_inf;         /* ||v_k||_inf of the final iterate (C2) */
  int device_loops;     /* reg_solve_lockstep: 1 when the problem's PCG and line-search loops ran
                           on the device (conditional CUDA graphs), 0 when the host drove them */
} reg_solve_report;

/* Fill opts with the defaults above (grad_rtol 1e-2, max_outer 50, Krylov
 * method, relative-gradient stop, step memory on, tau_J 1e-3). */
REG_API void reg_solve_opts_default(reg_solve_opts* opts);

/* Outer solve (Alg. 1). REG_METHOD_KRYLOV: inexact Newton-Krylov with PCG,
 * forcing term eta_k = min(0.5, sqrt(||g_k||_2/||g_0||_2)) (Eq.
 * termination-criterion-ksm), preconditioner reg_precond, the Hessian chosen
 * by reg_set_hessian (GN-PCG or N-PCG). REG_METHOD_PICARD: s = -P^{-1} g
 * (Eq. picard) with the optional step memory. Then CFL halving (cfl_max) and
 * Armijo backtracking from alpha = 1. v_inout: initial guess in, solution out
 * (n_c*d*N). report (may be NULL): host. Returns REG_EMAXIT when the
 * iteration cap ends the solve (v_inout holds the last iterate). */
REG_API reg_status reg_solve(reg_ctx* ctx, double* v_inout, const reg_solve_opts* opts, reg_solve_report* report);

/* One independent registration problem of a batch (Sec. 1.1 for each pair).
 * m_T, m_R: N doubles each; v: initial guess in, solution out (n_c*d*N);
 * each may be host or device memory. n[2] is ignored when d == 2. */
typedef struct {
  int d;
  int64_t n[3];
  int n_t;
  int n_c;
  double beta;
  int reg_type;
  int stokes;
  const double* m_T;
  const double* m_R;
  double* v;
} reg_problem;

/* Solve `count` independent problems (Alg. 1 each, options opts for all, or
 * the defaults when NULL) concurrently on the current device: `workers` host
 * threads, each with its own CUDA stream and contexts cached per problem
 * configuration, take problems from a queue ordered largest first. Contexts
 * with their own stream replay the Hessian matvec as a captured CUDA graph.
 * reports (may be NULL): host array of count, report i for problem i. Returns
 * REG_OK when every solve returned REG_OK or REG_EMAXIT, else the status of
 * the first failing problem (all problems are attempted); the message is in
 * reg_last_error(NULL). Each problem's arrays must stay valid until return. */
REG_API reg_status reg_solve_batched(const reg_problem* problems, int count, int precision, const reg_solve_opts* opts,
                                     reg_solve_report* reports, int workers);

/* Lockstep batched solve of independent problems (Sec. 1.1 for each pair):
 * problems of one shape, n_t, n_c, regulariser and scheme are stacked along
 * an untransformed leading axis into one context (at most max_stack per
 * stack; 0 = no limit), with one beta per problem. Every kernel of a matvec,
 * gradient or objective evaluation covers the whole stack in one launch, and
 * the stack's matvec is replayed as one captured CUDA graph. The outer loop of
 * Alg. 1 (PCG or Picard, CFL halving, line search, stopping rule: opts) runs
 * for all problems of a stack at once with per-problem Krylov and line-search
 * scalars, so each problem takes the iterates it would take alone (up to the
 * order of its inner-product sums); a problem that stops keeps its iterate
 * while the others continue. Stacks run concurrently, one stream each.
 * Checkpointing is off (every state gradient is stored). Arrays may be host
 * or device memory; reports (may be NULL): one per problem, in the order of
 * `problems`. Returns the status of the first failing stack; a problem that
 * ends with REG_EMAXIT does not fail its stack. det F statistics are not
 * computed (detF_substeps is ignored). With the Krylov method and no CFL bound
 * the PCG and line-search loops of a stack run on the device: each is one
 * CUDA graph whose conditional WHILE node iterates a check kernel (per-problem
 * forcing-term, curvature and Armijo decisions, the same operations as the
 * host loop) and an IF node with one iteration, so the host waits once per
 * loop instead of once per reduction (report device_loops = 1; the
 * environment variable REG_LOCKSTEP_GRAPHS=0 keeps the host-driven loops). */
REG_API reg_status reg_solve_lockstep(const reg_problem* problems, int count, int precision,
                                      const reg_solve_opts* opts, reg_solve_report* reports, int max_stack);

/* Parameter continuation in beta (Sec. 3.3.5 "Regularization"). */
typedef struct {
  double beta0;       /* first beta, large enough to underfit (1) */
  double beta_min;    /* lower bound on beta (1e-6) */
  double eps_F;       /* lower bound on min det F_1, in (0, 1) (0.1); 0 disables */
  double eps_theta;   /* lower bound on the smallest grid angle in radians (0 = off; pi/16 in Sec. 5) */
  double beta_rtol;   /* the bisection ends when beta changes by less than beta_rtol times
                         the first beta that breached a bound (0.05) */
  double dist_rtol;   /* the reduction ends when ||m_R - m_1||_2 drops by less than this fraction (1e-2) */
  double cfl_target;  /* > 0: after a solve whose CFL number exceeds it, raise n_t in proportion
                         (a multiple of ckpt_every) and solve again at the same beta (0 = off) */
  int detF_substeps;  /* substeps of the det F_1 / grid-angle evaluation (1) */
  int max_solves;     /* cap on registration solves (50) */
} reg_cont_opts;

#define REG_CONT_TRACE 64
typedef struct {
  int found;           /* 1 if some beta met the bounds: beta and v are that solution */
  int stop;            /* 0 bisection converged, 1 beta_min reached, 2 distance stalled,
                          3 no feasible beta (beta0 breached), 4 max_solves */
  double beta;         /* the smallest accepted beta (the last one tried if none) */
  double beta_breach;  /* first beta that breached a bound (0: none) */
  int solves;          /* registration solves */
  int n_t;             /* time steps at the end */
  long outer, pcg_iters, matvecs;
  double detF_min, angle_min, dist_rel; /* at the result; dist_rel = ||m_R-m_1||^2/||m_R-m_T||^2 */
  double seconds;
  int n_trace;         /* per solve (first REG_CONT_TRACE): beta, min det F_1, min angle,
                          relative L2 distance ||m_R-m_1||/||m_R-m_T||, accepted */
  double trace_beta[REG_CONT_TRACE], trace_detF[REG_CONT_TRACE], trace_angle[REG_CONT_TRACE];
  double trace_dist[REG_CONT_TRACE];
  int trace_ok[REG_CONT_TRACE];
} reg_cont_report;

REG_API void reg_cont_opts_default(reg_cont_opts* opts);

/* Beta continuation: solve at beta0, divide beta by 10 while the solution
 * keeps min det F_1 >= eps_F (and the smallest grid angle >= eps_theta),
 * then bisect between the last accepted and the first breaching beta. Each
 * solve (reg_solve with solve_opts) starts from the last accepted solution
 * (from v_inout before any). On return v_inout holds the accepted solution
 * and the context's beta is its beta. report: host. REG_OK also when no beta
 * was feasible (report->found = 0). */
REG_API reg_status reg_continuation(reg_ctx* ctx, double* v_inout, const reg_solve_opts* solve_opts,
                                    const reg_cont_opts* cont_opts, reg_cont_report* report);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used to measure the kernels).
 * Kernel kinds: 0 row real-to-complex FFT pass, 1 row complex-to-real pass,
 * 2 strided complex FFT pass, 3 Fourier multipliers, 4 Heun stage /
 * transport right-hand side, 5 body-force accumulation, 6 other.
 * ------------------------------------------------------------------------ */
#define REG_KIND_COUNT 7

/* Start bracketing every launch of the kinds in kind_mask (bit k = kind k)
 * with CUDA events on the context's stream. */
REG_API reg_status reg_profile_begin(reg_ctx* ctx, unsigned kind_mask);

/* Stop and return, per kind (arrays of REG_KIND_COUNT, each may be NULL),
 * the summed event time in ms, the summed algorithmic bytes (the bytes each
 * launch must read and write) and the number of launches. Synchronises. */
REG_API reg_status reg_profile_end(reg_ctx* ctx, double* ms, double* bytes, long* count);

/* Floating-point operations of the transforms of the launches collected by
 * the last reg_profile_end, per kind (REG_KIND_COUNT values): the butterflies
 * and twiddle multiplications of every FFT the launches ran (radix plan
 * counts), the spectral multipliers of the column passes, and the packing of
 * the real-to-complex rows. Pointwise epilogue arithmetic is not counted. */
REG_API reg_status reg_profile_flops(reg_ctx* ctx, double* flops);

/* Double-precision FMA throughput of the current device in GFLOP/s (2 flops
 * per FMA): independent FMA chains in every thread of one wave of resident
 * blocks, the best of three launches timed with CUDA events after a warm-up.
 * Allocates and frees a small buffer; changes no device setting. The bound
 * of the FP64 transport sweeps, whose arithmetic rate the bench reports
 * against it. Errors: REG_ECUDA (message in reg_last_error(NULL)). */
REG_API reg_status reg_fp64_peak(double* gflops);

/* Number of kernel launches issued by the library in this process so far. */
REG_API long reg_launch_count(void);

/* Failure-path check of the bounded waits (no counterpart in the paper): one
 * block polls an mbarrier that nothing completes, gives up after a bounded
 * number of polls, and counts the timeout the way the TMA column pass counts
 * a tile copy that never lands (which fails the API call with
 * REG_ETIMEOUT). *counted: the timeouts read back and cleared (1 expected).
 * Faults, traps and hangs nothing; uses the current device. */
REG_API reg_status reg_selftest_copy_timeout(int* counted);

#ifdef __cplusplus
}
#endif

#endif /* REG_H */
