/*
 * fde.h — C ABI of libfde: symbol-based tau-preconditioned Krylov solves of
 * shifted-Grunwald fractional diffusion systems on one GB300 (sm_103a).
 *
 * Method: Barakitis, Ekstrom, Vassalos, "Preconditioners for Fractional
 * Diffusion Equations Based on the Spectral Symbol".
 *
 *   1D (Sec. 1.2, eq. for M_{alpha,n}):  M = c0 I + D_+ T + D_- T^T,
 *       T = T_{alpha,n} = -[g_{i-j+1}] (first-order weights g_k = (-1)^k binom(alpha,k))
 *       or S_{alpha,n} = -[w_{i-j+1}] (second-order WSGD weights, Sec. 1.3);
 *       c0 = nu = h^alpha / dt for implicit Euler.
 *   2D (Sec. 1.4 and Sec. 3.2):  M = c0 I + D_+(I (x) T_a) + D_-(I (x) T_a^T)
 *                                 + sr [E_+(T_b (x) I) + E_-(T_b^T (x) I)],
 *       x-fastest ordering u[i + j*n1]; implicit Euler c0 = h_x^alpha/dt,
 *       sr = h_x^alpha / h_y^beta (Crank-Nicolson: c0 = 1/r = 2 h_x^alpha/dt, same sr).
 *   Preconditioner (Sec. 3.1 eq. P_F, Sec. 3.2 eq. for the 2D P):
 *       P = D tau(F) or tau(F) D, tau(F) = S diag(F(theta)) S (DST-I, Sec. 1),
 *       F = F_alpha (1D) or F_a(theta_1) + sr F_b(theta_2) (2D), D = mean of the
 *       diffusion coefficients; with tau_shift the constant-coefficient shifted
 *       symbols of Sec. 3.1.1 (Case I) and Sec. 3.2 (P_hat, no D).
 *
 * Conventions for every entry point:
 *   - All vector arguments are DEVICE pointers (cudaMalloc / torch CUDA memory)
 *     unless stated; the caller owns them and the workspace.  The library
 *     owns only the small host-side plan struct.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*,
 *     NULL = legacy default stream); no call allocates device memory or
 *     synchronises the host, except fde_assemble_symbol's one-time kernel
 *     attribute setup on first use.
 *   - Arguments are validated before any launch; invalid input returns
 *     FDE_EINVAL and launches nothing.  A failed launch returns FDE_ECUDA.
 *     Convergence failures are reported per solve in fde_solve_info (device
 *     memory), never by aborting; no C++ exception crosses the ABI.
 *   - Grid sizes: n1 + 1 (and n2 + 1 in 2D) must be powers of two, 1 <= n+1.
 */
#ifndef FDE_H
#define FDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDE_OK = 0,
    FDE_EINVAL = 1,        /* invalid argument (checked before any launch) */
    FDE_ENOMEM = 2,        /* workspace smaller than fde_workspace_size() */
    FDE_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    FDE_ENOCONV = 4,       /* iteration cap reached; best iterate left in x */
    FDE_EBREAKDOWN = 5,    /* PCG p^T A p <= 0, or a non-positive preconditioner */
    FDE_ETIMEOUT = 6,      /* an inter-CTA barrier wait exceeded its bound */
    FDE_ENONFINITE = 7     /* NaN/Inf met in a reduction */
} fde_status;

typedef enum { FDE_F64 = 0, FDE_F32 = 1 } fde_dtype;
typedef enum { FDE_WEIGHTS_GL1 = 0, FDE_WEIGHTS_WSGD2 = 1 } fde_weights;
/* The preconditioner: P = tau(F) D, P = D tau(F) (Sec. 3.1), P_F-tilde =
   S diag(D_j F(theta_j)) S (Sec. 4, Table 2; 1D): D sampled on the tau grid and
   folded into the symbol, or P_tri (Sec. 4, Table 2; 1D, no shift): the three
   main diagonals of M, solved by parallel cyclic reduction on the device. */
typedef enum { FDE_ORDER_TAU_D = 0, FDE_ORDER_D_TAU = 1, FDE_ORDER_TAU_DF = 2, FDE_ORDER_TRI = 3 } fde_order;
typedef enum { FDE_SCHEME_IMPLICIT_EULER = 0, FDE_SCHEME_CRANK_NICOLSON = 1 } fde_scheme;
typedef enum { FDE_PCG = 0, FDE_GMRES = 1 } fde_method;
typedef enum {
    FDE_PREC_F64 = 0,      /* every vector, transform and reduction in FP64 */
    FDE_PREC_F32 = 1,      /* FP32 vectors and transforms; FP64 dots and scalars; no refinement */
    FDE_PREC_F32_IR = 2    /* FP32 inner solves, FP64 outer residual r = b - A x and update */
} fde_precision;
typedef enum { FDE_SIDE_RIGHT = 0, FDE_SIDE_LEFT = 1 } fde_side;

/*
 * The problem of one time step, in the paper's terms (Sec. 1.2-1.4).
 * Coefficient arrays: device FP64, length n1*n2, x fastest; a NULL array means
 * the matching *_const scalar is used everywhere.
 */
typedef struct {
    int dim;               /* 1 or 2 */
    int n1, n2;            /* interior points per axis (n2 ignored in 1D); n+1 = 2^k */
    double alpha, beta;    /* fractional orders in (1,2); beta ignored in 1D */
    double len1, len2;     /* domain lengths R-L, so h = len/(n+1) */
    double dt;             /* time step h_t > 0 */
    int scheme;            /* fde_scheme: sets c0 = h^alpha/dt or 2 h^alpha/dt */
    int weights;           /* fde_weights */
    const double *dp, *dm, *ep, *em;        /* d_+, d_-, e_+, e_- (device) or NULL */
    double dp_const, dm_const, ep_const, em_const;
    int tau_shift;         /* 1: shifted symbol (needs constant, equal coefficients) */
    int order;             /* fde_order: P = tau(F) D (default), D tau(F), P_F-tilde or P_tri (1D, no shift) */
} fde_problem;

typedef struct {
    int method;            /* fde_method */
    int restart;           /* GMRES(m) restart length m, 1..64 */
    double tol;            /* stop when ||b - A x||_2 <= tol ||b||_2 (right precond.) */
    int max_iters;         /* cap on products with M (inner iterations), >= 1 */
    int precision;         /* fde_precision */
    double inner_tol;      /* FDE_PREC_F32_IR: relative tolerance of each inner solve,
                              loosened to min(0.5, 0.3 tol ||b|| / ||r||) when that is larger
                              (the last correction closes only the remaining gap); an
                              inner solve also stops after 2m products (GMRES(m)) or 50
                              (PCG), and the refinement loop then measures the correction
                              by how much it shrank the FP64 residual */
    int max_outer;         /* FDE_PREC_F32_IR: cap on refinement steps */
    int side;              /* fde_side (GMRES only; PCG ignores it) */
    int balance;           /* fde_krylov_solve with count > 1: 0 splits the GPU evenly over the
                              instances; 1 sizes each instance's team in proportion to
                              N log2(L) times the iteration count that info_dev[i] holds from
                              the previous solve of the same plans, in the same order (zeros:
                              even split).  Time stepping keeps the counts stable from step
                              to step. */
} fde_solve_opts;

/* Per-solve result, written by the device into caller memory. */
typedef struct {
    int32_t status;        /* fde_status */
    int32_t iterations;    /* products with M inside the Krylov loops (inner, all restarts) */
    int32_t outer;         /* refinement steps (FDE_PREC_F32_IR), else 0 */
    int32_t restarts;      /* GMRES restarts */
    double relres;         /* final true ||b - A x||_2/||b||_2, FP64 */
    double relres_est;     /* the Krylov loop's own last residual estimate */
    /* work counters, for accounting the bytes a solve moved: */
    int32_t basis_sum;     /* sum over GMRES steps of the basis vectors the step orthogonalised against */
    int32_t reorth;        /* GMRES steps that took a second Gram-Schmidt pass */
    int32_t cycles;        /* Krylov cycles started from a true residual (restarts + 1 per Krylov solve) */
    int32_t residuals64;   /* FP64 true residuals of the FP32 and refinement modes */
    int32_t iterations64;  /* of `iterations`, those on FP64 vectors (all in FDE_PREC_F64; in
                              FDE_PREC_F32_IR those of an FP64 finish) */
    int32_t reserved;      /* 0 */
} fde_solve_info;

typedef struct fde_plan fde_plan;

/* Default options: GMRES(30), tol 1e-8, 5000 iterations, FP64, right side. */
void fde_default_opts(fde_solve_opts* opts);

/*
 * Bytes of device workspace that a plan for (prob, opts) needs: symbol data
 * (circulant eigenvalues of T, tau samples, twiddles, D^{-1}), Krylov vectors
 * and transform intermediates.  Host-only; touches no device memory.
 * Returns FDE_EINVAL for an invalid problem or options.
 */
fde_status fde_workspace_size(const fde_problem* prob, const fde_solve_opts* opts, size_t* bytes);

/*
 * Assemble the symbol data of `prob` into `workspace` (device, >= bytes from
 * fde_workspace_size, 256-byte aligned) on `stream` and return a host plan.
 * Computes on the device, in FP64: the weights g_k or w_k (Sec. 1.2/1.3), the
 * eigenvalues of the 2(n+1)-circulant that embeds T (FFT of its first
 * column), the tau samples F(theta_j) (Thm 2; shifted per Sec. 3.1.1 / 3.2),
 * D^{-1}, and FP32 copies of all of them.  The coefficient arrays in `prob`
 * must stay valid for the plan's lifetime.  `opts` fixes the solver
 * workspace layout; later solves must use the same method/precision/restart.
 */
fde_status fde_assemble_symbol(const fde_problem* prob, const fde_solve_opts* opts,
                               void* workspace, size_t bytes, fde_plan** plan, void* stream);

/*
 * y = M x (Sec. 1.2 eq. for M_{alpha,n}; Sec. 3.2 eq. for M_(alpha,beta),N):
 * the Toeplitz products by circulant embedding and FFT, with c0, D_+-, E_+-
 * and sr fused.  x, y: device arrays of n1*n2 elements of `dtype`; x != y.
 */
fde_status fde_toeplitz_matvec(const fde_plan* plan, int dtype, const void* x, void* y, void* stream);

/*
 * z = P^{-1} r (Sec. 3.1 eq. P_F; Sec. 3.2): DST-I, division by the symbol
 * samples, DST-I (per axis in 2D), with D^{-1} before or after per `order`;
 * for FDE_ORDER_TRI the tridiagonal solve with P_tri (Sec. 4, Table 2).
 * r, z: device arrays of n1*n2 elements of `dtype`; r != z.
 */
fde_status fde_tau_solve(const fde_plan* plan, int dtype, const void* r, void* z, void* stream);

/*
 * Solve M_i x_i = b_i for count >= 1 independent plans in ONE persistent
 * cooperative launch.  b[i], x[i]: device FP64 arrays; x[i] holds the initial
 * guess on entry and the solution on exit.  `b` and `x` are HOST arrays of
 * device pointers.  info_dev: device array of `count` fde_solve_info.
 * All plans must have been assembled with the same opts->method/precision and
 * restart; opts->tol/max_iters/inner_tol/max_outer may differ from assembly.
 */
fde_status fde_krylov_solve(const fde_plan* const* plans, int count, const double* const* b,
                            double* const* x, const fde_solve_opts* opts,
                            fde_solve_info* info_dev, void* stream);

/*
 * Right-hand side of one time step, per the plan's scheme:
 *   implicit Euler (Sec. 1.2):    b = c0 u_prev + h^alpha f        (c0 = h^alpha / dt)
 *   Crank-Nicolson (Sec. 1.4):    b = (2 c0 I - M) u_prev + 2 h^alpha f
 *                                 (c0 = 1/r = 2 h^alpha / dt; f at the half step),
 * the explicit operator applied with the plan's FP64 matvec.  f may be NULL
 * (f = 0).  Device FP64 arrays of n1*n2 elements; u_prev != b.
 */
fde_status fde_step_rhs(const fde_plan* plan, const double* u_prev, const double* f,
                        double* b, void* stream);

/*
 * y = M x for a 1D problem (Sec. 1.2, eq. for M_{alpha,n}: c0 x + D_+ T x +
 * D_- T^T x, T applied by 2(n+1)-circulant embedding and FFT), in FP64, with
 * no plan, no workspace and no allocation.  The paper has no counterpart of
 * this entry point: it gives callers that cannot allocate device memory a
 * product with M.  Such callers are, for instance, a time-stepping code whose
 * device memory is held by another allocator (a caching allocator such as
 * PyTorch's may have reserved nearly all of it, so cudaMalloc fails), or a
 * loop with work in flight on other streams (cudaFree synchronises the whole
 * device and would stall them).
 *
 * The symbol data (twiddles, weights g_k or w_k, circulant eigenvalues) and
 * the transform buffers live in one fixed static device array of
 * FDE_MATVEC_NOALLOC_SCRATCH_BYTES bytes, sized for n1 <= FDE_MATVEC_NOALLOC_MAX_N.
 *   prob: 1D problem as for fde_assemble_symbol (coefficient arrays device
 *         FP64 or NULL for the constants; tau_shift and order are ignored).
 *   x, y: device FP64 arrays of n1 elements, x != y; the caller owns them.
 * Errors (nothing is launched): NULL prob/x/y, x == y, dim != 1 or an invalid
 * problem -> FDE_EINVAL; n1 > FDE_MATVEC_NOALLOC_MAX_N -> FDE_ENOMEM (the
 * problem does not fit the fixed scratch).  FDE_ECUDA if setup or a launch
 * fails.
 * Setup: the first call on each device (made with that device current)
 * resolves the scratch's device address with cudaGetSymbolAddress, once, and
 * caches it under the id of the current CUDA context; make that first call
 * before any stream capture.  After cudaDeviceReset (or with another context
 * current on the device) the context id differs, and the next call resolves
 * the address again; that call too should come before any capture.
 * No part of the scratch needs to start at zero: every call writes each
 * scratch word it reads before reading it.
 * Calls that overlap in time on one device (on different streams, or from
 * different host threads) share the scratch and race; order them on one
 * stream.  Three single-CTA launches on `stream`: meant for occasional
 * products; the solvers use fde_toeplitz_matvec with a plan.
 */
#define FDE_MATVEC_NOALLOC_MAX_N 4095
#define FDE_MATVEC_NOALLOC_SCRATCH_BYTES 640256
fde_status fde_toeplitz_matvec_noalloc(const fde_problem* prob, const double* x, double* y, void* stream);

/*
 * Transform schedule of a plan (no counterpart in the paper; the paper fixes
 * the method, not its mapping to the GPU).
 *   ctas:   CTAs that cooperate on this plan in single-plan solves and operator
 *           calls (0 = all co-resident CTAs); batched solves size their teams
 *           themselves.
 *   log_p1: 1D only.  0: a CTA holds each whole line where it fits in shared
 *           memory (else the line is split with P1 = 2^floor(log2(n1+1)/2));
 *           k >= 4: the line is split across the CTAs as a four-step FFT of
 *           n1 + 1 = P1 x P2 points, P1 = 2^k <= P2.  2D: must be 0.
 * FDE_EINVAL if the split does not fit shared memory for the plan's
 * precisions.  Rewrites the device copy of the plan on `stream`.
 */
fde_status fde_plan_set_schedule(fde_plan* plan, int ctas, int log_p1, void* stream);

/*
 * Autotuner (no counterpart in the paper): times one tau solve plus one
 * matvec -- the operators of an iteration -- in the plan's solver precision
 * on the plan's own scratch vectors for every feasible schedule
 * (fde_plan_set_schedule: ctas in {16, 32, 64, ..., all}; 1D: whole lines per
 * CTA, and every split 2^4 <= P1 <= P2) and keeps the fastest.  The choice is
 * cached per (dim, n1, n2, precision, method, restart) for the process, so a
 * later plan of the same shape takes it without timing.  Synchronises
 * `stream` (CUDA events); allocates no device memory; overwrites the plan's
 * Krylov scratch (call it between solves).  *ctas and *log_p1 (may be NULL)
 * receive the choice.
 */
fde_status fde_autotune(fde_plan* plan, void* stream, int* ctas, int* log_p1);

/*
 * Failure-path self-test (no counterpart in the paper) of the bounded team
 * barrier and of the launch-wide wind-down after a timeout.  Two CTAs each
 * enter a two-CTA team barrier of their own on the plan's sync area; the
 * partners are never launched.  CTA 0 waits with a bound of 2e6 clock cycles
 * (about 1 ms): its wait runs out and raises the launch's abort flag.  CTA 1
 * waits with the solver's full bound (about 2 s) but must see the abort flag
 * on its next poll and return too.  status_dev: device array of 2 ints that
 * receive FDE_ETIMEOUT for each CTA, the status a solve reports when a team
 * member stops arriving; the launch ends within about 1 ms plus one poll, not
 * after CTA 1's full bound.  The sync area is cleared before and after.
 * Asynchronous on `stream`.
 */
fde_status fde_selftest_barrier_timeout(const fde_plan* plan, int* status_dev, void* stream);

/*
 * Measurement helper (no counterpart in the paper): the FP64 FMA rate of the
 * current device in TFLOP/s, from one launch of eight independent DFMA
 * chains per thread over every SM (the denominator of the FP64 rooflines).
 * Synchronises `stream`; *tflops is host memory.
 */
fde_status fde_measure_fp64_rate(double* tflops, void* stream);

/* Scalars the plan derived from the problem: c0, sr, h1^alpha. */
fde_status fde_plan_scalars(const fde_plan* plan, double* c0, double* sr, double* h_alpha);

void fde_plan_destroy(fde_plan* plan);
const char* fde_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* FDE_H */
