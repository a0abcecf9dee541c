/*
 * sfac.h - C ABI of libsfac: the time step of the two-level Strang splitting
 * scheme for the d-dimensional (d = 1, 2, 3) spatial fractional Allen-Cahn
 * equation u_t = eps^2 L^alpha u + u - u^3 on [a, b]^d with zero Dirichlet data
 * (Cai, Fang, Chen, Sun, arXiv 2209.08437, eq. (FAC)), on one NVIDIA GB300.
 *
 * One step (eq. (finalstrang), Sec. 2.2) is
 *     u <- J^Q_{tau/2}  [ prod_l e^{tau/2 C_l} e^{tau S_l} e^{tau/2 C_l} ]  J^Q_{tau/2} u
 * where B_l = C_l + S_l is the symmetric Toeplitz Riesz matrix of axis l
 * (eq. (B), with eps^2 inside B), C_l its circulant part and S_l its
 * skew-circulant part (eqs. (C), (S)), and J^Q_s the exact flow of v' = v - v^3
 * (eq. (nonlinear_operator)). Each exponential is applied along every grid line
 * of its axis as FFT -> multiply by exp(t * eigenvalue) -> inverse FFT, the skew
 * part between the twist diag(e^{i pi k / n}) and its inverse (Remark 1).
 *
 * Conventions shared by every entry point
 * - Field layout: a contiguous array of n[0] * n[1] * n[2] reals (only the first
 *   `dim` extents are used) holding the interior unknowns, axis 1 (x^(1))
 *   fastest: element (i1, i2, i3) sits at i1 + n[0] * (i2 + n[1] * i3). This is
 *   the lexicographic ordering of Sec. 2.1; the zero boundary is implicit.
 * - Reals are double for SFAC_FP64 plans and float for SFAC_FP32 plans.
 * - Device pointers are CUDA device memory of the current device; `stream` is a
 *   cudaStream_t (NULL = the legacy default stream). Calls are stream-ordered
 *   and asynchronous unless stated otherwise.
 * - Every call returns an sfac_status. Argument errors are detected on the host
 *   before anything is enqueued and leave the field untouched. Launch errors
 *   come back as SFAC_ECUDA; asynchronous device faults surface on a later call
 *   or synchronisation. No exception crosses the ABI. sfac_last_error() gives a
 *   message for the calling thread's most recent failure.
 * - Input range: the maximum principle (Theorem 1, Sec. 3) holds for
 *   max|u0| <= 1; other values are accepted and stay finite for tau > 0.
 */
#ifndef SFAC_H
#define SFAC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFAC_OK = 0,
    SFAC_EINVAL = 1,        /* bad argument (NULL, alpha outside (1,2), eps/tau <= 0, b <= a, ...) */
    SFAC_EUNSUPPORTED = 2,  /* valid but not implemented (e.g. an unsupported grid length) */
    SFAC_ENOMEM = 3,        /* device or host allocation failed */
    SFAC_ECUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    SFAC_ETIMEOUT = 5       /* a bounded wait gave up */
} sfac_status;

typedef enum { SFAC_FP64 = 0, SFAC_FP32 = 1 } sfac_precision;

/* Problem description (Sec. 2.1). n[l] is the number of interior unknowns of
 * axis l+1, i.e. m_l - 1 for m_l mesh intervals, so h_l = (b - a) / (n[l] + 1).
 * alpha[l] in (1, 2) is the Riesz order of axis l+1. Extents beyond `dim` are
 * ignored. `prec` selects the arithmetic of the device passes; the tables
 * (Riesz weights, eigenvalues, their exponentials, twists, twiddles and the
 * nonlinear-flow constants) are always computed in FP64 on the host and
 * rounded once for FP32 plans. */
typedef struct sfac_params {
    int dim;          /* 1, 2 or 3 */
    int n[3];         /* interior points per axis */
    double alpha[3];  /* Riesz orders, each in (1, 2) */
    double eps;       /* interface parameter, > 0 */
    double tau;       /* time step, > 0 */
    double a, b;      /* domain [a, b]^dim, b > a */
    int prec;         /* sfac_precision */
    int reserved;     /* must be 0 */
} sfac_params;

typedef struct sfac_plan sfac_plan;

/* Build a plan: per-axis FP64 precompute on the host (omega_k by eqs. (g_coe),
 * (omega_coe); b_k by eq. (B); c_k, s_k by eqs. (C), (S); circulant eigenvalues
 * lambda_j = sum_k c_k e^{-2 pi i jk/n} and skew-circulant eigenvalues
 * mu_j = sum_k s_k e^{i pi k/n} e^{-2 pi i jk/n} by Remark 1; the tables
 * e^{tau/2 lambda_j}/n, e^{tau mu_j}/n, e^{i pi k/n}, e^{-2 pi i m/n}), then one
 * upload of those tables to the current device on `stream`.
 * Supported grid lengths: every n[l] a power of two with 4 <= n[l] <= 4096.
 * Other lengths return SFAC_EUNSUPPORTED. The plan owns its device tables and
 * any staging buffer; free it with sfac_plan_destroy. On success *out is set;
 * on failure *out is NULL. The call synchronises `stream` once (upload). */
sfac_status sfac_plan_create(const sfac_params* params, void* stream, sfac_plan** out);

/* Release a plan and its device memory. Synchronises the device first so that no
 * enqueued work still reads the tables. NULL is accepted (no-op). */
sfac_status sfac_plan_destroy(sfac_plan* plan);

/* Advance the device field u_dev (layout above, plan precision) by `nsteps`
 * complete steps of eq. (finalstrang) on `stream`; nsteps = 0 is a no-op.
 * Each axis is one fused pass over the field (load, J^Q if first, six FFTs
 * with the eigenvalue multiplies and the twist, J^Q if last, store); inside one
 * call the closing J^Q_{tau/2} of a step and the opening J^Q_{tau/2} of the
 * next are applied together as J^Q_{tau} (exact: J^Q is a flow). u_dev is
 * updated in place and must not be accessed by other streams until the work
 * completes. Returns SFAC_EINVAL for NULL pointers or nsteps < 0. */
sfac_status sfac_step(sfac_plan* plan, void* u_dev, long long nsteps, void* stream);

/* sfac_step with nsteps = T / tau. T / tau must be within 1e-9 relative of an
 * integer (the partition t_n = n tau <= T of Sec. 2.2 takes whole steps only);
 * otherwise SFAC_EINVAL. */
sfac_status sfac_solve(sfac_plan* plan, void* u_dev, double T, void* stream);

/* One fused pass of the linear factor along one axis: every grid line of axis
 * `axis` (0-based, < dim) of u_dev is replaced by e^{tau/2 C} e^{tau S} e^{tau/2 C}
 * applied to it (eq. (hatv), per axis by the Kronecker-sum form of eq.
 * (newlinear)). jq_in / jq_out select the nonlinear flow applied pointwise on
 * load / store: 0 none, 1 J^Q_{tau/2}, 2 J^Q_{tau} (eq. (nonlinear_operator)).
 * sfac_step(plan, u, 1) launches exactly axis_pass(0, 1, 0), axis_pass(1, 0, 0),
 * ..., axis_pass(dim-1, 0, 1) (for dim = 1: axis_pass(0, 1, 1)); this entry point
 * exposes one such launch so that callers can time or test it alone.
 * SFAC_EINVAL for a bad axis, mode or pointer. */
sfac_status sfac_axis_pass(sfac_plan* plan, void* u_dev, int axis, int jq_in, int jq_out, void* stream);

/* End-to-end variant on HOST memory: copy u_host (plan precision, layout above)
 * to a plan-owned device buffer, advance it by nsteps, copy it back into u_host.
 * u_host may be pageable or pinned; pinned memory gives full copy bandwidth.
 * Blocks until the result is in u_host. The staging buffer is allocated on the
 * first call and kept by the plan. Not safe to call concurrently on one plan. */
sfac_status sfac_step_host(sfac_plan* plan, void* u_host, long long nsteps, void* stream);

/* Host-only: the FP64 tables sfac_plan_create computes for axis `axis` (0-based)
 * of `params`, without touching any GPU. Each output pointer may be NULL; a
 * non-NULL one must hold n = params->n[axis] doubles:
 *   lambda[j]   circulant eigenvalues of C_axis       (Remark 1)
 *   mu[j]       skew-circulant eigenvalues of S_axis  (Remark 1)
 *   bcol[k]     first column b_k of B_axis            (eq. (B))
 * and jq[4] (if non-NULL) receives {e^{-tau}, 1 - e^{-tau}, e^{-2 tau},
 * 1 - e^{-2 tau}}, the constants of J^Q_{tau/2} and J^Q_{tau} (eq. (nonlinear_operator)). */
sfac_status sfac_plan_tables(const sfac_params* params, int axis, double* lambda, double* mu,
                             double* bcol, double* jq);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* sfac_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int sfac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SFAC_H */
