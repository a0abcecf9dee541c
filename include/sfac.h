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

#include <stddef.h>

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
 * Supported grid lengths: powers of two 4 <= n[l] <= 4096 (FFTs of length n),
 * and any 2 <= n[l] <= 2048 otherwise: then e^{tau/2 C} and e^{tau S}, both
 * symmetric Toeplitz matrices, are applied as linear convolutions with their
 * first columns, zero-padded to a power of two L >= 2n - 1 (real multipliers,
 * no twist); an axis whose stride is odd takes that path too. Other lengths
 * return SFAC_EUNSUPPORTED. The plan owns its device tables and
 * any staging buffer; free it with sfac_plan_destroy. On success *out is set;
 * on failure *out is NULL. The call synchronises `stream` once (upload). */
sfac_status sfac_plan_create(const sfac_params* params, void* stream, sfac_plan** out);

/* How the plan runs axis `axis` (0-based): *fft_len receives the FFT length of
 * its pass (n, or the padded length L) and *padded 1 for the zero-padded
 * convolution pass, 0 for the spectral pass with the twist. */
sfac_status sfac_plan_info(const sfac_plan* plan, int axis, int* fft_len, int* padded);

/* Kernels of an axis pass (sfac_plan_kernel). The paper has no counterpart;
 * these describe only how libsfac maps the pass of Sec. 2.2 onto the GPU. */
#define SFAC_KERNEL_CTA 0    /* lines spread over a CTA, CTA-wide exchanges (FP64; FP32 N >= 1024, persistent CTAs from 2048) */
#define SFAC_KERNEL_WARP 1   /* FP32, 32 <= N <= 512: lines held inside one warp, persistent CTAs */
#define SFAC_KERNEL_STAGED 2 /* the warp kernel fed by TMA tile copies (FP32 strided axes) */

/* Which kernel a pass of axis `axis` would use for the field at u_dev: *kind
 * receives one of SFAC_KERNEL_*. The staged kernel needs an FP32 plan, a
 * spectral (not zero-padded) pass of length 32..512 on a strided axis (axis >= 1)
 * whose stride, the product of the earlier extents, is a multiple of 4 and at
 * least the tile width W (32 floats; 16 from length 256), at least as many
 * tiles (W columns of one slab) as the device has SMs, and u_dev 16-byte
 * aligned; otherwise the pass runs the warp or CTA kernel, with the same
 * arithmetic. Host-only; nothing is enqueued. */
sfac_status sfac_plan_kernel(const sfac_plan* plan, int axis, const void* u_dev, int* kind);

/* How sfac_step runs a call of nsteps steps (sfac_plan_step_kernel). The paper
 * has no counterpart. */
#define SFAC_STEP_PASSES 0 /* one launch per axis pass */
#define SFAC_STEP_WHOLE 1  /* small grids: the whole call in one cooperative launch */

/* *kind receives SFAC_STEP_WHOLE if sfac_step(plan, u, nsteps) runs the whole
 * call in one cooperative launch: two steps or more, every axis a spectral
 * (not zero-padded) pass of 32..256 points, at most 65536 unknowns, and every
 * line's warp resident at once on the device (one 32-thread CTA per line pair,
 * N/32 values per thread). The CTAs meet at a grid-wide barrier between passes;
 * each wait on it is bounded by the plan's wait limit (sfac_plan_set_wait_limit,
 * whose hold hook makes the first wait of every CTA run out), and a wait that
 * runs out is reported by sfac_plan_check. Otherwise SFAC_STEP_PASSES: one
 * launch per axis pass. Host-only. */
sfac_status sfac_plan_step_kernel(const sfac_plan* plan, long long nsteps, int* kind);

/* Synchronise `stream`, then report whether an axis pass of this plan gave up
 * on one of its bounded waits since the last check: SFAC_ETIMEOUT if so (the
 * field written by that pass is not valid; the flag is cleared), SFAC_OK
 * otherwise. The staged kernel waits on its tile copies and the whole-call
 * launch of small grids on its grid barrier (about two seconds at most per
 * wait); sfac_step_host checks automatically. The paper has no counterpart. */
sfac_status sfac_plan_check(sfac_plan* plan, void* stream);

/* Limit of each bounded wait of the plan's passes, in SM clock cycles
 * (default 2^32, about two seconds at 2.07 GHz; must be >= 1). hold != 0 is a
 * test hook: the first wait of every CTA of a staged pass then waits for a
 * barrier that nothing completes, so it runs out after wait_cycles, the pass
 * records the timeout (see sfac_plan_check) and leaves the field partly
 * updated. Host-only. The paper has no counterpart. */
sfac_status sfac_plan_set_wait_limit(sfac_plan* plan, long long wait_cycles, int hold);

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

/* Monitoring reductions (Examples 4 and 5, Sec. 5): out[0] = max |u| and
 * out[1] = the discrete energy E(u) = h^d ( (1/4) sum (u^2 - 1)^2
 * - (1/2) u^T A u ), h^d the product of the axes' h, A u = sum_l B_l along axis l.
 * u^T A u is accumulated line by line as x . B_l x with B_l x formed through the
 * spectra of C_l and S_l (zero-padded axes: one linear convolution with B_l's
 * column); FP64 arithmetic for both precisions; partial sums are added in a
 * fixed order (deterministic). u_dev is read only. Synchronises `stream`. */
sfac_status sfac_diagnostics(sfac_plan* plan, const void* u_dev, double* out, void* stream);

/* End-to-end variant on HOST memory: advance u_host (plan precision, layout
 * above) by nsteps through a plan-owned device buffer and leave the result in
 * u_host. u_host may be pageable or pinned; the route (sfac_plan_host_route)
 * is one of
 *   SFAC_HOST_COPY       cudaMemcpyAsync in, the steps, cudaMemcpyAsync out;
 *   SFAC_HOST_MAPPED     the first pass of the call loads the field from u_host
 *                        and the last pass stores the result into it: pinned
 *                        memory is mapped into the device's address space, so
 *                        the transfers ride inside those two passes (over
 *                        NVLink-C2C on GB300) and no copy runs;
 *   SFAC_HOST_MAPPED_IN  the first pass loads from u_host, a copy brings the
 *                        result back.
 * Every route gives the same bits as sfac_step on a device field. Blocks until
 * the result is in u_host. The staging buffer is allocated on the first call
 * and kept by the plan. Not safe to call concurrently on one plan. Errors:
 * SFAC_EINVAL (NULL plan or u_host, nsteps < 0), SFAC_ENOMEM (the staging
 * buffer), SFAC_ECUDA (a copy, launch or synchronisation), SFAC_ETIMEOUT (a
 * pass gave up a bounded wait, as sfac_plan_check reports; u_host then holds
 * a field that is not valid). The paper has no counterpart. */
sfac_status sfac_step_host(sfac_plan* plan, void* u_host, long long nsteps, void* stream);

#define SFAC_HOST_COPY 0
#define SFAC_HOST_MAPPED 1
#define SFAC_HOST_MAPPED_IN 2

/* *route receives the SFAC_HOST_* route sfac_step_host(plan, u_host, nsteps)
 * takes. A mapped route needs pinned (page-locked, CUDA-registered) u_host,
 * 16-byte aligned, nsteps >= 1, the per-pass launches (not the whole-call
 * launch of small grids) and at least 4096 complex lines (line pairs) in both
 * the first and the last pass, so that the link's latency hides behind other
 * lines' work; otherwise SFAC_HOST_COPY. It is SFAC_HOST_MAPPED_IN for an FP32
 * plan whose last axis has an FFT length above 512 (whose pass would write
 * rows too narrow for the link). Host-only; nothing is enqueued. SFAC_EINVAL
 * for a NULL plan, u_host or route, or nsteps < 0. The paper has no
 * counterpart. */
sfac_status sfac_plan_host_route(const sfac_plan* plan, const void* u_host, long long nsteps, int* route);

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

/* ------------------------------------------------------------------------ */
/* Batched runner: many independent problems in one persistent launch.       */
/* ------------------------------------------------------------------------ */

/* A batch of `count` independent problems, each advanced by eq. (finalstrang)
 * with its own grid, alpha, eps, tau and step count. One persistent kernel
 * runs every instance: its work items (groups of lines of one axis pass of one
 * instance at one step) are claimed by warps in an order that respects each
 * instance's pass order; a warp starts an item once every item of the same
 * instance's previous pass has finished (per-instance completion counters).
 * The batch owns its tables, schedule and scratch counters; the caller owns
 * the fields. */
typedef struct sfac_batch sfac_batch;

/* Build a batch: params[i] describes instance i (dim 2 or 3; every n[l] a power
 * of two in [32, 512]; one precision for all). The spectral factors of each
 * instance and axis are computed in FP64 on the host (as in sfac_plan_create);
 * the twists and twiddles, which depend on the line length only, are held once
 * per batch for every length. Both are uploaded on `stream` (synchronised).
 * SFAC_EUNSUPPORTED for other shapes. */
sfac_status sfac_batch_create(const sfac_params* params, int count, void* stream, sfac_batch** out);

/* Release the batch (synchronises the device first). NULL is a no-op. */
sfac_status sfac_batch_destroy(sfac_batch* batch);

/* Bind fields and step counts: u_dev[i] is instance i's device field (layout of
 * sfac_step, 16-byte aligned), nsteps[i] >= 0 its number of steps. Builds the
 * phase schedule on the host and uploads it (synchronises `stream`). */
sfac_status sfac_batch_prepare(sfac_batch* batch, void* const* u_dev, const long long* nsteps, void* stream);

/* Enqueue the prepared run on `stream`: reset the scratch counters, launch the
 * persistent kernel, copy its status flag to host memory. Asynchronous, with no
 * host synchronisation and no allocation, so it can be captured in a CUDA
 * graph and replayed (each replay advances every field again). */
sfac_status sfac_batch_launch(sfac_batch* batch, void* stream);

/* Synchronise `stream` and report the status of the last launch: SFAC_ETIMEOUT
 * if a dependency wait gave up (the kernel then returns early and fields may be
 * partly advanced), SFAC_ECUDA for a CUDA error. */
sfac_status sfac_batch_wait(sfac_batch* batch, void* stream);

/* prepare + launch + wait. */
sfac_status sfac_batch_step(sfac_batch* batch, void* const* u_dev, const long long* nsteps, void* stream);

/* Autotuner: time every kernel shape (warps per CTA, values per thread, i.e. the
 * radix schedule of lines up to 256 points, and line groups per work item) on
 * copies of the prepared fields for min(nsteps, max_steps) steps, keep the
 * fastest and re-prepare. Requires a prepared batch; the fields are not
 * changed. *choice (may be NULL) receives the chosen shape's index. */
sfac_status sfac_batch_autotune(sfac_batch* batch, int max_steps, void* stream, int* choice);

/* Select a kernel shape by index in [0, sfac_batch_num_configs()) (takes effect
 * at the next prepare) and read back the current one. */
sfac_status sfac_batch_set_config(sfac_batch* batch, int config);
sfac_status sfac_batch_get_config(const sfac_batch* batch, int* config, int* warps_per_cta,
                                  int* values_per_thread, int* groups_per_item);
int sfac_batch_num_configs(void);

/* Failure-detection controls: every dependency wait polls at most spin_limit
 * times (about 100 ns apart) before the launch gives up with SFAC_ETIMEOUT.
 * hold_instance >= 0 makes that instance's second pass wait for a completion
 * count that is never reached, to exercise the bounded wait (-1: off). Takes
 * effect at the next prepare. */
sfac_status sfac_batch_set_wait_limit(sfac_batch* batch, long long spin_limit, int hold_instance);

/* Largest batch sfac_batch_launch_noalloc accepts. */
#define SFAC_NOALLOC_MAX_INSTANCES 8192

/* No counterpart in the paper: a deployment convenience. Same as
 * sfac_batch_launch, but allocating nothing: the persistent kernel's work
 * counter, per-instance completion counters and status word live in one fixed
 * array of (SFAC_NOALLOC_MAX_INSTANCES + 2) * 8 bytes = 64 KiB of device memory
 * that the library holds on every GPU it is loaded on until the process exits.
 * For callers that must not call cudaMalloc when they launch work (an
 * allocator that owns all device memory, latency-critical loops where
 * allocation may synchronise the device, fixed memory budgets). The batch must
 * be prepared (its tables and schedule were allocated by sfac_batch_create and
 * sfac_batch_prepare); the caller's fields are the inputs and outputs. Batches
 * of more than SFAC_NOALLOC_MAX_INSTANCES instances are rejected with
 * SFAC_EINVAL. All calls on a device share the array: each call clears the
 * counters first, and calls whose work overlaps on the GPU race, so serialise
 * them. The first call on each device looks up the array's device address
 * (with the batch's device made current); make that first call before any
 * stream capture. The address is kept per device and context: after a context
 * reset (e.g. cudaDeviceReset) the next call on that device looks it up again,
 * so make that call before any capture too. Report status with sfac_batch_wait
 * as for sfac_batch_launch. */
sfac_status sfac_batch_launch_noalloc(sfac_batch* batch, void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of requests of different sizes.              */
/* ------------------------------------------------------------------------ */

/* A server owns one device arena of `arena_bytes`. An admitted request gets a
 * slot whose field and per-axis spectral factors (as in sfac_plan_create) stay
 * resident in the arena until its result is fetched; twists and twiddles are
 * held once per server for every line length. A round advances every active slot by
 * up to `chunk` steps in one persistent launch of the batched kernel, so
 * requests admitted while rounds run join a later round. Up to two rounds may
 * be in flight: the second is enqueued behind the first (each has its own
 * schedule, counters and status word), so the caller can collect the first
 * round's finished requests while the device runs the second. A slot always
 * advances in whole chunks counted from its own first step, so its result does
 * not depend on which other requests share its rounds. */
typedef struct sfac_server sfac_server;

/* Create a server with `max_slots` slots for problems of precision `prec`.
 * Allocates the arena, the scratch counters and an internal copy stream. */
sfac_status sfac_server_create(size_t arena_bytes, int max_slots, int prec, void* stream, sfac_server** out);

/* Release everything (synchronises the device first). NULL is a no-op. */
sfac_status sfac_server_destroy(sfac_server* server);

/* Arena bytes one request with these parameters occupies (field + the two
 * spectral factors per axis). */
sfac_status sfac_server_request_bytes(const sfac_params* params, size_t* bytes);

/* Admit a request: dim 2 or 3, every n[l] a power of two in [32, 512], the
 * server's precision; u0_host holds its initial field (layout of sfac_step);
 * nsteps >= 0. Computes its FP64 tables on the host and copies field and tables
 * into the arena on the internal copy stream (synchronised), which may overlap
 * a round in flight. Returns SFAC_ENOMEM, and admits nothing, when no slot or
 * no arena block is free: admission is by device memory, the caller keeps the
 * request queued and retries after results are fetched. *slot receives the slot. */
sfac_status sfac_server_admit(sfac_server* server, const sfac_params* params, const void* u0_host,
                              long long nsteps, int* slot);

/* Enqueue one round on `stream`: every slot with steps left that no round in
 * flight already covers advances by min(chunk, those steps) steps (kernel
 * shape `shape`, an index as in sfac_batch_set_config). Asynchronous: the
 * schedule goes up through pinned memory, so the call does not wait for a
 * round in flight; the new round starts on the device after that round ends
 * (also on another stream). At most two rounds in flight (SFAC_EINVAL
 * otherwise). *launched (may be NULL) receives 1 if a round was enqueued, 0 if
 * no slot had open steps (then nothing is enqueued). */
sfac_status sfac_server_round(sfac_server* server, long long chunk, int shape, void* stream, int* launched);

/* Wait for the oldest round in flight (host wait on its completion event; a
 * later round keeps running) and list the slots that have no steps left and
 * no round in flight: up to max_finished slot numbers go to finished[],
 * *nfinished receives their count. With no round in flight: SFAC_OK and none.
 * If a dependency wait of the round gave up, every slot of that round is
 * marked failed (its field is partly advanced), the call returns SFAC_ETIMEOUT
 * and still lists the slots that are finished, the failed ones among them once
 * no round in flight holds them; later rounds skip failed slots. */
sfac_status sfac_server_wait(sfac_server* server, void* stream, int* finished, int max_finished,
                             int* nfinished);

/* Copy a slot's field to u_host (if not NULL; on the internal copy stream,
 * synchronised, so it may overlap rounds in flight that do not include the
 * slot) and, if release != 0, free its slot and arena block. SFAC_EINVAL if a
 * round in flight still holds the slot. For a failed slot nothing is copied
 * and the call returns SFAC_ETIMEOUT (after freeing the slot if release != 0). */
sfac_status sfac_server_fetch(sfac_server* server, int slot, void* u_host, int release);

/* Failure-detection controls of the server's rounds, as sfac_batch_set_wait_limit:
 * every dependency wait polls at most spin_limit times; hold_slot >= 0 makes
 * the next round that advances that slot wait on a count that is never reached
 * in the slot's second pass, so the round gives up (-1: off; the hook acts on
 * one round only). Host-only. The paper has no counterpart. */
sfac_status sfac_server_set_wait_limit(sfac_server* server, long long spin_limit, int hold_slot);

/* Free arena bytes, largest free block, slots in use and slot capacity (each
 * pointer may be NULL). */
sfac_status sfac_server_info(const sfac_server* server, size_t* free_bytes, size_t* largest_free,
                             int* active, int* capacity);

/* ------------------------------------------------------------------------ */
/* Measurement                                                               */
/* ------------------------------------------------------------------------ */

/* Microbenchmark of the SMs' multiply-add rate: the ALU roofline the FP64 and
 * FP32 axis passes are reported against. The paper has no counterpart.
 * Enqueues one kernel of `blocks` CTAs of 256 threads on `stream`; every thread
 * runs 8 independent chains x <- fma(x, a, b) for 16 * iters rounds and writes
 * one value to out_dev[thread], which must hold blocks * 256 elements (double
 * for kind 0, float otherwise). kind 0: FP64 fma; 1: FP32 fmaf; 2: the packed
 * two-lane FP32 multiply-add (each chain a pair of floats). The launch executes
 * blocks * 256 * 8 * 16 * iters multiply-adds (kind 2: twice as many lanes),
 * 2 flops each. Asynchronous: time it with events on `stream`.
 * SFAC_EINVAL for an unknown kind, blocks < 1, iters < 1 or a NULL buffer. */
sfac_status sfac_probe_fma(int kind, int blocks, long long iters, void* out_dev, void* stream);

/* The nonlinear flow J^Q_s(v) = v / sqrt(E + (1 - E) v^2), E = e^{-2s} (the
 * exact solution of u' = u - u^3 over time s, Sec. 2.2), evaluated on n values
 * by the very device code the passes use: v times the double reciprocal
 * square root of E + (1 - E) v^2 in the FP64 passes, v plus the increment of
 * the FP32 passes (which use 1 - E only). It lets a test measure that code's error value by value; the paper
 * has no counterpart. prec SFAC_FP64 / SFAC_FP32 sets the element type of
 * v_dev and out_dev (n elements each, device memory, may be the same buffer);
 * E in (0, 1] and one_minus_E = 1 - E as the plans compute them. Enqueued on
 * `stream`, asynchronous. SFAC_EINVAL for another prec, n < 0 or n > 2^36,
 * NULL buffers with n > 0, or E outside (0, 1]; n = 0 enqueues nothing. */
sfac_status sfac_probe_jq(int prec, const void* v_dev, void* out_dev, long long n, double E,
                          double one_minus_E, void* stream);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* sfac_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int sfac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SFAC_H */
