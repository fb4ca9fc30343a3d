/*
 * spring_ising.h -- C ABI of the GB300 (sm_103a) Spring-Ising hot path.
 *
 * The Spring-Ising Algorithm (arXiv 2305.07187) treats every Ising spin as a
 * mass on a zero-length spring driven by the coupling force F = J q (+ h) and
 * iterates (Eq. 8, walls of Eq. 6)
 *
 *     p <- clip(p + dt_n ( -k (q - q0) + zeta_n F ),  -p_max, p_max)
 *     q <- clip(q + (dt_n / m) p,                       -q_max, q_max)
 *
 * for R independent replicas ("parallel tests", Fig. 3), then reads the spins
 * as sign(q) and scores them with the Ising energy of Eq. 1.
 *
 * General conventions
 *   - Every pointer argument may be host or device memory; the library tells
 *     them apart with cudaPointerGetAttributes.  Host inputs are copied in on
 *     the context's stream; host outputs are copied out.  si_run and
 *     si_energy are asynchronous with respect to the host when all of their
 *     array arguments are device memory (or NULL): they return once their
 *     work is enqueued on the context's stream, and a device-side error of
 *     that work (a timed-out wait) is reported by the next call that
 *     synchronises, which also drops the run's state (no continuing, no
 *     readout of its spins).  A call with any host input or host output
 *     returns only after its work has finished, so the caller may reuse or
 *     free its host buffers (pinned ones included) as soon as it returns.
 *     The other computing calls (si_grad, si_hamiltonian, si_get_state,
 *     si_run_group, si_group_energy) always return after their work has
 *     finished: they end by reading the device error word.  si_synchronize
 *     waits for a context's work and reports its pending device error.
 *   - The caller owns every buffer it passes.  The context owns its device
 *     copy of J, the integrator state, the operand buffers and the
 *     checkpoints, all allocated in si_create and freed in si_destroy.
 *   - Layouts: J is n x n row-major (J[i*n + j]); per-replica arrays are
 *     replica-major, x[r*n + i].
 *   - No call aborts the process.  Each returns an si_status; si_last_error()
 *     gives a message for the last failure on the calling thread.  A device
 *     wait that exceeds its time limit ends the kernel cooperatively and is
 *     reported as SI_ERR_TIMEOUT; the context stays usable.  After an
 *     error status the contents of the call's outputs are unspecified.
 */
#ifndef SPRING_ISING_H
#define SPRING_ISING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct si_ctx si_ctx;

typedef enum {
    SI_OK = 0,
    SI_ERR_INVALID_ARG = 1,   /* bad size, NULL where required, bad enum    */
    SI_ERR_CUDA = 2,          /* a CUDA runtime call failed                 */
    SI_ERR_OOM = 3,           /* device allocation failed                   */
    SI_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out         */
    SI_ERR_UNSUPPORTED = 5,   /* valid request this build cannot serve      */
    SI_ERR_NOT_SYMMETRIC = 6  /* J not symmetric, or non-zero diagonal      */
} si_status;

/* Arithmetic of the hot path.  The paper does not state its precision. */
typedef enum {
    SI_PREC_FP32 = 0,          /* J, q, p, F in FP32 on CUDA cores           */
    SI_PREC_FP64 = 1,          /* debug: everything FP64 (slow on GB300)     */
    SI_PREC_J_FP8_Q_BF16 = 2,  /* J validated exact in e4m3 (e.g. +-1),
                                  q rounded to bf16 as the tensor-core
                                  operand, FP32 accumulation and state      */
    SI_PREC_J_BF16_Q_BF16 = 3  /* J rounded once to bf16 (Gaussian J),
                                  otherwise as above                        */
} si_prec;

/* Update order of one time step. */
typedef enum {
    SI_ORDER_KICK_DRIFT = 0,   /* Eq. 8: p from q(t_n), then q from new p    */
    SI_ORDER_EULER = 1         /* Eq. 5 literally: both from the old state   */
} si_order;

typedef struct {
    int32_t n;              /* number of spins, >= 1                          */
    int32_t replicas;       /* R, independent runs, >= 1                      */
    int32_t steps;          /* T, length of the schedules given to si_run     */
    float   k;              /* spring constant (paper: 0.5)                   */
    float   m;              /* mass (paper: 1)                                */
    float   q0;             /* spring origin (paper: 0)                       */
    float   q_max;          /* position wall, Eq. 6 (paper: sqrt 2)           */
    float   p_max;          /* momentum wall (paper: 2)                       */
    int32_t prec;           /* si_prec                                        */
    int32_t update_order;   /* si_order                                       */
    int32_t wall_zero_p;    /* 1: zero p of a spin whose q was clipped        */
    int32_t ckpt_every;     /* si_grad checkpoint interval (0: 50)            */
    int32_t tile_n;         /* tensor-core replica tile (0: autotuned)        */
    int32_t fused_readout;  /* 1: a tensor-path si_run also sums sigma^T J
                               sigma of its final spins inside the step
                               kernel (one more pass over J), so that the
                               next si_energy with spins NULL only finishes
                               E and the cut (Eq. 1, 2); 0: off.  Contexts
                               served by the grouped kernel, with the e4m3
                               operand or on CTA pairs ignore it.            */
    int32_t reserved[3];    /* must be zero                                   */
} si_params;

/* Fill *p with the paper's parameters (k=0.5, m=1, q0=0, q_max=sqrt 2,
 * p_max=2, kick-drift, FP32) and n = replicas = steps = 0. */
void si_default_params(si_params *p);

/*
 * Create a context for one Ising instance.
 *   J      n*n floats, row-major; must be symmetric with a zero diagonal
 *          (Eq. 1 sums over pairs i < j; the force of Eq. 4 uses full rows),
 *          else SI_ERR_NOT_SYMMETRIC.  SI_PREC_J_FP8_Q_BF16 additionally
 *          requires every entry to be exact in e4m3, else SI_ERR_INVALID_ARG.
 *   h      n floats (external field of Eq. 1) or NULL for h = 0.
 *   stream cudaStream_t (as void*) on which all work of this context is
 *          enqueued; NULL is the legacy default stream.
 * J and h are copied (and converted to the storage precision) before the call
 * returns; the caller may free them afterwards.
 */
si_status si_create(si_ctx **out, const si_params *prm, const float *J,
                    const float *h, void *stream);

/*
 * Run prm.steps time steps of Eq. 8 (or Eq. 5) for all replicas.
 *   zeta    [steps]  coupling coefficient zeta(t_n) (the dynamic-equilibrium
 *                    ramp of the paper is a host-built schedule)
 *   dt      [steps]  time step Delta_n
 *   q_init  [R][n]   initial positions; or NULL to continue from the
 *                    context's state at its working precision (the final
 *                    state of the last successful si_run, or of the forward
 *                    sweep of the last si_grad), with p_init NULL too;
 *                    SI_ERR_INVALID_ARG if there is no such state.  A
 *                    segmented run continued this way equals one run over the
 *                    concatenated schedules.
 *   p_init  [R][n]   initial momenta, or NULL for zero
 *   q_out   [R][n]   final positions, or NULL
 *   p_out   [R][n]   final momenta, or NULL
 *   spins_out [R][n] final spins sign(q) in {-1,+1} as int8 (sign(0) = +1),
 *                    or NULL
 * The run is deterministic: the same inputs give bit-identical outputs.
 */
si_status si_run(si_ctx *ctx, const float *zeta, const float *dt,
                 const float *q_init, const float *p_init, float *q_out,
                 float *p_out, int8_t *spins_out);

/*
 * si_run with a watch on the energy (the time-to-target use of the method):
 * after every `every` steps, and after the last one, the exact Ising energy
 * of Eq. 1 of every replica's spins sign(q) is summed inside the step kernel
 * (one more pass over J with the spins as the operand), and the run stops at
 * the first such readout at which some replica's energy is at most
 * target_energy.  A target cut C of the MAX-CUT instance with w_ij = -J_ij
 * (and h = 0) is the energy -2 C - sum_{i<j} J_ij.  Every CTA takes the same
 * decision at the same readout, so all replicas stop at the same step.
 *   zeta, dt, q_init, p_init   as for si_run (prm.steps entries; the run
 *                    reads only those of the steps it makes)
 *   every           readout interval in steps, >= 1
 *   q_out, p_out, spins_out    the state at the stop (or after prm.steps
 *                    steps), as for si_run; a continuing call (q_init NULL)
 *                    of si_run or si_run_watch starts from it
 *   steps_done      [1] steps made: min(prm.steps, (k + 1) every) for the
 *                    stopping readout k; host memory; or NULL
 *   energy_out      [R] int32 energies of the last readout, host or device,
 *                    or NULL
 * The call returns after the run has completed (it needs the decision).
 * Requires a context whose steps all run in one tensor-core kernel (the
 * bf16 operand of SI_PREC_J_FP8_Q_BF16 or SI_PREC_J_BF16_Q_BF16 on single
 * CTAs) with J and h integer-valued, |J_ij|, |h_i| <= 127; else
 * SI_ERR_UNSUPPORTED.  Deterministic: the same inputs give the same stop and
 * bit-identical outputs, equal to those of si_run over the steps made.
 */
si_status si_run_watch(si_ctx *ctx, const float *zeta, const float *dt,
                       const float *q_init, const float *p_init, int32_t every,
                       int64_t target_energy, float *q_out, float *p_out,
                       int8_t *spins_out, int32_t *steps_done,
                       int32_t *energy_out);

/*
 * Change the integrator parameters of an existing context without copying J
 * again: k, m, q0, q_max, p_max, update_order, wall_zero_p, ckpt_every and
 * fused_readout take the values in *prm for every later call (e.g. the spring constant
 * being tuned by gradient descent).  n, replicas, steps, prec and tile_n
 * must equal the context's (else SI_ERR_INVALID_ARG); the other fields are
 * checked as in si_create.  The context's state, J and h are kept, so a
 * run may continue (q_init NULL) under the new parameters.  Work already
 * enqueued keeps the values it was launched with.
 */
si_status si_set_params(si_ctx *ctx, const si_params *prm);

/*
 * Copy the state after the last si_run at the context's working precision,
 * widened to double: q_out, p_out [R][n] (either may be NULL).  Used by the
 * FP64 debug mode, whose state would lose digits through si_run's float
 * outputs.  Returns SI_ERR_INVALID_ARG if no run has completed.
 */
si_status si_get_state(si_ctx *ctx, double *q_out, double *p_out);

/*
 * Ising energy of Eq. 1 and cut value for R spin vectors.
 *   spins      [R][n] int8 in {-1,+1}; or NULL for the sign readout of the
 *              final state of the last si_run on this context (R must then
 *              equal the context's replica count; SI_ERR_INVALID_ARG if no
 *              si_run has completed since creation or since the last si_grad)
 *   energy_out [R] exact int32 energy; requires J and h integer-valued with
 *              |J_ij|, |h_i| <= 127 (else SI_ERR_UNSUPPORTED); or NULL
 *   cut_out    [R] exact int32 cut of the MAX-CUT instance with weights
 *              w_ij = -J_ij (same integrality requirement); or NULL
 *   energy_f   [R] energy as double for any J; exact (the integer energy)
 *              when J and h are integer-valued, else computed in FP32;
 *              or NULL
 * R may differ from the context's replica count.  With spins NULL after a
 * run whose step kernel summed sigma^T J sigma itself (si_params
 * fused_readout), only E and the cut are finished here (one small kernel);
 * the results are the same, bit for bit.
 */
si_status si_energy(si_ctx *ctx, const int8_t *spins, int32_t R,
                    int32_t *energy_out, int32_t *cut_out, double *energy_f);

/*
 * Gradient of the relaxed Ising energy at the final step,
 *   L = sum_r ( -1/2 q_r^T J q_r - h^T q_r ),  q_r after prm.steps steps,
 * with respect to the schedules and the spring constant, by an adjoint sweep
 * that integrates the equation of motion backwards (checkpoints every
 * prm.ckpt_every steps, recomputation in between).  The derivative of each
 * wall clamp is taken as 1 strictly inside and 0 on or beyond the wall.
 *   zeta, dt  [steps] float, host or device
 *   q_init    [R][n] float; p_init [R][n] float or NULL (zero momenta)
 *   g_zeta [steps], g_dt [steps], g_k [1], objective [1] float, host or
 *   device; any may be NULL.
 * FP32 contexts whose J is exact in bf16 compute the products J X^T on the
 * tensor cores from a three-piece bf16 split of the FP32 operand (exact
 * products, FP32 accumulation); otherwise, and for SI_PREC_FP64, on CUDA
 * cores.  SI_ADJOINT_SIMT=1 in the environment forces the CUDA cores.  After
 * the call si_get_state returns the final state of the forward sweep.
 * Deterministic: repeated calls give bit-identical results, whatever
 * ckpt_every is.  Supported for SI_PREC_FP32 and SI_PREC_FP64, kick-drift
 * order, without wall_zero_p (else SI_ERR_UNSUPPORTED).
 */
si_status si_grad(si_ctx *ctx, const float *zeta, const float *dt,
                  const float *q_init, const float *p_init, float *g_zeta,
                  float *g_dt, float *g_k, float *objective);

/*
 * Hamiltonian of the spring system, evaluated in FP64 for drift monitoring:
 *   H_r = sum_i p_ri^2/(2m) + k/2 sum_i (q_ri - q0)^2
 *         + zeta * ( -1/2 q_r^T J q_r - h^T q_r )
 * (kinetic energy and spring potential of Eqs. 2-3, coupling potential of
 * Eq. 4 whose force is zeta (J q + h); the field term follows Eq. 1).  J and
 * h are the context's working copies, so for SI_PREC_J_BF16_Q_BF16 J is the
 * bf16-rounded matrix the kernels integrate.
 *   q, p   [R][n] float, host or device (e.g. si_run's q_out, p_out)
 *   zeta   the coupling coefficient of the stretch being monitored
 *   H_out  [R] double, host or device
 * Every product and sum is FP64 in a fixed order (deterministic).  R may
 * differ from the context's replica count; R = 0 does nothing (the pointers
 * may then be NULL).  Returns SI_ERR_INVALID_ARG for R < 0, or for NULL q, p
 * or H_out when R > 0.
 */
si_status si_hamiltonian(si_ctx *ctx, const float *q, const float *p, int32_t R,
                         double zeta, double *H_out);

/*
 * Kernel timing.  With timing enabled, si_run records CUDA events on the
 * context's stream immediately before and after the launch(es) of the
 * time-step kernel (the coupling force fused with the integrator) and
 * si_last_kernel_time returns their elapsed time in milliseconds.  Off by
 * default; the events cost two records per si_run.  si_last_kernel_time
 * waits for the run; if that run ended on a device error (a timed-out wait)
 * it returns that error, as si_synchronize would, instead of a time.
 */
si_status si_enable_timing(si_ctx *ctx, int32_t on);
si_status si_last_kernel_time(const si_ctx *ctx, float *ms);

/*
 * Wait until all work enqueued by this context has finished and report a
 * pending device-side error of it (SI_ERR_TIMEOUT for a wait that ran out;
 * the run's state is then dropped), else SI_OK.
 */
si_status si_synchronize(si_ctx *ctx);

/*
 * Allocation-free single-replica run.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (a
 * plugin whose host application owns every device allocation, a real-time
 * loop that must not enter the allocator, code running while a memory pool
 * is captured or exhausted).  It runs prm->steps steps of the FP32 plain
 * path for ONE replica (prm->replicas must be 1, prm->prec SI_PREC_FP32)
 * and calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (two position vectors, a step counter, an error word) is a fixed device
 * array of 256 + 8 * SI_NOALLOC_MAX_N bytes inside the library, which every
 * GPU that loads the library holds until the process exits.
 *   J          device, n*n floats, row-major, symmetric with zero diagonal
 *              (not re-checked here)
 *   h          device, n floats, or NULL
 *   zeta, dt   device, [steps]
 *   q, p       device, [n], initial state in, final state out
 *   spins_out  device, [n] int8 sign(q) after the last step, or NULL
 *   stream     cudaStream_t as void*
 * n > SI_NOALLOC_MAX_N is rejected with SI_ERR_INVALID_ARG.  On
 * SI_ERR_TIMEOUT (an inter-CTA step wait ran out) q still holds its input
 * positions, but p, which the kernel updates in place, is unspecified.  The first call
 * on a device looks up the scratch array's device address (once per device),
 * so make that first call before any stream capture.  All calls share the
 * one scratch array and it keeps the last call's contents (the call clears
 * what must start at zero), so calls whose work overlaps on the GPU race:
 * serialise them, e.g. on one stream.  The call synchronises the stream
 * before it returns (it reads the device error word).
 */
#define SI_NOALLOC_MAX_N 16384
si_status si_run_noalloc(const si_params *prm, const float *J, const float *h,
                         const float *zeta, const float *dt, float *q, float *p,
                         int8_t *spins_out, void *stream);

/*
 * Grouped batch of independent instances of uneven size (many "parallel
 * tests" of Fig. 3 at once, each its own J).  All members share steps and the
 * integrator parameters (k, m, q0, q_max, p_max, update_order, wall_zero_p)
 * and use a tensor-core precision (SI_PREC_J_FP8_Q_BF16 or
 * SI_PREC_J_BF16_Q_BF16); n and replicas may differ.  Each time step is one
 * grouped launch over all members' tiles (replayed from a CUDA graph); the
 * tile width per member is chosen by an autotuner on the first run and
 * cached by group shape.
 *   prm[count], J[count] (n_i*n_i floats, host or device), h NULL or
 *   h[count] with NULL entries allowed.
 */
typedef struct si_group si_group;
si_status si_create_group(si_group **out, int32_t count, const si_params *prm,
                          const float *const *J, const float *const *h,
                          void *stream);
/*
 * Run steps time steps for every member.  zeta, dt [steps]; q_init[i] and
 * optional p_init[i], q_out[i], p_out[i], spins_out[i] are [R_i][n_i] (host
 * or device); any of the output arrays, or p_init, may be NULL.
 */
si_status si_run_group(si_group *g, const float *zeta, const float *dt,
                       const float *const *q_init, const float *const *p_init,
                       float *const *q_out, float *const *p_out,
                       int8_t *const *spins_out);
/* si_energy for member `index` of the group. */
si_status si_group_energy(si_group *g, int32_t index, const int8_t *spins,
                          int32_t R, int32_t *energy_out, int32_t *cut_out,
                          double *energy_f);
si_status si_group_enable_timing(si_group *g, int32_t on);
si_status si_group_last_kernel_time(const si_group *g, float *ms);
si_status si_group_describe(const si_group *g, char *buf, int32_t len);
int32_t si_group_last_launch_count(const si_group *g);
void si_destroy_group(si_group *g);

/* Short description of the kernel path and tile shape the context uses. */
si_status si_describe(const si_ctx *ctx, char *buf, int32_t len);

/* Number of kernel launches the last si_run / si_energy / si_grad made. */
int32_t si_last_launch_count(const si_ctx *ctx);

/* Message for the last failing call on this thread ("" if none). */
const char *si_last_error(void);

/* Release everything the context owns.  NULL is ignored. */
void si_destroy(si_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPRING_ISING_H */
