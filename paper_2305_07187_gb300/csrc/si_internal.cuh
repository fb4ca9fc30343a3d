// Internal declarations shared by the translation units of libspring_ising.
// Nothing here is part of the public ABI (include/spring_ising.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

#include "spring_ising.h"
#include <nvtx3/nvToolsExt.h>

namespace si {

// ------------------------------------------------------------ error plumbing
void set_error(const std::string &msg);

#define SI_CUDA_TRY(expr)                                                      \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess) {                                               \
            ::si::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); \
            return _e == cudaErrorMemoryAllocation ? SI_ERR_OOM : SI_ERR_CUDA; \
        }                                                                      \
    } while (0)

// Every device allocation of the library goes through si_dev_malloc.  With
// SI_DEBUG_FAIL_ALLOC=k in the environment the k-th allocation after the
// last si_create / si_create_group entry fails with
// cudaErrorMemoryAllocation (fault injection for the error paths; host-side
// only, nothing reaches the GPU).
cudaError_t dev_malloc_raw(void **p, size_t bytes);
void alloc_fault_reset();
template <typename P>
inline cudaError_t si_dev_malloc(P **p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

// Device error word values (written by kernels, read by the host).
enum : int {
    DEV_OK = 0,
    DEV_TIMEOUT_BARRIER = 1,   // inter-CTA step barrier ran out of time
    DEV_TIMEOUT_MBAR = 2,      // an mbarrier wait ran out of time
    DEV_BAD_CONFIG = 3         // launch shape the kernel cannot serve
};

// Integrator parameters, identical for every kernel family.
struct StepParams {
    float k, m, q0, q_max, p_max;
    int order;          // 0 kick-drift (Eq. 8), 1 literal Eq. 5
    int wall_zero_p;
};

enum class Path { PLAIN_PERSISTENT, SIMT_TILED, TENSOR };
struct AdjTc;
struct Group;

struct Ctx {
    si_params prm;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int n = 0, R = 0;
    Path path = Path::SIMT_TILED;
    bool integer_j = false;      // every J_ij integer in [-127, 127]
    bool integer_h = true;       // h NULL or integer in [-127, 127]
    bool bf16_j = false;         // every J_ij exact in bf16
    bool has_h = false;
    long long s_upper = 0;       // sum_{i<j} J_ij (integer J only)
    long long spin_limit_ns = 2000000000LL;
    // Failure-detection test hook: at this step the inter-CTA wait targets a
    // count that no CTA will ever reach, so the bounded wait must run out and
    // the call must return SI_ERR_TIMEOUT (-1: off).  Set from
    // SI_DEBUG_STALL_STEP at creation.
    int stall_step = -1;
    int stall_rank = -1;       // CTA pairs: only the CTAs of this pair rank stall (-1: all)

    // Storage of J.  FP32/FP64 paths: [n][ldj] in the state precision.
    // Tensor path: [mpad][ldk], zero padded, bf16 or (j_e4m3) e4m3 bytes.
    int ldj = 0;                 // row stride (elements) of the SIMT J copy
    int ldk = 0, mpad = 0;       // tensor path padding
    void *dJ = nullptr;          // J in working precision
    int8_t *dJ8 = nullptr;       // int8 copy for the exact energy
    int ld8 = 0;                 // row stride of dJ8 (multiple of 16)
    void *dh = nullptr;          // h in state precision (float or double)
    float *dhf = nullptr;        // h in FP32 (energy readout)
    int8_t *dh8 = nullptr;       // integer h for the exact energy

    // State and operand buffers.
    void *dq = nullptr, *dp = nullptr;   // [R][n] state precision
    void *dqbuf = nullptr;               // q exchange / operand double buffer
    size_t qbuf_bytes = 0;
    // FP32 plain path: q exchanged between CTAs as (value bits, step tag)
    // words, [2][R][ldj] x 8 bytes
    unsigned long long *dxch = nullptr;
    size_t xch_bytes = 0;
    // FP32 tiled path (R > 4): spin-major q (two planes) and p during a run,
    // [3][ldj][round_up(R, 128)]
    float *dqT = nullptr;
    float *dzeta = nullptr, *ddt = nullptr;  // schedules [steps]
    unsigned *dbar = nullptr;            // inter-CTA barrier counters
    int nbar = 0;
    int *derr = nullptr;                 // device error word
    int *herr = nullptr;                 // pinned host copy of it (the read at the end of a call is a DMA)
    int8_t *dspins = nullptr;            // [R][ld8]
    int8_t *dspins_in = nullptr;         // staging for si_energy
    int spins_in_cap = 0;                // replicas the staging holds
    int32_t *dE = nullptr, *dC = nullptr;
    double *dEf = nullptr;
    int e_cap = 0;
    float *dstage = nullptr;             // host-input staging [R][n] x 2
    int launches = 0;
    int cur_parity = 0;                  // q exchange buffer holding q(t_T)
    bool have_run = false;               // a run completed since creation
    bool run_spins_valid = false;        // dspins holds the sign readout of the last si_run
    bool timing = false;                 // record events around the step kernel
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ev_valid = false;

    // Tensor path configuration.
    int tile_n = 0;                      // replicas per CTA
    bool j_e4m3 = false;                 // dJ holds e4m3 bytes [mpad][ldk] (else bf16)
    bool tc_pair = false;                // k_tc_run on CTA pairs (cta_group::2, M = 256)
    int tc_plane = -1;                   // operand plane holding bf16 q of the state (-1: not current)
    int tc_p0 = 0;                       // operand plane the next k_tc_run starts from
    bool tc_readout = false;             // the launch also sums sigma^T J sigma of its final spins
    bool fused_valid = false;            // e_sum holds those sums for the last run's spins
    // watched run (si_run_watch): readout interval (0: none) and target energy
    int tc_watch_every = 0;
    long long tc_watch_target = 0;
    int tc_per_sm[2] = {0, 0};           // co-resident CTAs per SM of the step kernel without / with
                                         // readout passes (0: not yet queried)
    int stages = 0;
    int rpad = 0;                        // R rounded up to tile_n
    CUtensorMap mapA, mapB;              // J tiles, q operand tiles
    // Tensor contexts whose persistent grid would not be co-resident run on
    // the grouped per-step kernel as a one-member group that owns J and the
    // state (dJ, dq, dp alias its buffers).
    Group *grp = nullptr;

    // Tensor-core energy readout workspace (allocated lazily).
    void *e_sig = nullptr;               // bf16 spin operand
    size_t e_sig_bytes = 0;
    unsigned long long *e_sum = nullptr; // per-replica sigma^T J sigma
    int e_sum_cap = 0;
    // watched run: per-readout sums [nread][R], evaluation counters
    // [nread][rblocks], then the finished evaluations and the first readout
    // that reached the target
    unsigned long long *w_sum = nullptr;
    size_t w_sum_cap = 0;
    unsigned *w_ctl = nullptr;
    size_t w_ctl_cap = 0;

    // Gradient workspace (allocated lazily by si_grad).
    void *g_ws = nullptr;
    size_t g_ws_bytes = 0;
    // Tensor-core adjoint products (FP32 contexts with bf16-exact J),
    // created by the first si_grad, owned by the context.
    AdjTc *g_tc = nullptr;
    cudaGraphExec_t g_graph = nullptr;   // captured adjoint sweep
    int g_graph_key = -1;
    void *g_graph_ws = nullptr;
    int g_graph_launches = 0;
    int g_path = 0;              // 0: no si_grad yet, 1: CUDA cores, 2: tensor cores
};

// NVTX range over one public call (header-only NVTX 3: free unless a
// profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------ helpers
bool is_device_ptr(const void *p);
inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
inline int round_up(int a, int b) { return cdiv(a, b) * b; }

// FP64 Hamiltonian for drift monitoring, si_monitor.cu (device pointers).
si_status monitor_hamiltonian(Ctx *c, const float *q, const float *p, int R, double zeta, double *H);

// SIMT (FP32 / FP64) paths, si_simt.cu.
si_status simt_run(Ctx *c, int steps, int8_t *spins_dev);
si_status simt_energy(Ctx *c, const int8_t *spins_dev, int R, int ld,
                      int32_t *E, int32_t *C, double *Ef);
si_status simt_convert_j(Ctx *c, const float *J_dev, int n);
si_status simt_validate(const float *J_dev, const float *h_dev, int n,
                        int prec, unsigned long long *flags_host,
                        long long *s_upper, cudaStream_t st);
// Writes sign(q) for R replicas of the state into spins [R][ld].
si_status simt_spins(Ctx *c, int8_t *spins, int ld);
si_status simt_init_state(Ctx *c, const float *q_init, const float *p_init);
// Start the next run from the state the last one left (exchange buffer of
// parity cur_parity, p in place).
si_status simt_continue_state(Ctx *c);
// int8 copy of J for the exact energy.
si_status convert_j8(Ctx *c, const float *J_dev);
// int8 copy of an integer-valued field.
si_status h_to_int8(const float *h_dev, int n, int8_t *out, cudaStream_t st);
// Copies the state of the current run into q_out / p_out (device, [R][n]).
si_status simt_copy_state(Ctx *c, float *q_out, float *p_out);
si_status simt_copy_state_f64(Ctx *c, double *q_out, double *p_out);

// Tensor-core path, si_tc.cu.
// True when the persistent all-steps kernel can serve the context (its grid
// of M tiles x replica blocks is co-resident and within the step flags).
bool tc_persistent_fits(Ctx *c);
si_status tc_prepare(Ctx *c, const float *J_dev);
si_status tc_run(Ctx *c, int steps, int8_t *spins_dev);
si_status tc_copy_state(Ctx *c, float *q_out, float *p_out);
si_status tc_copy_state_f64(Ctx *c, double *q_out, double *p_out);
si_status tc_init_state(Ctx *c, const float *q_init, const float *p_init);
// Start the next run from the FP32 state in place: rebuild the bf16 operand
// plane of step 0 from it.
si_status tc_continue_state(Ctx *c);
si_status tc_spins(Ctx *c, int8_t *spins, int ld);
// Exact energy/cut on the tensor cores (integer J, tensor-path contexts);
// SI_ERR_UNSUPPORTED when it does not apply.
// E and cut from per-replica totals s_r = sigma^T J sigma (64-bit), with the
// integer field term, one CTA of 128 threads per replica.
__global__ void k_energy_finish(const unsigned long long *sum, const int8_t *h8, const int8_t *s, int lds, int n,
                                int R, long long s_upper, int32_t *E, int32_t *C);
si_status tc_energy(Ctx *c, const int8_t *spins_dev, int R, int ld, int32_t *E, int32_t *C);
// The per-replica sums the step kernel's readout pass left in c->e_sum: E and
// the cut of the last run's spins (c->dspins).
si_status tc_energy_finish(Ctx *c, int R, int32_t *E, int32_t *C);
// c->e_sum with room for the context's replicas.
si_status tc_readout_buffer(Ctx *c);
// Whether a run of this context can sum its final energies in the step kernel.
bool tc_readout_supported(const Ctx *c);
// Buffers of a watched run of `steps` steps with a readout every `every`.
si_status tc_watch_buffers(Ctx *c, int steps, int every);
// Energies (Eq. 1) of the stopping readout of the last watched run (of
// nread) into E [R] (device); the kernel reads the stop itself.
si_status tc_watch_energy(Ctx *c, int nread, int32_t *E);
const char *tc_describe(const Ctx *c, char *buf, int len);
// 2D tensor map of e4m3 (1-byte) tiles of 64 x box_outer with the 64-byte swizzle.
si_status tc_make_map_e4m3(CUtensorMap *m, void *base, int inner, int outer, int box_outer);
// J (fp32 n x n, e4m3-exact) -> e4m3 [mpad][ldk], zero padded.
si_status tc_convert_j_e4m3(const float *J_dev, int n, void *out, int ldk, int mpad, int sms, cudaStream_t st);
// 2D bf16 tensor map with the 128-byte swizzle (inner dimension contiguous).
si_status tc_make_map_bf16(CUtensorMap *m, void *base, int inner, int outer, int box_inner,
                           int box_outer);
// J (fp32 n x n) -> bf16 [mpad][ldk], zero padded.
si_status tc_convert_j(const float *J_dev, int n, void *out, int ldk, int mpad, int sms,
                       cudaStream_t st);

// One-member grouped service of a tensor context, si_group.cu.
si_status group_ctx_create(Ctx *c, const float *J_dev, const float *h_dev);
si_status group_ctx_prepare(Ctx *c, int steps);
si_status group_ctx_run(Ctx *c, int steps);
void group_ctx_params(Ctx *c);
void group_ctx_describe(const Ctx *c, char *buf, int len);
void group_ctx_free(Ctx *c);

// Adjoint, si_adjoint.cu.
// Tensor-core products of the adjoint sweep, si_adjoint_tc.cu.
si_status adj_tc_prepare(Ctx *c, AdjTc **out);
// Operand layout of the tensor-core adjoint: replica blocks of 64, each as
// three bf16 pieces (rows [rb][piece][64][ldk]).
constexpr int ADJ_TC_RB = 64, ADJ_TC_BN = 3 * ADJ_TC_RB;
// Product J X^T of the sweep: X's pieces are read from operand buffer xin
// (split from X first when `split`); a forward product writes the pieces of
// q_{t+1} into buffer xout (>= 0).
si_status adj_tc_gemm(Ctx *c, AdjTc *a, int mode, const float *X, const float *P, float *Qn, float *Pn,
                      float *Fo, const float *LB, float *LQ, float *LP, float *obj_part, int t, int xin,
                      bool split, int xout);
__nv_bfloat16 *adj_tc_xs(const AdjTc *a, int buf);
int adj_tc_ldk(const AdjTc *a);
int adj_tc_nobj(const AdjTc *a);
int adj_tc_splits(const AdjTc *a);
void adj_tc_free(AdjTc *a);

// Persistent sweep (k_adj_run): one launch runs one or two chains of
// products, each over every (M tile, replica block, K split) CTA.
struct AdjChain {
    int reverse;                 // 0: forward products, 1: reverse steps of one segment
    int t_start, len;            // forward: steps t_start .. t_start+len-1; reverse: t_start+len-1 down to t_start
    int buf0;                    // first of the chain's two operand buffers
    unsigned *flags;             // [mtiles * nrb] slices published (zeroed by adj_tc_run)
    const float *q_in, *p_in;    // forward: state at t_start, [R][ld]
    float *sq[2], *sp[2], *sF[2];   // slot sets (segment parity): q, p [K+1] planes, F [K] planes
    float *ckq, *ckp;            // forward: checkpoint planes written at segment ends, or null
    float *lq, *lp;              // reverse: adjoint state at t_start+len on entry, at t_start on exit
    float *part;                 // reverse: gradient partials [T][3][nparts]
};
// Cluster size of the persistent sweep (0: not available for this context,
// the per-step kernels run instead), whether two chains run side by side,
// the number of gradient partials per step, and a chain's step counters.
int adj_tc_run_splits(const AdjTc *a);
bool adj_tc_run_pair(const AdjTc *a);
int adj_tc_run_nparts(const AdjTc *a);
unsigned *adj_tc_run_flags(const AdjTc *a, int chain);
si_status adj_tc_run(Ctx *c, AdjTc *a, const AdjChain *chains, int nch, int K);

si_status adjoint_grad(Ctx *c, int steps, float *g_zeta, float *g_dt,
                       float *g_k, float *objective, const float *q_init,
                       const float *p_init);

// Validation flags (bit set = property violated / present).
enum : unsigned long long {
    VF_ASYM = 1ull << 0,
    VF_DIAG = 1ull << 1,
    VF_NONFINITE = 1ull << 2,
    VF_NOT_INT8 = 1ull << 3,
    VF_NOT_E4M3 = 1ull << 4,
    VF_H_NOT_INT8 = 1ull << 5,
    VF_H_NONFINITE = 1ull << 6,
    VF_NOT_BF16 = 1ull << 7
};

}  // namespace si
