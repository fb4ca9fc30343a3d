// Tensor-core path of the Spring-Ising hot path (sm_103a, tcgen05 + TMA).
//
// One persistent launch runs all T steps.  CTA (mt, rb) owns the output tile
// F[mt*128 .. +128][rb*BN .. +BN] of F = J Q^T (rows = spins, columns =
// replicas) for the whole run:
//   warp 0      TMA producers in lanes 0 and 1: J tile (128 x 64 bf16) and q
//               tile (BN x 64 bf16) per K block into the two halves of an
//               S-stage shared-memory ring (128B swizzle), lane 0 the even
//               and lane 1 the odd positions of the K loop
//   warps 1, 2  issue tcgen05.mma (M=128, N=BN, K=16) for alternating K
//               blocks into two FP32 accumulators in TMEM (warp 1 also
//               allocates TMEM)
//   warps 3..10 epilogue: tcgen05.ld of the accumulators, the spring
//               integrator of Eq. 8 with the walls of Eq. 6 on the q, p state
//               that lives in TMEM next to the accumulators, and the bf16
//               copy of the new q (the next step's MMA operand), stored by
//               the epilogue threads straight into the operand plane
// CTAs of one replica block exchange q through the double-buffered operand
// array in L2.  There is no step barrier: each CTA publishes a per-CTA step
// counter after writing its rows of q, and a consumer waits only for the
// owner of the K block it is about to load (dataflow), starting its K loop at
// its own rows.  CTAs of different replica blocks never wait on each other.
// Every wait (mbarrier or counter) has a time limit; on expiry the kernel
// raises the device error word, drains its own copies and MMAs, frees TMEM
// and returns.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cstdlib>

#include "si_tcgen05.cuh"

namespace si {

constexpr int TC_BM = 128;       // spins per CTA (MMA M)
constexpr int TC_BK = 64;        // K elements per stage (128 bytes of bf16)
// Threads: producer warp, 2 MMA-issuing warps, EPI epilogue warps (4 or 8),
// with e4m3 J storage four converter warps, and the warp that mirrors the
// owners' step flags into shared memory.
template <int EPI, bool E4>
constexpr int tc_threads() { return 32 * (4 + EPI + (E4 ? 4 : 0)); }
template <int EPI, bool E4>
constexpr int tc_poll_warp() { return 3 + EPI + (E4 ? 4 : 0); }
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;

struct TcArgs {
    int n, R, steps;
    int mtiles, rblocks, kblocks;
    int ldk, rpad;
    const float *zeta, *dt, *h;
    float *q_state, *p_state;    // [R][n], initial in / final out
    __nv_bfloat16 *qop;          // [3][rpad][ldk]: bf16 q of step t in plane (t + p0) & 1, sign(q(T)) in plane 2
    int8_t *spins;               // [R][lds] or null
    int lds;
    unsigned *bar;               // [rblocks * mtiles] published-step flags
    int *err;
    long long limit_ns;
    StepParams sp;
    int stall_step;              // failure-detection test hook (-1: off)
    int stall_rank;              // CTA pairs: only this pair rank stalls (-1: every CTA)
    int smem_bytes;              // dynamic shared memory the launch provides
    int p0;                      // operand plane holding q(0)
    // Readout passes: after every `every` steps and after the last one, one
    // more pass over J with sign(q) as the operand sums sigma^T J sigma per
    // replica (0: no readout; `steps`: only the final one).
    int every;
    unsigned long long *e_sum;   // [number of readouts][R], zeroed by the caller
    // Watch: readout k of replica block rb is evaluated by the last of its
    // M-tile CTAs to add its part (w_cnt); the run stops after the first
    // readout at which some replica's energy is at most `target` (w_hit:
    // first such readout, atomic minimum; w_done: evaluations finished, all
    // replica blocks of readout k once it reaches rblocks (k + 1)).  The
    // readout then adds 2 h_i sigma_i per spin (integer h8), so that the
    // energy of Eq. 1 is minus half the sum.
    int watch;
    long long target;
    unsigned *w_cnt;             // [number of readouts][rblocks]
    unsigned *w_done;
    int *w_hit;
    const int8_t *h8;            // integer h, or null
};

// Pass schedule of one launch: step t of the iteration, or a readout pass
// (after every `every` steps and after the last).  Passes are what the
// step flags count.
struct TcPasses {
    int E, nread, npass;
    __device__ __forceinline__ TcPasses(int steps, int every)
        : E(every), nread(every > 0 ? (steps + every - 1) / every : 0), npass(steps + nread) {}
    __device__ __forceinline__ bool readout(int p) const {
        return E > 0 && ((p + 1) % (E + 1) == 0 || p == npass - 1);
    }
    __device__ __forceinline__ int step(int p) const { return E > 0 ? p - p / (E + 1) : p; }
    __device__ __forceinline__ int index(int p) const { return p / (E + 1); }   // readout number of pass p
    // the first readout pass at or after pass p (npass if there is none)
    __device__ __forceinline__ int next_readout(int p) const {
        if (E <= 0) return npass;
        const int r = p + (E - p % (E + 1));
        return r < npass - 1 ? r : npass - 1;
    }
};

// Walk over the passes in order without a division per pass: the step of
// the current pass, the next readout pass, and the latest readout passed.
struct TcWalk {
    int st = 0, next_ro, k = 0, last_ro = -3, last_k = -1;
    __device__ __forceinline__ explicit TcWalk(const TcPasses &P) : next_ro(P.next_readout(0)) {}
    __device__ __forceinline__ bool readout(int t) const { return t == next_ro; }
    __device__ __forceinline__ void advance(const TcPasses &P, int t) {   // after pass t
        if (t == next_ro) {
            last_ro = t;
            last_k = k++;
            next_ro = P.next_readout(t + 1);
        } else {
            ++st;
        }
    }
};

// ------------------------------------------------------------------ kernel
// Shared memory: S ring stages (J tile + q tile), then the mbarriers and the
// mirrored step flags.
//
// With e4m3 J storage (E4) a stage holds the J tile as 8 KB of e4m3 (64-byte
// swizzle) and four converter warps widen it into tensor memory, where the
// MMAs read their A operand: the J tile then costs 8 KB of TMA traffic and
// 8 KB of shared-memory reads instead of 16 + 16 KB.  Tensor memory holds
// the two accumulators, q and NA A slots, so the momenta p move to shared
// memory ([replica][spin] within the tile).
template <int BN, int S, bool E4, bool CG2 = false>
struct TcSmem {
    static constexpr int B_BYTES = (CG2 ? BN / 2 : BN) * TC_BK * 2;   // a CTA pair holds half of q each
    static constexpr int A_STAGE = E4 ? TC_BM * TC_BK : TC_A_BYTES;   // J tile in its storage type
    static constexpr int STAGE_BYTES = A_STAGE + B_BYTES;
    static constexpr int TX_BYTES = STAGE_BYTES;          // bytes TMA delivers per stage
    static constexpr int TILES = S * STAGE_BYTES;
    static constexpr int PTILE = TILES;                   // p of the tile (E4), [BN][128] floats
    static constexpr int BARS = PTILE + (E4 ? BN * TC_BM * 4 : 0);
    static constexpr int NA = E4 ? 4 : 0;                 // A slots in tensor memory (two per MMA warp)
    // full[S], empty[S], accf, tmem_empty, epi_done, drain, afull[NA], aempty[NA]
    static constexpr int NBARS = 2 * S + 4 + 2 * NA;
    static constexpr int SEEN = BARS + NBARS * 8 + 16;     // after the tmem slot and abort flag
    static constexpr int CNT = SEEN + 68 * 4;              // mirrored step flags of up to 64 owners, their minimum
    static constexpr int TOTAL = CNT + 4 * 4;              // pair: stages issued per ring by each CTA
    static constexpr int TMEM_COLS = (E4 || 4 * BN > 256) ? 512 : 256;
};

constexpr int TC_MMA_WARPS = 2;
constexpr int TC_EPI_WARP0 = 1 + TC_MMA_WARPS;             // first epilogue warp

// EPI: epilogue warps (8 in both tile instantiations; a CTA that allocates
// tensor memory occupies its SM alone, so a lighter CTA buys no second CTA).
//
// CG2: CTA pairs.  The two CTAs of a cluster (consecutive M tiles of one
// replica block) share each MMA of M = 256 (tcgen05 cta_group::2): each loads
// its own 128 rows of J and half of the q tile (BN/2 replicas), so a K block
// costs a CTA 24 KB of TMA traffic instead of 32 KB.  The even CTA issues the
// MMAs.  The copies of both CTAs complete on the even CTA's full barrier
// (TMA cta_group::2), which the even CTA's producer arms for the bytes of
// both; the odd CTA's producer only waits for its stage to be free.  The MMA
// completions are multicast to the empty and accumulator barriers of both
// CTAs; the odd CTA's epilogue frees the accumulators on the even CTA's
// barrier.  At the end each producer leaves the number of stages it issued
// in the even CTA's shared memory; after a cluster barrier (no copy is
// issued after it) the even CTA settles every stage that only one CTA filled
// (it arms the ones the odd CTA filled alone and counts the bytes that were
// never sent) and waits until every copy of both CTAs has landed.  Both
// CTAs then meet at a second cluster barrier before TMEM is freed, so that
// neither leaves while a copy or an arrival may still reach its shared
// memory.
// Epilogue of a readout pass (one warp): the accumulators hold G = J sigma
// (integers below 2^24, exact in FP32).  sigma_i (G_ir + h2) per element,
// h2 = 2 h_i on a watched run (else 0), is added over the warp's 32 rows by
// a transposing shuffle reduction (lane j ends with column j), and each warp
// adds its column sums to the readout's per-replica totals `es` in 64-bit
// integers.  Unless this is the final pass, the pass is published, and on a
// watched run the last M-tile CTA of the replica block to add its part
// evaluates the readout (any replica at or below the target: atomic minimum
// of the readout index into w_hit, then one release increment of w_done).
// The grid's decision is waited for later, before the next step's update.
// Returns 0 to go on with the next pass, 2 after the final pass.
template <int BN, int CPH, bool CG2>
__device__ __forceinline__ int tc_readout_epi(uint32_t tl, int c_begin, bool two_acc, bool row_ok, int h2,
                                           unsigned long long *es, int r0, int R, int lane, bool pub_warp,
                                           bool final_pass, uint32_t tmem_empty_bar, uint32_t epi_done_bar,
                                           bool remote_tmem_empty, int t, unsigned *flag, int watch, unsigned *w_cnt,
                                           unsigned last_cta, long long target, unsigned *w_done, int *w_hit,
                                           int k, int *err, volatile int *abort_flag, long long limit_ns) {
    constexpr uint32_t COL_ACC0 = 0, COL_ACC1 = BN, COL_Q = 2 * BN;
#pragma unroll 1
    for (int c = c_begin; c < c_begin + CPH; ++c) {
        // two 32-register arrays at a time (G in place, then q into the other)
        uint32_t vf[32], vg[32];
        tmem_ld32(tl + COL_ACC0 + c * 32, vf);
        if (two_acc) {
            tmem_ld32(tl + COL_ACC1 + c * 32, vg);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) vf[j] = __float_as_uint(__uint_as_float(vf[j]) + __uint_as_float(vg[j]));
        }
        tmem_ld32(tl + COL_Q + c * 32, vg);
        tmem_wait_ld();
        int v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            v[j] = row_ok ? ((int)__uint_as_float(vf[j]) + h2) * (int)spin_of(__uint_as_float(vg[j])) : 0;
        column_sums32(v, lane);
        const int r = r0 + c * 32 + lane;
        if (r < R && v[0] != 0) atomicAdd(es + r, (unsigned long long)(long long)v[0]);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
        if (!final_pass) {
            if (remote_tmem_empty) mbar_arrive_remote(mapa_shared(tmem_empty_bar, 0u));
            else mbar_arrive(tmem_empty_bar);
        }
        mbar_arrive(epi_done_bar);
    }
    if (final_pass) return 2;
    if (pub_warp) {
        bool lastc = false;
        if (lane == 0) {
            if (mbar_wait(epi_done_bar, (uint32_t)(t & 1), err, abort_flag, limit_ns)) {
                red_release_gpu_add(flag, 1u);
                if (watch) lastc = atom_add_acq_rel_gpu(w_cnt, 1u) == last_cta;
            }
        }
        lastc = __shfl_sync(0xffffffffu, lastc ? 1 : 0, 0) != 0;
        if (lastc) {
            // every CTA's additions are ordered before this acquire
            (void)ld_acquire_gpu(w_cnt);
            bool hit = false;
#pragma unroll
            for (int j = 0; j < BN / 32; ++j) {
                const int r = r0 + j * 32 + lane;
                if (r < R) {
                    const long long sum = (long long)ld_relaxed_gpu_u64(es + r);
                    hit = hit || (-(sum / 2) <= target);
                }
            }
            hit = __any_sync(0xffffffffu, hit);
            if (lane == 0) {
                if (hit) atomicMin(w_hit, k);
                red_release_gpu_add(w_done, 1u);
            }
        }
    }
    return 0;
}

// The state in tensor memory as the run's final state (a watched run that
// stops after a readout: the state of the readout's step), one warp's rows
// (E4: p from the shared-memory tile).  Every lane takes part in the
// tensor-memory loads (.sync.aligned); only the stores depend on the row.
template <int BN, bool E4>
__device__ __forceinline__ void tc_write_state(uint32_t tl, int c_begin, int cph, bool row_ok, int r0, int R, int n,
                                            int i, int row, float *q_state, float *p_state, int8_t *spins, int lds,
                                            const float *p_tile) {
    constexpr uint32_t COL_Q = 2 * BN, COL_P = 3 * BN;
#pragma unroll 1
    for (int c = c_begin; c < c_begin + cph; ++c) {
        uint32_t vq[32], vp[32];
        tmem_ld32(tl + COL_Q + c * 32, vq);
        if constexpr (!E4) tmem_ld32(tl + COL_P + c * 32, vp);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int r = r0 + c * 32 + j;
            if (row_ok && r < R) {
                const float qv = __uint_as_float(vq[j]);
                q_state[(size_t)r * n + i] = qv;
                if constexpr (E4) p_state[(size_t)r * n + i] = p_tile[(c * 32 + j) * TC_BM + row];
                else p_state[(size_t)r * n + i] = __uint_as_float(vp[j]);
                if (spins) spins[(size_t)r * lds + i] = spin_of(qv);
            }
        }
    }
}

// RO: the launch may have readout passes (a fused final readout or a
// watched run).  The steps' loop of the instantiation without them carries
// no readout code, which its register allocation and schedule would pay
// for (about 5 % per step).
template <int BN, int S, int EPI, bool E4, bool CG2 = false, bool RO = false>
__global__ void __launch_bounds__(tc_threads<EPI, E4>(), 1)
    k_tc_run(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
             TcArgs a) {
    static_assert(!(E4 && CG2), "CTA pairs take the bf16 J operand");
    using L = TcSmem<BN, S, E4, CG2>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    // The 128-byte swizzled tiles need a 1024-aligned base; the launch provides
    // only a little slack, so check that the aligned layout fits before
    // touching any barrier or TMEM (uniform for the whole CTA).
    if ((int)(smem - smem_raw) + L::TOTAL > a.smem_bytes) {
        if (threadIdx.x == 0) atomicCAS(a.err, 0, DEV_BAD_CONFIG);
        return;
    }
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + L::BARS;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    const uint32_t accf_bar = bar0 + 8u * (2 * S);
    const uint32_t tmem_empty_bar = bar0 + 8u * (2 * S + 1);
    const uint32_t epi_done_bar = bar0 + 8u * (2 * S + 2);
    const uint32_t drain_bar = bar0 + 8u * (2 * S + 3);
    auto afull_bar = [&](int k) { return bar0 + 8u * (2 * S + 4 + k); };
    auto aempty_bar = [&](int k) { return bar0 + 8u * (2 * S + 4 + L::NA + k); };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::BARS + L::NBARS * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L::BARS + L::NBARS * 8 + 4);
    const uint32_t seen = sbase + L::SEEN;   // mirrored step flags of the owners
    const TcPasses P(a.steps, a.every);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x % a.mtiles, rb = blockIdx.x / a.mtiles;
    const int m0 = mt * TC_BM, r0 = rb * BN;
    const uint32_t crank = CG2 ? cluster_ctarank() : 0u;   // rank in the CTA pair (mt & 1)
    const bool leader = crank == 0u;
    // TMEM columns: two partial accumulators, then the q and p state (E4:
    // q, then the A slots of 32 columns; p lives in shared memory).
    constexpr uint32_t COL_ACC0 = 0, COL_ACC1 = BN, COL_Q = 2 * BN, COL_P = 3 * BN, COL_A = 3 * BN;
    constexpr int NAR = L::NA / 2;   // A slots per MMA warp

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);   // pair: the even CTA's arming counts the bytes of both CTAs
            mbar_init(empty_bar(s), 1);
        }
        for (int k = 0; k < L::NA; ++k) {
            mbar_init(afull_bar(k), 4);
            mbar_init(aempty_bar(k), 1);
        }
        mbar_init(accf_bar, TC_MMA_WARPS);
        mbar_init(tmem_empty_bar, CG2 ? 2 * EPI : EPI);   // pair: both CTAs' epilogues
        mbar_init(epi_done_bar, EPI);
        mbar_init(drain_bar, TC_MMA_WARPS);
        *abort_flag = 0;
        // mirrored owners' flags and minimum: 0; decisions final: 0; first
        // readout at the target: none
        for (int o = 0; o <= MIRROR_HIT; ++o)
            reinterpret_cast<unsigned *>(smem + L::SEEN)[o] = o == MIRROR_HIT ? 0x7fffffffu : 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    if (warp == 1) {
        if constexpr (CG2) {
            // one warp of each CTA of the pair allocates, collectively
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "n"(L::TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "n"(L::TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    // pair: both CTAs' barriers are initialised before either signals the other
    if constexpr (CG2) cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producers (lanes 0 and 1)
        // Step t needs the positions q(t) of its replica block.  The K block kb
        // (spins 64kb .. 64kb+63) of q(t) is written by the CTA owning M tile
        // kb/2 at the end of its step t-1 and announced through that CTA's flag
        // (number of steps published), which the poller warp mirrors into
        // shared memory.  The K loop starts at this CTA's own rows; the copy
        // is read only when the next block's owner is not yet known to be
        // ready.  J tiles do not depend on the step and are issued before the
        // wait.
        // Stages are split into two rings, the even stages filled by lane 0
        // for the even positions of the K loop and consumed only by MMA warp
        // 1, the odd stages filled by lane 1 and consumed only by MMA warp 2,
        // so that every stage has one in-order producer and consumer and no
        // waiter can run two phases ahead of a stage's barrier.  One thread's
        // chain of barrier wait, arming and two TMA instructions per K block
        // takes about as long as the K block's MMAs; the two lanes run that
        // chain side by side (positions 2i and 2i+1, whose q blocks have the
        // same owner), so a K block costs half of it.
        constexpr int HS = S / 2;
        static_assert(S % 2 == 0, "stage count must be even");
        if (lane < 2) {
            const int ring = lane;
            uint32_t cnt = 0u;   // stages armed in this ring
            bool ok = true;
            // pair: both CTAs walk the K blocks in the same order (the pair's rows first)
            const int kb0 = (CG2 ? (mt & ~1) : mt) * (TC_BM / TC_BK);
            TcWalk W(P);
            for (int t = 0; t < P.npass && ok; W.advance(P, t), ++t) {
                // Watch: the grid's decision after readout pass t - 2 (one for
                // the grid).  The pass right after a readout is loaded and
                // multiplied before the decision is known, so that waiting for
                // it overlaps that pass; its update is applied only if the run
                // goes on (the epilogue waits for the decision before it).
                if (a.watch && t == W.last_ro + 2) {
                    bool stop = false;
                    if (!wait_decision(seen, W.last_k, stop, a.err, abort_flag, a.limit_ns)) { ok = false; break; }
                    if (stop) break;
                }
                unsigned long long ready = t == 0 ? ~0ull : 0ull;   // owners known to have published pass t
                const bool stall = t == a.stall_step && (a.stall_rank < 0 || a.stall_rank == (int)crank);
                const unsigned need = (unsigned)t + (stall ? 1000000u : 0u);
                // q of step s in plane (s + p0) & 1; a readout pass reads sign(q) in plane 2
                const int yb = (W.readout(t) ? 2 : ((W.st + a.p0) & 1)) * a.rpad + r0 + (int)crank * (BN / 2);
                for (int j = ring; j < a.kblocks; j += 2) {
                    int kb = kb0 + j;
                    if (kb >= a.kblocks) kb -= a.kblocks;
                    const int s = 2 * (int)(cnt % HS) + ring;
                    const uint32_t ph = (cnt / HS) & 1u;
                    const uint32_t dA = sbase + s * L::STAGE_BYTES;
                    if (!mbar_wait(empty_bar(s), ph ^ 1u, a.err, abort_flag, a.limit_ns)) { ok = false; break; }
                    if (CG2 && !leader) {
                        tma_load_2d_pair(dA, &mapA, mapa_shared(full_bar(s), 0u), kb * TC_BK, m0);
                    } else {
                        mbar_arrive_expect_tx(full_bar(s), (uint32_t)(CG2 ? 2 * L::TX_BYTES : L::TX_BYTES));
                        tma_load_2d(dA, &mapA, full_bar(s), kb * TC_BK, m0);
                    }
                    ++cnt;
                    const int mo = kb >> 1;
                    bool have = ((ready >> mo) & 1ull) != 0ull;
                    if (!have) {
                        if (!CG2 && mo == mt && t > 0 && t != a.stall_step) {
                            // This CTA's own rows, written by its epilogue of
                            // pass t - 1: its barrier orders those stores, and
                            // the proxy fence makes them visible to the copy,
                            // without waiting for the published flag.
                            have = mbar_wait(epi_done_bar, (uint32_t)((t - 1) & 1), a.err, abort_flag, a.limit_ns);
                            if (have) fence_proxy_async_global();
                        } else {
                            have = wait_owner(seen, mo, need, ready, a.err, abort_flag, a.limit_ns);
                        }
                    }
                    // The q tile is issued even on abort so that the stage's
                    // transaction count completes and the drain below ends.
                    if (CG2 && !leader)
                        tma_load_2d_pair(dA + L::A_STAGE, &mapB, mapa_shared(full_bar(s), 0u), kb * TC_BK, yb);
                    else
                        tma_load_2d(dA + L::A_STAGE, &mapB, full_bar(s), kb * TC_BK, yb);
                    if (!have) { ok = false; break; }
                }
            }
            if constexpr (CG2) {
                // pair: the stages issued, for the even CTA's settlement at the end
                st_shared_cluster_u32(mapa_shared(sbase + L::CNT + 4u * (2u * crank + (uint32_t)ring), 0u), cnt);
                cnt = 0u;   // the even CTA waits for the copies of both CTAs
            }
            // Let every copy this thread issued land before the CTA exits.
            const uint32_t first = cnt > (uint32_t)HS ? cnt - HS : 0u;
            for (uint32_t k = first; k < cnt; ++k) {
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait(full_bar(2 * (int)(k % HS) + ring), (k / HS) & 1u)) {
                    if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                        atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                        break;
                    }
                }
            }
        }
    } else if (warp == tc_poll_warp<EPI, E4>()) {
        // ------------------------------------------------ step-flag mirror
        if (P.npass > 1)
            mirror_flags(a.bar + (size_t)rb * a.mtiles, a.mtiles, (unsigned)(P.npass - 1), seen, lane, a.err,
                         abort_flag, a.limit_ns, a.watch ? a.w_done : nullptr, a.w_hit, (unsigned)a.rblocks);
    } else if (warp <= TC_MMA_WARPS) {
        // ------------------------------------------------ MMA issuers
        // Warp 1 takes the even positions of the K loop into accumulator 0,
        // warp 2 the odd ones into accumulator 1; the epilogue adds the two.
        // Two issuing threads keep the tensor pipe fed: one thread alone
        // issues a 128x128x16 MMA no faster than the pipe executes it.
        // In the odd CTA of a pair the two warps have nothing to do.
        if (lane == 0 && !(CG2 && !leader)) {
            const int w = warp - 1;
            constexpr uint32_t idesc = idesc_bf16(CG2 ? 2 * TC_BM : TC_BM, BN);
            const uint32_t d_tmem = tmem + (w == 0 ? COL_ACC0 : COL_ACC1);
            constexpr int HS = S / 2;
            uint32_t c = 0;  // this warp's position in its ring of stages
            bool ok = true;
            // pair barriers receive arrivals from the other CTA: acquire at cluster scope
            auto wait_bar = [&](uint32_t bar, uint32_t parity) {
                return CG2 ? mbar_wait_cluster(bar, parity, a.err, abort_flag, a.limit_ns)
                           : mbar_wait(bar, parity, a.err, abort_flag, a.limit_ns);
            };
            TcWalk W(P);
            for (int t = 0; t < P.npass && ok; W.advance(P, t), ++t) {
                if (a.watch && t == W.last_ro + 2) {
                    bool stop = false;
                    if (!wait_decision(seen, W.last_k, stop, a.err, abort_flag, a.limit_ns)) break;
                    if (stop) break;
                }
                if (t > 0) {
                    if (!wait_bar(tmem_empty_bar, (uint32_t)((t - 1) & 1))) break;
                }
                tc_fence_after();
                for (int j = w; j < a.kblocks; j += TC_MMA_WARPS, ++c) {
                    const int s = 2 * (int)(c % HS) + w;
                    const uint32_t ph = (c / HS) & 1u;
                    if (!wait_bar(full_bar(s), ph)) { ok = false; break; }
                    if constexpr (E4) {
                        // A from the tensor-memory slot the converters filled
                        const int as = 2 * (int)(c % NAR) + w;
                        if (!mbar_wait(afull_bar(as), (c / NAR) & 1u, a.err, abort_flag, a.limit_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t bd = sdesc_sw128(sbase + s * L::STAGE_BYTES + L::A_STAGE);
                        const uint32_t at = tmem + COL_A + 32u * (uint32_t)as;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk)
                            mma_bf16_tmem_a(d_tmem, at + 8u * kk, bd + 2u * kk, idesc,
                                            (j != w || kk != 0) ? 1u : 0u);
                        mma_commit(empty_bar(s));
                        mma_commit(aempty_bar(as));
                    } else {
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(sbase + s * L::STAGE_BYTES);
                        const uint64_t bd = ad + (uint64_t)(TC_A_BYTES >> 4);
                        if constexpr (CG2) {
#pragma unroll
                            for (int kk = 0; kk < TC_BK / 16; ++kk)
                                mma_bf16_pair(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc,
                                              (j != w || kk != 0) ? 1u : 0u);
                            mma_commit_pair(empty_bar(s));
                        } else {
#pragma unroll
                            for (int kk = 0; kk < TC_BK / 16; ++kk)
                                mma_bf16(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc, (j != w || kk != 0) ? 1u : 0u);
                            mma_commit(empty_bar(s));
                        }
                    }
                }
                if (ok) {
                    if constexpr (CG2) mma_commit_pair(accf_bar);
                    else mma_commit(accf_bar);
                }
            }
            // Drain: wait until every MMA this thread issued has completed.
            if constexpr (CG2) mma_commit_pair_local(drain_bar);
            else mma_commit(drain_bar);
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(drain_bar, 0u)) {
                if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                    atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                    break;
                }
            }
        }
    } else if (warp < TC_EPI_WARP0 + EPI) {
        // ------------------------------------------------ epilogue (8 warps)
        // Warp w reads TMEM lanes 32*(w%4) .. +31 (one spin per thread) and
        // half (w-3)/4 of the replica columns.
        const int quad = warp & 3;
        const int half = (warp - TC_EPI_WARP0) >> 2;
        constexpr int CPH = BN / 32 / (EPI / 4);    // 32-column chunks per warp
        const int c_begin = half * CPH;
        const int row = quad * 32 + lane;
        const int i = m0 + row;
        const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
        const bool row_ok = i < a.n;
        const bool two_acc = a.kblocks > 1;
        const float hi = (a.h && row_ok) ? a.h[i] : 0.f;
        const bool publisher = (warp == TC_EPI_WARP0 && lane == 0);
        // E4: p of this thread's spin at p_tile[col * 128 + row] (a warp's
        // 32 consecutive rows are consecutive words: no bank conflicts)
        float *p_tile = reinterpret_cast<float *>(smem + L::PTILE);
        // Load the initial state into TMEM (E4: p into shared memory).
#pragma unroll 1
        for (int c = c_begin; c < c_begin + CPH; ++c) {
            uint32_t vq[32], vp[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int r = r0 + c * 32 + j;
                const bool ok = row_ok && r < a.R;
                vq[j] = __float_as_uint(ok ? a.q_state[(size_t)r * a.n + i] : 0.f);
                vp[j] = __float_as_uint(ok ? a.p_state[(size_t)r * a.n + i] : 0.f);
            }
            tmem_st32(tl + COL_Q + c * 32, vq);
            if constexpr (E4) {
#pragma unroll
                for (int j = 0; j < 32; ++j) p_tile[(c * 32 + j) * TC_BM + row] = __uint_as_float(vp[j]);
            } else {
                tmem_st32(tl + COL_P + c * 32, vp);
            }
        }
        tmem_wait_st();
        // Normal passes run in an inner loop up to the next readout pass, so
        // that its body carries no readout code: the register allocation and
        // schedule of the steps' loop would pay for it at every step.
        int t = 0;
        bool run = true;
#pragma unroll 1
        while (run && t < P.npass) {
            const int t_end = RO ? P.next_readout(t) : P.npass;
            int st = P.step(t);
#pragma unroll 1
            for (; t < t_end; ++t, ++st) {
                bool ok = true;
                if (lane == 0)
                    ok = CG2 ? mbar_wait_cluster(accf_bar, (uint32_t)(t & 1), a.err, abort_flag, a.limit_ns)
                             : mbar_wait(accf_bar, (uint32_t)(t & 1), a.err, abort_flag, a.limit_ns);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    run = false;
                    break;
                }
                tc_fence_after();
                const float zt = a.zeta[st], dtt = a.dt[st];
                const float dtm = dtt / a.sp.m;
                const bool last = (st == a.steps - 1);
                const bool pre_ro = RO && t + 1 == t_end && t_end < P.npass;   // the next pass reads sign(q) of this step
                // The chunk loop, instantiated once with the update order and the
                // wall variant as run-time parameters and once for the default
                // (kick-drift, no momentum zeroing) so that the integrator does
                // not test them per element.
                auto chunks = [&](auto mode_tag) {
                constexpr int MODE = decltype(mode_tag)::value;
    #pragma unroll 1
                for (int c = c_begin; c < c_begin + CPH; ++c) {
                    uint32_t vf[32], vp[32], vq[32];
                    tmem_ld32(tl + COL_ACC0 + c * 32, vf);
                    if (two_acc) {
                        tmem_ld32(tl + COL_ACC1 + c * 32, vp);
                        tmem_wait_ld();
    #pragma unroll
                        for (int j = 0; j < 32; ++j)
                            vf[j] = __float_as_uint(__uint_as_float(vf[j]) + __uint_as_float(vp[j]));
                    }
                    tmem_ld32(tl + COL_Q + c * 32, vq);
                    if constexpr (E4) {
    #pragma unroll
                        for (int j = 0; j < 32; ++j) vp[j] = __float_as_uint(p_tile[(c * 32 + j) * TC_BM + row]);
                    } else {
                        tmem_ld32(tl + COL_P + c * 32, vp);
                    }
                    tmem_wait_ld();
                    if constexpr (MODE == 1) {
    #pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            float F0 = __uint_as_float(vf[j]), F1 = __uint_as_float(vf[j + 1]);
                            F0 = __fadd_rn(F0, hi);
                            F1 = __fadd_rn(F1, hi);
                            float q0o, q1o, p0o, p1o;
                            integrate2_kd(__uint_as_float(vq[j]), __uint_as_float(vq[j + 1]), __uint_as_float(vp[j]),
                                          __uint_as_float(vp[j + 1]), F0, F1, zt, dtt, dtm, a.sp, q0o, q1o, p0o, p1o);
                            vq[j] = __float_as_uint(q0o);
                            vq[j + 1] = __float_as_uint(q1o);
                            vp[j] = __float_as_uint(p0o);
                            vp[j + 1] = __float_as_uint(p1o);
                        }
                    } else {
    #pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float F = __uint_as_float(vf[j]);
                            float qo, po;
                            integrate<float, MODE>(__uint_as_float(vq[j]), __uint_as_float(vp[j]), __fadd_rn(F, hi), zt,
                                                   dtt, dtm, a.sp, qo, po);
                            vq[j] = __float_as_uint(qo);
                            vp[j] = __float_as_uint(po);
                        }
                    }
                    tmem_st32(tl + COL_Q + c * 32, vq);
                    if constexpr (E4) {
    #pragma unroll
                        for (int j = 0; j < 32; ++j) p_tile[(c * 32 + j) * TC_BM + row] = __uint_as_float(vp[j]);
                    } else {
                        tmem_st32(tl + COL_P + c * 32, vp);
                    }
                    {
                        // bf16 copy into the operand plane of step t+1 (after the
                        // last step: the plane a continuing run starts from),
                        // written directly: a warp's 32 consecutive spins of one
                        // replica are 64 contiguous bytes.  Entries outside n x R
                        // are never written and keep the zeros of the initial fill.
                        __nv_bfloat16 *dst =
                            a.qop + ((size_t)((st + 1 + a.p0) & 1) * a.rpad + (size_t)(r0 + c * 32)) * a.ldk + i;
                        if (row_ok && r0 + c * 32 + 32 <= a.R) {
    #pragma unroll
                            for (int j = 0; j < 32; ++j) dst[(size_t)j * a.ldk] = __float2bfloat16_rn(__uint_as_float(vq[j]));
                        } else if (row_ok) {
    #pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (r0 + c * 32 + j < a.R)
                                    dst[(size_t)j * a.ldk] = __float2bfloat16_rn(__uint_as_float(vq[j]));
                        }
                    }
                    if (last && row_ok) {
    #pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int r = r0 + c * 32 + j;
                            if (r < a.R) {
                                const float qv = __uint_as_float(vq[j]);
                                a.q_state[(size_t)r * a.n + i] = qv;
                                a.p_state[(size_t)r * a.n + i] = __uint_as_float(vp[j]);
                                if (a.spins) a.spins[(size_t)r * a.lds + i] = spin_of(qv);
                            }
                        }
                    }
                }
                };
                if (a.sp.order == 0 && !a.sp.wall_zero_p)
                    chunks(std::integral_constant<int, 1>{});
                else
                    chunks(std::integral_constant<int, 0>{});
                tmem_wait_st();
                if constexpr (RO) {
                    // sign(q) of this step as the operand of the readout pass
                    // that follows (plane 2), from the q just stored in tensor
                    // memory: a pass of its own, so that the chunk loop of every
                    // step does not carry it
                    if (pre_ro) {
#pragma unroll 1
                        for (int c = c_begin; c < c_begin + CPH; ++c) {
                            uint32_t vq[32];
                            tmem_ld32(tl + COL_Q + c * 32, vq);
                            tmem_wait_ld();
                            if (row_ok) {
                                __nv_bfloat16 *dst = a.qop + ((size_t)2 * a.rpad + (size_t)(r0 + c * 32)) * a.ldk + i;
#pragma unroll
                                for (int j = 0; j < 32; ++j)
                                    if (r0 + c * 32 + j < a.R)
                                        dst[(size_t)j * a.ldk] = __float2bfloat16_rn((float)spin_of(__uint_as_float(vq[j])));
                            }
                        }
                    }
                }
                tc_fence_before();
                // The warp's stores of q are ordered before lane 0's arrivals
                // (warp barrier), the arrivals (release, CTA scope) before the
                // publisher's wait (acquire), and that before its release
                // increment at GPU scope, which the consumers' acquire loads read.
                __syncwarp();
                if (lane == 0) {
                    if (CG2 && !leader) mbar_arrive_remote(mapa_shared(tmem_empty_bar, 0u));
                    else mbar_arrive(tmem_empty_bar);
                    mbar_arrive(epi_done_bar);
                }
                if (publisher && t + 1 < P.npass) {
                    // All 8 warps have written their part of q(t+1) (or sign(q(T))): publish.
                    if (mbar_wait(epi_done_bar, (uint32_t)(t & 1), a.err, abort_flag, a.limit_ns))
                        red_release_gpu_add(a.bar + (size_t)rb * a.mtiles + mt, 1u);
                }
            }
            if constexpr (RO) {
                if (!run || t >= P.npass) break;
                // Readout pass t.
                {
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait(accf_bar, (uint32_t)(t & 1), a.err, abort_flag, a.limit_ns);
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) break;
                }
                tc_fence_after();
                const int k = P.index(t);
                const int rc = tc_readout_epi<BN, CPH, CG2>(
                    tl, c_begin, two_acc, row_ok, (a.watch && a.h8 && row_ok) ? 2 * (int)a.h8[i] : 0,
                    a.e_sum + (size_t)k * a.R, r0, a.R, lane, warp == TC_EPI_WARP0, t == P.npass - 1, tmem_empty_bar,
                    epi_done_bar, CG2 && !leader, t, a.bar + (size_t)rb * a.mtiles + mt, a.watch,
                    a.w_cnt ? a.w_cnt + (size_t)k * a.rblocks + rb : nullptr, (unsigned)(a.mtiles - 1), a.target,
                    a.w_done, a.w_hit, k, a.err, abort_flag, a.limit_ns);
                if (rc != 0) break;
                ++t;
                if (a.watch) {
                    // The grid's decision after this readout, while the next
                    // pass's MMAs run (its producers and MMA warps wait for the
                    // decision only one pass later): on a stop, the state stays
                    // that of the readout's step and the next update is not made.
                    bool okd = true, stop = false;
                    if (lane == 0) okd = wait_decision(seen, k, stop, a.err, abort_flag, a.limit_ns);
                    okd = __shfl_sync(0xffffffffu, okd ? 1 : 0, 0) != 0;
                    stop = __shfl_sync(0xffffffffu, stop ? 1 : 0, 0) != 0;
                    if (!okd) break;
                    if (stop) {
                        tc_write_state<BN, E4>(tl, c_begin, CPH, row_ok, r0, a.R, a.n, i, row, a.q_state, a.p_state,
                                               a.spins, a.lds, p_tile);
                        break;
                    }
                }
            } else {
                break;
            }
        }
    } else if constexpr (E4) {
        // ------------------------------------------------ e4m3 converters (4 warps)
        // Widen every J tile into a tensor-memory A slot, stage by stage in
        // the order the producer fills them (the same two rings; slot ring w
        // feeds MMA warp w).  Warp w writes TMEM lanes 32*(w%4) .. +31, so
        // thread = row of the tile; the four warps work independently and
        // the MMA warp waits for all four (afull counts 4 arrivals).  Every
        // lane waits itself and the warp goes on only if all lanes saw the
        // stage, so the .sync.aligned tensor-memory store stays convergent.
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);
        constexpr int HS = S / 2;
        uint32_t cnt0 = 0u, cnt1 = 0u;
        bool ok = true;
        for (int t = 0; t < P.npass && ok; ++t) {
            for (int j = 0; j < a.kblocks; ++j) {
                const int ring = j & 1;
                const uint32_t c = ring ? cnt1 : cnt0;
                const int s = 2 * (int)(c % HS) + ring;
                const int as = 2 * (int)(c % NAR) + ring;
                bool okl = mbar_wait(full_bar(s), (c / HS) & 1u, a.err, abort_flag, a.limit_ns);
                okl = okl && mbar_wait(aempty_bar(as), ((c / NAR) & 1u) ^ 1u, a.err, abort_flag, a.limit_ns);
                if (!__all_sync(0xffffffffu, okl)) { ok = false; break; }
                if (ring) ++cnt1; else ++cnt0;
                tc_fence_after();
                uint32_t w[16], o[32];
                e4m3_row_load(sbase + s * L::STAGE_BYTES, row, w);
                e4m3_row_to_bf16x2(w, o);
                tmem_st32(tq + COL_A + 32u * (uint32_t)as, o);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(afull_bar(as));
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if constexpr (CG2) {
        // No copy is issued after this barrier, and both CTAs' counts of
        // issued stages are in the even CTA's shared memory.
        cluster_sync_all();
        if (leader && warp == 0 && lane < 2) {
            // Ring `lane`: stage k of the ring (k-th arming or issue) is filled
            // by both CTAs in the same order, and a CTA fills stage k only after
            // the MMAs of stage k - S/2 have consumed the same slot, so each
            // slot has at most one unfinished phase, that of the largest k
            // mapped to it.  Settle the stages that only one CTA filled, then
            // wait for the last phase of every slot.
            constexpr int HS = S / 2;
            const int ring = lane;
            const volatile unsigned *cnts = reinterpret_cast<const volatile unsigned *>(smem + L::CNT);
            const uint32_t own = cnts[ring], odd = cnts[2 + ring];
            const uint32_t lo = own < odd ? own : odd, hi = own < odd ? odd : own;
            for (uint32_t k = lo; k < hi; ++k) {
                const uint32_t bar = full_bar(2 * (int)(k % HS) + ring);
                if (k >= own) mbar_arrive_expect_tx(bar, (uint32_t)(2 * L::TX_BYTES));   // filled by the odd CTA alone
                mbar_complete_tx(bar, (uint32_t)L::TX_BYTES);                              // the bytes never sent
            }
            const uint32_t first = hi > (uint32_t)HS ? hi - HS : 0u;
            for (uint32_t k = first; k < hi; ++k) {
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait_cluster(full_bar(2 * (int)(k % HS) + ring), (k / HS) & 1u)) {
                    if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                        atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                        break;
                    }
                }
            }
        }
        __syncwarp();
        // neither CTA frees TMEM or leaves while a copy or an arrival of the
        // other may still reach its shared memory
        cluster_sync_all();
    }
    tc_fence_after();
    if (warp == 1) {
        if constexpr (CG2) {
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(L::TMEM_COLS)
                         : "memory");
        } else {
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(L::TMEM_COLS)
                         : "memory");
        }
    }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                     const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                     const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                     CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    }
    return fn;
}

si_status tc_make_map_bf16(CUtensorMap *m, void *base, int inner, int outer, int box_inner,
                          int box_outer) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return SI_ERR_CUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[96];
        std::snprintf(msg, sizeof msg, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        set_error(msg);
        return SI_ERR_CUDA;
    }
    return SI_OK;
}

// 2D tensor map of the e4m3 J copy (1-byte elements, [outer][inner]) with
// the 64-byte swizzle: boxes of 64 K elements (64 bytes) x box_outer rows.
si_status tc_make_map_e4m3(CUtensorMap *m, void *base, int inner, int outer, int box_outer) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return SI_ERR_CUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner};
    cuuint32_t box[2] = {64u, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char msg[96];
        std::snprintf(msg, sizeof msg, "cuTensorMapEncodeTiled (e4m3) failed (%d)", (int)r);
        set_error(msg);
        return SI_ERR_CUDA;
    }
    return SI_OK;
}

// J (fp32 n x n, every entry exact in e4m3) -> e4m3 [mpad][ldk], zero padded.
// Saturating round-to-nearest conversion; the values were validated exact, so
// nothing rounds.
__global__ void k_convert_j_e4m3(const float *J, int n, __nv_fp8_storage_t *out, int ldk, int mpad) {
    const long long total = (long long)mpad * ldk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldk), j = (int)(e % ldk);
        const float v = (i < n && j < n) ? J[(size_t)i * n + j] : 0.f;
        out[e] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

si_status tc_convert_j_e4m3(const float *J_dev, int n, void *out, int ldk, int mpad, int sms, cudaStream_t st) {
    k_convert_j_e4m3<<<std::min(8 * sms, cdiv((long long)mpad * ldk, 256)), 256, 0, st>>>(
        J_dev, n, (__nv_fp8_storage_t *)out, ldk, mpad);
    SI_CUDA_TRY(cudaGetLastError());
    return SI_OK;
}

__global__ void k_convert_j_bf16(const float *J, int n, __nv_bfloat16 *out, int ldk, int mpad) {
    const long long total = (long long)mpad * ldk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldk), j = (int)(e % ldk);
        out[e] = __float2bfloat16_rn((i < n && j < n) ? J[(size_t)i * n + j] : 0.f);
    }
}

si_status tc_convert_j(const float *J_dev, int n, void *out, int ldk, int mpad, int sms, cudaStream_t st) {
    k_convert_j_bf16<<<std::min(8 * sms, cdiv((long long)mpad * ldk, 256)), 256, 0, st>>>(
        J_dev, n, (__nv_bfloat16 *)out, ldk, mpad);
    SI_CUDA_TRY(cudaGetLastError());
    return SI_OK;
}

__global__ void k_tc_init(const float *q_init, const float *p_init, int n, int R, float *q_state,
                          float *p_state, __nv_bfloat16 *qop, int ldk) {
    const long long total = (long long)R * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), i = (int)(e % n);
        const float q = q_init[e];
        q_state[e] = q;
        p_state[e] = p_init ? p_init[e] : 0.f;
        qop[(size_t)r * ldk + i] = __float2bfloat16_rn(q);
    }
}

// bf16 operand plane of step 0 from the FP32 positions in place.
__global__ void k_tc_operand(const float *q_state, int n, int R, __nv_bfloat16 *qop, int ldk) {
    const long long total = (long long)R * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), i = (int)(e % n);
        qop[(size_t)r * ldk + i] = __float2bfloat16_rn(q_state[e]);
    }
}

template <typename O>
__global__ void k_tc_copy(const float *q_state, const float *p_state, long long total, O *q_out,
                          O *p_out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        if (q_out) q_out[e] = (O)q_state[e];
        if (p_out) p_out[e] = (O)p_state[e];
    }
}

__global__ void k_tc_spins(const float *q_state, int n, int R, int8_t *spins, int ld) {
    const long long total = (long long)R * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ld), i = (int)(e % ld);
        spins[e] = i < n ? spin_of(q_state[(size_t)r * n + i]) : (int8_t)0;
    }
}

template <int BN, int S, int EPI, bool E4, bool CG2 = false, bool RO = false>
static si_status tc_launch_t(Ctx *c, int steps, int8_t *spins_dev) {
    using L = TcSmem<BN, S, E4, CG2>;
    TcArgs a;
    a.n = c->n;
    a.R = c->R;
    a.steps = steps;
    a.mtiles = c->mpad / TC_BM;
    a.rblocks = c->rpad / BN;
    a.kblocks = c->ldk / TC_BK;
    a.ldk = c->ldk;
    a.rpad = c->rpad;
    a.zeta = c->dzeta;
    a.dt = c->ddt;
    a.h = c->has_h ? c->dhf : nullptr;
    a.q_state = (float *)c->dq;
    a.p_state = (float *)c->dp;
    a.qop = (__nv_bfloat16 *)c->dqbuf;
    a.spins = spins_dev;
    a.lds = c->ld8;
    a.bar = c->dbar;
    a.err = c->derr;
    a.limit_ns = c->spin_limit_ns;
    a.stall_step = c->stall_step;
    a.stall_rank = c->stall_rank;
    a.sp = StepParams{c->prm.k, c->prm.m, c->prm.q0, c->prm.q_max, c->prm.p_max,
                      c->prm.update_order, c->prm.wall_zero_p};
    a.p0 = c->tc_p0;
    const bool watch = c->tc_watch_every > 0;
    a.every = watch ? c->tc_watch_every : (c->tc_readout ? steps : 0);
    a.watch = watch ? 1 : 0;
    a.target = c->tc_watch_target;
    const int nread = a.every > 0 ? cdiv(steps, a.every) : 0;
    a.e_sum = watch ? c->w_sum : c->e_sum;
    a.w_cnt = watch ? c->w_ctl + 2 : nullptr;
    a.w_done = watch ? c->w_ctl : nullptr;
    a.w_hit = watch ? reinterpret_cast<int *>(c->w_ctl + 1) : nullptr;
    a.h8 = c->has_h ? c->dh8 : nullptr;
    if ((watch || a.every > 0) && (CG2 || E4 || !RO)) {
        set_error("tensor path: readout passes need the bf16 operand on single CTAs");
        return SI_ERR_UNSUPPORTED;
    }
    const int grid = a.mtiles * a.rblocks;
    if (a.rblocks * a.mtiles > c->nbar || a.mtiles > 64) {
        set_error("tensor path: too many tiles for the step flags (n <= 8192 per context)");
        return SI_ERR_UNSUPPORTED;
    }
    const int smem = L::TOTAL + 1024;
    a.smem_bytes = smem;
    auto kern = k_tc_run<BN, S, EPI, E4, CG2, RO>;
    // launch attributes and the co-residency check once per context (its
    // device and tile are fixed)
    if (c->tc_per_sm[RO ? 1 : 0] <= 0) {
        SI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        SI_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared));
        int per_sm = 0;
        SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tc_threads<EPI, E4>(), smem));
        if (CG2 && per_sm > 0) {
            // every pair of the grid must be resident at once (the CTAs wait on each other)
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(tc_threads<EPI, E4>());
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int clusters = 0;
            SI_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg));
            if (2 * clusters < grid) per_sm = 0;
        }
        c->tc_per_sm[RO ? 1 : 0] = per_sm;
    }
    const int per_sm = c->tc_per_sm[RO ? 1 : 0];
    if (per_sm * c->num_sms < grid) {
        set_error("tensor path: grid cannot be co-resident (reduce replicas per context)");
        return SI_ERR_UNSUPPORTED;
    }
    SI_CUDA_TRY(cudaMemsetAsync(c->dbar, 0, sizeof(unsigned) * grid, c->stream));
    if (nread > 0)
        SI_CUDA_TRY(cudaMemsetAsync(a.e_sum, 0, sizeof(unsigned long long) * (size_t)nread * c->R, c->stream));
    if (watch) {
        // finished evaluations 0, first hit "none" (0x7f7f7f7f), counters 0
        SI_CUDA_TRY(cudaMemsetAsync(c->w_ctl, 0, sizeof(unsigned) * (2 + (size_t)nread * a.rblocks), c->stream));
        SI_CUDA_TRY(cudaMemsetAsync(c->w_ctl + 1, 0x7f, sizeof(unsigned), c->stream));
    }
    if constexpr (CG2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(tc_threads<EPI, E4>());
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        SI_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, c->mapA, c->mapB, a));
    } else {
        void *args[] = {(void *)&c->mapA, (void *)&c->mapB, (void *)&a};
        SI_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(tc_threads<EPI, E4>()), args,
                                                smem, c->stream));
    }
    c->launches += 1;
    return SI_OK;
}

bool tc_readout_supported(const Ctx *c) {
    return !c->grp && !c->j_e4m3 && !c->tc_pair && c->integer_j && (!c->has_h || c->integer_h);
}

si_status tc_watch_buffers(Ctx *c, int steps, int every) {
    const size_t nread = (size_t)cdiv(steps, every);
    // counters for the smallest replica tile (64): room for any tile choice
    const size_t ns = nread * c->R, nc = 2 + nread * (size_t)(c->rpad / 64);
    if (ns > c->w_sum_cap) {
        if (c->w_sum) cudaFree(c->w_sum);
        c->w_sum = nullptr;
        c->w_sum_cap = 0;
        SI_CUDA_TRY(si_dev_malloc((void **)&c->w_sum, sizeof(unsigned long long) * ns));
        c->w_sum_cap = ns;
    }
    if (nc > c->w_ctl_cap) {
        if (c->w_ctl) cudaFree(c->w_ctl);
        c->w_ctl = nullptr;
        c->w_ctl_cap = 0;
        SI_CUDA_TRY(si_dev_malloc((void **)&c->w_ctl, sizeof(unsigned) * nc));
        c->w_ctl_cap = nc;
    }
    return SI_OK;
}

// E = -(sigma^T J sigma + 2 h^T sigma) / 2 of the stopping readout (exact:
// the sum is even), which the kernel picks itself: the first readout that
// reached the target, else the last one.
__global__ void k_watch_energy(const unsigned long long *sums, const int *hit, int nread, int R, int32_t *E) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = *hit;
    const int k = (h >= 0 && h < nread) ? h : nread - 1;
    if (r < R) E[r] = (int32_t)(-((long long)sums[(size_t)k * R + r] / 2));
}

si_status tc_watch_energy(Ctx *c, int nread, int32_t *E) {
    k_watch_energy<<<cdiv(c->R, 256), 256, 0, c->stream>>>(c->w_sum, reinterpret_cast<const int *>(c->w_ctl + 1),
                                                           nread, c->R, E);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

si_status tc_run(Ctx *c, int steps, int8_t *spins_dev) {
    if (steps == 0) return SI_OK;
    if (c->j_e4m3) {
        switch (c->tile_n) {
            case 64: return tc_launch_t<64, 8, 8, true>(c, steps, spins_dev);
            case 128: return tc_launch_t<128, 4, 8, true>(c, steps, spins_dev);
            default: break;
        }
    } else if (c->tc_pair) {
        return tc_launch_t<128, 8, 8, false, true>(c, steps, spins_dev);
    } else if (c->tc_readout || c->tc_watch_every > 0) {
        switch (c->tile_n) {
            case 64: return tc_launch_t<64, 8, 8, false, false, true>(c, steps, spins_dev);
            case 128: return tc_launch_t<128, 6, 8, false, false, true>(c, steps, spins_dev);
            default: break;
        }
    } else {
        switch (c->tile_n) {
            case 64: return tc_launch_t<64, 8, 8, false>(c, steps, spins_dev);
            case 128: return tc_launch_t<128, 6, 8, false>(c, steps, spins_dev);
            default: break;
        }
    }
    set_error("tensor path: unsupported tile");
    return SI_ERR_UNSUPPORTED;
}

template <int BN, int S, int EPI, bool E4>
static int tc_occupancy() {
    using L = TcSmem<BN, S, E4>;
    const int smem = L::TOTAL + (EPI == 4 ? 256 : 1024);
    if (cudaFuncSetAttribute(k_tc_run<BN, S, EPI, E4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return 0;
    if (cudaFuncSetAttribute(k_tc_run<BN, S, EPI, E4>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_run<BN, S, EPI, E4>, tc_threads<EPI, E4>(),
                                                      smem) != cudaSuccess)
        return 0;
    return per_sm;
}

// Replica tile: 128 when the grid of 128-wide tiles is co-resident, else 64,
// unless the caller fixed tile_n.  Returns the CTAs per SM of the choice.
static int choose_tile(const Ctx *c, int *per_sm) {
    const int mtiles = c->mpad / TC_BM;
    const int occ128 = c->j_e4m3 ? tc_occupancy<128, 4, 8, true>() : tc_occupancy<128, 6, 8, false>();
    const int occ64 = c->j_e4m3 ? tc_occupancy<64, 8, 8, true>() : tc_occupancy<64, 8, 8, false>();
    int bn;
    if (c->prm.tile_n == 64 || c->prm.tile_n == 128) {
        bn = c->prm.tile_n;
    } else if (c->R > 64 && mtiles * cdiv(c->R, 128) <= occ128 * c->num_sms) {
        bn = 128;
    } else {
        bn = 64;
    }
    *per_sm = bn == 128 ? occ128 : occ64;
    return bn;
}

// Operand of J for the persistent kernel.  Its J tiles are re-read from L2
// at every step, so it keeps J as bf16: widening each e4m3 tile at every step
// (into tensor memory, the fastest of the forms measured) costs more time
// than the 8 KB of L2 traffic it saves per 128 x 64 tile.  SI_TC_J_E4M3=1
// selects the e4m3 operand with per-tile widening (same results, bit for
// bit).  The grouped per-step kernel, which streams J from HBM, reads e4m3.
static bool tc_e4m3_operand(const Ctx *c) {
    if (c->prm.prec != SI_PREC_J_FP8_Q_BF16) return false;
    const char *e = std::getenv("SI_TC_J_E4M3");
    return e && std::atoi(e) == 1;
}

// Pairs of consecutive 128-row tiles sharing each MMA (k_tc_run with CG2)
// for the 128-replica tile that the library chose itself on a bf16 J
// operand, when every pair of the grid (J rows padded to 256) can be
// resident at once.  SI_TC_PAIR=1 turns them on.
static bool tc_pair_choice(const Ctx *c) {
    const char *e = std::getenv("SI_TC_PAIR");
    if (!(e && std::atoi(e) == 1)) return false;
    if (c->j_e4m3 || c->prm.tile_n != 0 || c->tile_n != 128) return false;
    using L = TcSmem<128, 8, false, true>;
    auto kern = k_tc_run<128, 8, 8, false, true>;
    const int smem = L::TOTAL + 1024;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(tc_threads<8, false>());
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int mtiles = round_up(c->n, 2 * TC_BM) / TC_BM;
    const long long grid = (long long)mtiles * cdiv(c->R, 128);
    return mtiles <= 64 && grid <= 2LL * clusters;
}

bool tc_persistent_fits(Ctx *c) {
    c->ldk = round_up(c->n, TC_BK);
    c->mpad = round_up(c->n, TC_BM);
    c->j_e4m3 = tc_e4m3_operand(c);
    const int mtiles = c->mpad / TC_BM;
    int per_sm = 0;
    const int bn = choose_tile(c, &per_sm);
    const long long grid = (long long)mtiles * cdiv(c->R, bn);
    return mtiles <= 64 && grid <= 4096 && per_sm > 0 && grid <= (long long)per_sm * c->num_sms;
}

si_status tc_prepare(Ctx *c, const float *J_dev) {
    const int n = c->n;
    c->ldk = round_up(n, TC_BK);
    c->mpad = round_up(n, TC_BM);
    c->j_e4m3 = tc_e4m3_operand(c);
    int per_sm = 0;
    c->tile_n = choose_tile(c, &per_sm);
    c->rpad = round_up(c->R, c->tile_n);
    c->tc_pair = tc_pair_choice(c);
    if (c->tc_pair) {
        c->mpad = round_up(n, 2 * TC_BM);   // whole pairs of 128-row tiles
        per_sm = 1;
    }
    SI_CUDA_TRY(si_dev_malloc(&c->dJ, (size_t)c->mpad * c->ldk * (c->j_e4m3 ? 1 : 2)));
    si_status sc = c->j_e4m3 ? tc_convert_j_e4m3(J_dev, n, c->dJ, c->ldk, c->mpad, c->num_sms, c->stream)
                             : tc_convert_j(J_dev, n, c->dJ, c->ldk, c->mpad, c->num_sms, c->stream);
    if (sc != SI_OK) return sc;
    c->qbuf_bytes = 3ull * c->rpad * c->ldk * 2;   // planes 0, 1: q; plane 2: sign(q(T)) for the readout pass
    SI_CUDA_TRY(si_dev_malloc(&c->dqbuf, c->qbuf_bytes));
    SI_CUDA_TRY(cudaMemsetAsync(c->dqbuf, 0, c->qbuf_bytes, c->stream));
    SI_CUDA_TRY(si_dev_malloc(&c->dq, sizeof(float) * (size_t)c->R * n));
    SI_CUDA_TRY(si_dev_malloc(&c->dp, sizeof(float) * (size_t)c->R * n));
    si_status s = c->j_e4m3 ? tc_make_map_e4m3(&c->mapA, c->dJ, c->ldk, c->mpad, TC_BM)
                            : tc_make_map_bf16(&c->mapA, c->dJ, c->ldk, c->mpad, TC_BK, TC_BM);
    if (s != SI_OK) return s;
    // pairs load half of the q tile per CTA
    s = tc_make_map_bf16(&c->mapB, c->dqbuf, c->ldk, 3 * c->rpad, TC_BK, c->tc_pair ? c->tile_n / 2 : c->tile_n);
    if (s != SI_OK) return s;
    const int mtiles = c->mpad / TC_BM;
    const int grid = mtiles * (c->rpad / c->tile_n);
    if (grid > per_sm * c->num_sms) {
        set_error("tensor path: n x replicas too large for one co-resident launch");
        return SI_ERR_UNSUPPORTED;
    }
    return SI_OK;
}

si_status tc_init_state(Ctx *c, const float *q_init, const float *p_init) {
    const long long total = (long long)c->R * c->n;
    k_tc_init<<<std::min(8 * c->num_sms, cdiv(total, 256)), 256, 0, c->stream>>>(
        q_init, p_init, c->n, c->R, (float *)c->dq, (float *)c->dp, (__nv_bfloat16 *)c->dqbuf, c->ldk);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

si_status tc_continue_state(Ctx *c) {
    const long long total = (long long)c->R * c->n;
    k_tc_operand<<<std::min(8 * c->num_sms, cdiv(total, 256)), 256, 0, c->stream>>>(
        (const float *)c->dq, c->n, c->R, (__nv_bfloat16 *)c->dqbuf, c->ldk);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

si_status tc_copy_state(Ctx *c, float *q_out, float *p_out) {
    const long long total = (long long)c->R * c->n;
    k_tc_copy<float><<<std::min(8 * c->num_sms, cdiv(total, 256)), 256, 0, c->stream>>>(
        (const float *)c->dq, (const float *)c->dp, total, q_out, p_out);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

si_status tc_copy_state_f64(Ctx *c, double *q_out, double *p_out) {
    const long long total = (long long)c->R * c->n;
    k_tc_copy<double><<<std::min(8 * c->num_sms, cdiv(total, 256)), 256, 0, c->stream>>>(
        (const float *)c->dq, (const float *)c->dp, total, q_out, p_out);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

si_status tc_spins(Ctx *c, int8_t *spins, int ld) {
    const long long total = (long long)c->R * ld;
    k_tc_spins<<<std::min(8 * c->num_sms, cdiv(total, 256)), 256, 0, c->stream>>>(
        (const float *)c->dq, c->n, c->R, spins, ld);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

const char *tc_describe(const Ctx *c, char *buf, int len) {
    std::snprintf(buf, len,
                  "tcgen05 prec=%s J=%s n=%d R=%d tile=128x%d%s stages=%d grid=%d (mtiles=%d rblocks=%d) kblocks=%d",
                  c->prm.prec == SI_PREC_J_FP8_Q_BF16 ? "j_fp8_q_bf16" : "j_bf16_q_bf16",
                  c->j_e4m3 ? "e4m3(1B)" : "bf16(2B)", c->n, c->R, c->tile_n,
                  c->tc_pair ? " cta_pairs(M=256)" : "", c->tile_n == 128 ? (c->j_e4m3 ? 4 : (c->tc_pair ? 8 : 6)) : 8,
                  (c->mpad / TC_BM) * (c->rpad / c->tile_n), c->mpad / TC_BM, c->rpad / c->tile_n, c->ldk / TC_BK);
    return buf;
}

}  // namespace si
