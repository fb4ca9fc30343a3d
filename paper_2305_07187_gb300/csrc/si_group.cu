// Grouped batch: many independent Ising instances of uneven size (the
// paper's parallel tests, Fig. 3, generalised to many problems at once) run
// the tensor-core step together.
//
// One launch performs one time step for every instance.  Its CTAs walk a
// list of (instance, M tile, replica block) tiles ordered by decreasing cost;
// each tile is a tcgen05 GEMM F = J Q^T over the instance's K range (its own
// TMA tensor maps, read from device memory) with the integrator of Eq. 8 and
// the walls of Eq. 6 fused into the epilogue.  The launch boundary is the
// step barrier for all instances; the T launches are captured once into a
// CUDA graph and replayed.  The operand ring runs across tile boundaries, and
// TMEM holds two accumulator slots so that the epilogue of one tile overlaps
// the MMAs of the next.  J of all instances does not fit in L2, so this path
// streams J from HBM every step.
//
// Tile width (64 or 128 replicas per tile, per instance) is chosen by an
// autotuner that times a few steps of each candidate policy on the actual
// group and caches the winner by group shape.
//
// Members of precision SI_PREC_J_FP8_Q_BF16 keep J in HBM as 1-byte e4m3
// (validated exact), so the step streams half the J bytes of a bf16 member.
// Four converter warps widen each e4m3 J tile to bf16: under the policy
// "whole-instance-tmem-a" into tensor memory, where the MMA reads its A
// operand (one accumulator slot of up to 256 columns, the other 256 columns
// hold eight A slots), under every other policy in place in shared memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "si_tcgen05.cuh"

namespace si {

constexpr int GR_BM = 128, GR_BK = 64;
// Warps: producer of the even stages, 2 MMA issuers, GR_EPI epilogue warps
// (three per TMEM lane quadrant), in groups with e4m3 members (CONV) 4
// converter warps, then the producer of the odd stages.
constexpr int GR_EPI = 12;
template <bool CONV>
constexpr int gr_threads() { return 32 * (4 + GR_EPI + (CONV ? 4 : 0)); }
template <bool CONV>
constexpr int gr_prod1_warp() { return 3 + GR_EPI + (CONV ? 4 : 0); }
constexpr int GR_A_BYTES = GR_BM * GR_BK * 2;
constexpr int GR_SMAX = 8;                       // most ring stages of any policy
constexpr int GR_TILES = 196608;                 // shared memory for the ring
constexpr int GR_NA = 8;                          // tensor-memory A slots (single-accumulator policy)
constexpr int GR_NBARS = 3 * GR_SMAX + 2 + 2 + 1 + GR_NA;  // full, empty, accf[2], tmem_empty[2], drain, conv, aempty

// TMEM column of A slot k (tensor-memory A policy: one accumulator slot in
// columns 0 .. 255, the A slots after it).
__device__ __forceinline__ uint32_t gr_acol(int k) { return 256u + 32u * k; }
constexpr int GR_SMEM = GR_TILES + GR_NBARS * 8 + 16 + 1024;

struct GroupInst {
    int n, R, ldk, rpad, mtiles, rblocks, kblocks, bn;
    int e4m3;                  // J stored as e4m3 bytes (else bf16)
    int lds;                   // row stride of spins
    const float *h;            // [n] or null
    float *q_state, *p_state;  // [R][n]
    __nv_bfloat16 *qop;        // [2][rpad][ldk]
    int8_t *spins;             // [R][lds]
};

struct GroupTile {
    int inst, mt, r0, bn;      // replicas r0 .. r0 + bn - 1 (bn: the instance's width or half of it)
    int cost;
    int kb_off, kb_cnt;        // the M tile's non-zero K blocks: kbl[kb_off .. kb_off + kb_cnt)
};

struct GroupArgs {
    const GroupInst *inst;
    const GroupTile *tiles;
    int ntiles;
    const CUtensorMap *maps;   // [3*count]: J map, q map (width bn), q map (width bn/2) of each instance
    const int *kbl;            // K-block lists of all (instance, M tile)
    const float *zeta, *dt;
    int t, last;
    StepParams sp;
    int *err;
    long long limit_ns;
    int single;                // 1: one accumulator per tile (N = bn <= 256), one MMA warp
    int tmem_a;                // 1 (single mode, one slot): e4m3 J tiles widened into TMEM A slots
    int nslots;                // accumulator slots in TMEM (2: the epilogue of tile u overlaps tile u+1)
    int stages;                // ring stages (even, <= GR_SMAX)
    int stage_bytes;           // A tile + largest B tile of the policy (multiple of 1024)
};

template <bool CONV>
__global__ void __launch_bounds__(gr_threads<CONV>(), 1) k_group_step(const __grid_constant__ GroupArgs a) {
    constexpr int GR_CONV_WARP0 = 3 + GR_EPI;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + GR_TILES;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (GR_SMAX + s); };
    auto accf_bar = [&](int k) { return bar0 + 8u * (2 * GR_SMAX + k); };
    auto tmem_empty_bar = [&](int k) { return bar0 + 8u * (2 * GR_SMAX + 2 + k); };
    const uint32_t drain_bar = bar0 + 8u * (2 * GR_SMAX + 4);
    auto conv_bar = [&](int s) { return bar0 + 8u * (2 * GR_SMAX + 5 + s); };
    auto aempty_bar = [&](int k) { return bar0 + 8u * (3 * GR_SMAX + 5 + k); };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + GR_TILES + GR_NBARS * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + GR_TILES + GR_NBARS * 8 + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.stages, HS = a.stages / 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GR_SMAX; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
            mbar_init(conv_bar(s), 4);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(accf_bar(k), 2);
            mbar_init(tmem_empty_bar(k), GR_EPI);
        }
        mbar_init(drain_bar, 2);
        for (int k = 0; k < GR_NA; ++k) mbar_init(aempty_bar(k), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "n"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int plane_in = a.t & 1;
    // The hot loops track (index within the ring, phase) incrementally: split
    // mode has two rings (even / odd stages, one per MMA warp), single mode
    // one ring of all stages.
    const int ring_len = a.single ? S : HS;
    auto ring_stage = [&](int k, int ring) -> int { return a.single ? k : 2 * k + ring; };

    if (warp == 0 || warp == gr_prod1_warp<CONV>()) {
        // ---------------------------------------------- TMA producers (warp 0, last warp)
        // One thread's chain of barrier wait, arming and two TMA issues per K
        // block takes about as long as the K block's MMAs, so two producers
        // fill the ring, producer l the stages 2i + l.  In split mode that is
        // ring l (the K blocks of parity l within a tile, for MMA warp l + 1);
        // in single mode the one consumer takes the stages in order, the g-th
        // K block of this CTA in stage g mod S (S even), so producer l takes
        // the K blocks g of parity l.  The two are in separate warps, so that
        // neither waits for the other's stage (in single mode those come one
        // MMA apart).
        if (lane == 0) {
            const int ring = warp == 0 ? 0 : 1;
            uint32_t cnt = 0u;   // stages armed by this producer
            int rk = 0;          // next index within this producer's stages
            uint32_t rph = 0u;   // and its phase parity
            int gpar = 0;        // single mode: parity of this CTA's K blocks before the tile
            bool ok = true;
            for (int k = blockIdx.x; k < a.ntiles && ok; k += gridDim.x) {
                const GroupTile tl = a.tiles[k];
                const GroupInst &in = a.inst[tl.inst];
                const CUtensorMap *mJ = a.maps + 3 * tl.inst;
                const CUtensorMap *mQ = mJ + (tl.bn == in.bn ? 1 : 2);
                const uint32_t bytes = (uint32_t)((in.e4m3 ? GR_BM * GR_BK : GR_A_BYTES) + tl.bn * GR_BK * 2);
                const uint32_t a_off = in.e4m3 ? (uint32_t)E4M3_TILE_OFFSET : 0u;
                const int yq = plane_in * in.rpad + tl.r0;
                const int j0 = a.single ? (ring ^ gpar) : ring;
                for (int j = j0; j < tl.kb_cnt; j += 2) {
                    const int kb = a.kbl[tl.kb_off + j];
                    const int s = 2 * rk + ring;
                    if (!mbar_wait(empty_bar(s), rph ^ 1u, a.err, abort_flag, a.limit_ns)) { ok = false; break; }
                    ++cnt;
                    if (++rk == HS) {
                        rk = 0;
                        rph ^= 1u;
                    }
                    const uint32_t dA = sbase + s * a.stage_bytes;
                    mbar_arrive_expect_tx(full_bar(s), bytes);
                    tma_load_2d(dA + a_off, mJ, full_bar(s), kb * GR_BK, tl.mt * GR_BM);
                    tma_load_2d(dA + GR_A_BYTES, mQ, full_bar(s), kb * GR_BK, yq);
                }
                gpar = (gpar + tl.kb_cnt) & 1;
            }
            // Let every copy this producer issued land before the CTA exits.
            const uint32_t first = cnt > (uint32_t)HS ? cnt - HS : 0u;
            for (uint32_t k = first; k < cnt; ++k) {
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait(full_bar(2 * (int)(k % (uint32_t)HS) + ring), (k / (uint32_t)HS) & 1u)) {
                    if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                        atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                        break;
                    }
                }
            }
        }
    } else if (warp <= 2) {
        // ---------------------------------------------- MMA issuers
        // Split mode: warp 1 takes even K blocks into acc0, warp 2 odd ones
        // into acc1, of TMEM slot (u & 1).  Single mode: warp 1 issues every
        // K block into one accumulator of up to 256 columns; warp 2 only keeps
        // the per-tile handshake.
        if (lane == 0) {
            const int w = warp - 1;
            int rk = 0;          // index within this warp's ring of stages
            uint32_t rph = 0u;   // and its phase parity
            uint32_t ce = 0u;    // e4m3 K blocks taken from TMEM A slots so far
            bool ok = true;
            int u = 0;
            for (int k = blockIdx.x; k < a.ntiles && ok; k += gridDim.x, ++u) {
                const GroupTile tl = a.tiles[k];
                const int slot = a.nslots == 2 ? (u & 1) : 0;
                const int use = a.nslots == 2 ? (u >> 1) : u;   // earlier tiles in this slot
                if (use >= 1) {
                    if (!mbar_wait(tmem_empty_bar(slot), (uint32_t)((use - 1) & 1), a.err, abort_flag,
                                   a.limit_ns)) {
                        ok = false;
                        break;
                    }
                }
                tc_fence_after();
                const uint32_t idesc = idesc_bf16(GR_BM, tl.bn);
                if (a.single) {
                    if (w == 0) {
                        const uint32_t d_tmem = tmem + (uint32_t)slot * 256u;
                        const bool ta = a.tmem_a && a.inst[tl.inst].e4m3;
                        for (int kb = 0; kb < tl.kb_cnt; ++kb) {
                            const int s = ring_stage(rk, 0);
                            if (!mbar_wait(full_bar(s), rph, a.err, abort_flag, a.limit_ns) ||
                                (CONV && !mbar_wait(conv_bar(s), rph, a.err, abort_flag, a.limit_ns))) {
                                ok = false;
                                break;
                            }
                            if (++rk == ring_len) {
                                rk = 0;
                                rph ^= 1u;
                            }
                            tc_fence_after();
                            const uint64_t ad = sdesc_sw128(sbase + s * a.stage_bytes);
                            const uint64_t bd = ad + (uint64_t)(GR_A_BYTES >> 4);
                            if (ta) {
                                // A from the tensor-memory slot the converters filled
                                // (conv_bar of this stage came after their store)
                                const int as = (int)(ce % GR_NA);
                                ++ce;
                                const uint32_t at = tmem + gr_acol(as);
#pragma unroll
                                for (int kk = 0; kk < GR_BK / 16; ++kk)
                                    mma_bf16_tmem_a(d_tmem, at + 8u * kk, bd + 2u * kk, idesc,
                                                    (kb != 0 || kk != 0) ? 1u : 0u);
                                mma_commit(empty_bar(s));
                                mma_commit(aempty_bar(as));
                            } else {
#pragma unroll
                                for (int kk = 0; kk < GR_BK / 16; ++kk)
                                    mma_bf16(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc,
                                             (kb != 0 || kk != 0) ? 1u : 0u);
                                mma_commit(empty_bar(s));
                            }
                        }
                    }
                } else {
                    const uint32_t d_tmem = tmem + (uint32_t)slot * 256u + (w == 0 ? 0u : 128u);
                    for (int kb = w; kb < tl.kb_cnt; kb += 2) {
                        const int s = ring_stage(rk, w);
                        if (!mbar_wait(full_bar(s), rph, a.err, abort_flag, a.limit_ns) ||
                            (CONV && !mbar_wait(conv_bar(s), rph, a.err, abort_flag, a.limit_ns))) {
                            ok = false;
                            break;
                        }
                        if (++rk == ring_len) {
                            rk = 0;
                            rph ^= 1u;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(sbase + s * a.stage_bytes);
                        const uint64_t bd = ad + (uint64_t)(GR_A_BYTES >> 4);
#pragma unroll
                        for (int kk = 0; kk < GR_BK / 16; ++kk)
                            mma_bf16(d_tmem, ad + 2u * kk, bd + 2u * kk, idesc, (kb != w || kk != 0) ? 1u : 0u);
                        mma_commit(empty_bar(s));
                    }
                }
                if (ok) mma_commit(accf_bar(slot));
            }
            mma_commit(drain_bar);
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(drain_bar, 0u)) {
                if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                    atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                    break;
                }
            }
        }
    } else if (warp < GR_CONV_WARP0) {
        // ---------------------------------------------- epilogue (GR_EPI warps)
        // Warp w reads TMEM lanes 32*(w%4) .. +31 (one spin per thread) and
        // share (w-3)/4 of the tile's 16-column chunks.
        const int quad = warp & 3;
        const int half = (warp - 3) >> 2;   // which share of the chunks (0 .. GR_EPI/4 - 1)
        const int row = quad * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        const float zt = a.zeta[a.t], dtt = a.dt[a.t];
        const float dtm = dtt / a.sp.m;
        int u = 0;
        for (int k = blockIdx.x; k < a.ntiles; k += gridDim.x, ++u) {
            const GroupTile tl = a.tiles[k];
            const GroupInst &in = a.inst[tl.inst];
            const int slot = a.nslots == 2 ? (u & 1) : 0;
            const int use = a.nslots == 2 ? (u >> 1) : u;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(accf_bar(slot), (uint32_t)(use & 1), a.err, abort_flag, a.limit_ns);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            const int i = tl.mt * GR_BM + row;
            const bool row_ok = i < in.n;
            const float hi = (in.h && row_ok) ? in.h[i] : 0.f;
            const bool two_acc = !a.single && tl.kb_cnt > 1;
            const int nch = tl.bn / 16;
            constexpr int NPART = GR_EPI / 4;
            const int c0 = (nch * half + NPART - 1) / NPART;
            const int c1 = (nch * (half + 1) + NPART - 1) / NPART;
            const uint32_t tacc = tmem + lane_off + (uint32_t)slot * 256u;
            __nv_bfloat16 *qn = in.qop + (size_t)(plane_in ^ 1) * in.rpad * in.ldk;
            for (int c = c0; c < c1; ++c) {
                uint32_t vf[16], vg[16];
                tmem_ld16(tacc + c * 16, vf);
                if (two_acc) tmem_ld16(tacc + 128 + c * 16, vg);
                tmem_wait_ld();
                if (row_ok) {
                    // load the 16 replicas' state before the first store, so
                    // the loads overlap instead of queueing behind the stores
                    float qv[16], pv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int r = tl.r0 + c * 16 + j;
                        const size_t e = (size_t)r * in.n + i;
                        qv[j] = r < in.R ? in.q_state[e] : 0.f;
                        pv[j] = r < in.R ? in.p_state[e] : 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int r = tl.r0 + c * 16 + j;
                        if (r >= in.R) continue;
                        float F = __uint_as_float(vf[j]);
                        if (two_acc) F += __uint_as_float(vg[j]);
                        const size_t e = (size_t)r * in.n + i;
                        float qo, po;
                        integrate<float>(qv[j], pv[j], F + hi, zt, dtt, dtm, a.sp, qo, po);
                        in.q_state[e] = qo;
                        in.p_state[e] = po;
                        if (!a.last) qn[(size_t)r * in.ldk + i] = __float2bfloat16_rn(qo);
                        else if (in.spins) in.spins[(size_t)r * in.lds + i] = spin_of(qo);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty_bar(slot));
        }
    } else if constexpr (CONV) {
        // ---------------------------------------------- converters (4 warps)
        // Walk the stages in the producer's order.  Every use of a stage is
        // released to the MMA warp through conv_bar, after its e4m3 J tile
        // (if the member stores J as e4m3) has been widened in place; bf16
        // tiles pass straight through.  Waiting for the stage's TMA first
        // keeps conv_bar one phase behind full_bar, so no waiter can see a
        // phase two ahead.  Every thread waits itself; the four warps agree
        // on success through one reducing barrier.
        // Warp w writes TMEM lanes 32*(w%4) .. +31: thread = row (w%4)*32 + lane.
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);
        int rk0 = 0, rk1 = 0;
        uint32_t rph0 = 0u, rph1 = 0u;
        uint32_t ce = 0u;   // e4m3 K blocks widened into TMEM A slots so far
        bool ok = true;
        for (int k = blockIdx.x; k < a.ntiles && ok; k += gridDim.x) {
            const GroupTile tl = a.tiles[k];
            const int e4 = a.inst[tl.inst].e4m3;
            const bool ta = a.tmem_a && e4;
            for (int j = 0; j < tl.kb_cnt; ++j) {
                const int ring = a.single ? 0 : (j & 1);
                int &rk = ring ? rk1 : rk0;
                uint32_t &rph = ring ? rph1 : rph0;
                const int s = ring_stage(rk, ring);
                const uint32_t ph = rph;
                const int as = (int)(ce % GR_NA);
                bool okl = mbar_wait(full_bar(s), ph, a.err, abort_flag, a.limit_ns);
                if (ta) okl = okl && mbar_wait(aempty_bar(as), ((ce / GR_NA) & 1u) ^ 1u, a.err, abort_flag, a.limit_ns);
                if (!named_barrier_and(2, 128, okl ? 1 : 0)) { ok = false; break; }
                if (++rk == ring_len) {
                    rk = 0;
                    rph ^= 1u;
                }
                if (ta) {
                    tc_fence_after();
                    uint32_t wv[16], o[32];
                    e4m3_row_load(sbase + s * a.stage_bytes + (uint32_t)E4M3_TILE_OFFSET, row, wv);
                    e4m3_row_to_bf16x2(wv, o);
                    tmem_st32(tq + gr_acol(as), o);
                    tmem_wait_st();
                    tc_fence_before();
                    ++ce;
                } else if (e4) {
                    widen_e4m3_tile(sbase + s * a.stage_bytes, row, 2);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(conv_bar(s));
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(512) : "memory");
    }
}

// q_state -> bf16 operand plane 0 for every instance (blockIdx.y = instance).
__global__ void k_group_init(const GroupInst *inst) {
    const GroupInst in = inst[blockIdx.y];
    const long long total = (long long)in.R * in.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / in.n), i = (int)(e % in.n);
        in.qop[(size_t)r * in.ldk + i] = __float2bfloat16_rn(in.q_state[e]);
    }
}

// ============================================================ host side
struct GroupMember {
    int n, R;
    bool e4m3 = false;          // J stored as e4m3 bytes (SI_PREC_J_FP8_Q_BF16), else bf16
    void *J = nullptr;          // [mpad][ldk], e4m3 or bf16
    int ldk = 0, mpad = 0;
    float *h = nullptr;
    float *q = nullptr, *p = nullptr;
    __nv_bfloat16 *qop = nullptr;
    int rpad_max = 0;
    int8_t *spins = nullptr;
    int lds = 0;                // row stride of spins (n, or the serving context's padded stride)
    bool own_spins = true;
    Ctx energy;                 // readout view (int8 J, h copies)
    std::vector<int> kb_off, kb_cnt;   // per M tile: its non-zero K blocks in Group::kbl
};

constexpr int kMaxPolicies = 8;   // room in the per-policy tables (kPolicies are used)

struct Group {
    int count = 0, steps = 0;
    // Set when the group serves one si_create context whose persistent grid
    // would not be co-resident: the member then writes the context's spin
    // buffer and error word, and the context does the readouts.
    Ctx *host = nullptr;
    si_params common;
    cudaStream_t stream = nullptr;
    int device = 0, sms = 0;
    long long limit_ns = 2000000000LL;
    std::vector<GroupMember> m;
    GroupInst *d_inst = nullptr;
    GroupTile *d_tiles = nullptr;
    int ntiles = 0;
    // per tile policy (kPolicies of them)
    int pol_tiles_off[kMaxPolicies] = {}, pol_ntiles[kMaxPolicies] = {};
    int pol_stages[kMaxPolicies] = {}, pol_stage_bytes[kMaxPolicies] = {};
    CUtensorMap *d_maps = nullptr;
    std::vector<int> kbl;       // K-block lists of every (member, M tile), host copy
    int *d_kbl = nullptr;
    float *d_zeta = nullptr, *d_dt = nullptr;
    int *d_err = nullptr;
    int *h_err = nullptr;   // pinned host copy of the error word
    int policy = -1;            // chosen tile policy
    bool any_e4m3 = false;      // some member stores J as e4m3
    int grid = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1;
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ev_valid = false;
    int launches = 0;
};

static const char *kPolicyName[] = {"bn64-if-R<=64-else-128", "all-64", "all-128", "whole-instance",
                                    "whole-instance-tmem-a"};
constexpr int kPolicies = 5;
static_assert(kPolicies <= kMaxPolicies, "per-policy tables too small");
constexpr int kPolicyWhole = 3;
constexpr int kPolicyWholeTmemA = 4;   // whole-instance tiles, e4m3 J widened into TMEM, one accumulator slot

// Replicas per tile of a member under a policy.  "whole-instance" covers all
// R replicas of the member in one tile (R <= 256, a multiple of 16), so each
// J slab is read once per step, and larger R in tiles of 256; it runs the
// single-accumulator mode (one MMA of N up to 256 per K step).
static int policy_bn(int policy, int R, bool any_e4m3) {
    if (policy == 1) return 64;
    if (policy == 2) return 128;
    (void)any_e4m3;
    if (policy == kPolicyWhole || policy == kPolicyWholeTmemA) return round_up(R, 16) <= 256 ? round_up(R, 16) : 256;
    return R <= 64 ? 64 : 128;
}

// Ring geometry of a policy: stage = A tile + the largest B tile (rounded to
// 1024 bytes), as many even stages as fit the ring's shared memory.
static void policy_ring(int policy, const std::vector<int> &bns, int *stages, int *stage_bytes) {
    int bmax = 16;
    for (int b : bns) bmax = std::max(bmax, b);
    int sb = GR_BM * GR_BK * 2 + round_up(bmax * GR_BK * 2, 1024);
    int st = std::min(GR_SMAX, GR_TILES / sb);
    st &= ~1;
    if (policy == kPolicyWhole || policy == kPolicyWholeTmemA) st = std::max(st, 2);
    *stages = st;
    *stage_bytes = sb;
}

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;
static bool g_tune_file_loaded = false;

// Autotuner results persist across processes in the text file named by
// SI_TUNE_CACHE (one "key policy" line per group shape; later lines win).
// Without the variable the cache lives in the process only.  Callers hold
// g_tune_mu.
static void tune_file_load_locked() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char *path = std::getenv("SI_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[8192];
    while (std::fgets(line, sizeof line, f)) {
        char *sp = std::strrchr(line, ' ');
        if (!sp) continue;
        const int pol = std::atoi(sp + 1);
        *sp = '\0';
        if (pol >= 0 && pol < kPolicies && line[0]) g_tune_cache[line] = pol;
    }
    std::fclose(f);
}

static void tune_file_store_locked(const std::string &key, int pol) {
    const char *path = std::getenv("SI_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), pol);
    std::fclose(f);
}

static bool tune_cache_find(const std::string &key, int *pol) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_file_load_locked();
    auto it = g_tune_cache.find(key);
    if (it == g_tune_cache.end()) return false;
    *pol = it->second;
    return true;
}

static std::string group_key(const Group *g) {
    int drv = 0;
    cudaDriverGetVersion(&drv);
    std::string k = "sm" + std::to_string(g->sms) + "-drv" + std::to_string(drv) + ":";
    for (const auto &x : g->m) {
        long long nb = 0;
        for (int v : x.kb_cnt) nb += v;
        k += std::to_string(x.n) + "x" + std::to_string(x.R) + "b" + std::to_string(nb) + (x.e4m3 ? "e" : "") + ",";
    }
    return k;
}

// Which 128 x 64 blocks of J (bf16 when E is unsigned short, e4m3 when it is
// unsigned char) hold a non-zero coupling: one CTA per block,
// mask[mt * kblocks + kb].
template <typename E>
__global__ void k_block_nonzero(const E *J, int ldk, int kblocks, unsigned char *mask) {
    const int mt = blockIdx.y, kb = blockIdx.x;
    const unsigned absmask = sizeof(E) == 1 ? 0x7Fu : 0x7FFFu;   // +0 and -0 count as zero
    int nz = 0;
    for (int e = threadIdx.x; e < GR_BM * GR_BK; e += blockDim.x) {
        const int r = e / GR_BK, cidx = e % GR_BK;
        const unsigned v = J[(size_t)(mt * GR_BM + r) * ldk + kb * GR_BK + cidx];
        nz |= (v & absmask) != 0u;
    }
    nz = __syncthreads_or(nz);
    if (threadIdx.x == 0) mask[(size_t)mt * kblocks + kb] = nz ? 1 : 0;
}

// K-block lists of a member from its block mask; an M tile without any
// non-zero block keeps block 0 (all zero) so that its accumulator is written.
static si_status member_block_lists(Group *g, GroupMember &x) {
    const int mtiles = x.mpad / GR_BM, kblocks = x.ldk / GR_BK;
    unsigned char *d_mask = nullptr;
    SI_CUDA_TRY(si_dev_malloc((void **)&d_mask, (size_t)mtiles * kblocks));
    if (x.e4m3)
        k_block_nonzero<unsigned char><<<dim3(kblocks, mtiles), 256, 0, g->stream>>>(
            (const unsigned char *)x.J, x.ldk, kblocks, d_mask);
    else
        k_block_nonzero<unsigned short><<<dim3(kblocks, mtiles), 256, 0, g->stream>>>(
            (const unsigned short *)x.J, x.ldk, kblocks, d_mask);
    cudaError_t e = cudaGetLastError();
    std::vector<unsigned char> mask((size_t)mtiles * kblocks);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mask.data(), d_mask, mask.size(), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFree(d_mask);
    SI_CUDA_TRY(e);
    x.kb_off.assign(mtiles, 0);
    x.kb_cnt.assign(mtiles, 0);
    for (int mt = 0; mt < mtiles; ++mt) {
        x.kb_off[mt] = (int)g->kbl.size();
        for (int kb = 0; kb < kblocks; ++kb)
            if (mask[(size_t)mt * kblocks + kb]) g->kbl.push_back(kb);
        if ((int)g->kbl.size() == x.kb_off[mt]) g->kbl.push_back(0);
        x.kb_cnt[mt] = (int)g->kbl.size() - x.kb_off[mt];
    }
    return SI_OK;
}

// Tile cost model: a K block moves its J tile and bn replica rows through
// shared memory twice (TMA write, MMA read), 16 KB + bn * 128 B each way.
static int tile_cost(int kb_cnt, int bn) { return kb_cnt * (128 + bn); }
static bool half_width(int bn) { return bn % 32 == 0 && bn >= 32; }

// Round-robin makespan of a cost-sorted tile list on `grid` CTAs (the kernel
// walks the list with stride gridDim.x).
static long long rr_makespan(const std::vector<GroupTile> &t, int grid) {
    std::vector<long long> load((size_t)grid, 0);
    for (size_t k = 0; k < t.size(); ++k) load[k % grid] += t[k].cost;
    return *std::max_element(load.begin(), load.end());
}

static void sort_tiles(std::vector<GroupTile> &t) {
    // Longest first; tiles of one M slab stay adjacent so that concurrent
    // replica blocks share the J slab through L2.
    std::stable_sort(t.begin(), t.end(), [](const GroupTile &x, const GroupTile &y) { return x.cost > y.cost; });
}

// The last wave of equal tiles leaves most CTAs idle (N=32768, R=512: 512
// tiles on 152 CTAs, 4 waves for some, 3 for the rest), and a list shorter
// than the grid leaves CTAs without work.  Splitting the cheapest s tiles
// into two tiles of half the replicas fills them: try a range of s and keep
// the list with the smallest round-robin makespan.
static void balance_tiles(std::vector<GroupTile> &tiles, int grid) {
    sort_tiles(tiles);
    if (grid <= 0 || tiles.empty()) return;
    std::vector<GroupTile> best = tiles;
    long long best_ms = rr_makespan(tiles, grid);
    const int T = (int)tiles.size();
    const int step = std::max(1, T / 128);
    for (int sidx = step; sidx <= T; sidx += step) {
        std::vector<GroupTile> cand;
        cand.reserve((size_t)T + sidx);
        int split = 0;
        for (int k = T - 1; k >= 0; --k) {
            const GroupTile &x = tiles[k];
            if (split < sidx && half_width(x.bn)) {
                GroupTile a = x, b = x;
                a.bn = b.bn = x.bn / 2;
                b.r0 = x.r0 + a.bn;
                a.cost = b.cost = tile_cost(x.kb_cnt, a.bn);
                cand.push_back(a);
                cand.push_back(b);
                ++split;
            } else {
                cand.push_back(x);
            }
        }
        sort_tiles(cand);
        const long long ms = rr_makespan(cand, grid);
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    tiles.swap(best);
}

// Build, once at creation, the instance table, tensor maps and tile list of
// every tile policy (device tables are never rewritten after a launch used
// them); group_apply_policy only selects one.
static si_status group_build_policies(Group *g) {
    const int c = g->count;
    std::vector<GroupInst> inst((size_t)kPolicies * c);
    std::vector<CUtensorMap> maps((size_t)kPolicies * 3 * c);
    std::vector<std::vector<GroupTile>> tiles(kPolicies);
    for (int pol = 0; pol < kPolicies; ++pol) {
        std::vector<int> bns;
        for (int i = 0; i < c; ++i) bns.push_back(policy_bn(pol, g->m[i].R, g->any_e4m3));
        policy_ring(pol, bns, &g->pol_stages[pol], &g->pol_stage_bytes[pol]);
        for (int i = 0; i < c; ++i) {
            GroupMember &x = g->m[i];
            GroupInst &d = inst[(size_t)pol * c + i];
            d.n = x.n;
            d.R = x.R;
            d.ldk = x.ldk;
            d.bn = policy_bn(pol, x.R, g->any_e4m3);
            d.rpad = x.rpad_max;
            d.mtiles = x.mpad / GR_BM;
            d.rblocks = cdiv(x.R, d.bn);
            d.kblocks = x.ldk / GR_BK;
            d.e4m3 = x.e4m3 ? 1 : 0;
            d.h = x.h;
            d.q_state = x.q;
            d.p_state = x.p;
            d.qop = x.qop;
            d.spins = x.spins;
            d.lds = x.lds;
            CUtensorMap *mp = &maps[((size_t)pol * c + i) * 3];
            si_status s = x.e4m3 ? tc_make_map_e4m3(mp, x.J, x.ldk, x.mpad, GR_BM)
                                 : tc_make_map_bf16(mp, x.J, x.ldk, x.mpad, GR_BK, GR_BM);
            if (s != SI_OK) return s;
            s = tc_make_map_bf16(mp + 1, x.qop, x.ldk, 2 * x.rpad_max, GR_BK, d.bn);
            if (s != SI_OK) return s;
            s = tc_make_map_bf16(mp + 2, x.qop, x.ldk, 2 * x.rpad_max, GR_BK, half_width(d.bn) ? d.bn / 2 : d.bn);
            if (s != SI_OK) return s;
            for (int mt = 0; mt < d.mtiles; ++mt)
                for (int rb = 0; rb < d.rblocks; ++rb)
                    tiles[pol].push_back(GroupTile{i, mt, rb * d.bn, d.bn, tile_cost(x.kb_cnt[mt], d.bn),
                                                   x.kb_off[mt], x.kb_cnt[mt]});
        }
        balance_tiles(tiles[pol], g->sms);
    }
    size_t ntot = 0;
    for (auto &v : tiles) ntot += v.size();
    SI_CUDA_TRY(si_dev_malloc((void **)&g->d_inst, sizeof(GroupInst) * inst.size()));
    SI_CUDA_TRY(si_dev_malloc((void **)&g->d_maps, sizeof(CUtensorMap) * maps.size()));
    SI_CUDA_TRY(si_dev_malloc((void **)&g->d_tiles, sizeof(GroupTile) * ntot));
    SI_CUDA_TRY(si_dev_malloc((void **)&g->d_kbl, sizeof(int) * std::max<size_t>(1, g->kbl.size())));
    SI_CUDA_TRY(cudaMemcpyAsync(g->d_kbl, g->kbl.data(), sizeof(int) * g->kbl.size(), cudaMemcpyHostToDevice,
                                g->stream));
    SI_CUDA_TRY(cudaMemcpyAsync(g->d_inst, inst.data(), sizeof(GroupInst) * inst.size(), cudaMemcpyHostToDevice,
                                g->stream));
    SI_CUDA_TRY(cudaMemcpyAsync(g->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                                g->stream));
    size_t off = 0;
    for (int pol = 0; pol < kPolicies; ++pol) {
        SI_CUDA_TRY(cudaMemcpyAsync(g->d_tiles + off, tiles[pol].data(), sizeof(GroupTile) * tiles[pol].size(),
                                    cudaMemcpyHostToDevice, g->stream));
        g->pol_tiles_off[pol] = (int)off;
        g->pol_ntiles[pol] = (int)tiles[pol].size();
        off += tiles[pol].size();
    }
    SI_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return SI_OK;
}

static si_status group_apply_policy(Group *g, int policy) {
    g->policy = policy;
    g->ntiles = g->pol_ntiles[policy];
    if (g->graph) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
        g->graph_steps = -1;
    }
    return SI_OK;
}

static si_status group_launch_step(Group *g, int t, int steps) {
    GroupArgs a;
    a.inst = g->d_inst + (size_t)g->policy * g->count;
    a.tiles = g->d_tiles + g->pol_tiles_off[g->policy];
    a.ntiles = g->ntiles;
    a.maps = g->d_maps + (size_t)g->policy * 3 * g->count;
    a.kbl = g->d_kbl;
    a.zeta = g->d_zeta;
    a.dt = g->d_dt;
    a.t = t;
    a.last = (t == steps - 1) ? 1 : 0;
    a.sp = StepParams{g->common.k, g->common.m, g->common.q0, g->common.q_max, g->common.p_max,
                      g->common.update_order, g->common.wall_zero_p};
    a.err = g->d_err;
    a.limit_ns = g->limit_ns;
    a.single = (g->policy == kPolicyWhole || g->policy == kPolicyWholeTmemA) ? 1 : 0;
    a.tmem_a = g->policy == kPolicyWholeTmemA ? 1 : 0;
    a.nslots = g->policy == kPolicyWholeTmemA ? 1 : 2;
    a.stages = g->pol_stages[g->policy];
    a.stage_bytes = g->pol_stage_bytes[g->policy];
    if (g->any_e4m3) k_group_step<true><<<g->grid, gr_threads<true>(), GR_SMEM, g->stream>>>(a);
    else k_group_step<false><<<g->grid, gr_threads<false>(), GR_SMEM, g->stream>>>(a);
    SI_CUDA_TRY(cudaGetLastError());
    return SI_OK;
}

// Capture the T step launches into a CUDA graph (once per step count/policy).
static si_status group_graph(Group *g, int steps) {
    if (g->graph && g->graph_steps == steps) return SI_OK;
    if (g->graph) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    cudaStream_t cs;
    SI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = g->stream;
    g->stream = cs;
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    si_status s = SI_OK;
    if (e == cudaSuccess) {
        for (int t = 0; t < steps && s == SI_OK; ++t) s = group_launch_step(g, t, steps);
        e = cudaStreamEndCapture(cs, &graph);
    }
    g->stream = saved;
    cudaStreamDestroy(cs);
    if (s != SI_OK) return s;
    SI_CUDA_TRY(e);
    e = cudaGraphInstantiate(&g->graph, graph, 0);
    cudaGraphDestroy(graph);
    SI_CUDA_TRY(e);
    g->graph_steps = steps;
    return SI_OK;
}

static si_status group_check_err(Group *g) {
    int local = 0;
    int *dst = g->h_err ? g->h_err : &local;
    SI_CUDA_TRY(cudaMemcpyAsync(dst, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    SI_CUDA_TRY(cudaStreamSynchronize(g->stream));
    const int herr = *dst;
    if (herr != DEV_OK) {
        SI_CUDA_TRY(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream));
        SI_CUDA_TRY(cudaStreamSynchronize(g->stream));
        set_error("grouped step: an mbarrier wait timed out");
        return SI_ERR_TIMEOUT;
    }
    return SI_OK;
}

// Time `steps` uncaptured launches of a policy (autotuner).
static si_status group_time_policy(Group *g, int policy, int steps, float *ms) {
    si_status s = group_apply_policy(g, policy);
    if (s != SI_OK) return s;
    cudaEvent_t e0, e1;
    SI_CUDA_TRY(cudaEventCreate(&e0));
    SI_CUDA_TRY(cudaEventCreate(&e1));
    // warm-up step, then timed steps (states evolve; timing does not depend on values)
    s = group_launch_step(g, 0, g->steps + 1);
    SI_CUDA_TRY(cudaEventRecord(e0, g->stream));
    for (int t = 0; t < steps && s == SI_OK; ++t) s = group_launch_step(g, t % std::max(1, g->steps), g->steps + 1);
    SI_CUDA_TRY(cudaEventRecord(e1, g->stream));
    SI_CUDA_TRY(cudaEventSynchronize(e1));
    SI_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != SI_OK) return s;
    return group_check_err(g);
}

// SI_GROUP_POLICY=<index> pins the tile policy (over the autotuner and its
// cache); a negative value skips the timing and takes policy 0.
static int forced_policy() {
    const char *env = std::getenv("SI_GROUP_POLICY");
    if (!env) return -1;
    const int v = std::atoi(env);
    return v < kPolicies ? v : -1;
}

static si_status group_autotune(Group *g) {
    const std::string key = group_key(g);
    {
        int cached = -1;
        if (tune_cache_find(key, &cached)) return group_apply_policy(g, cached);
    }
    int best = 0;
    const char *env = std::getenv("SI_GROUP_POLICY");
    if (env && std::atoi(env) >= 0 && std::atoi(env) < kPolicies) {
        best = std::atoi(env);
    } else if (!(env && std::atoi(env) < 0)) {
        float best_ms = 1e30f;
        for (int pol = 0; pol < kPolicies; ++pol) {
            if (pol == kPolicyWholeTmemA && !g->any_e4m3) continue;   // only differs for e4m3 members
            float ms = 0.f;
            si_status s = group_time_policy(g, pol, 3, &ms);
            if (s != SI_OK) return s;
            if (ms < best_ms) {
                best_ms = ms;
                best = pol;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
        if (!env) tune_file_store_locked(key, best);
    }
    return group_apply_policy(g, best);
}

static void free_group(Group *g) {
    if (!g) return;
    for (auto &x : g->m) {
        void *ptrs[] = {x.J, x.h, x.q, x.p, x.qop, x.own_spins ? x.spins : nullptr, x.energy.dJ8, x.energy.dh8,
                        x.energy.dspins_in, x.energy.e_sig, x.energy.e_sum};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    void *ptrs[] = {g->d_inst, g->d_tiles, g->d_maps, g->d_kbl, g->d_zeta, g->d_dt, g->host ? nullptr : g->d_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (g->h_err) cudaFreeHost(g->h_err);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

static si_status group_create_impl(Group *g, const si_params *prm, const float *const *J,
                                   const float *const *h) {
    SI_CUDA_TRY(cudaGetDevice(&g->device));
    SI_CUDA_TRY(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device));
    if (const char *e = std::getenv("SI_SPIN_LIMIT_NS")) {
        long long v = std::atoll(e);
        if (v > 0) g->limit_ns = v;
    }
    g->m.resize(g->count);
    for (int i = 0; i < g->count; ++i) {
        GroupMember &x = g->m[i];
        const int n = prm[i].n;
        x.n = n;
        x.R = prm[i].replicas;
        x.ldk = round_up(n, GR_BK);
        x.mpad = round_up(n, GR_BM);
        x.rpad_max = std::max(round_up(x.R, 128), round_up(x.R, 16) <= 256 ? round_up(x.R, 16) : round_up(x.R, 256));
        const float *Jp = J[i];
        const float *hp = h ? h[i] : nullptr;
        // device copies of host J / h for this member, freed on every exit
        struct DevTmp {
            void *p = nullptr;
            ~DevTmp() {
                if (p) cudaFree(p);
            }
        } Jtmp, htmp;
        if (!is_device_ptr(Jp)) {
            SI_CUDA_TRY(si_dev_malloc(&Jtmp.p, sizeof(float) * (size_t)n * n));
            SI_CUDA_TRY(cudaMemcpyAsync(Jtmp.p, Jp, sizeof(float) * (size_t)n * n, cudaMemcpyDefault, g->stream));
            Jp = (const float *)Jtmp.p;
        }
        if (hp && !is_device_ptr(hp)) {
            SI_CUDA_TRY(si_dev_malloc(&htmp.p, sizeof(float) * n));
            SI_CUDA_TRY(cudaMemcpyAsync(htmp.p, hp, sizeof(float) * n, cudaMemcpyDefault, g->stream));
            hp = (const float *)htmp.p;
        }
        unsigned long long flags = 0;
        long long s_upper = 0;
        si_status s = simt_validate(Jp, hp, n, prm[i].prec, &flags, &s_upper, g->stream);
        if (s != SI_OK) return s;
        if (flags & (VF_NONFINITE | VF_H_NONFINITE)) {
            set_error("group member " + std::to_string(i) + ": J or h holds a non-finite value");
            return SI_ERR_INVALID_ARG;
        }
        if (flags & (VF_ASYM | VF_DIAG)) {
            set_error("group member " + std::to_string(i) + ": J must be symmetric with a zero diagonal");
            return SI_ERR_NOT_SYMMETRIC;
        }
        if (prm[i].prec == SI_PREC_J_FP8_Q_BF16 && (flags & VF_NOT_E4M3)) {
            set_error("group member " + std::to_string(i) + ": SI_PREC_J_FP8_Q_BF16 needs J exact in e4m3");
            return SI_ERR_INVALID_ARG;
        }
        x.e4m3 = prm[i].prec == SI_PREC_J_FP8_Q_BF16;
        SI_CUDA_TRY(si_dev_malloc(&x.J, (size_t)x.mpad * x.ldk * (x.e4m3 ? 1 : 2)));
        s = x.e4m3 ? tc_convert_j_e4m3(Jp, n, x.J, x.ldk, x.mpad, g->sms, g->stream)
                   : tc_convert_j(Jp, n, x.J, x.ldk, x.mpad, g->sms, g->stream);
        if (s != SI_OK) return s;
        // block sparsity: all-zero 128 x 64 blocks of J are never loaded
        s = member_block_lists(g, x);
        if (s != SI_OK) return s;
        SI_CUDA_TRY(si_dev_malloc((void **)&x.q, sizeof(float) * (size_t)x.R * n));
        SI_CUDA_TRY(si_dev_malloc((void **)&x.p, sizeof(float) * (size_t)x.R * n));
        if (g->host) {
            x.spins = g->host->dspins;
            x.lds = g->host->ld8;
            x.own_spins = false;
        } else {
            SI_CUDA_TRY(si_dev_malloc((void **)&x.spins, (size_t)x.R * n));
            x.lds = n;
        }
        const size_t qb = 2ull * x.rpad_max * x.ldk * 2;
        SI_CUDA_TRY(si_dev_malloc((void **)&x.qop, qb));
        SI_CUDA_TRY(cudaMemsetAsync(x.qop, 0, qb, g->stream));
        // readout view for si_group_energy
        Ctx &c = x.energy;
        c.prm = prm[i];
        c.stream = g->stream;
        c.device = g->device;
        c.num_sms = g->sms;
        c.n = n;
        c.R = x.R;
        c.path = Path::TENSOR;
        c.integer_j = !(flags & VF_NOT_INT8);
        c.has_h = hp != nullptr;
        c.integer_h = !(flags & VF_H_NOT_INT8);
        c.s_upper = c.integer_j ? s_upper : 0;
        c.ld8 = round_up(n, 16);
        c.dJ = x.J;
        c.j_e4m3 = x.e4m3;
        c.ldk = x.ldk;
        c.mpad = x.mpad;
        SI_CUDA_TRY(si_dev_malloc((void **)&x.h, sizeof(float) * n));
        if (hp) SI_CUDA_TRY(cudaMemcpyAsync(x.h, hp, sizeof(float) * n, cudaMemcpyDeviceToDevice, g->stream));
        else SI_CUDA_TRY(cudaMemsetAsync(x.h, 0, sizeof(float) * n, g->stream));
        c.dhf = x.h;
        if (c.integer_j && !g->host) {
            SI_CUDA_TRY(si_dev_malloc((void **)&c.dJ8, (size_t)n * c.ld8));
            s = convert_j8(&c, Jp);
            if (s != SI_OK) return s;
        }
        if (c.has_h && c.integer_h && !g->host) {
            SI_CUDA_TRY(si_dev_malloc((void **)&c.dh8, n));
            s = h_to_int8(hp, n, c.dh8, g->stream);
            if (s != SI_OK) return s;
        }
        SI_CUDA_TRY(cudaStreamSynchronize(g->stream));
        if (!hp) {
            cudaFree(x.h);
            x.h = nullptr;
            c.dhf = nullptr;
        }
    }
    for (const auto &x : g->m) g->any_e4m3 = g->any_e4m3 || x.e4m3;
    si_status sb = group_build_policies(g);
    if (sb != SI_OK) return sb;
    SI_CUDA_TRY(si_dev_malloc((void **)&g->d_zeta, sizeof(float) * std::max(1, g->steps)));
    SI_CUDA_TRY(si_dev_malloc((void **)&g->d_dt, sizeof(float) * std::max(1, g->steps)));
    if (g->host) {
        g->d_err = g->host->derr;
    } else {
        SI_CUDA_TRY(si_dev_malloc((void **)&g->d_err, sizeof(int)));
        SI_CUDA_TRY(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream));
    }
    if (cudaHostAlloc((void **)&g->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();   // optional: the read then goes through pageable memory
        g->h_err = nullptr;
    }
    for (auto &x : g->m) {            // readout views share the group's error word
        x.energy.derr = g->d_err;
        x.energy.spin_limit_ns = g->limit_ns;
    }
    // the converter warps exist only in groups with e4m3 members
    int per_sm = 0;
    if (g->any_e4m3) {
        SI_CUDA_TRY(cudaFuncSetAttribute(k_group_step<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, GR_SMEM));
        SI_CUDA_TRY(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group_step<true>, gr_threads<true>(), GR_SMEM));
    } else {
        SI_CUDA_TRY(cudaFuncSetAttribute(k_group_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, GR_SMEM));
        SI_CUDA_TRY(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group_step<false>, gr_threads<false>(), GR_SMEM));
    }
    if (per_sm < 1) {
        set_error("grouped step kernel does not fit on an SM");
        return SI_ERR_UNSUPPORTED;
    }
    g->grid = per_sm * g->sms;
    return group_apply_policy(g, 0);
}

// ------------------------------------------------ serving one si_create context
// A tensor-precision context whose persistent grid would not be co-resident
// (many M tiles x replica blocks, e.g. n = 32768) runs on this grouped step
// kernel as a one-member group: one launch per time step from a CUDA graph.
// The member's J copy and FP32 state are the context's (c->dJ, c->dq, c->dp
// point at them), its last step writes the context's padded spin buffer, and
// its waits raise the context's error word, so every other call of the
// context (readouts, state copies, continuation) works unchanged.
si_status group_ctx_create(Ctx *c, const float *J_dev, const float *h_dev) {
    Group *g = new (std::nothrow) Group();
    if (!g) return SI_ERR_OOM;
    c->grp = g;   // released by group_ctx_free, also after a failure below
    g->count = 1;
    g->steps = c->prm.steps;
    g->common = c->prm;
    g->stream = c->stream;
    g->host = c;
    const float *Js[1] = {J_dev};
    const float *hs[1] = {h_dev};
    si_status s = group_create_impl(g, &c->prm, Js, h_dev ? hs : nullptr);
    if (s != SI_OK) return s;
    GroupMember &x = g->m[0];
    c->dJ = x.J;
    c->j_e4m3 = x.e4m3;
    c->ldk = x.ldk;
    c->mpad = x.mpad;
    c->dq = x.q;
    c->dp = x.p;
    c->rpad = x.rpad_max;
    // Choose the tile policy now, on zeroed scratch state (timing does not
    // depend on the values; the first si_run loads its own state).
    const size_t bytes = sizeof(float) * (size_t)x.R * x.n;
    SI_CUDA_TRY(cudaMemsetAsync(x.q, 0, bytes, g->stream));
    SI_CUDA_TRY(cudaMemsetAsync(x.p, 0, bytes, g->stream));
    SI_CUDA_TRY(cudaMemsetAsync(g->d_zeta, 0, sizeof(float) * std::max(1, g->steps), g->stream));
    SI_CUDA_TRY(cudaMemsetAsync(g->d_dt, 0, sizeof(float) * std::max(1, g->steps), g->stream));
    int cached = forced_policy();
    if (cached < 0) tune_cache_find(group_key(g), &cached);
    if (cached >= 0) return group_apply_policy(g, cached);
    if (g->steps == 0) return group_apply_policy(g, 0);
    return group_autotune(g);
}

// Start a run: the FP32 state is already in c->dq / c->dp (loaded by the
// caller, or left by the last run); copy the schedule and build the bf16
// operand plane of step 0 from the positions.
si_status group_ctx_prepare(Ctx *c, int steps) {
    Group *g = c->grp;
    if (steps > 0) {
        SI_CUDA_TRY(cudaMemcpyAsync(g->d_zeta, c->dzeta, sizeof(float) * steps, cudaMemcpyDeviceToDevice, g->stream));
        SI_CUDA_TRY(cudaMemcpyAsync(g->d_dt, c->ddt, sizeof(float) * steps, cudaMemcpyDeviceToDevice, g->stream));
    }
    const GroupMember &x = g->m[0];
    dim3 grid(std::min(8 * g->sms, std::max(1, cdiv((long long)x.R * x.n, 256))), 1);
    k_group_init<<<grid, 256, 0, g->stream>>>(g->d_inst + (size_t)g->policy * g->count);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

// The `steps` time steps (one graph launch; asynchronous).
si_status group_ctx_run(Ctx *c, int steps) {
    Group *g = c->grp;
    if (steps == 0) return SI_OK;
    si_status s = group_graph(g, steps);
    if (s != SI_OK) return s;
    SI_CUDA_TRY(cudaGraphLaunch(g->graph, g->stream));
    c->launches += steps;
    return SI_OK;
}

// After si_set_params: the captured steps hold the old integrator values.
void group_ctx_params(Ctx *c) {
    Group *g = c->grp;
    g->common = c->prm;
    if (g->graph) {
        cudaStreamSynchronize(g->stream);
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
        g->graph_steps = -1;
    }
}

void group_ctx_describe(const Ctx *c, char *buf, int len) {
    const Group *g = c->grp;
    const GroupMember &x = g->m[0];
    std::snprintf(buf, len,
                  "tcgen05 grouped-step prec=%s J=%s n=%d R=%d tiles=%d grid=%d policy=%s (one launch per step, "
                  "CUDA graph)",
                  c->prm.prec == SI_PREC_J_FP8_Q_BF16 ? "j_fp8_q_bf16" : "j_bf16_q_bf16",
                  x.e4m3 ? "e4m3(1B)" : "bf16(2B)", c->n, c->R, g->ntiles, g->grid,
                  g->policy >= 0 ? kPolicyName[g->policy] : "none");
}

void group_ctx_free(Ctx *c) {
    if (!c->grp) return;
    // the member owns J and the state that the context's pointers alias
    c->dJ = nullptr;
    c->dq = nullptr;
    c->dp = nullptr;
    free_group(c->grp);
    c->grp = nullptr;
}

}  // namespace si

using namespace si;

extern "C" {

si_status si_create_group(si_group **out, int32_t count, const si_params *prm, const float *const *J,
                          const float *const *h, void *stream) {
    NvtxRange nvtx_range("si_create_group");
    alloc_fault_reset();
    set_error("");
    if (!out || count < 1 || !prm || !J) {
        set_error("si_create_group: out, count >= 1, prm[count] and J[count] are required");
        return SI_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const si_params &p = prm[i];
        if (!J[i] || p.n < 1 || p.replicas < 1 || p.steps < 0) {
            set_error("si_create_group: member " + std::to_string(i) + " needs J, n >= 1, replicas >= 1");
            return SI_ERR_INVALID_ARG;
        }
        if (p.prec != SI_PREC_J_FP8_Q_BF16 && p.prec != SI_PREC_J_BF16_Q_BF16) {
            set_error("si_create_group: members use the tensor-core precisions");
            return SI_ERR_UNSUPPORTED;
        }
        if (p.steps != prm[0].steps || p.k != prm[0].k || p.m != prm[0].m || p.q0 != prm[0].q0 ||
            p.q_max != prm[0].q_max || p.p_max != prm[0].p_max || p.update_order != prm[0].update_order ||
            p.wall_zero_p != prm[0].wall_zero_p) {
            set_error("si_create_group: steps and integrator parameters must be equal across members");
            return SI_ERR_INVALID_ARG;
        }
        if (!(p.m > 0.f) || !(p.q_max > 0.f) || !(p.p_max > 0.f) || (p.update_order != 0 && p.update_order != 1)) {
            set_error("si_create_group: need m, q_max, p_max > 0 and order 0 or 1");
            return SI_ERR_INVALID_ARG;
        }
    }
    Group *g = new (std::nothrow) Group();
    if (!g) return SI_ERR_OOM;
    g->count = count;
    g->steps = prm[0].steps;
    g->common = prm[0];
    g->stream = (cudaStream_t)stream;
    si_status s = group_create_impl(g, prm, J, h);
    if (s != SI_OK) {
        free_group(g);
        return s;
    }
    *out = reinterpret_cast<si_group *>(g);
    return SI_OK;
}

si_status si_run_group(si_group *grp, const float *zeta, const float *dt, const float *const *q_init,
                       const float *const *p_init, float *const *q_out, float *const *p_out,
                       int8_t *const *spins_out) {
    NvtxRange nvtx_range("si_run_group");
    set_error("");
    Group *g = reinterpret_cast<Group *>(grp);
    if (!g || !q_init || (g->steps > 0 && (!zeta || !dt))) {
        set_error("si_run_group: group, q_init[count], zeta and dt are required");
        return SI_ERR_INVALID_ARG;
    }
    for (int i = 0; i < g->count; ++i)
        if (!q_init[i]) {
            set_error("si_run_group: q_init[" + std::to_string(i) + "] is NULL");
            return SI_ERR_INVALID_ARG;
        }
    g->launches = 0;
    const int steps = g->steps;
    if (steps > 0) {
        SI_CUDA_TRY(cudaMemcpyAsync(g->d_zeta, zeta, sizeof(float) * steps, cudaMemcpyDefault, g->stream));
        SI_CUDA_TRY(cudaMemcpyAsync(g->d_dt, dt, sizeof(float) * steps, cudaMemcpyDefault, g->stream));
    }
    auto load_state = [&]() -> si_status {
        for (int i = 0; i < g->count; ++i) {
            GroupMember &x = g->m[i];
            const size_t bytes = sizeof(float) * (size_t)x.R * x.n;
            SI_CUDA_TRY(cudaMemcpyAsync(x.q, q_init[i], bytes, cudaMemcpyDefault, g->stream));
            if (p_init && p_init[i]) SI_CUDA_TRY(cudaMemcpyAsync(x.p, p_init[i], bytes, cudaMemcpyDefault, g->stream));
            else SI_CUDA_TRY(cudaMemsetAsync(x.p, 0, bytes, g->stream));
        }
        int maxnr = 1;
        for (auto &x : g->m) maxnr = std::max(maxnr, x.R * x.n);
        dim3 grid(std::min(64, cdiv(maxnr, 256)), g->count);
        k_group_init<<<grid, 256, 0, g->stream>>>(g->d_inst);
        SI_CUDA_TRY(cudaGetLastError());
        g->launches += 1;
        return SI_OK;
    };
    si_status s;
    if (steps > 0) {
        int cached = forced_policy();
        if (cached < 0) {
            tune_cache_find(group_key(g), &cached);
        }
        if (cached < 0) {
            // autotune once per group shape, on the real data as scratch state
            if ((s = load_state()) != SI_OK) return s;
            if ((s = group_autotune(g)) != SI_OK) return s;
        } else if (g->policy != cached) {
            if ((s = group_apply_policy(g, cached)) != SI_OK) return s;
        }
    }
    if ((s = load_state()) != SI_OK) return s;
    g->ev_valid = false;
    if (steps > 0) {
        if ((s = group_graph(g, steps)) != SI_OK) return s;
        if (g->timing) SI_CUDA_TRY(cudaEventRecord(g->ev0, g->stream));
        SI_CUDA_TRY(cudaGraphLaunch(g->graph, g->stream));
        if (g->timing) {
            SI_CUDA_TRY(cudaEventRecord(g->ev1, g->stream));
            g->ev_valid = true;
        }
        g->launches += steps;
    }
    if ((s = group_check_err(g)) != SI_OK) return s;
    for (int i = 0; i < g->count; ++i) {
        GroupMember &x = g->m[i];
        const size_t bytes = sizeof(float) * (size_t)x.R * x.n;
        if (q_out && q_out[i]) SI_CUDA_TRY(cudaMemcpyAsync(q_out[i], x.q, bytes, cudaMemcpyDefault, g->stream));
        if (p_out && p_out[i]) SI_CUDA_TRY(cudaMemcpyAsync(p_out[i], x.p, bytes, cudaMemcpyDefault, g->stream));
        if (spins_out && spins_out[i]) {
            if (steps == 0) {
                set_error("si_run_group: spins need steps >= 1");
                return SI_ERR_INVALID_ARG;
            }
            SI_CUDA_TRY(cudaMemcpyAsync(spins_out[i], x.spins, (size_t)x.R * x.n, cudaMemcpyDefault, g->stream));
        }
    }
    SI_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return SI_OK;
}

si_status si_group_energy(si_group *grp, int32_t index, const int8_t *spins, int32_t R, int32_t *energy_out,
                          int32_t *cut_out, double *energy_f) {
    NvtxRange nvtx_range("si_group_energy");
    Group *g = reinterpret_cast<Group *>(grp);
    if (!g || index < 0 || index >= g->count) {
        set_error("si_group_energy: bad group or index");
        return SI_ERR_INVALID_ARG;
    }
    return si_energy(reinterpret_cast<si_ctx *>(&g->m[index].energy), spins, R, energy_out, cut_out, energy_f);
}

si_status si_group_enable_timing(si_group *grp, int32_t on) {
    Group *g = reinterpret_cast<Group *>(grp);
    if (!g) return SI_ERR_INVALID_ARG;
    if (on && !g->ev0) {
        SI_CUDA_TRY(cudaEventCreate(&g->ev0));
        SI_CUDA_TRY(cudaEventCreate(&g->ev1));
    }
    g->timing = on != 0;
    return SI_OK;
}

si_status si_group_last_kernel_time(const si_group *grp, float *ms) {
    const Group *g = reinterpret_cast<const Group *>(grp);
    if (!g || !ms || !g->ev_valid) {
        set_error("si_group_last_kernel_time: no timed run");
        return SI_ERR_INVALID_ARG;
    }
    SI_CUDA_TRY(cudaEventSynchronize(g->ev1));
    SI_CUDA_TRY(cudaEventElapsedTime(ms, g->ev0, g->ev1));
    return SI_OK;
}

si_status si_group_describe(const si_group *grp, char *buf, int32_t len) {
    const Group *g = reinterpret_cast<const Group *>(grp);
    if (!g || !buf || len <= 0) return SI_ERR_INVALID_ARG;
    long long macs = 0, jbytes = 0;
    for (const auto &x : g->m) {
        const int bn = policy_bn(g->policy, x.R, g->any_e4m3);
        macs += (long long)x.n * x.n * x.R;
        long long nb = 0;
        for (int v : x.kb_cnt) nb += v;
        jbytes += nb * GR_BM * GR_BK * (x.e4m3 ? 1 : 2) * cdiv(x.R, bn);
    }
    std::snprintf(buf, len, "grouped tcgen05 count=%d tiles=%d grid=%d policy=%s graph-steps=%d macs/step=%lld jbytes/step=%lld",
                  g->count, g->ntiles, g->grid, g->policy >= 0 ? kPolicyName[g->policy] : "none", g->graph_steps,
                  macs, jbytes);
    return SI_OK;
}

int32_t si_group_last_launch_count(const si_group *grp) {
    const Group *g = reinterpret_cast<const Group *>(grp);
    return g ? g->launches : 0;
}

void si_destroy_group(si_group *grp) {
    Group *g = reinterpret_cast<Group *>(grp);
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    free_group(g);
}

}  // extern "C"
