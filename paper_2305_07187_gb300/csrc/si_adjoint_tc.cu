// Tensor-core products of the adjoint sweep (FP32 contexts whose J is exact
// in bf16, e.g. +-1 or bf16-rounded Gaussian couplings).
//
// Each step of the reverse sweep needs G = J X^T twice (the recomputed
// forward force J q_t and the adjoint product J lambda_a) over R replicas.
// With J exact in bf16, the FP32 operand X is split into three bf16 pieces
// x = x_hi + x_mid + x_lo (each the round-to-nearest bf16 of the remaining
// residual, so the pieces carry the 24-bit significand); every product
// J_ij * piece is exact in FP32 and the tensor cores accumulate in FP32.  The
// result carries the rounding of an FP32 dot product, against the bf16 error
// that a single-piece operand would add.
//
// Tile: 128 rows of J x 64 replicas; the B operand holds the three pieces of
// the 64 replicas as 192 rows, so one kind::f16 MMA of N = 192 computes all
// three partial products into one TMEM accumulator and the epilogue adds
// them, (hi + mid) + lo.  The K dimension is split over the CTAs of a thread
// block cluster to fill the GPU (N = 2000, R = 64 has only 16 tiles): each
// split leaves its FP32 partial tile in its own shared memory, and after a
// cluster barrier every CTA adds, through distributed shared memory and in
// split order (deterministic), the partials of its own slice of replicas
// and applies the step's epilogue to that slice: the forward integrator
// step, the terminal adjoint, or the adjoint update.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "si_device.cuh"
#include "si_tcgen05.cuh"

namespace si {

constexpr int AT_BM = 128, AT_BK = 64, AT_RB = ADJ_TC_RB;
constexpr int AT_BN = ADJ_TC_BN;                         // 192 MMA columns: 64 replicas x 3 pieces
constexpr int AT_A_BYTES = AT_BM * AT_BK * 2;            // 16 KB
constexpr int AT_B_BYTES = AT_BN * AT_BK * 2;            // 24 KB
constexpr int AT_STAGE = AT_A_BYTES + AT_B_BYTES;        // 40 KB, multiple of 1024
constexpr int AT_S = 4;
constexpr int AT_THREADS = 192;                          // producer, MMA, 4 epilogue warps
constexpr int AT_TILES = AT_S * AT_STAGE;
constexpr int AT_NBARS = 2 * AT_S + 2;                   // full, empty, accf, drain
constexpr int AT_MISC = 1024;                            // barriers, flags, reduction scratch
constexpr int AT_RECV = AT_RB * AT_BM * 4;               // 32 KB: partials pushed by the cluster
constexpr int AT_SMEM = AT_TILES + AT_MISC + AT_RECV + 1024;
static_assert(AT_NBARS * 8 + 16 + AT_BM * 4 <= AT_MISC, "misc area too small");
static_assert(AT_STAGE % 1024 == 0, "stages must keep the 1024-byte swizzle alignment");

enum { AT_FORWARD = 0, AT_TERMINAL = 1, AT_ADJOINT = 2 };

struct AdjTc {
    int n, R, ld, ldk, mpad, mtiles, nrb, kblocks, kb_per, splits;
    // persistent sweep (k_adj_run): cluster size, K blocks per split, and
    // whether a recompute chain and a reverse chain fit side by side
    int run_splits = 0, run_kb_per = 0;
    bool run_pair = false;
    unsigned *run_flags = nullptr;  // [2][mtiles * nrb] slices published, per chain
    __nv_bfloat16 *jb = nullptr;    // [mpad][ldk]
    // [4][nrb * 192][ldk]: per-step sweep: forward chain (buffers 0, 1),
    // lambda_a (2); persistent sweep: forward chain (0, 1), reverse chain (2, 3)
    __nv_bfloat16 *xs = nullptr;
    CUtensorMap mapA, mapB;
};

struct AdjTcArgs {
    int n, R, ld, nrb, kblocks, kb_per, splits;   // splits = cluster size (1, 2, 4 or 8)
    int xin;                                       // operand buffer of X (0, 1 or 2)
    int ldk;
    __nv_bfloat16 *xs_out;                         // forward: pieces of q_{t+1} for the next product, or null
    const float *h;
    const float *X, *P;
    float *Qn, *Pn, *Fo;
    const float *LB;
    float *LQ, *LP;
    float *obj_part;                               // terminal: [tiles][splits]
    StepParams sp;
    const float *zeta, *dt;
    int t;
    int *err;
    long long limit_ns;
};

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Cluster barrier halves (every thread of every CTA of the cluster takes
// part; not .aligned, so warps need not be converged).
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// 16-byte store into CTA `rank`'s shared memory at this CTA's address
// `local_addr` (fire and forget; the next cluster barrier orders it).
__device__ __forceinline__ void st_dsmem_v4(uint32_t local_addr, uint32_t rank, float4 v) {
    asm volatile(
        "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %0, %1;\n\t"
        "st.shared::cluster.v4.f32 [ra], {%2, %3, %4, %5};\n\t}" ::"r"(local_addr),
        "r"(rank), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
        : "memory");
}

// Epilogue of 16 replicas r0 .. r0+15 of spin i from G = (J X^T)_ir.  The
// inputs of all 16 are loaded before the first store (X, P and LB are never
// written by this kernel), so the loads overlap instead of waiting behind
// the stores one element at a time.
template <int MODE, int CNT = 16>
__device__ __forceinline__ void at_apply16(const AdjTcArgs &a, int i, int r0, const float *G, float hi, float zt,
                                           float dtt, float dtm, float &objp) {
    float u0[CNT], u1[CNT];
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
        const int r = r0 + u;
        const size_t e = (size_t)r * a.ld + i;
        const bool v = r < a.R;
        u0[u] = v ? __ldg(a.X + e) : 0.f;
        if (MODE == AT_FORWARD) u1[u] = v ? __ldg(a.P + e) : 0.f;
        if (MODE == AT_ADJOINT) u1[u] = v ? __ldg(a.LB + e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
        const int r = r0 + u;
        if (r >= a.R) continue;
        const size_t e = (size_t)r * a.ld + i;
        if (MODE == AT_FORWARD) {
            const float F = G[u] + hi;
            float qo, po;
            integrate<float>(u0[u], u1[u], F, zt, dtt, dtm, a.sp, qo, po);
            a.Qn[e] = qo;
            a.Pn[e] = po;
            a.Fo[e] = F;
            if (a.xs_out) {
                __nv_bfloat16 p0, p1, p2;
                bf16_split3(qo, p0, p1, p2);
                __nv_bfloat16 *xb = a.xs_out + ((size_t)(r / AT_RB) * AT_BN + (r % AT_RB)) * a.ldk + i;
                xb[0] = p0;
                xb[(size_t)AT_RB * a.ldk] = p1;
                xb[(size_t)2 * AT_RB * a.ldk] = p2;
            }
        } else if (MODE == AT_TERMINAL) {
            const float x = u0[u];
            a.LQ[e] = -(G[u] + hi);
            a.LP[e] = 0.f;
            objp += -0.5f * x * G[u] - hi * x;
        } else {
            const float la = u0[u];
            a.LQ[e] = adj_lq(u1[u], la, G[u], dtt, zt, a.sp.k);
            a.LP[e] = la;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(AT_THREADS, 1)
    k_adj_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
             const __grid_constant__ AdjTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + AT_TILES;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (AT_S + s); };
    const uint32_t accf_bar = bar0 + 8u * (2 * AT_S);
    const uint32_t drain_bar = bar0 + 8u * (2 * AT_S + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + AT_TILES + AT_NBARS * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + AT_TILES + AT_NBARS * 8 + 4);
    float *red = reinterpret_cast<float *>(smem + AT_TILES + AT_NBARS * 8 + 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int mn = blockIdx.x / a.splits, ks = blockIdx.x % a.splits;
    const int mt = mn / a.nrb, rb = mn % a.nrb;
    const int kb0 = ks * a.kb_per;
    const int nk = min(a.kblocks, kb0 + a.kb_per) - kb0;   // >= 1 by construction

    if (threadIdx.x == 0) {
        for (int s = 0; s < AT_S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(accf_bar, 1);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "n"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // The setup above overlaps the previous kernel of the sweep; every read of
    // its results comes after this wait.
    grid_dep_wait();
    grid_dep_launch();
    // phase 1 of the cluster barrier: every CTA of the cluster has started
    // (its shared memory may receive partials once the phase completes)
    if (a.splits > 1) cluster_arrive_relaxed();

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int c = 0; c < nk; ++c) {
                const int s = c % AT_S;
                const uint32_t ph = (uint32_t)(c / AT_S) & 1u;
                if (!mbar_wait(empty_bar(s), ph ^ 1u, a.err, abort_flag, a.limit_ns)) break;
                const uint32_t dA = sbase + s * AT_STAGE;
                mbar_arrive_expect_tx(full_bar(s), (uint32_t)AT_STAGE);
                tma_load_2d(dA, &mapA, full_bar(s), (kb0 + c) * AT_BK, mt * AT_BM);
                tma_load_2d(dA + AT_A_BYTES, &mapB, full_bar(s), (kb0 + c) * AT_BK, (a.xin * a.nrb + rb) * AT_BN);
                ++issued;
            }
            // Let every copy land before the CTA exits.
            const int first = issued > AT_S ? issued - AT_S : 0;
            for (int c = first; c < issued; ++c) {
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait(full_bar(c % AT_S), (uint32_t)(c / AT_S) & 1u)) {
                    if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                        atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(AT_BM, AT_BN);
            bool ok = true;
            for (int c = 0; c < nk; ++c) {
                const int s = c % AT_S;
                if (!mbar_wait(full_bar(s), (uint32_t)(c / AT_S) & 1u, a.err, abort_flag, a.limit_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(sbase + s * AT_STAGE);
                const uint64_t bd = sdesc_sw128(sbase + s * AT_STAGE + AT_A_BYTES);
#pragma unroll
                for (int kk = 0; kk < AT_BK / 16; ++kk)
                    mma_bf16(tmem, ad + 2u * kk, bd + 2u * kk, idesc, (c != 0 || kk != 0) ? 1u : 0u);
                mma_commit(empty_bar(s));
            }
            if (ok) mma_commit(accf_bar);
            mma_commit(drain_bar);
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(drain_bar, 0u)) {
                if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                    atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                    break;
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue (4 warps)
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const int et = threadIdx.x - 64;             // 0..127 among the epilogue threads
        const int i = mt * AT_BM + row;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        bool ok = true;
        if (lane == 0) ok = mbar_wait(accf_bar, 0u, a.err, abort_flag, a.limit_ns);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        // all four warps agree on success before any partial is used
        epi_bar();
        if (!ok) *abort_flag = 1;
        epi_bar();
        ok = (*abort_flag == 0);
        tc_fence_after();
        const float hi = (a.h && i < a.n) ? a.h[i] : 0.f;
        float zt = 0.f, dtt = 0.f, dtm = 0.f;
        if (MODE != AT_TERMINAL) {
            zt = a.zeta[a.t];
            dtt = a.dt[a.t];
            dtm = dtt / a.sp.m;
        }
        float objp = 0.f;
        // Split-K partials are pushed to their owners: replicas [j S, j S + S)
        // of the tile belong to cluster rank j, S = 64 / splits.  The
        // receive buffer of rank j holds [source rank][S / 4][128 rows] of
        // four-replica chunks.
        const int S = AT_RB / a.splits;
        const uint32_t recv = sbase + AT_TILES + AT_MISC;
        if (a.splits > 1) cluster_wait_acquire();   // phase 1: all peers are running
        if (ok) {
#pragma unroll 1
            for (int ch = 0; ch < AT_RB / 32; ++ch) {
                uint32_t v0[32], v1[32], v2[32];
                tmem_ld32(tmem + lane_off + ch * 32, v0);
                tmem_ld32(tmem + lane_off + AT_RB + ch * 32, v1);
                tmem_ld32(tmem + lane_off + 2 * AT_RB + ch * 32, v2);
                tmem_wait_ld();
                float G[32];
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    G[j] = (__uint_as_float(v0[j]) + __uint_as_float(v1[j])) + __uint_as_float(v2[j]);
                if (a.splits > 1) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int rl = ch * 32 + 4 * q;          // first replica of the chunk
                        const int owner = rl / S, c4 = (rl % S) / 4;
                        const uint32_t off = (uint32_t)(((ks * (S / 4) + c4) * AT_BM + row) * 16);
                        st_dsmem_v4(recv + off, (uint32_t)owner,
                                    make_float4(G[4 * q], G[4 * q + 1], G[4 * q + 2], G[4 * q + 3]));
                    }
                } else if (i < a.n) {
                    at_apply16<MODE>(a, i, rb * AT_RB + ch * 32, G, hi, zt, dtt, dtm, objp);
                    at_apply16<MODE>(a, i, rb * AT_RB + ch * 32 + 16, G + 16, hi, zt, dtt, dtm, objp);
                }
            }
        }
        if (MODE == AT_TERMINAL && a.splits == 1) {
            red[et] = objp;
            epi_bar();
            if (et == 0) {
                CompSum<float> s;
                s.init();
                for (int w = 0; w < AT_BM; ++w) s.add(red[w]);
                a.obj_part[mn] = s.value();
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (a.splits > 1) {
        // The epilogue warps took phase 1 before pushing; the others take it
        // here.  Phase 2: every push of the cluster has landed.
        if (warp < 2) cluster_wait_acquire();
        cluster_arrive_release();
        cluster_wait_acquire();
        if (warp >= 2) {
            const int quad = warp & 3;
            const int row = quad * 32 + lane;
            const int et = threadIdx.x - 64;
            const int i = mt * AT_BM + row;
            const float hi = (a.h && i < a.n) ? a.h[i] : 0.f;
            float zt = 0.f, dtt = 0.f, dtm = 0.f;
            if (MODE != AT_TERMINAL) {
                zt = a.zeta[a.t];
                dtt = a.dt[a.t];
                dtm = dtt / a.sp.m;
            }
            float objp = 0.f;
            const int S = AT_RB / a.splits;
            const int nc = S / 4;
            const float4 *rv = reinterpret_cast<const float4 *>(smem + AT_TILES + AT_MISC);
            // add the pushed partials of this CTA's replicas in source-rank order
            float G[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) G[u] = 0.f;
            for (int p = 0; p < a.splits; ++p) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (q < nc) {
                        const float4 v = rv[(p * nc + q) * AT_BM + row];
                        G[4 * q] += v.x;
                        G[4 * q + 1] += v.y;
                        G[4 * q + 2] += v.z;
                        G[4 * q + 3] += v.w;
                    }
                }
            }
            const int rl0 = ks * S;
            if (*abort_flag == 0 && i < a.n) {
                if (S == 32) {
                    at_apply16<MODE, 32>(a, i, rb * AT_RB + rl0, G, hi, zt, dtt, dtm, objp);
                } else if (S == 16) {
                    at_apply16<MODE, 16>(a, i, rb * AT_RB + rl0, G, hi, zt, dtt, dtm, objp);
                } else {
                    at_apply16<MODE, 8>(a, i, rb * AT_RB + rl0, G, hi, zt, dtt, dtm, objp);
                }
            }
            if (MODE == AT_TERMINAL) {
                float *red = reinterpret_cast<float *>(smem + AT_TILES + AT_NBARS * 8 + 16);
                red[et] = objp;
                epi_bar();
                if (et == 0) {
                    CompSum<float> s;
                    s.init();
                    for (int w = 0; w < AT_BM; ++w) s.add(red[w]);
                    a.obj_part[mn * a.splits + ks] = s.value();
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(256) : "memory");
    }
}

// ------------------------------------------------------------------ persistent sweep
// k_adj_run runs a stretch of the sweep in one launch: the forward products
// of consecutive steps (the first forward pass, which also writes the
// checkpoints, or the recomputation of one segment), the reverse steps of
// one segment, or a recomputation and a reverse sweep side by side (segment
// s-1 is recomputed into the other set of slots while segment s is swept
// back).  A chain's CTAs are the (M tile, replica block, K split) CTAs of
// k_adj_tc with the same products and the same split-K reduction through
// distributed shared memory, so every value equals the per-step kernels'.
// The state of a CTA's slice (128 spins x 64/S replicas) stays in registers
// for the whole launch: q, p on a forward chain; lambda_a, lambda_b on a
// reverse chain, where the elementwise part of the next reverse step is
// fused into the epilogue of each adjoint product.
//
// Consecutive products exchange their operand pieces through two buffers
// per chain in L2: product u reads buffer u & 1 and its epilogue writes the
// pieces of the next operand into the other one.  Each CTA publishes its
// slice with a release increment of its tile's counter; a producer waits
// until the counters of the M tiles its K range covers show all S slices of
// the step (dataflow, no grid barrier).  The cluster barrier of every step
// makes the double buffer safe: a cluster's epilogue of product u comes
// after the MMAs of product u in all its CTAs, whose K ranges cover every
// M tile, so every tile has published the operand of product u and thus
// finished reading buffer (u - 1) & 1 before it is overwritten.
//
// Every thread of a CTA takes part in one cluster barrier per product (and
// one at the start), whatever happens, so the barriers cannot hang; every
// other wait has a time limit, after which the kernel raises the device
// error word and skips the remaining work.
constexpr int AR_RECV = AT_RB * AT_BM * 4;               // 32 KB: one buffer of pushed partials
constexpr int AR_NBARS = 2 * AT_S + 4;                   // full, empty, accf, drain, pub, red
constexpr int AR_EPI = 16;                               // epilogue warps
constexpr int AR_THREADS = 32 * (2 + AR_EPI);            // producer, MMA issuer, epilogue
constexpr int AR_SMEM = AT_TILES + AT_MISC + 2 * AR_RECV + 1024;
static_assert(AR_NBARS * 8 + 16 + AR_EPI * 6 * 4 <= AT_MISC, "misc area too small");
static_assert(AR_SMEM <= 232448, "persistent sweep exceeds the shared memory of a CTA");

struct AdjRunArgs {
    int n, R, ld, ldk, nrb, mtiles, kblocks, kb_per, splits, K, nparts;
    size_t plane;                // R * ld
    const float *h;
    StepParams sp;
    const float *zeta, *dt;
    __nv_bfloat16 *xs;           // operand buffers [4][nrb * 192][ldk]
    AdjChain ch[2];
    int *err;
    long long limit_ns;
};

template <int SR>
__global__ void __launch_bounds__(AR_THREADS, 1)
    k_adj_run(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ AdjRunArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + AT_TILES;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (AT_S + s); };
    const uint32_t accf_bar = bar0 + 8u * (2 * AT_S);
    const uint32_t drain_bar = bar0 + 8u * (2 * AT_S + 1);
    const uint32_t pub_bar = bar0 + 8u * (2 * AT_S + 2);
    const uint32_t red_bar = bar0 + 8u * (2 * AT_S + 3);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + AT_TILES + AR_NBARS * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + AT_TILES + AR_NBARS * 8 + 4);
    float *red = reinterpret_cast<float *>(smem + AT_TILES + AR_NBARS * 8 + 16);   // [16 warps][3 sums][hi, lo]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int per_chain = a.mtiles * a.nrb * a.splits;
    const AdjChain &ch = a.ch[blockIdx.x / per_chain];
    const int local = blockIdx.x % per_chain;            // index of the CTA's gradient partials
    const int mn = local / a.splits, ks = local % a.splits;
    const int mt = mn / a.nrb, rb = mn % a.nrb;
    const int S = a.splits;                               // == AT_RB / SR
    const int kb0 = ks * a.kb_per;
    const int nk = min(a.kblocks, kb0 + a.kb_per) - kb0;   // >= 1 by construction
    const int len = ch.len;

    if (threadIdx.x == 0) {
        for (int s = 0; s < AT_S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(accf_bar, 1);
        mbar_init(drain_bar, 1);
        mbar_init(pub_bar, AR_EPI);
        mbar_init(red_bar, AR_EPI);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "n"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // every CTA of the cluster is running before any pushes partials to it
    cluster_arrive_relaxed();
    cluster_wait_acquire();

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        // Lanes 0 .. nown-1 wait for the counters of the M tiles that the
        // CTA's K range covers (K block kb holds spins of M tile kb / 2);
        // lane 0 then issues the J tile and the operand tile of every K block.
        // The J tiles do not depend on the step: the first min(nk, S)
        // stages are armed and their J tiles issued before the wait (every
        // stage is free by then: the previous product has completed), and
        // only the operand tiles follow it.
        const int o0 = kb0 >> 1, nown = ((kb0 + nk - 1) >> 1) - o0 + 1;
        const int npre = min(nk, AT_S);
        uint32_t cnt = 0;
        bool ok = true;
        for (int u = 0; u < len; ++u) {
            if (ok) {
                int armed = 0;
                if (lane == 0) {
                    for (; armed < npre; ++armed) {
                        const uint32_t k = cnt + (uint32_t)armed;
                        const int s = (int)(k % AT_S);
                        if (!mbar_wait(empty_bar(s), ((k / AT_S) & 1u) ^ 1u, a.err, abort_flag, a.limit_ns)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(full_bar(s), (uint32_t)AT_STAGE);
                        tma_load_2d(sbase + s * AT_STAGE, &mapA, full_bar(s), (kb0 + armed) * AT_BK, mt * AT_BM);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                bool mine = true;
                if (ok && lane < nown)
                    mine = wait_counter_geq(ch.flags + (size_t)(o0 + lane) * a.nrb + rb, (unsigned)(S * (u + 1)),
                                            a.err, a.limit_ns);
                const bool ready = ok && __all_sync(0xffffffffu, mine);
                // orders every lane's acquire before lane 0's copies
                __syncwarp();
                if (lane == 0) {
                    // The operand tiles of the armed stages are issued even
                    // after a failed wait, so that their transaction counts
                    // complete and the drain below ends.
                    if (ready) fence_proxy_async_global();
                    const int yb = ((ch.buf0 + (u & 1)) * a.nrb + rb) * AT_BN;
                    for (int c = 0; c < nk; ++c, ++cnt) {
                        const int s = (int)(cnt % AT_S);
                        const uint32_t dA = sbase + s * AT_STAGE;
                        if (c >= armed) {
                            if (!ready) break;
                            if (!mbar_wait(empty_bar(s), ((cnt / AT_S) & 1u) ^ 1u, a.err, abort_flag, a.limit_ns)) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(full_bar(s), (uint32_t)AT_STAGE);
                            tma_load_2d(dA, &mapA, full_bar(s), (kb0 + c) * AT_BK, mt * AT_BM);
                        }
                        tma_load_2d(dA + AT_A_BYTES, &mapB, full_bar(s), (kb0 + c) * AT_BK, yb);
                    }
                    ok = ok && ready;
                }
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            }
            cluster_arrive_relaxed();
            cluster_wait_acquire();
        }
        // Let every copy land before the CTA exits.
        if (lane == 0) {
            const uint32_t first = cnt > (uint32_t)AT_S ? cnt - AT_S : 0u;
            for (uint32_t c = first; c < cnt; ++c) {
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait(full_bar((int)(c % AT_S)), (c / AT_S) & 1u)) {
                    if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                        atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        uint32_t c = 0;
        bool ok = true;
        constexpr uint32_t idesc = idesc_bf16(AT_BM, AT_BN);
        for (int u = 0; u < len; ++u) {
            if (ok) {
                if (lane == 0) {
                    // after the previous step's cluster barrier: the epilogue has read the accumulator
                    tc_fence_after();
                    for (int cc = 0; cc < nk; ++cc, ++c) {
                        const int s = (int)(c % AT_S);
                        if (!mbar_wait(full_bar(s), (c / AT_S) & 1u, a.err, abort_flag, a.limit_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc_sw128(sbase + s * AT_STAGE);
                        const uint64_t bd = sdesc_sw128(sbase + s * AT_STAGE + AT_A_BYTES);
#pragma unroll
                        for (int kk = 0; kk < AT_BK / 16; ++kk)
                            mma_bf16(tmem, ad + 2u * kk, bd + 2u * kk, idesc, (cc != 0 || kk != 0) ? 1u : 0u);
                        mma_commit(empty_bar(s));
                    }
                    if (ok) mma_commit(accf_bar);
                }
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            }
            cluster_arrive_relaxed();
            cluster_wait_acquire();
        }
        // Drain: every MMA this thread issued has completed.
        if (lane == 0) {
            mma_commit(drain_bar);
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(drain_bar, 0u)) {
                if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                    atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                    break;
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue (16 warps)
        // Warp w reads TMEM lanes 32 (w % 4) .. +31 (thread = spin i); the four
        // warps of a lane quadrant (sub = 0..3) take a quarter of the columns
        // when pushing partials and W = SR/4 replicas of the CTA's slice
        // afterwards, so that four warps per SM sub-partition hide each
        // other's latencies.
        constexpr int W = SR / 4;
        const int e = warp - 2;
        const int quad = warp & 3, sub = e >> 2;
        const int row = quad * 32 + lane;
        const int i = mt * AT_BM + row;
        const bool row_ok = i < a.n;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        const int rl0 = ks * SR + sub * W;                    // first replica of the thread, within the tile
        const int rs0 = rb * AT_RB + rl0;
        const int nv = row_ok ? max(0, min(W, a.R - rs0)) : 0;
        const float hi = (!ch.reverse && a.h && row_ok) ? a.h[i] : 0.f;
        const size_t pl = a.plane;
        const float kq = a.sp.k, mq = a.sp.m, q0 = a.sp.q0, qmax = a.sp.q_max, pmax = a.sp.p_max;
        const int zrev = (ch.t_start / a.K) & 1;             // slot set of a reverse chain's segment
        float x0[W], x1[W];      // forward: q, p; reverse: lambda_a, lambda_b
#pragma unroll
        for (int u = 0; u < W; ++u) x0[u] = x1[u] = 0.f;
        uint32_t pubs = 0;
        bool ok = true;
        auto eidx = [&](int u) { return (size_t)(rs0 + u) * a.ld + i; };
        // bf16 pieces of x0 as rows of the B operand in buffer `buf`
        auto pieces = [&](int buf) {
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (u < nv) {
                    __nv_bfloat16 p0, p1, p2;
                    bf16_split3(x0[u], p0, p1, p2);
                    __nv_bfloat16 *xb =
                        a.xs + ((size_t)(buf * a.nrb + rb) * AT_BN + (size_t)(rl0 + u)) * a.ldk + i;
                    xb[0] = p0;
                    xb[(size_t)AT_RB * a.ldk] = p1;
                    xb[(size_t)2 * AT_RB * a.ldk] = p2;
                }
            }
        };
        // The warps' stores of the next operand are ordered before lane 0's
        // arrivals (warp barrier), the arrivals before thread 0's wait, and
        // that before its release increment of the tile's counter.
        uint32_t reds = 0;
        auto publish = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(pub_bar);
            if (e == 0 && lane == 0) {
                if (mbar_wait(pub_bar, pubs & 1u, a.err, abort_flag, a.limit_ns))
                    red_release_gpu_add(ch.flags + (size_t)mt * a.nrb + rb, 1u);
            }
            ++pubs;
        };
        // The CTA's gradient partials of step tau: warp shuffle trees of the
        // compensated sums, then the 16 warps in order (off the critical path:
        // after the publication).
        auto partials = [&](CompSum<float> *g, int tau) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const float oh = __shfl_down_sync(0xffffffffu, g[j].hi, off);
                    const float ol = __shfl_down_sync(0xffffffffu, g[j].lo, off);
                    g[j].merge(oh, ol);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    red[(e * 3 + j) * 2] = g[j].hi;
                    red[(e * 3 + j) * 2 + 1] = g[j].lo;
                }
                mbar_arrive(red_bar);
            }
            if (e == 0 && lane == 0) {
                if (mbar_wait(red_bar, reds & 1u, a.err, abort_flag, a.limit_ns)) {
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        CompSum<float> sm;
                        sm.init();
                        for (int w = 0; w < AR_EPI; ++w) sm.merge(red[(w * 3 + j) * 2], red[(w * 3 + j) * 2 + 1]);
                        ch.part[(size_t)tau * 3 * a.nparts + (size_t)j * a.nparts + local] = sm.value();
                    }
                }
            }
            ++reds;
        };
        // Slot values of reverse step tau (slot jj of the segment): q_{tau+1},
        // p_{tau+1} (the clamp indicators, lb p'/m), q_tau and F_tau.
        float pre[4][W];
        auto fetch = [&](int jj) {
            const float *sqz = ch.sq[zrev], *spz = ch.sp[zrev], *sFz = ch.sF[zrev];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (u < nv) {
                    const size_t x = eidx(u);
                    pre[0][u] = sqz[(size_t)(jj + 1) * pl + x];
                    pre[1][u] = spz[(size_t)(jj + 1) * pl + x];
                    pre[2][u] = sqz[(size_t)jj * pl + x];
                    pre[3][u] = sFz[(size_t)jj * pl + x];
                }
            }
        };
        // Elementwise part of reverse step tau from the adjoint state (lq, lp)
        // of step tau + 1 and the fetched slot values, in two halves: lambda_a
        // and lambda_b into x0, x1 (needed for the next operand), and, after
        // that operand is published, the gradient terms into g.
        auto elem = [&](int tau, const float *lqv, const float *lpv) {
            const float dtm = a.dt[tau] / mq;
#pragma unroll
            for (int u = 0; u < W; ++u)
                if (u < nv) adj_clamps(lqv[u], lpv[u], pre[0][u], pre[1][u], qmax, pmax, dtm, x0[u], x1[u]);
        };
        auto terms = [&](int tau, CompSum<float> *g) {
            const float zt = a.zeta[tau], dtt = a.dt[tau];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (u < nv) {
                    float g0, g1, g2;
                    adj_terms(x0[u], x1[u], pre[2][u], pre[3][u], pre[1][u], q0, kq, mq, zt, dtt, g0, g1, g2);
                    g[0].add(g0);
                    g[1].add(g1);
                    g[2].add(g2);
                }
            }
        };

        // ---------------- prologue: the operand of product 0
        if (!ch.reverse) {
#pragma unroll
            for (int u = 0; u < W; ++u)
                if (u < nv) {
                    x0[u] = ch.q_in[eidx(u)];
                    x1[u] = ch.p_in[eidx(u)];
                }
            pieces(ch.buf0);
            publish();
        } else {
            float lqv[W], lpv[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                lqv[u] = u < nv ? ch.lq[eidx(u)] : 0.f;
                lpv[u] = u < nv ? ch.lp[eidx(u)] : 0.f;
            }
            fetch(len - 1);
            CompSum<float> g[3];
            g[0].init();
            g[1].init();
            g[2].init();
            const int tau = ch.t_start + len - 1;
            elem(tau, lqv, lpv);
            pieces(ch.buf0);
            publish();
            terms(tau, g);
            partials(g, tau);
        }

        // ---------------- products
#pragma unroll 1
        for (int u = 0; u < len; ++u) {
            // a reverse chain's slot values for the next elementwise step load
            // while the product runs
            if (ch.reverse && u + 1 < len) fetch(len - 2 - u);
            bool okw = true;
            if (ok && lane == 0) okw = mbar_wait(accf_bar, (uint32_t)(u & 1), a.err, abort_flag, a.limit_ns);
            ok = ok && __shfl_sync(0xffffffffu, okw ? 1 : 0, 0) != 0;
            tc_fence_after();
            const uint32_t recv = sbase + AT_TILES + AT_MISC + (uint32_t)(u & 1) * AR_RECV;
            if (ok) {
                // this warp's 16 replicas of the tile, pieces added (hi + mid) + lo;
                // replicas [j SR, j SR + SR) go to cluster rank j as [source][SR / 4][row] float4
                uint32_t v0[16], v1[16], v2[16];
                tmem_ld16(tmem + lane_off + sub * 16, v0);
                tmem_ld16(tmem + lane_off + AT_RB + sub * 16, v1);
                tmem_ld16(tmem + lane_off + 2 * AT_RB + sub * 16, v2);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float G4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        G4[j] = (__uint_as_float(v0[4 * q + j]) + __uint_as_float(v1[4 * q + j])) +
                                __uint_as_float(v2[4 * q + j]);
                    const int rl = sub * 16 + 4 * q;
                    const int owner = rl / SR, c4 = (rl % SR) / 4;
                    const uint32_t off = (uint32_t)(((ks * (SR / 4) + c4) * AT_BM + row) * 16);
                    st_dsmem_v4(recv + off, (uint32_t)owner, make_float4(G4[0], G4[1], G4[2], G4[3]));
                }
            }
            tc_fence_before();
            cluster_arrive_release();
            cluster_wait_acquire();
            // one decision per warp (the abort word may change between its lanes' reads)
            ok = ok && !__any_sync(0xffffffffu, *abort_flag != 0);
            if (!ok) continue;
            // the partials of this thread's replicas, added in source-rank order
            float G[W];
#pragma unroll
            for (int u2 = 0; u2 < W; ++u2) G[u2] = 0.f;
            const float4 *rv = reinterpret_cast<const float4 *>(smem + AT_TILES + AT_MISC + (u & 1) * AR_RECV);
            for (int p = 0; p < S; ++p) {
                if constexpr (W >= 4) {
#pragma unroll
                    for (int cc = 0; cc < W / 4; ++cc) {
                        const float4 v = rv[(p * (SR / 4) + sub * (W / 4) + cc) * AT_BM + row];
                        G[4 * cc] += v.x;
                        G[4 * cc + 1] += v.y;
                        G[4 * cc + 2] += v.z;
                        G[4 * cc + 3] += v.w;
                    }
                } else {
                    // W == 2: half of the chunk (sub / 2)
                    const float4 v = rv[(p * (SR / 4) + (sub >> 1)) * AT_BM + row];
                    G[0] += (sub & 1) ? v.z : v.x;
                    G[1] += (sub & 1) ? v.w : v.y;
                }
            }
            if (!ch.reverse) {
                // forward step t: Eq. 8 with the walls of Eq. 6
                const int t = ch.t_start + u, sg = t / a.K, j = t - sg * a.K, z = sg & 1;
                const float zt = a.zeta[t], dtt = a.dt[t];
                const float dtm = dtt / a.sp.m;
                float *sqz = ch.sq[z], *spz = ch.sp[z], *sFz = ch.sF[z];
                const bool ck_end = ch.ckq != nullptr && (t + 1 == ch.t_start + len || j + 1 == a.K);
                float Fv[W], qv[W], pv[W];   // F_t and the state before the step
#pragma unroll
                for (int u2 = 0; u2 < W; ++u2) {
                    Fv[u2] = G[u2] + hi;
                    qv[u2] = x0[u2];
                    pv[u2] = x1[u2];
                    integrate<float>(qv[u2], pv[u2], Fv[u2], zt, dtt, dtm, a.sp, x0[u2], x1[u2]);
                }
                // the next operand first, then the slots of the sweep
                if (u + 1 < len) {
                    pieces(ch.buf0 + ((u + 1) & 1));
                    publish();
                }
#pragma unroll
                for (int u2 = 0; u2 < W; ++u2) {
                    if (u2 < nv) {
                        const size_t x = eidx(u2);
                        if (j == 0) {
                            sqz[x] = qv[u2];
                            spz[x] = pv[u2];
                        }
                        sFz[(size_t)j * pl + x] = Fv[u2];
                        sqz[(size_t)(j + 1) * pl + x] = x0[u2];
                        spz[(size_t)(j + 1) * pl + x] = x1[u2];
                        if (ck_end) {
                            ch.ckq[(size_t)(sg + 1) * pl + x] = x0[u2];
                            ch.ckp[(size_t)(sg + 1) * pl + x] = x1[u2];
                        }
                    }
                }
            } else {
                // adjoint product of step t, then the elementwise part of step t - 1
                const int t = ch.t_start + len - 1 - u;
                const float zt = a.zeta[t], dtt = a.dt[t];
                float lqv[W], lpv[W];
#pragma unroll
                for (int u2 = 0; u2 < W; ++u2) {
                    lqv[u2] = adj_lq(x1[u2], x0[u2], G[u2], dtt, zt, kq);
                    lpv[u2] = x0[u2];
                }
                if (u + 1 < len) {
                    CompSum<float> g[3];
                    g[0].init();
                    g[1].init();
                    g[2].init();
                    elem(t - 1, lqv, lpv);
                    pieces(ch.buf0 + ((u + 1) & 1));
                    publish();
                    terms(t - 1, g);
                    partials(g, t - 1);
                } else {
#pragma unroll
                    for (int u2 = 0; u2 < W; ++u2)
                        if (u2 < nv) {
                            ch.lq[eidx(u2)] = lqv[u2];
                            ch.lp[eidx(u2)] = lpv[u2];
                        }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(256) : "memory");
    }
}

// Split of the FP32 operand X [R][ld] into bf16 pieces, laid out as the B
// operand rows [rb][piece][64][ldk] (zero for padded replicas and spins).
__global__ void k_adj_split(const float *X, int n, int R, int ld, int nrb, int ldk, __nv_bfloat16 *xs) {
    grid_dep_wait();
    grid_dep_launch();
    const long long total = (long long)nrb * AT_RB * ldk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ldk);
        const int rr = (int)(e / ldk);               // rb * 64 + rl
        const int rb = rr / AT_RB, rl = rr % AT_RB;
        const float x = (rr < R && j < n) ? X[(size_t)rr * ld + j] : 0.f;
        __nv_bfloat16 p0, p1, p2;
        bf16_split3(x, p0, p1, p2);
        __nv_bfloat16 *base = xs + ((size_t)rb * AT_BN + rl) * ldk + j;
        base[0] = p0;
        base[(size_t)AT_RB * ldk] = p1;
        base[(size_t)2 * AT_RB * ldk] = p2;
    }
}

__global__ void k_adj_jb(const float *J, int n, int ld, __nv_bfloat16 *out, int ldk, int mpad) {
    const long long total = (long long)mpad * ldk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldk), j = (int)(e % ldk);
        out[e] = __float2bfloat16_rn((i < n && j < n) ? J[(size_t)i * ld + j] : 0.f);
    }
}

void adj_tc_free(AdjTc *t) {
    if (!t) return;
    if (t->jb) cudaFree(t->jb);
    if (t->xs) cudaFree(t->xs);
    if (t->run_flags) cudaFree(t->run_flags);
    delete t;
}

int adj_tc_nobj(const AdjTc *t) { return t->mtiles * t->nrb * t->splits; }
int adj_tc_splits(const AdjTc *t) { return t ? t->splits : 0; }

template <int MODE>
static cudaError_t launch_adj(const AdjTc *t, const AdjTcArgs &a, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(t->mtiles * t->nrb * t->splits));
    cfg.blockDim = dim3(AT_THREADS);
    cfg.dynamicSmemBytes = AT_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)t->splits;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_adj_tc<MODE>, t->mapA, t->mapB, a);
}

si_status adj_tc_prepare(Ctx *c, AdjTc **out) {
    if (c->g_tc) {
        *out = c->g_tc;
        return SI_OK;
    }
    AdjTc *t = new AdjTc();
    t->n = c->n;
    t->R = c->R;
    t->ld = c->ldj;
    t->ldk = round_up(c->n, AT_BK);
    t->mpad = round_up(c->n, AT_BM);
    t->mtiles = t->mpad / AT_BM;
    t->nrb = cdiv(c->R, AT_RB);
    t->kblocks = t->ldk / AT_BK;
    const int tiles = t->mtiles * t->nrb;
    auto fail = [&](si_status e) {
        adj_tc_free(t);
        return e;
    };
    for (int mode = 0; mode < 3; ++mode) {
        cudaError_t e = mode == 0 ? cudaFuncSetAttribute(k_adj_tc<AT_FORWARD>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, AT_SMEM)
                        : mode == 1 ? cudaFuncSetAttribute(k_adj_tc<AT_TERMINAL>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, AT_SMEM)
                                    : cudaFuncSetAttribute(k_adj_tc<AT_ADJOINT>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, AT_SMEM);
        if (e != cudaSuccess) {
            set_error("si_grad: cannot reserve shared memory for the tensor-core kernel");
            return fail(SI_ERR_CUDA);
        }
    }
    // K split = cluster size in {1, 2, 4, 8}: about one wave of CTAs (one per
    // SM), every split non-empty, and all clusters resident at once (an
    // 8-CTA cluster needs 8 free SMs of one GPC).
    int splits = 8;
    while (splits > 1 && (tiles * splits > c->num_sms || (splits - 1) * cdiv(t->kblocks, splits) >= t->kblocks))
        splits >>= 1;
    while (splits > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(tiles * splits));
        cfg.blockDim = dim3(AT_THREADS);
        cfg.dynamicSmemBytes = AT_SMEM;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)splits;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_adj_tc<AT_FORWARD>, &cfg) == cudaSuccess &&
            nclusters >= tiles)
            break;
        cudaGetLastError();
        splits >>= 1;
    }
    t->splits = splits;
    t->kb_per = cdiv(t->kblocks, splits);
    // Persistent sweep: cluster size S in {8, 4, 2} (64/S replicas per CTA
    // in registers), every split non-empty, and all clusters of one chain
    // (and, for side-by-side chains, of two) resident at once, since the
    // chains' CTAs wait on each other's step counters.
    {
        const char *pe = std::getenv("SI_ADJOINT_PERSISTENT");
        const char *pp = std::getenv("SI_ADJOINT_PAIR");
        const bool allow = !(pe && std::atoi(pe) == 0);
        auto fits = [&](int S, int nch) -> bool {
            if (nch * tiles * S > c->num_sms || (S - 1) * cdiv(t->kblocks, S) >= t->kblocks) return false;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(nch * tiles * S));
            cfg.blockDim = dim3(AR_THREADS);
            cfg.dynamicSmemBytes = AR_SMEM;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)S;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            cudaError_t e = S == 8   ? cudaOccupancyMaxActiveClusters(&nclusters, k_adj_run<8>, &cfg)
                            : S == 4 ? cudaOccupancyMaxActiveClusters(&nclusters, k_adj_run<16>, &cfg)
                                     : cudaOccupancyMaxActiveClusters(&nclusters, k_adj_run<32>, &cfg);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            return nclusters >= nch * tiles;
        };
        int rs = 0;
        if (allow &&
            cudaFuncSetAttribute(k_adj_run<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, AR_SMEM) == cudaSuccess &&
            cudaFuncSetAttribute(k_adj_run<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, AR_SMEM) == cudaSuccess &&
            cudaFuncSetAttribute(k_adj_run<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, AR_SMEM) == cudaSuccess) {
            for (int S = 8; S >= 2 && rs == 0; S >>= 1)
                if (fits(S, 1)) rs = S;
        }
        cudaGetLastError();
        t->run_splits = rs;
        t->run_kb_per = rs ? cdiv(t->kblocks, rs) : 0;
        t->run_pair = rs && !(pp && std::atoi(pp) == 0) && fits(rs, 2);
    }
    if (si_dev_malloc((void **)&t->jb, sizeof(__nv_bfloat16) * (size_t)t->mpad * t->ldk) != cudaSuccess ||
        si_dev_malloc((void **)&t->xs, sizeof(__nv_bfloat16) * 4 * (size_t)t->nrb * AT_BN * t->ldk) != cudaSuccess ||
        si_dev_malloc((void **)&t->run_flags, sizeof(unsigned) * 2 * (size_t)tiles) != cudaSuccess) {
        cudaGetLastError();
        set_error("si_grad: out of device memory for the tensor-core workspace");
        return fail(SI_ERR_OOM);
    }
    if (cudaMemsetAsync(t->xs, 0, sizeof(__nv_bfloat16) * 4 * (size_t)t->nrb * AT_BN * t->ldk, c->stream) !=
        cudaSuccess) {
        set_error("si_grad: cudaMemsetAsync failed");
        return fail(SI_ERR_CUDA);
    }
    k_adj_jb<<<std::min(4096, cdiv((long long)t->mpad * t->ldk, 256)), 256, 0, c->stream>>>(
        (const float *)c->dJ, c->n, c->ldj, t->jb, t->ldk, t->mpad);
    if (cudaGetLastError() != cudaSuccess) {
        set_error("si_grad: J conversion launch failed");
        return fail(SI_ERR_CUDA);
    }
    si_status s;
    if ((s = tc_make_map_bf16(&t->mapA, t->jb, t->ldk, t->mpad, AT_BK, AT_BM)) != SI_OK) return fail(s);
    if ((s = tc_make_map_bf16(&t->mapB, t->xs, t->ldk, 4 * t->nrb * AT_BN, AT_BK, AT_BN)) != SI_OK) return fail(s);
    c->launches += 1;
    c->g_tc = t;
    *out = t;
    return SI_OK;
}

int adj_tc_run_splits(const AdjTc *t) { return t ? t->run_splits : 0; }
bool adj_tc_run_pair(const AdjTc *t) { return t && t->run_pair; }
int adj_tc_run_nparts(const AdjTc *t) { return t->mtiles * t->nrb * t->run_splits; }
unsigned *adj_tc_run_flags(const AdjTc *t, int chain) { return t->run_flags + (size_t)chain * t->mtiles * t->nrb; }

template <int SR>
static cudaError_t launch_run(const AdjTc *t, const AdjRunArgs &a, int nch, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nch * t->mtiles * t->nrb * t->run_splits));
    cfg.blockDim = dim3(AR_THREADS);
    cfg.dynamicSmemBytes = AR_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)t->run_splits;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_adj_run<SR>, t->mapA, t->mapB, a);
}

si_status adj_tc_run(Ctx *c, AdjTc *t, const AdjChain *chains, int nch, int K) {
    if (!t->run_splits || nch < 1 || nch > 2 || (nch == 2 && !t->run_pair)) {
        set_error("si_grad: persistent sweep not available for this context");
        return SI_ERR_UNSUPPORTED;
    }
    AdjRunArgs a{};
    a.n = t->n;
    a.R = t->R;
    a.ld = t->ld;
    a.ldk = t->ldk;
    a.nrb = t->nrb;
    a.mtiles = t->mtiles;
    a.kblocks = t->kblocks;
    a.kb_per = t->run_kb_per;
    a.splits = t->run_splits;
    a.K = K;
    a.nparts = adj_tc_run_nparts(t);
    a.plane = (size_t)t->R * t->ld;
    a.h = c->has_h ? c->dhf : nullptr;
    a.sp = StepParams{c->prm.k, c->prm.m, c->prm.q0, c->prm.q_max, c->prm.p_max, 0, 0};
    a.zeta = c->dzeta;
    a.dt = c->ddt;
    a.xs = t->xs;
    a.err = c->derr;
    a.limit_ns = c->spin_limit_ns;
    for (int k = 0; k < nch; ++k) {
        a.ch[k] = chains[k];
        if (chains[k].len < 1) {
            set_error("si_grad: empty chain in the persistent sweep");
            return SI_ERR_INVALID_ARG;
        }
        SI_CUDA_TRY(cudaMemsetAsync(chains[k].flags, 0, sizeof(unsigned) * (size_t)t->mtiles * t->nrb, c->stream));
    }
    cudaError_t e = t->run_splits == 8   ? launch_run<8>(t, a, nch, c->stream)
                    : t->run_splits == 4 ? launch_run<16>(t, a, nch, c->stream)
                                         : launch_run<32>(t, a, nch, c->stream);
    SI_CUDA_TRY(e);
    c->launches += 1;
    return SI_OK;
}

__nv_bfloat16 *adj_tc_xs(const AdjTc *t, int buf) {
    return t->xs + (size_t)buf * t->nrb * AT_BN * t->ldk;
}
int adj_tc_ldk(const AdjTc *t) { return t->ldk; }

si_status adj_tc_gemm(Ctx *c, AdjTc *t, int mode, const float *X, const float *P, float *Qn, float *Pn,
                      float *Fo, const float *LB, float *LQ, float *LP, float *obj_part, int tstep, int xin,
                      bool split, int xout) {
    if (split) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)std::min(2048, cdiv((long long)t->nrb * AT_RB * t->ldk, 256)));
        cfg.blockDim = dim3(256);
        cfg.stream = c->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_adj_split, X, t->n, t->R, t->ld, t->nrb, t->ldk, adj_tc_xs(t, xin)));
        c->launches += 1;
    }
    AdjTcArgs a{};
    a.n = t->n;
    a.R = t->R;
    a.ld = t->ld;
    a.nrb = t->nrb;
    a.kblocks = t->kblocks;
    a.kb_per = t->kb_per;
    a.splits = t->splits;
    a.xin = xin;
    a.ldk = t->ldk;
    a.xs_out = (mode == AT_FORWARD && xout >= 0) ? adj_tc_xs(t, xout) : nullptr;
    a.h = c->has_h ? c->dhf : nullptr;
    a.X = X;
    a.P = P;
    a.Qn = Qn;
    a.Pn = Pn;
    a.Fo = Fo;
    a.LB = LB;
    a.LQ = LQ;
    a.LP = LP;
    a.obj_part = obj_part;
    a.sp = StepParams{c->prm.k, c->prm.m, c->prm.q0, c->prm.q_max, c->prm.p_max, 0, 0};
    a.zeta = c->dzeta;
    a.dt = c->ddt;
    a.t = tstep;
    a.err = c->derr;
    a.limit_ns = c->spin_limit_ns;
    cudaError_t e = mode == AT_FORWARD    ? launch_adj<AT_FORWARD>(t, a, c->stream)
                    : mode == AT_TERMINAL ? launch_adj<AT_TERMINAL>(t, a, c->stream)
                                          : launch_adj<AT_ADJOINT>(t, a, c->stream);
    SI_CUDA_TRY(e);
    c->launches += 1;
    return SI_OK;
}

}  // namespace si
