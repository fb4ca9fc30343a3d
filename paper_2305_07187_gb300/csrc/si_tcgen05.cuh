// tcgen05 / TMA / mbarrier helpers shared by the tensor-core kernels
// (inline PTX for sm_103a).
#pragma once

#include "si_device.cuh"

namespace si {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity.  Returns false
// (and raises the error word on timeout) if the run is being aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err,
                                          volatile int *abort_flag, long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 0) {
            if (*abort_flag || (err && ld_volatile_int(err) != 0)) {
                *abort_flag = 1;
                return false;
            }
            if ((long long)(globaltimer_ns() - t0) > limit_ns) {
                if (err) atomicCAS(err, 0, DEV_TIMEOUT_MBAR);
                *abort_flag = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire_cta_shared(uint32_t addr) {
    unsigned v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_cta_shared(uint32_t addr, unsigned v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Atomic add with acquire-release semantics at GPU scope (returns the old value).
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Step flags of the CTAs that own the q blocks of a replica block, mirrored
// into shared memory by one warp of the consuming CTA (mirror_flags), so that
// the TMA producers test a shared-memory word instead of polling global
// memory on their critical path.  Lane o (and o + 32) reads owner o's flag
// with an acquire load, all lanes at once (one memory round trip per sweep),
// and stores every new value with a release store; a producer that reads the
// copy with an acquire load is then ordered after the owner's published q
// block (the two synchronisations compose).  Word MIRROR_MIN holds the
// smallest flag of all owners, stored by lane 0 after a warp barrier that
// orders every lane's acquire loads before it, so that one test of it shows
// a producer every owner ready.  The warp stops once every owner has
// published `last` steps, when the run is being aborted, or when no flag has
// moved for limit_ns (the waiting producer raises the error then).
//
// A watched run (w_done non-null) also mirrors the grid's stop decision:
// lane 0 reads the number of finished readout evaluations with a relaxed
// load issued with the owners' loads (an acquire load there would hold them
// back and slow every step's flag propagation); when it has moved, lane 0
// reads it again with acquire semantics, then the first readout that
// reached the target, stores the latter in word MIRROR_HIT and then
// (release) the number of readouts whose decision is final,
// floor(w_done / rblocks), in word MIRROR_FINAL.  Once a final readout has
// reached the target the run ends after it, and the warp stops.
constexpr int MIRROR_MIN = 64;     // word index of the minimum (words 0..63: owners)
constexpr int MIRROR_FINAL = 65;   // readouts whose stop decision is final
constexpr int MIRROR_HIT = 66;     // first readout that reached the target (large: none yet)

__device__ __forceinline__ void mirror_flags(const unsigned *flags, int nown, unsigned last, uint32_t seen,
                                             int lane, int *err, volatile int *abort_flag, long long limit_ns,
                                             const unsigned *w_done = nullptr, const int *w_hit = nullptr,
                                             unsigned rblocks = 1u) {
    unsigned m0 = 0u, m1 = 0u, mmin = 0u;   // last values mirrored by this lane
    unsigned mfin = 0u;
    unsigned long long t_last = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        bool moved = false, done = true, decided = false;
        unsigned wd = 0u;
        if (w_done && lane == 0) wd = ld_relaxed_gpu_u32(w_done);
        unsigned vmin = 0xffffffffu;
        if (lane < nown) {
            const unsigned v = ld_acquire_gpu(flags + lane);
            if (v != m0) {
                st_release_cta_shared(seen + 4u * lane, v);
                m0 = v;
                moved = true;
            }
            done = (int)(v - last) >= 0;
            vmin = v;
        }
        if (lane + 32 < nown) {
            const unsigned v = ld_acquire_gpu(flags + lane + 32);
            if (v != m1) {
                st_release_cta_shared(seen + 4u * (lane + 32), v);
                m1 = v;
                moved = true;
            }
            done = done && (int)(v - last) >= 0;
            vmin = min(vmin, v);
        }
        if (w_done && lane == 0 && wd / rblocks != mfin) {
            const unsigned fin = ld_acquire_gpu(w_done) / rblocks;
            const int h = ld_volatile_int(w_hit);
            st_release_cta_shared(seen + 4u * MIRROR_HIT, (unsigned)h);
            st_release_cta_shared(seen + 4u * MIRROR_FINAL, fin);
            mfin = fin;
            moved = true;
            decided = h < (int)fin;
        }
        if (__any_sync(0xffffffffu, decided)) return;
        vmin = __reduce_min_sync(0xffffffffu, vmin);
        __syncwarp();
        if (lane == 0 && vmin != mmin) {
            st_release_cta_shared(seen + 4u * MIRROR_MIN, vmin);
            mmin = vmin;
        }
        if (__all_sync(0xffffffffu, done)) return;
        const unsigned long long now = globaltimer_ns();
        if (__any_sync(0xffffffffu, moved)) t_last = now;
        if ((it & 7u) == 0u) {
            int stop = 0;
            if (lane == 0) stop = (*abort_flag || ld_volatile_int(err) != 0) ? 1 : 0;
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop || (long long)(now - t_last) > limit_ns) return;
        }
    }
}

// A producer's bounded wait until the mirrored flags show that owner mo has
// published step `need` (acquire loads of the shared copies), followed by
// the proxy fence that orders its next TMA loads after the published data.
// When the mirrored minimum shows the step, every owner is marked ready.
// Returns false on abort or timeout (raising DEV_TIMEOUT_BARRIER).
__device__ __forceinline__ bool wait_owner(uint32_t seen, int mo, unsigned need, unsigned long long &ready,
                                           int *err, volatile int *abort_flag, long long limit_ns) {
    const uint32_t addr = seen + 4u * (uint32_t)mo;
    const uint32_t amin = seen + 4u * MIRROR_MIN;
    auto test = [&]() -> bool {
        if ((int)(ld_acquire_cta_shared(amin) - need) >= 0) {
            ready = ~0ull;
            return true;
        }
        if ((int)(ld_acquire_cta_shared(addr) - need) >= 0) {
            ready |= 1ull << mo;
            return true;
        }
        return false;
    };
    if (!test()) {
        const unsigned long long t0 = globaltimer_ns();
        for (unsigned it = 1;; ++it) {
            if (test()) break;
            if ((it & 15u) == 0u) {
                if (*abort_flag || ld_volatile_int(err) != 0) {
                    *abort_flag = 1;
                    return false;
                }
                if ((long long)(globaltimer_ns() - t0) > limit_ns) {
                    atomicCAS(err, 0, DEV_TIMEOUT_BARRIER);
                    *abort_flag = 1;
                    return false;
                }
            }
        }
    }
    fence_proxy_async_global();
    return true;
}

// Bounded wait until the mirrored decision of readout k is final; `stop` is
// then whether the run reached its target at a readout <= k.  Returns false
// on abort or timeout (raising DEV_TIMEOUT_BARRIER).
__device__ __forceinline__ bool wait_decision(uint32_t seen, int k, bool &stop, int *err, volatile int *abort_flag,
                                              long long limit_ns) {
    const uint32_t afin = seen + 4u * MIRROR_FINAL;
    const unsigned need = (unsigned)k + 1u;
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        if ((int)(ld_acquire_cta_shared(afin) - need) >= 0) {
            stop = (int)ld_acquire_cta_shared(seen + 4u * MIRROR_HIT) <= k;
            return true;
        }
        if (it == 0) t0 = globaltimer_ns();
        if ((it & 15u) == 15u) {
            if (*abort_flag || ld_volatile_int(err) != 0) {
                *abort_flag = 1;
                return false;
            }
            if ((long long)(globaltimer_ns() - t0) > limit_ns) {
                atomicCAS(err, 0, DEV_TIMEOUT_BARRIER);
                *abort_flag = 1;
                return false;
            }
        }
    }
}

// Column sums of a warp's 32 x 32 block (lane = row, v[j] = column j): a
// transposing butterfly of 31 shuffles, after which v[0] of lane j holds the
// sum of column j.  At the round of width s a lane keeps the half of its
// current columns selected by bit s of its index and adds its partner's
// copy of that half.
__device__ __forceinline__ void column_sums32(int (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const int give = upper ? v[j] : v[j + s];
            const int keep = upper ? v[j + s] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, give, s);
        }
    }
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major bf16 tile whose rows are 128
// bytes, written by TMA with the 128-byte swizzle: 8-row groups are 1024
// bytes apart (stride byte offset), version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D fp32, A bf16, B bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// ------------------------------------------------ CTA pairs (cta_group::2)
// Two CTAs of a cluster share one MMA of M = 256: the even CTA (rank 0)
// issues it; its A operand is the 128 rows of each CTA's shared memory and
// its B operand N/2 columns from each, at the same shared-memory offsets; the
// accumulator rows of each CTA land in that CTA's tensor memory.

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared::cluster address of the object at local shared address `addr` in
// the CTA of cluster rank `rank`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Arrive (release, cluster scope) on an mbarrier of another CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// 2D TMA tile load into this CTA's shared memory whose bytes are counted on
// an mbarrier of either CTA of the pair (cta_group::2): `bar_cluster` is the
// shared::cluster address of that barrier (mapa_shared).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar_cluster, int x,
                                                 int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}

// Count `bytes` of the current phase's transactions of a barrier of this CTA
// as done without a copy (for copies that were never issued).
__device__ __forceinline__ void mbar_complete_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Store a word into the shared memory of a CTA of the cluster.
__device__ __forceinline__ void st_shared_cluster_u32(uint32_t cluster_addr, unsigned v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// mbar_wait with acquire at cluster scope (barriers that the other CTA of
// the pair arrives on).
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, int *err,
                                                  volatile int *abort_flag, long long limit_ns) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 15u) == 0) {
            if (*abort_flag || (err && ld_volatile_int(err) != 0)) {
                *abort_flag = 1;
                return false;
            }
            if ((long long)(globaltimer_ns() - t0) > limit_ns) {
                if (err) atomicCAS(err, 0, DEV_TIMEOUT_MBAR);
                *abort_flag = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier at shared offset `bar` of both CTAs of the pair
// once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    const uint16_t mask = 3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(mask)
        : "memory");
}

// Arrive on this CTA's mbarrier `bar` once every MMA this thread issued has
// completed (pair kernels).
__device__ __forceinline__ void mma_commit_pair_local(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

#define TC_REG32(a)                                                                          \
    "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]),      \
        "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]),           \
        "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(a[16]), "=r"(a[17]), "=r"(a[18]),        \
        "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]), "=r"(a[24]),        \
        "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]),        \
        "=r"(a[31])
#define TC_IN32(a)                                                                             \
    "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),    \
        "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]),      \
        "r"(a[15]), "r"(a[16]), "r"(a[17]), "r"(a[18]), "r"(a[19]), "r"(a[20]), "r"(a[21]),    \
        "r"(a[22]), "r"(a[23]), "r"(a[24]), "r"(a[25]), "r"(a[26]), "r"(a[27]), "r"(a[28]),    \
        "r"(a[29]), "r"(a[30]), "r"(a[31])

// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : TC_REG32(v)
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        TC_IN32(v)
        : "memory");
}

#define TC_REG16(a)                                                                          \
    "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]),      \
        "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]),           \
        "=r"(a[13]), "=r"(a[14]), "=r"(a[15])

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : TC_REG16(v)
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}


// ------------------------------------------------------------ e4m3 J tiles
// A J tile of 128 rows x 64 K elements stored as e4m3 (1 byte each) is loaded
// by TMA with the 64-byte swizzle into the upper half of the 16 KB bf16 A
// region of a ring stage: row r at byte 8192 + 64 r, its 16-byte chunk c (K
// elements 16c .. 16c+15) at chunk position c ^ ((r >> 1) & 3).  Four
// converter warps (128 threads, thread = row) widen it in place to the bf16
// tile that the MMA descriptors read, in the 128-byte swizzled layout TMA
// gives a bf16 tile: row r at byte 128 r, chunk c (K elements 8c .. 8c+7) at
// chunk position c ^ (r & 7).  Every thread first reads its whole e4m3 row
// into registers; only after a barrier of the four warps does any of them
// write, because bf16 rows 64..127 overwrite the e4m3 rows.  Every e4m3 value
// (3 mantissa bits, magnitudes 2^-9 .. 448) is exact in bf16, so the widening
// is exact.
constexpr int E4M3_TILE_OFFSET = 8192;   // e4m3 tile inside the 16 KB A region

// Four e4m3 values (bytes of w, lowest first) -> two bf16x2 words, on the
// integer and FMA pipes (no conversion-unit instructions).  For a byte
// s eeee mmm, PRMT builds the 16-bit word ssssssss s eeee mmm (the high
// byte replicates the sign); shifted left by 4 and masked with 0x87F0 it is
// s 0000 eeee mmm 0000: as bf16 that is the sign with exponent field eeee
// and mantissa mmm, i.e. the e4m3 magnitude times 2^(7 - 127) (for eeee = 0
// the bf16 subnormal m 2^-3 2^-126 is the e4m3 subnormal m 2^-9 times
// 2^-120 as well).  One exact bf16 multiply by 2^120 restores the value;
// zeros keep their sign.
__device__ __forceinline__ void e4m3x4_to_bf16x4(uint32_t w, uint32_t &lo, uint32_t &hi) {
    uint32_t z0, z1;
    asm("prmt.b32 %0, %1, 0, 0x9180;" : "=r"(z0) : "r"(w));   // bytes a0, sign(a0), a1, sign(a1)
    asm("prmt.b32 %0, %1, 0, 0xB3A2;" : "=r"(z1) : "r"(w));   // bytes a2, sign(a2), a3, sign(a3)
    z0 = (z0 << 4) & 0x87F087F0u;
    z1 = (z1 << 4) & 0x87F087F0u;
    const uint32_t two120 = 0x7B807B80u;                       // bf16 2^120 in both halves
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(lo) : "r"(z0), "r"(two120));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(hi) : "r"(z1), "r"(two120));
}

// Row r (64 e4m3 bytes, 64-byte swizzle) of the e4m3 tile at `tile` into 16
// registers: word m holds K elements 4m .. 4m+3, lowest first.
__device__ __forceinline__ void e4m3_row_load(uint32_t tile, int r, uint32_t (&w)[16]) {
    const uint32_t row = tile + (uint32_t)r * 64u;
    const uint32_t sw = (uint32_t)((r >> 1) & 3);
#pragma unroll
    for (int c = 0; c < 4; ++c)
        asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(w[4 * c]), "=r"(w[4 * c + 1]), "=r"(w[4 * c + 2]), "=r"(w[4 * c + 3])
                     : "r"(row + ((((uint32_t)c) ^ sw) << 4))
                     : "memory");
}

// Row r of the bf16 tile at a_region from the 16 e4m3 words of e4m3_row_load.
__device__ __forceinline__ void bf16_row_store(uint32_t a_region, int r, const uint32_t (&w)[16]) {
    const uint32_t row = a_region + (uint32_t)r * 128u;
    const uint32_t sw = (uint32_t)(r & 7);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        // bf16 chunk c holds K elements 8c .. 8c+7 = e4m3 words 2c, 2c+1
        uint32_t o0, o1, o2, o3;
        e4m3x4_to_bf16x4(w[2 * c], o0, o1);
        e4m3x4_to_bf16x4(w[2 * c + 1], o2, o3);
        asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(row + ((((uint32_t)c) ^ sw) << 4)), "r"(o0),
                     "r"(o1), "r"(o2), "r"(o3)
                     : "memory");
    }
}

// One row of 64 e4m3 values (16 words of e4m3_row_load) as 32 bf16x2 words,
// word m holding K elements 2m, 2m+1: the layout of one lane of a 128 x 64
// bf16 A operand in tensor memory (row = lane, two K elements per column).
__device__ __forceinline__ void e4m3_row_to_bf16x2(const uint32_t (&w)[16], uint32_t (&o)[32]) {
#pragma unroll
    for (int m = 0; m < 16; ++m) e4m3x4_to_bf16x4(w[m], o[2 * m], o[2 * m + 1]);
}

// MMA with the A operand (M = 128 rows x K = 16 bf16) read from tensor memory
// at column a_tmem (lane = row, 8 columns of two K elements each) and B from
// shared memory.
__device__ __forceinline__ void mma_bf16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void named_barrier_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Named barrier over `threads` threads that also ANDs a predicate: every
// participant gets true iff every participant passed a non-zero value.
__device__ __forceinline__ bool named_barrier_and(int id, int threads, int pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

// Widen one e4m3 J tile in place (all 128 threads of the four converter
// warps call this, thread t converting row t; barrier id `bar_id` is private
// to them).  The generic-proxy stores are then made visible to the tensor
// cores (async proxy) before the caller signals the MMA issuer.
__device__ __forceinline__ void widen_e4m3_tile(uint32_t a_region, int row, int bar_id) {
    uint32_t w[16];
    e4m3_row_load(a_region + (uint32_t)E4M3_TILE_OFFSET, row, w);
    named_barrier_sync(bar_id, 128);
    bf16_row_store(a_region, row, w);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}

}  // namespace si
