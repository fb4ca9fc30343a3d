// Exact Ising energy (Eq. 1) on the tensor cores for tensor-path contexts.
//
// s_r = sigma_r^T J sigma_r is computed as G = J Sigma^T with sigma in {-1,+1}
// as bf16 operands (exact) and integer-valued J in bf16 (exact for |J_ij| <=
// 256); every product and partial sum is an integer of magnitude below 2^24,
// so the FP32 tensor-core accumulation is exact.  The epilogue multiplies
// G_ir by sigma_ir, reduces the 128 rows of the tile per replica and adds the
// tile's integer sum into a 64-bit per-replica total; a finishing kernel
// forms E = -s/2 - h.sigma and cut = (s - 2 S_upper)/4 (weights w = -J).
// When the context stores J as e4m3, the four epilogue warps, idle during the
// mainloop, first widen each J tile to bf16 in shared memory (exactly).
#include <algorithm>
#include <cstdio>

#include "si_tcgen05.cuh"

namespace si {

constexpr int TE_BM = 128, TE_BN = 128, TE_BK = 64, TE_S = 4, TE_THREADS = 192;
constexpr int TE_A_BYTES = TE_BM * TE_BK * 2, TE_B_BYTES = TE_BN * TE_BK * 2;
constexpr int TE_STAGE = TE_A_BYTES + TE_B_BYTES;
constexpr int TE_BARS = TE_S * TE_STAGE;
constexpr int TE_NBARS = 3 * TE_S + 1;   // full[S], empty[S], accf, conv[S]
constexpr int TE_SMEM = TE_BARS + TE_NBARS * 8 + 16 + 1024;

struct TeArgs {
    int n, R, kblocks;
    const int8_t *spins;   // [R][lds]
    int lds;
    unsigned long long *sum;  // [R] (zeroed before the launch)
    int *err;
    long long limit_ns;
};

template <bool E4>
__global__ void __launch_bounds__(TE_THREADS, 1)
    k_tc_sigma_j_sigma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapS,
                       TeArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + TE_BARS;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (TE_S + s); };
    const uint32_t accf_bar = bar0 + 8u * (2 * TE_S);
    auto conv_bar = [&](int s) { return bar0 + 8u * (2 * TE_S + 1 + s); };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + TE_BARS + TE_NBARS * 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + TE_BARS + TE_NBARS * 8 + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TE_BM, r0 = blockIdx.y * TE_BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TE_S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
            mbar_init(conv_bar(s), 4);
        }
        mbar_init(accf_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
                const int s = it % TE_S;
                const uint32_t ph = (it / TE_S) & 1u;
                if (!mbar_wait(empty_bar(s), ph ^ 1u, a.err, abort_flag, a.limit_ns)) break;
                const uint32_t d = sbase + s * TE_STAGE;
                mbar_arrive_expect_tx(full_bar(s), (uint32_t)(E4 ? TE_BM * TE_BK + TE_B_BYTES : TE_STAGE));
                tma_load_2d(E4 ? d + (uint32_t)E4M3_TILE_OFFSET : d, &mapA, full_bar(s), kb * TE_BK, m0);
                tma_load_2d(d + TE_A_BYTES, &mapS, full_bar(s), kb * TE_BK, r0);
            }
            const uint32_t first = it > (uint32_t)TE_S ? it - TE_S : 0u;
            for (uint32_t k = first; k < it; ++k) {
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait(full_bar(k % TE_S), (k / TE_S) & 1u)) {
                    if ((long long)(globaltimer_ns() - t0) > a.limit_ns) {
                        atomicCAS(a.err, 0, DEV_TIMEOUT_MBAR);
                        break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(TE_BM, TE_BN);
            bool ok = true;
            for (int kb = 0; kb < a.kblocks; ++kb) {
                const int s = kb % TE_S;
                const uint32_t ph = (kb / TE_S) & 1u;
                if (!mbar_wait(full_bar(s), ph, a.err, abort_flag, a.limit_ns)) { ok = false; break; }
                if (E4 && !mbar_wait(conv_bar(s), ph, a.err, abort_flag, a.limit_ns)) { ok = false; break; }
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(sbase + s * TE_STAGE);
                const uint64_t bd = ad + (uint64_t)(TE_A_BYTES >> 4);
#pragma unroll
                for (int kk = 0; kk < TE_BK / 16; ++kk)
                    mma_bf16(tmem, ad + 2u * kk, bd + 2u * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
                mma_commit(empty_bar(s));
            }
            if (ok) mma_commit(accf_bar);   // on abort the epilogue sees the abort flag instead
        }
    } else {
        // epilogue: warps 2..5, TMEM lane quadrant warp%4, one spin per
        // thread.  The products G_ir sigma_ir go to shared memory as
        // [replica][row] (the operand ring is free once the accumulator is
        // complete: every stage has been loaded and read by the MMAs); after
        // a barrier of the four warps, thread t adds the 128 rows of replica
        // column t and issues one 64-bit add for the tile.  Integer sums:
        // exact in any order.
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const int i = m0 + row;
        int *prod = reinterpret_cast<int *>(smem);   // [TE_BN][TE_BM + 1]
        bool ok = true;
        if (E4) {
            // widen the e4m3 J tiles in place, in the order they arrive (thread
            // (warp - 2) * 32 + lane converts that row of every tile)
            const int crow = (warp - 2) * 32 + lane;
            for (int kb = 0; kb < a.kblocks; ++kb) {
                const int s = kb % TE_S;
                const uint32_t ph = (kb / TE_S) & 1u;
                const int okw = mbar_wait(full_bar(s), ph, a.err, abort_flag, a.limit_ns) ? 1 : 0;
                if (!named_barrier_and(2, 128, okw)) break;
                widen_e4m3_tile(sbase + s * TE_STAGE, crow, 2);
                __syncwarp();
                if (lane == 0) mbar_arrive(conv_bar(s));
            }
        }
        if (lane == 0) ok = mbar_wait(accf_bar, 0u, a.err, abort_flag, a.limit_ns);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
            tc_fence_after();
            const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < TE_BN / 32; ++c) {
                uint32_t v[32];
                int sg[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int r = r0 + c * 32 + j;
                    sg[j] = (i < a.n && r < a.R) ? (int)a.spins[(size_t)r * a.lds + i] : 0;
                }
                tmem_ld32(tl + c * 32, v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) prod[(c * 32 + j) * (TE_BM + 1) + row] = (int)__uint_as_float(v[j]) * sg[j];
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
        if (ok) {
            const int rl = row;                  // replica column of this thread
            const int r = r0 + rl;
            long long x = 0;
            const int *col = prod + rl * (TE_BM + 1);
#pragma unroll 8
            for (int w = 0; w < TE_BM; ++w) x += col[w];
            if (r < a.R && x != 0) atomicAdd(a.sum + r, (unsigned long long)x);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
    }
}

// spins int8 [R][lds] -> bf16 operand [rpad][ldk] (zero padded).
__global__ void k_spins_to_bf16(const int8_t *s, int lds, int n, int R, __nv_bfloat16 *out, int ldk, int rpad) {
    const long long total = (long long)rpad * ldk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ldk), i = (int)(e % ldk);
        out[e] = __float2bfloat16_rn((r < R && i < n) ? (float)s[(size_t)r * lds + i] : 0.f);
    }
}

__global__ void k_energy_finish(const unsigned long long *sum, const int8_t *h8, const int8_t *s, int lds, int n,
                                int R, long long s_upper, int32_t *E, int32_t *C) {
    const int r = blockIdx.x;
    __shared__ long long hs[32];
    long long part = 0;
    if (h8)
        for (int i = threadIdx.x; i < n; i += blockDim.x) part += (long long)h8[i] * s[(size_t)r * lds + i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) hs[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long hsum = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) hsum += hs[w];
        const long long sr = (long long)sum[r];
        if (E) E[r] = (int32_t)(-(sr / 2) - hsum);
        if (C) C[r] = (int32_t)((sr - 2 * s_upper) / 4);
    }
}

si_status tc_readout_buffer(Ctx *c) {
    if (c->R > c->e_sum_cap) {
        if (c->e_sum) cudaFree(c->e_sum);
        c->e_sum = nullptr;
        c->e_sum_cap = 0;
        SI_CUDA_TRY(si_dev_malloc((void **)&c->e_sum, sizeof(unsigned long long) * c->R));
        c->e_sum_cap = c->R;
    }
    return SI_OK;
}

si_status tc_energy_finish(Ctx *c, int R, int32_t *E, int32_t *C) {
    k_energy_finish<<<R, 128, 0, c->stream>>>(c->e_sum, c->has_h ? c->dh8 : nullptr, c->dspins, c->ld8, c->n, R,
                                              c->s_upper, E, C);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

// Exact energy/cut of R spin vectors (staged in spins_dev [R][ld], ld == c->ld8)
// for a tensor-path context with integer J.  Returns SI_ERR_UNSUPPORTED when
// the tensor readout does not apply (the caller falls back to dp4a).
si_status tc_energy(Ctx *c, const int8_t *spins_dev, int R, int ld, int32_t *E, int32_t *C) {
    if (c->path != Path::TENSOR || !c->integer_j || !c->dJ || !c->derr) return SI_ERR_UNSUPPORTED;
    const int rpad = round_up(R, TE_BN);
    const size_t bytes = (size_t)rpad * c->ldk * 2;
    if (bytes > c->e_sig_bytes) {
        if (c->e_sig) cudaFree(c->e_sig);
        c->e_sig = nullptr;
        c->e_sig_bytes = 0;
        SI_CUDA_TRY(si_dev_malloc(&c->e_sig, bytes));
        c->e_sig_bytes = bytes;
    }
    if (R > c->e_sum_cap) {
        if (c->e_sum) cudaFree(c->e_sum);
        c->e_sum = nullptr;
        c->e_sum_cap = 0;
        SI_CUDA_TRY(si_dev_malloc((void **)&c->e_sum, sizeof(unsigned long long) * R));
        c->e_sum_cap = R;
    }
    const int grid1 = std::min(8 * c->num_sms, cdiv((long long)rpad * c->ldk, 256));
    k_spins_to_bf16<<<grid1, 256, 0, c->stream>>>(spins_dev, ld, c->n, R, (__nv_bfloat16 *)c->e_sig, c->ldk, rpad);
    SI_CUDA_TRY(cudaGetLastError());
    CUtensorMap mapS;
    si_status s = tc_make_map_bf16(&mapS, c->e_sig, c->ldk, rpad, TE_BK, TE_BN);
    if (s != SI_OK) return s;
    CUtensorMap mapA;
    s = c->j_e4m3 ? tc_make_map_e4m3(&mapA, c->dJ, c->ldk, c->mpad, TE_BM)
                  : tc_make_map_bf16(&mapA, c->dJ, c->ldk, c->mpad, TE_BK, TE_BM);
    if (s != SI_OK) return s;
    SI_CUDA_TRY(cudaMemsetAsync(c->e_sum, 0, sizeof(unsigned long long) * R, c->stream));
    TeArgs a;
    a.n = c->n;
    a.R = R;
    a.kblocks = c->ldk / TE_BK;
    a.spins = spins_dev;
    a.lds = ld;
    a.sum = c->e_sum;
    a.err = c->derr;
    a.limit_ns = c->spin_limit_ns;
    dim3 grid(c->mpad / TE_BM, rpad / TE_BN);
    if (c->j_e4m3) {
        SI_CUDA_TRY(cudaFuncSetAttribute(k_tc_sigma_j_sigma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TE_SMEM));
        k_tc_sigma_j_sigma<true><<<grid, TE_THREADS, TE_SMEM, c->stream>>>(mapA, mapS, a);
    } else {
        SI_CUDA_TRY(cudaFuncSetAttribute(k_tc_sigma_j_sigma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TE_SMEM));
        k_tc_sigma_j_sigma<false><<<grid, TE_THREADS, TE_SMEM, c->stream>>>(mapA, mapS, a);
    }
    SI_CUDA_TRY(cudaGetLastError());
    k_energy_finish<<<R, 128, 0, c->stream>>>(c->e_sum, c->has_h ? c->dh8 : nullptr, spins_dev, ld, c->n, R,
                                              c->s_upper, E, C);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 3;
    return SI_OK;
}

}  // namespace si
