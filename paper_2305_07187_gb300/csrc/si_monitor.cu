// Hamiltonian of the spring system in FP64, for drift monitoring.
//
// H_r = sum_i p_ri^2 / (2m) + k/2 sum_i (q_ri - q0)^2 + zeta * U(q_r),
// U(q) = -1/2 q^T J q - h^T q,
// i.e. the kinetic energy and spring potential of Eq. 2 / Eq. 3 plus the
// coupling potential of Eq. 4 (its force is zeta (J q + h)), with the field
// term of Eq. 1 included.  The integrator does not conserve H exactly; the
// monitor reports how far it moves over a stretch of constant zeta.
//
// One CTA per HM_R replicas; warps over rows of J, lanes over columns.  J is
// the context's working copy (FP32, FP64, bf16 or e4m3), so H is the energy of the
// system the kernels actually integrate.  All sums are FP64 and reduced in a
// fixed order, so the result is deterministic.
#include <cuda_bf16.h>

#include "si_device.cuh"

namespace si {

constexpr int HM_R = 4;
constexpr int HM_THREADS = 512;

template <typename TJ>
__device__ __forceinline__ double to_f64(TJ x) { return (double)x; }
template <>
__device__ __forceinline__ double to_f64<__nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <>
__device__ __forceinline__ double to_f64<__nv_fp8_e4m3>(__nv_fp8_e4m3 x) { return (double)(float)x; }

template <typename TJ>
__global__ void __launch_bounds__(HM_THREADS) k_hamiltonian(const TJ *J, int ldj, const float *h, int n, int R,
                                                            const float *q, const float *p, double zeta,
                                                            double k, double m, double q0, double *H) {
    __shared__ double s_pair[HM_THREADS / 32][HM_R];
    __shared__ double s_loc[HM_THREADS / 32][HM_R];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int r0 = blockIdx.x * HM_R;
    const int nr = min(HM_R, R - r0);
    // pair[u] = sum over this warp's rows i of q_i (J q)_i for replica r0+u
    double pair[HM_R];
#pragma unroll
    for (int u = 0; u < HM_R; ++u) pair[u] = 0.0;
    for (int i = warp; i < n; i += nwarps) {
        const TJ *Jrow = J + (size_t)i * ldj;
        double dot[HM_R];
#pragma unroll
        for (int u = 0; u < HM_R; ++u) dot[u] = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double Jij = to_f64(Jrow[j]);
#pragma unroll
            for (int u = 0; u < HM_R; ++u)
                if (u < nr) dot[u] = fma(Jij, (double)__ldg(q + (size_t)(r0 + u) * n + j), dot[u]);
        }
#pragma unroll
        for (int u = 0; u < HM_R; ++u) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dot[u] += __shfl_down_sync(0xffffffffu, dot[u], off);
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < HM_R; ++u)
                if (u < nr) pair[u] = fma((double)q[(size_t)(r0 + u) * n + i], dot[u], pair[u]);
        }
    }
    // local terms: kinetic, spring and field, spread over all threads
    double loc[HM_R];
#pragma unroll
    for (int u = 0; u < HM_R; ++u) {
        loc[u] = 0.0;
        if (u < nr) {
            const float *qr = q + (size_t)(r0 + u) * n;
            const float *pr = p + (size_t)(r0 + u) * n;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const double qi = qr[i], pi = pr[i], d = qi - q0;
                double t = 0.5 * (pi / m) * pi + 0.5 * k * d * d;
                if (h) t -= zeta * (double)h[i] * qi;
                loc[u] += t;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) loc[u] += __shfl_down_sync(0xffffffffu, loc[u], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < HM_R; ++u) {
            s_pair[warp][u] = pair[u];
            s_loc[warp][u] = loc[u];
        }
    }
    __syncthreads();
    if (threadIdx.x < nr) {
        const int u = threadIdx.x;
        double a = 0.0, b = 0.0;
        for (int w = 0; w < nwarps; ++w) {
            a += s_pair[w][u];
            b += s_loc[w][u];
        }
        H[r0 + u] = b - 0.5 * zeta * a;
    }
}

si_status monitor_hamiltonian(Ctx *c, const float *q, const float *p, int R, double zeta, double *H) {
    const int grid = cdiv(R, HM_R);
    const float *h = c->has_h ? c->dhf : nullptr;
    const double k = c->prm.k, m = c->prm.m, q0 = c->prm.q0;
    if (c->path == Path::TENSOR && c->j_e4m3) {
        k_hamiltonian<__nv_fp8_e4m3><<<grid, HM_THREADS, 0, c->stream>>>(
            (const __nv_fp8_e4m3 *)c->dJ, c->ldk, h, c->n, R, q, p, zeta, k, m, q0, H);
    } else if (c->path == Path::TENSOR) {
        k_hamiltonian<__nv_bfloat16><<<grid, HM_THREADS, 0, c->stream>>>(
            (const __nv_bfloat16 *)c->dJ, c->ldk, h, c->n, R, q, p, zeta, k, m, q0, H);
    } else if (c->prm.prec == SI_PREC_FP64) {
        k_hamiltonian<double><<<grid, HM_THREADS, 0, c->stream>>>((const double *)c->dJ, c->ldj, h, c->n, R, q, p,
                                                                  zeta, k, m, q0, H);
    } else {
        k_hamiltonian<float><<<grid, HM_THREADS, 0, c->stream>>>((const float *)c->dJ, c->ldj, h, c->n, R, q, p,
                                                                 zeta, k, m, q0, H);
    }
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    return SI_OK;
}

}  // namespace si
