// Allocation-free entry point: si_run_noalloc.
//
// Some callers cannot allocate device memory at all: a plugin inside a host
// application that owns every device allocation and forbids others, a
// real-time control loop that must not enter the allocator, or code that
// runs while a memory pool is being captured or is already exhausted.  This
// entry point serves them with the single-replica FP32 run (the persistent
// matvec-plus-integrator kernel of the plain path) and takes its scratch --
// the double-buffered exchange vector of positions, the inter-CTA step
// counter and the device error word -- from a fixed array in this file
// instead of cudaMalloc.  The caller still provides J, the schedules and the
// state; nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <string>

#include "si_device.cuh"

namespace si {

constexpr int NOALLOC_MAX_N = SI_NOALLOC_MAX_N;
constexpr int NOALLOC_THREADS = 512;

// Scratch layout (bytes): [0, 4) step counter, [4, 8) error word,
// [256, 256 + 8 * NOALLOC_MAX_N) two position vectors of n floats.
constexpr size_t NOALLOC_HEADER = 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + 2 * sizeof(float) * (size_t)NOALLOC_MAX_N;

// Held by every GPU that loads the library, until the process exits.  In
// host code `g_noalloc_scratch` names a host-side shadow, not device memory:
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocArgs {
    const float *J;       // [n][n], row stride n
    const float *h;       // [n] or null
    int n, steps;
    const float *zeta, *dt;
    float *qbuf;          // scratch: [2][n], step t reads buffer t&1
    float *p;             // caller's momenta [n], updated in place
    int8_t *spins;        // caller's [n] or null (written after the last step)
    unsigned *bar;        // scratch counter
    int *err;             // scratch error word
    long long limit_ns;
    StepParams sp;
    int rows_per_block;
    int j_resident;
};

// Same algorithm and summation order as the plain persistent kernel, with
// scalar loads so that J may have any row stride n.  Lane l sums the chunks
// j = 4l + 128u, .. +3 as an FMA chain, chunk sums are accumulated with
// compensation and the warp tree carries the compensation.
__global__ void __launch_bounds__(NOALLOC_THREADS, 1) k_plain_noalloc(NoallocArgs a) {
    extern __shared__ __align__(16) float sm_f[];
    float *sq = sm_f;                 // [n]
    float *sJ = sm_f + a.n;           // [rows][n] when resident
    const int row0 = blockIdx.x * a.rows_per_block;
    const int nrows = max(0, min(a.rows_per_block, a.n - row0));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    if (a.j_resident && nrows > 0) {
        const float *src = a.J + (size_t)row0 * a.n;
        const int total = nrows * a.n;
        for (int e = threadIdx.x; e < total; e += blockDim.x) sJ[e] = src[e];
    }
    for (int t = 0; t < a.steps; ++t) {
        const float *qc = a.qbuf + (size_t)(t & 1) * a.n;
        float *qn = a.qbuf + (size_t)((t + 1) & 1) * a.n;
        for (int e = threadIdx.x; e < a.n; e += blockDim.x) sq[e] = __ldcg(qc + e);
        __syncthreads();
        const float zt = a.zeta[t], dtt = a.dt[t];
        const float dtm = dtt / a.sp.m;
        for (int rr = warp; rr < nrows; rr += nwarps) {
            const int i = row0 + rr;
            const float *Jrow = a.j_resident ? sJ + (size_t)rr * a.n : a.J + (size_t)i * a.n;
            CompSum<float> acc;
            acc.init();
            for (int j = lane * 4; j < a.n; j += 128) {
                float d = Jrow[j] * sq[j];
#pragma unroll
                for (int v = 1; v < 4; ++v) {
                    const float jv = (j + v < a.n) ? Jrow[j + v] : 0.f;
                    const float qv = (j + v < a.n) ? sq[j + v] : 0.f;
                    d = fmaf(jv, qv, d);
                }
                acc.add(d);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float oh = __shfl_down_sync(0xffffffffu, acc.hi, off);
                const float ol = __shfl_down_sync(0xffffffffu, acc.lo, off);
                acc.merge(oh, ol);
            }
            if (lane == 0) {
                const float hi = a.h ? a.h[i] : 0.f;
                float qo, po;
                integrate<float>(sq[i], a.p[i], acc.value() + hi, zt, dtt, dtm, a.sp, qo, po);
                qn[i] = qo;
                a.p[i] = po;
                if (a.spins && t == a.steps - 1) a.spins[i] = spin_of(qo);
            }
        }
        if (!grid_barrier(a.bar, (unsigned)(t + 1) * gridDim.x, a.err, a.limit_ns)) break;
    }
}

// Device address of the scratch array, resolved once per device.
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[128];
static bool g_noalloc_ready[128];

static si_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= 128) {
        set_error("si_run_noalloc: device ordinal out of range");
        return SI_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ready[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error(std::string("si_run_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return SI_ERR_CUDA;
        }
        g_noalloc_ptr[device] = ptr;
        g_noalloc_ready[device] = true;
    }
    *out = static_cast<unsigned char *>(g_noalloc_ptr[device]);
    return SI_OK;
}

}  // namespace si

using namespace si;

extern "C" si_status si_run_noalloc(const si_params *prm, const float *J, const float *h,
                                    const float *zeta, const float *dt, float *q, float *p,
                                    int8_t *spins_out, void *stream) {
    set_error("");
    if (!prm || !J || !q || !p || (prm->steps > 0 && (!zeta || !dt))) {
        set_error("si_run_noalloc: prm, J, q, p (and zeta, dt when steps > 0) are required");
        return SI_ERR_INVALID_ARG;
    }
    const int n = prm->n;
    if (n < 1 || prm->steps < 0 || prm->replicas != 1) {
        set_error("si_run_noalloc: needs n >= 1, steps >= 0 and replicas == 1");
        return SI_ERR_INVALID_ARG;
    }
    if (n > NOALLOC_MAX_N) {
        set_error("si_run_noalloc: n exceeds SI_NOALLOC_MAX_N (the fixed scratch holds two "
                  "position vectors of at most SI_NOALLOC_MAX_N floats)");
        return SI_ERR_INVALID_ARG;
    }
    if (prm->prec != SI_PREC_FP32 || !(prm->m > 0.f) || !(prm->q_max > 0.f) || !(prm->p_max > 0.f) ||
        (prm->update_order != 0 && prm->update_order != 1)) {
        set_error("si_run_noalloc: FP32 precision, m, q_max, p_max > 0 and order 0 or 1 required");
        return SI_ERR_INVALID_ARG;
    }
    const void *ptrs[] = {J, zeta, dt, q, p};
    for (const void *ptr : ptrs)
        if (ptr && !is_device_ptr(ptr)) {
            set_error("si_run_noalloc: J, zeta, dt, q, p must be device pointers");
            return SI_ERR_INVALID_ARG;
        }
    if ((h && !is_device_ptr(h)) || (spins_out && !is_device_ptr(spins_out))) {
        set_error("si_run_noalloc: h and spins_out must be device pointers");
        return SI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int device = 0, sms = 0, max_smem = 0;
    SI_CUDA_TRY(cudaGetDevice(&device));
    SI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    SI_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    unsigned char *scratch = nullptr;
    si_status s = noalloc_scratch(device, &scratch);
    if (s != SI_OK) return s;

    NoallocArgs a;
    a.J = J;
    a.h = h;
    a.n = n;
    a.steps = prm->steps;
    a.zeta = zeta;
    a.dt = dt;
    a.qbuf = reinterpret_cast<float *>(scratch + NOALLOC_HEADER);
    a.p = p;
    a.spins = spins_out;
    a.bar = reinterpret_cast<unsigned *>(scratch);
    a.err = reinterpret_cast<int *>(scratch + 4);
    a.limit_ns = 2000000000LL;
    if (const char *e = std::getenv("SI_SPIN_LIMIT_NS")) {
        long long v = std::atoll(e);
        if (v > 0) a.limit_ns = v;
    }
    a.sp = StepParams{prm->k, prm->m, prm->q0, prm->q_max, prm->p_max, prm->update_order, prm->wall_zero_p};
    int grid = sms;
    a.rows_per_block = cdiv(n, grid);
    grid = cdiv(n, a.rows_per_block);
    const size_t sq_bytes = sizeof(float) * (size_t)n;
    const size_t sj_bytes = sizeof(float) * (size_t)a.rows_per_block * n;
    a.j_resident = (sq_bytes + sj_bytes + 1024 <= (size_t)max_smem) ? 1 : 0;
    const size_t smem = sq_bytes + (a.j_resident ? sj_bytes : 0);
    SI_CUDA_TRY(cudaFuncSetAttribute(k_plain_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plain_noalloc, NOALLOC_THREADS, smem));
    if (per_sm * sms < grid) {
        set_error("si_run_noalloc: grid cannot be co-resident");
        return SI_ERR_UNSUPPORTED;
    }
    // The scratch keeps the previous call's contents: clear the counter and
    // the error word, and seed buffer 0 with the caller's positions.
    SI_CUDA_TRY(cudaMemsetAsync(scratch, 0, 8, st));
    SI_CUDA_TRY(cudaMemcpyAsync(a.qbuf, q, sq_bytes, cudaMemcpyDeviceToDevice, st));
    if (a.steps > 0) {
        void *args[] = {&a};
        SI_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_plain_noalloc, dim3(grid),
                                                dim3(NOALLOC_THREADS), args, smem, st));
    } else if (spins_out) {
        set_error("si_run_noalloc: spins_out needs steps >= 1");
        return SI_ERR_INVALID_ARG;
    }
    // Read the error word before the positions go back to the caller: a run
    // that timed out leaves q as it came in (p is updated in place and is
    // then unspecified).
    int herr = 0;
    SI_CUDA_TRY(cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr != DEV_OK) {
        set_error("si_run_noalloc: inter-CTA step barrier timed out");
        return SI_ERR_TIMEOUT;
    }
    SI_CUDA_TRY(cudaMemcpyAsync(q, a.qbuf + (size_t)(a.steps & 1) * n, sq_bytes, cudaMemcpyDeviceToDevice, st));
    SI_CUDA_TRY(cudaStreamSynchronize(st));
    return SI_OK;
}
