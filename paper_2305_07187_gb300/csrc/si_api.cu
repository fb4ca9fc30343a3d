// C ABI of the Spring-Ising hot path: context life cycle, argument checks,
// host/device staging and dispatch to the kernel families.
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <string>

#include "si_internal.cuh"

namespace si {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of a failed query
        return false;
    }
    if (attr.type == cudaMemoryTypeManaged) return true;
    if (attr.type != cudaMemoryTypeDevice) return false;
    // memory of another GPU is staged like host memory (copied with
    // cudaMemcpyDefault), so no kernel here dereferences a peer address
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess && attr.device == dev;
}

// A pointer argument staged on the device: either the caller's device
// pointer or a temporary copy of host data.
struct DevIn {
    const void *ptr = nullptr;
    void *owned = nullptr;
    ~DevIn() {
        if (owned) cudaFree(owned);
    }
};

static si_status stage_in(DevIn &d, const void *src, size_t bytes, cudaStream_t st) {
    if (!src) {
        d.ptr = nullptr;
        return SI_OK;
    }
    if (is_device_ptr(src)) {
        d.ptr = src;
        return SI_OK;
    }
    SI_CUDA_TRY(si_dev_malloc(&d.owned, bytes));
    SI_CUDA_TRY(cudaMemcpyAsync(d.owned, src, bytes, cudaMemcpyDefault, st));
    d.ptr = d.owned;
    return SI_OK;
}

// Output staging: device destination is written directly; a host destination
// gets a device temporary that is copied back by finish().
struct DevOut {
    void *host = nullptr;
    void *ptr = nullptr;
    void *owned = nullptr;
    size_t bytes = 0;
    ~DevOut() {
        if (owned) cudaFree(owned);
    }
};

static si_status stage_out(DevOut &d, void *dst, size_t bytes) {
    d.bytes = bytes;
    if (!dst) return SI_OK;
    if (is_device_ptr(dst)) {
        d.ptr = dst;
        return SI_OK;
    }
    SI_CUDA_TRY(si_dev_malloc(&d.owned, bytes));
    d.ptr = d.owned;
    d.host = dst;
    return SI_OK;
}

static si_status finish_out(DevOut &d, cudaStream_t st) {
    if (d.host) SI_CUDA_TRY(cudaMemcpyAsync(d.host, d.ptr, d.bytes, cudaMemcpyDefault, st));
    return SI_OK;
}

// Read and clear the device error word; synchronises the stream.
static si_status check_device_error(Ctx *c);

// End of a call: enqueue the copies to host outputs, then one synchronising
// read of the device error word covers them and every launch before.  A call
// that may return early (si_run, si_energy) and has neither a host output nor
// a host input returns once its work is enqueued: a device error of its
// kernels is reported by the next synchronising call.
// A call with a host input never returns early either: its copies from the
// caller's memory (pinned memory is read asynchronously) must have finished
// before the caller may reuse that memory.
static si_status finish_call(Ctx *c, std::initializer_list<DevOut *> outs, bool may_return_early = false,
                             bool host_in = false) {
    bool host_out = false;
    for (DevOut *d : outs) {
        si_status s = finish_out(*d, c->stream);
        if (s != SI_OK) return s;
        host_out = host_out || d->host != nullptr;
    }
    if (may_return_early && !host_out && !host_in) return SI_OK;
    if (c->derr) return check_device_error(c);
    SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SI_OK;
}

static si_status check_device_error(Ctx *c) {
    int local = 0;
    int *dst = c->herr ? c->herr : &local;
    SI_CUDA_TRY(cudaMemcpyAsync(dst, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const int herr = *dst;
    if (herr != DEV_OK) {
        // the error may come from an earlier call that returned early: no
        // state of a run is left to continue from or to read back
        c->have_run = false;
        c->run_spins_valid = false;
        SI_CUDA_TRY(cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream));
        SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (herr == DEV_BAD_CONFIG) {
            set_error("kernel rejected its launch configuration");
            return SI_ERR_UNSUPPORTED;
        }
        set_error(herr == DEV_TIMEOUT_BARRIER ? "inter-CTA step barrier timed out"
                                              : "mbarrier wait timed out");
        return SI_ERR_TIMEOUT;
    }
    return SI_OK;
}

static std::atomic<long> g_alloc_count{0};

cudaError_t dev_malloc_raw(void **p, size_t bytes) {
    if (const char *e = std::getenv("SI_DEBUG_FAIL_ALLOC")) {
        const long k = std::atol(e);
        if (k > 0 && g_alloc_count.fetch_add(1) + 1 == k) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

void alloc_fault_reset() { g_alloc_count = 0; }

static void free_ctx(Ctx *c) {
    if (!c) return;
    if (c->grp) {
        cudaStreamSynchronize(c->stream);
        group_ctx_free(c);   // also clears the pointers that alias its buffers
    }
    void *ptrs[] = {c->dJ, c->dJ8, c->dh, c->dhf, c->dh8, c->dq, c->dp, c->dqbuf,
                    c->dzeta, c->ddt, c->dbar, c->derr, c->dspins, c->dspins_in,
                    c->dE, c->dC, c->dEf, c->dstage, c->g_ws, c->e_sig, c->e_sum, c->dxch, c->dqT,
                    c->w_sum, c->w_ctl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->herr) cudaFreeHost(c->herr);
    adj_tc_free(c->g_tc);
    if (c->g_graph) cudaGraphExecDestroy(c->g_graph);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

static si_status check_params(const si_params *p) {
    if (!p) { set_error("params is NULL"); return SI_ERR_INVALID_ARG; }
    if (p->n < 1 || p->replicas < 1 || p->steps < 0) {
        set_error("need n >= 1, replicas >= 1, steps >= 0");
        return SI_ERR_INVALID_ARG;
    }
    if (p->prec < SI_PREC_FP32 || p->prec > SI_PREC_J_BF16_Q_BF16) {
        set_error("unknown precision");
        return SI_ERR_INVALID_ARG;
    }
    if (p->update_order != 0 && p->update_order != 1) {
        set_error("update_order must be 0 (kick-drift) or 1 (literal Eq. 5)");
        return SI_ERR_INVALID_ARG;
    }
    if (!(p->m > 0.f) || !(p->q_max > 0.f) || !(p->p_max > 0.f) || !std::isfinite(p->k) ||
        !std::isfinite(p->q0) || !std::isfinite(p->m) || !std::isfinite(p->q_max) ||
        !std::isfinite(p->p_max)) {
        set_error("need finite k, q0 and positive finite m, q_max, p_max");
        return SI_ERR_INVALID_ARG;
    }
    if (p->ckpt_every < 0 || p->tile_n < 0) {
        set_error("ckpt_every and tile_n must be >= 0");
        return SI_ERR_INVALID_ARG;
    }
    if (p->fused_readout != 0 && p->fused_readout != 1) {
        set_error("fused_readout must be 0 or 1");
        return SI_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3; ++i)
        if (p->reserved[i] != 0) {
            set_error("reserved fields must be zero");
            return SI_ERR_INVALID_ARG;
        }
    if ((long long)p->n * p->n > (1LL << 34)) {
        set_error("n too large");
        return SI_ERR_UNSUPPORTED;
    }
    return SI_OK;
}

template <typename T>
__global__ void k_copy_h(const float *h, int n, T *out, float *outf, int8_t *out8) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = h ? h[i] : 0.f;
        out[i] = (T)v;
        outf[i] = v;
        if (out8) out8[i] = (int8_t)v;
    }
}

static si_status create_impl(Ctx *c, const float *J, const float *h) {
    const si_params &p = c->prm;
    const int n = p.n;
    SI_CUDA_TRY(cudaGetDevice(&c->device));
    SI_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    if (const char *e = std::getenv("SI_SPIN_LIMIT_NS")) {
        long long v = std::atoll(e);
        if (v > 0) c->spin_limit_ns = v;
    }
    if (const char *e = std::getenv("SI_DEBUG_STALL_STEP")) c->stall_step = std::atoi(e);
    if (const char *e = std::getenv("SI_DEBUG_STALL_RANK")) c->stall_rank = std::atoi(e);
    DevIn Jd, hd;
    si_status s = stage_in(Jd, J, (size_t)n * n * sizeof(float), c->stream);
    if (s != SI_OK) return s;
    s = stage_in(hd, h, (size_t)n * sizeof(float), c->stream);
    if (s != SI_OK) return s;
    unsigned long long flags = 0;
    long long s_upper = 0;
    s = simt_validate((const float *)Jd.ptr, (const float *)hd.ptr, n, p.prec, &flags, &s_upper, c->stream);
    if (s != SI_OK) return s;
    if (flags & (VF_NONFINITE | VF_H_NONFINITE)) {
        set_error("J or h holds a non-finite value");
        return SI_ERR_INVALID_ARG;
    }
    if (flags & (VF_ASYM | VF_DIAG)) {
        set_error("J must be symmetric with a zero diagonal");
        return SI_ERR_NOT_SYMMETRIC;
    }
    if (p.prec == SI_PREC_J_FP8_Q_BF16 && (flags & VF_NOT_E4M3)) {
        set_error("SI_PREC_J_FP8_Q_BF16 needs every J entry exact in e4m3");
        return SI_ERR_INVALID_ARG;
    }
    c->integer_j = !(flags & VF_NOT_INT8);
    c->bf16_j = !(flags & VF_NOT_BF16);
    c->has_h = (h != nullptr);
    c->integer_h = !(flags & VF_H_NOT_INT8);
    c->s_upper = c->integer_j ? s_upper : 0;
    c->n = n;
    c->R = p.replicas;
    c->ld8 = round_up(n, 16);

    // Error word and spin readout buffer (the grouped service of a tensor
    // context writes both).
    SI_CUDA_TRY(si_dev_malloc((void **)&c->derr, sizeof(int)));
    SI_CUDA_TRY(cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream));
    // word 0: the device error word's copy; word 1: a watched run's first hit
    if (cudaHostAlloc((void **)&c->herr, 2 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();   // optional: the read then goes through pageable memory
        c->herr = nullptr;
    }
    SI_CUDA_TRY(si_dev_malloc((void **)&c->dspins, (size_t)c->R * c->ld8));
    SI_CUDA_TRY(cudaMemsetAsync(c->dspins, 0, (size_t)c->R * c->ld8, c->stream));

    // Coupling storage.
    const bool tensor = p.prec == SI_PREC_J_FP8_Q_BF16 || p.prec == SI_PREC_J_BF16_Q_BF16;
    const bool f64 = p.prec == SI_PREC_FP64;
    const size_t es = f64 ? 8 : 4;
    if (tensor) {
        c->path = Path::TENSOR;
        // one persistent launch for all steps when its grid is co-resident,
        // else one grouped launch per step
        s = tc_persistent_fits(c) ? tc_prepare(c, (const float *)Jd.ptr)
                                  : group_ctx_create(c, (const float *)Jd.ptr, (const float *)hd.ptr);
        if (s != SI_OK) return s;
    } else {
        c->path = (c->R <= 4) ? Path::PLAIN_PERSISTENT : Path::SIMT_TILED;
        s = simt_convert_j(c, (const float *)Jd.ptr, n);
        if (s != SI_OK) return s;
        SI_CUDA_TRY(si_dev_malloc(&c->dp, (size_t)c->R * n * es));
        c->qbuf_bytes = 2 * (size_t)c->R * c->ldj * es;
        SI_CUDA_TRY(si_dev_malloc(&c->dqbuf, c->qbuf_bytes));
        SI_CUDA_TRY(cudaMemsetAsync(c->dqbuf, 0, c->qbuf_bytes, c->stream));
        if (c->path == Path::PLAIN_PERSISTENT && !f64) {
            c->xch_bytes = 2 * (size_t)c->R * c->ldj * sizeof(unsigned long long);
            SI_CUDA_TRY(si_dev_malloc((void **)&c->dxch, c->xch_bytes));
        }
        if (c->path == Path::SIMT_TILED && !f64) {
            const size_t bytes = 3 * (size_t)c->ldj * round_up(c->R, 128) * sizeof(float);
            SI_CUDA_TRY(si_dev_malloc((void **)&c->dqT, bytes));
            SI_CUDA_TRY(cudaMemsetAsync(c->dqT, 0, bytes, c->stream));
        }
    }
    // int8 copy of J for the dp4a readout (tensor contexts read out on the
    // tensor cores and build it only if ever needed)
    if (c->integer_j && !tensor) SI_CUDA_TRY(si_dev_malloc((void **)&c->dJ8, (size_t)n * c->ld8));
    // h copies.
    SI_CUDA_TRY(si_dev_malloc((void **)&c->dhf, sizeof(float) * n));
    if (c->integer_h && c->has_h) SI_CUDA_TRY(si_dev_malloc((void **)&c->dh8, n));
    if (f64) {
        SI_CUDA_TRY(si_dev_malloc(&c->dh, sizeof(double) * n));
        k_copy_h<double><<<std::min(1024, cdiv(n, 256)), 256, 0, c->stream>>>(
            (const float *)hd.ptr, n, (double *)c->dh, c->dhf, c->dh8);
    } else {
        SI_CUDA_TRY(si_dev_malloc(&c->dh, sizeof(float) * n));
        k_copy_h<float><<<std::min(1024, cdiv(n, 256)), 256, 0, c->stream>>>(
            (const float *)hd.ptr, n, (float *)c->dh, c->dhf, c->dh8);
    }
    SI_CUDA_TRY(cudaGetLastError());
    if (!c->has_h) {
        // keep the pointers (zero field) but let kernels skip the add
        cudaFree(c->dh);
        c->dh = nullptr;
    }
    const int sched = std::max(1, p.steps);
    SI_CUDA_TRY(si_dev_malloc((void **)&c->dzeta, sizeof(float) * sched));
    SI_CUDA_TRY(si_dev_malloc((void **)&c->ddt, sizeof(float) * sched));
    c->nbar = 4096;
    SI_CUDA_TRY(si_dev_malloc((void **)&c->dbar, sizeof(unsigned) * c->nbar));
    if (c->dJ8) {
        si_status s8 = convert_j8(c, (const float *)Jd.ptr);
        if (s8 != SI_OK) return s8;
    }
    SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SI_OK;
}

// Kernel to pad-copy spins [R][n] (any pointer) into [R][ld] staging.
__global__ void k_pad_spins(const int8_t *src, int n, int R, int8_t *dst, int ld) {
    const long long total = (long long)R * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ld), i = (int)(e % ld);
        dst[e] = i < n ? src[(size_t)r * n + i] : (int8_t)0;
    }
}

__global__ void k_unpad_spins(const int8_t *src, int ld, int n, int R, int8_t *dst) {
    const long long total = (long long)R * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), i = (int)(e % n);
        dst[e] = src[(size_t)r * ld + i];
    }
}

}  // namespace si

using namespace si;

extern "C" {

void si_default_params(si_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->k = 0.5f;
    p->m = 1.0f;
    p->q0 = 0.0f;
    p->q_max = std::sqrt(2.0f);
    p->p_max = 2.0f;
    p->prec = SI_PREC_FP32;
    p->update_order = SI_ORDER_KICK_DRIFT;
}

si_status si_create(si_ctx **out, const si_params *prm, const float *J, const float *h,
                    void *stream) {
    NvtxRange nvtx_range("si_create");
    set_error("");
    alloc_fault_reset();
    if (!out || !J) {
        set_error("si_create: out and J are required");
        return SI_ERR_INVALID_ARG;
    }
    *out = nullptr;
    si_status s = check_params(prm);
    if (s != SI_OK) return s;
    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return SI_ERR_OOM;
    c->prm = *prm;
    c->stream = (cudaStream_t)stream;
    s = create_impl(c, J, h);
    if (s != SI_OK) {
        free_ctx(c);
        return s;
    }
    *out = reinterpret_cast<si_ctx *>(c);
    return SI_OK;
}

si_status si_run(si_ctx *ctx, const float *zeta, const float *dt, const float *q_init,
                 const float *p_init, float *q_out, float *p_out, int8_t *spins_out) {
    NvtxRange nvtx_range("si_run");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || (c->prm.steps > 0 && (!zeta || !dt))) {
        set_error("si_run: ctx, zeta and dt are required");
        return SI_ERR_INVALID_ARG;
    }
    const bool cont = (q_init == nullptr);
    if (cont && (p_init || !c->have_run)) {
        set_error("si_run: q_init NULL continues from the context's state: needs a completed si_run or si_grad, "
                  "and p_init NULL");
        return SI_ERR_INVALID_ARG;
    }
    c->launches = 0;
    const int steps = c->prm.steps, n = c->n, R = c->R;
    const size_t sb = sizeof(float) * std::max(steps, 1);
    const bool host_in = (steps > 0 && (!is_device_ptr(zeta) || !is_device_ptr(dt))) ||
                         (q_init && !is_device_ptr(q_init)) || (p_init && !is_device_ptr(p_init));
    if (steps > 0) {
        const cudaMemcpyKind kz = cudaMemcpyDefault, kd = cudaMemcpyDefault;
        SI_CUDA_TRY(cudaMemcpyAsync(c->dzeta, zeta, sizeof(float) * steps, kz, c->stream));
        SI_CUDA_TRY(cudaMemcpyAsync(c->ddt, dt, sizeof(float) * steps, kd, c->stream));
    }
    (void)sb;
    DevIn qi, pi;
    si_status s = stage_in(qi, q_init, sizeof(float) * (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    s = stage_in(pi, p_init, sizeof(float) * (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    DevOut qo, po, so;
    if ((s = stage_out(qo, q_out, sizeof(float) * (size_t)R * n)) != SI_OK) return s;
    if ((s = stage_out(po, p_out, sizeof(float) * (size_t)R * n)) != SI_OK) return s;
    if ((s = stage_out(so, spins_out, (size_t)R * n)) != SI_OK) return s;

    c->ev_valid = false;
    // the state is rewritten from here on: only a successful run leaves one
    // to continue from or to read back
    c->have_run = false;
    c->fused_valid = false;
    if (c->path == Path::TENSOR && c->grp) {
        if (!cont) {
            const size_t bytes = sizeof(float) * (size_t)R * n;
            SI_CUDA_TRY(cudaMemcpyAsync(c->dq, qi.ptr, bytes, cudaMemcpyDeviceToDevice, c->stream));
            if (pi.ptr) SI_CUDA_TRY(cudaMemcpyAsync(c->dp, pi.ptr, bytes, cudaMemcpyDeviceToDevice, c->stream));
            else SI_CUDA_TRY(cudaMemsetAsync(c->dp, 0, bytes, c->stream));
        }
        if ((s = group_ctx_prepare(c, steps)) != SI_OK) return s;
        if (c->timing) SI_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        if ((s = group_ctx_run(c, steps)) != SI_OK) return s;
    } else if (c->path == Path::TENSOR) {
        // A continuing run starts from the bf16 plane the last run left
        // (rebuilt from the FP32 state only when that plane is not current).
        if (!cont) {
            s = tc_init_state(c, (const float *)qi.ptr, (const float *)pi.ptr);
            c->tc_p0 = 0;
        } else if (c->tc_plane >= 0) {
            c->tc_p0 = c->tc_plane;
        } else {
            s = tc_continue_state(c);
            c->tc_p0 = 0;
        }
        if (s != SI_OK) return s;
        c->tc_plane = -1;
        c->tc_readout = c->prm.fused_readout == 1 && steps > 0 && tc_readout_supported(c);
        if (c->tc_readout && (s = tc_readout_buffer(c)) != SI_OK) return s;
        if (c->timing) SI_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        if ((s = tc_run(c, steps, c->dspins)) != SI_OK) return s;
        c->tc_plane = (steps + c->tc_p0) & 1;
    } else {
        s = cont ? simt_continue_state(c) : simt_init_state(c, (const float *)qi.ptr, (const float *)pi.ptr);
        if (s != SI_OK) return s;
        if (c->timing) SI_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        if ((s = simt_run(c, steps, c->dspins)) != SI_OK) return s;
        c->cur_parity = steps & 1;
    }
    if (c->timing) {
        SI_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
        c->ev_valid = true;
    }
    if (q_out || p_out) {
        if (c->path == Path::TENSOR) s = tc_copy_state(c, (float *)qo.ptr, (float *)po.ptr);
        else s = simt_copy_state(c, (float *)qo.ptr, (float *)po.ptr);
        if (s != SI_OK) return s;
    }
    if (steps == 0) {
        // no step ran: spins of the initial positions
        if (c->path == Path::TENSOR) {
            if ((s = tc_spins(c, c->dspins, c->ld8)) != SI_OK) return s;
        } else if ((s = simt_spins(c, c->dspins, c->ld8)) != SI_OK) {
            return s;
        }
    }
    c->run_spins_valid = false;
    if (spins_out) {
        k_unpad_spins<<<std::min(4096, cdiv((long long)R * n, 256)), 256, 0, c->stream>>>(
            c->dspins, c->ld8, n, R, (int8_t *)so.ptr);
        SI_CUDA_TRY(cudaGetLastError());
        c->launches += 1;
    }
    if ((s = finish_call(c, {&qo, &po, &so}, true, host_in)) != SI_OK) return s;
    c->have_run = true;
    c->run_spins_valid = true;
    c->fused_valid = c->path == Path::TENSOR && !c->grp && c->tc_readout;
    return SI_OK;
}

si_status si_run_watch(si_ctx *ctx, const float *zeta, const float *dt, const float *q_init,
                       const float *p_init, int32_t every, int64_t target_energy, float *q_out, float *p_out,
                       int8_t *spins_out, int32_t *steps_done, int32_t *energy_out) {
    NvtxRange nvtx_range("si_run_watch");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || (c->prm.steps > 0 && (!zeta || !dt)) || every < 1) {
        set_error("si_run_watch: ctx, zeta and dt are required, every >= 1");
        return SI_ERR_INVALID_ARG;
    }
    if (c->path != Path::TENSOR || !tc_readout_supported(c)) {
        set_error("si_run_watch: needs a tensor-path context (one kernel for all steps) with integer J and h");
        return SI_ERR_UNSUPPORTED;
    }
    const bool cont = (q_init == nullptr);
    if (cont && (p_init || !c->have_run)) {
        set_error("si_run_watch: q_init NULL continues from the context's state: needs a completed run, "
                  "and p_init NULL");
        return SI_ERR_INVALID_ARG;
    }
    c->launches = 0;
    const int steps = c->prm.steps, n = c->n, R = c->R;
    if (steps > 0) {
        SI_CUDA_TRY(cudaMemcpyAsync(c->dzeta, zeta, sizeof(float) * steps, cudaMemcpyDefault, c->stream));
        SI_CUDA_TRY(cudaMemcpyAsync(c->ddt, dt, sizeof(float) * steps, cudaMemcpyDefault, c->stream));
    }
    DevIn qi, pi;
    si_status s = stage_in(qi, q_init, sizeof(float) * (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    s = stage_in(pi, p_init, sizeof(float) * (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    DevOut qo, po, so, eo;
    if ((s = stage_out(qo, q_out, sizeof(float) * (size_t)R * n)) != SI_OK) return s;
    if ((s = stage_out(po, p_out, sizeof(float) * (size_t)R * n)) != SI_OK) return s;
    if ((s = stage_out(so, spins_out, (size_t)R * n)) != SI_OK) return s;
    if ((s = stage_out(eo, energy_out, sizeof(int32_t) * (size_t)R)) != SI_OK) return s;
    c->ev_valid = false;
    c->have_run = false;
    c->fused_valid = false;
    if (!cont) {
        s = tc_init_state(c, (const float *)qi.ptr, (const float *)pi.ptr);
        c->tc_p0 = 0;
    } else if (c->tc_plane >= 0) {
        c->tc_p0 = c->tc_plane;
    } else {
        s = tc_continue_state(c);
        c->tc_p0 = 0;
    }
    if (s != SI_OK) return s;
    c->tc_plane = -1;
    const int nread = steps > 0 ? cdiv(steps, every) : 0;
    int local = 0x7fffffff;
    int *hh = c->herr ? c->herr + 1 : &local;
    if (steps > 0) {
        if ((s = tc_watch_buffers(c, steps, every)) != SI_OK) return s;
        c->tc_readout = false;
        c->tc_watch_every = every;
        c->tc_watch_target = target_energy;
        if (c->timing) SI_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        s = tc_run(c, steps, c->dspins);
        c->tc_watch_every = 0;
        if (s != SI_OK) return s;
        if (c->timing) {
            SI_CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
            c->ev_valid = true;
        }
        // the first readout that reached the target (read after the one
        // synchronisation at the end of the call)
        SI_CUDA_TRY(cudaMemcpyAsync(hh, c->w_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    } else if ((s = tc_spins(c, c->dspins, c->ld8)) != SI_OK) {
        return s;
    }
    if (q_out || p_out) {
        if ((s = tc_copy_state(c, (float *)qo.ptr, (float *)po.ptr)) != SI_OK) return s;
    }
    if (spins_out) {
        k_unpad_spins<<<std::min(4096, cdiv((long long)R * n, 256)), 256, 0, c->stream>>>(c->dspins, c->ld8, n, R,
                                                                                        (int8_t *)so.ptr);
        SI_CUDA_TRY(cudaGetLastError());
        c->launches += 1;
    }
    if (energy_out) {
        if (nread == 0) {
            set_error("si_run_watch: no readout without steps");
            return SI_ERR_INVALID_ARG;
        }
        if ((s = tc_watch_energy(c, nread, (int32_t *)eo.ptr)) != SI_OK) return s;
    }
    if ((s = finish_call(c, {&qo, &po, &so, &eo}, false, true)) != SI_OK) return s;
    int done = steps;
    if (nread > 0) {
        const int hit = *hh;
        const int kstop = (hit >= 0 && hit < nread) ? hit : nread - 1;
        done = std::min(steps, (kstop + 1) * every);
    }
    c->tc_plane = (done + c->tc_p0) & 1;
    if (steps_done) *steps_done = done;
    c->have_run = true;
    c->run_spins_valid = true;
    return SI_OK;
}

si_status si_get_state(si_ctx *ctx, double *q_out, double *p_out) {
    NvtxRange nvtx_range("si_get_state");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (c && c->derr && c->have_run) {
        // a run that returned early may have failed since: report it first
        const si_status e = check_device_error(c);
        if (e != SI_OK) return e;
    }
    if (!c || !c->have_run) {
        set_error("si_get_state: no completed run");
        return SI_ERR_INVALID_ARG;
    }
    const size_t bytes = sizeof(double) * (size_t)c->R * c->n;
    DevOut qo, po;
    si_status s;
    if ((s = stage_out(qo, q_out, bytes)) != SI_OK) return s;
    if ((s = stage_out(po, p_out, bytes)) != SI_OK) return s;
    if (c->path == Path::TENSOR) s = tc_copy_state_f64(c, (double *)qo.ptr, (double *)po.ptr);
    else s = simt_copy_state_f64(c, (double *)qo.ptr, (double *)po.ptr);
    if (s != SI_OK) return s;
    if ((s = finish_out(qo, c->stream)) != SI_OK) return s;
    if ((s = finish_out(po, c->stream)) != SI_OK) return s;
    SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SI_OK;
}

si_status si_energy(si_ctx *ctx, const int8_t *spins, int32_t R, int32_t *energy_out,
                    int32_t *cut_out, double *energy_f) {
    NvtxRange nvtx_range("si_energy");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || R < 0) {
        set_error("si_energy: ctx is required, R >= 0");
        return SI_ERR_INVALID_ARG;
    }
    if (!spins && (!c->run_spins_valid || R != c->R)) {
        set_error("si_energy: spins NULL reads the last si_run's spins: needs a completed si_run and R = replicas");
        return SI_ERR_INVALID_ARG;
    }
    c->launches = 0;
    if (R == 0) return SI_OK;
    if ((energy_out || cut_out) && !c->integer_j) {
        set_error("exact int32 energy/cut needs integer J with |J_ij| <= 127");
        return SI_ERR_UNSUPPORTED;
    }
    if (energy_out && c->has_h && !c->integer_h) {
        set_error("exact int32 energy needs integer h with |h_i| <= 127");
        return SI_ERR_UNSUPPORTED;
    }
    const int n = c->n;
    si_status s;
    DevOut eo, co, fo;
    if ((s = stage_out(eo, energy_out, sizeof(int32_t) * R)) != SI_OK) return s;
    if ((s = stage_out(co, cut_out, sizeof(int32_t) * R)) != SI_OK) return s;
    if ((s = stage_out(fo, energy_f, sizeof(double) * R)) != SI_OK) return s;
    if (!spins && c->fused_valid && !energy_f) {
        // the step kernel already summed sigma^T J sigma of these spins
        s = tc_energy_finish(c, R, (int32_t *)eo.ptr, (int32_t *)co.ptr);
        if (s != SI_OK) return s;
        return finish_call(c, {&eo, &co, &fo}, true);
    }
    if (!spins) {
        // the last run's spins, already in the padded layout
        s = simt_energy(c, c->dspins, R, c->ld8, (int32_t *)eo.ptr, (int32_t *)co.ptr, (double *)fo.ptr);
        if (s != SI_OK) return s;
        return finish_call(c, {&eo, &co, &fo}, true);
    }
    DevIn sd;
    s = stage_in(sd, spins, (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    if (R > c->spins_in_cap) {
        if (c->dspins_in) cudaFree(c->dspins_in);
        c->dspins_in = nullptr;
        c->spins_in_cap = 0;
        SI_CUDA_TRY(si_dev_malloc((void **)&c->dspins_in, (size_t)R * c->ld8));
        c->spins_in_cap = R;
    }
    k_pad_spins<<<std::min(4096, cdiv((long long)R * c->ld8, 256)), 256, 0, c->stream>>>(
        (const int8_t *)sd.ptr, n, R, c->dspins_in, c->ld8);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    s = simt_energy(c, c->dspins_in, R, c->ld8, (int32_t *)eo.ptr, (int32_t *)co.ptr, (double *)fo.ptr);
    if (s != SI_OK) return s;
    return finish_call(c, {&eo, &co, &fo}, true, sd.owned != nullptr);
}

si_status si_hamiltonian(si_ctx *ctx, const float *q, const float *p, int32_t R, double zeta,
                         double *H_out) {
    NvtxRange nvtx_range("si_hamiltonian");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || R < 0 || (R > 0 && (!q || !p || !H_out))) {
        set_error("si_hamiltonian: ctx is required, R >= 0, and q, p, H_out when R > 0");
        return SI_ERR_INVALID_ARG;
    }
    c->launches = 0;
    if (R == 0) return SI_OK;
    const size_t bytes = sizeof(float) * (size_t)R * c->n;
    DevIn qd, pd;
    si_status s = stage_in(qd, q, bytes, c->stream);
    if (s != SI_OK) return s;
    if ((s = stage_in(pd, p, bytes, c->stream)) != SI_OK) return s;
    DevOut ho;
    if ((s = stage_out(ho, H_out, sizeof(double) * R)) != SI_OK) return s;
    s = monitor_hamiltonian(c, (const float *)qd.ptr, (const float *)pd.ptr, R, zeta, (double *)ho.ptr);
    if (s != SI_OK) return s;
    if ((s = finish_out(ho, c->stream)) != SI_OK) return s;
    SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SI_OK;
}

si_status si_grad(si_ctx *ctx, const float *zeta, const float *dt, const float *q_init,
                  const float *p_init, float *g_zeta, float *g_dt, float *g_k,
                  float *objective) {
    NvtxRange nvtx_range("si_grad");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !q_init || (c->prm.steps > 0 && (!zeta || !dt))) {
        set_error("si_grad: ctx, q_init, zeta and dt are required");
        return SI_ERR_INVALID_ARG;
    }
    if (c->path == Path::TENSOR || c->prm.update_order != 0 || c->prm.wall_zero_p) {
        set_error("si_grad supports FP32/FP64 contexts, kick-drift order, no wall_zero_p");
        return SI_ERR_UNSUPPORTED;
    }
    c->launches = 0;
    const int steps = c->prm.steps, n = c->n, R = c->R;
    if (steps > 0) {
        const cudaMemcpyKind kz = cudaMemcpyDefault, kd = cudaMemcpyDefault;
        SI_CUDA_TRY(cudaMemcpyAsync(c->dzeta, zeta, sizeof(float) * steps, kz, c->stream));
        SI_CUDA_TRY(cudaMemcpyAsync(c->ddt, dt, sizeof(float) * steps, kd, c->stream));
    }
    DevIn qi, pi;
    si_status s = stage_in(qi, q_init, sizeof(float) * (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    s = stage_in(pi, p_init, sizeof(float) * (size_t)R * n, c->stream);
    if (s != SI_OK) return s;
    DevOut gz, gd, gk, ob;
    if ((s = stage_out(gz, g_zeta, sizeof(float) * std::max(steps, 1))) != SI_OK) return s;
    if ((s = stage_out(gd, g_dt, sizeof(float) * std::max(steps, 1))) != SI_OK) return s;
    if ((s = stage_out(gk, g_k, sizeof(float))) != SI_OK) return s;
    if ((s = stage_out(ob, objective, sizeof(float))) != SI_OK) return s;
    c->run_spins_valid = false;   // the sweep replaces the context's state
    c->fused_valid = false;
    s = adjoint_grad(c, steps, (float *)gz.ptr, (float *)gd.ptr, (float *)gk.ptr, (float *)ob.ptr,
                     (const float *)qi.ptr, (const float *)pi.ptr);
    if (s != SI_OK) return s;
    return finish_call(c, {&gz, &gd, &gk, &ob});
}

si_status si_set_params(si_ctx *ctx, const si_params *prm) {
    NvtxRange nvtx_range("si_set_params");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) {
        set_error("si_set_params: ctx is required");
        return SI_ERR_INVALID_ARG;
    }
    si_status s = check_params(prm);
    if (s != SI_OK) return s;
    const si_params &o = c->prm;
    if (prm->n != o.n || prm->replicas != o.replicas || prm->steps != o.steps || prm->prec != o.prec ||
        prm->tile_n != o.tile_n) {
        set_error("si_set_params: n, replicas, steps, prec and tile_n are fixed at si_create");
        return SI_ERR_INVALID_ARG;
    }
    // Work already enqueued read the old values at launch; only the captured
    // gradient sweep holds them, so it is captured again on the next si_grad.
    c->prm = *prm;
    if (c->grp) group_ctx_params(c);
    if (c->g_graph) {
        SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
        cudaGraphExecDestroy(c->g_graph);
        c->g_graph = nullptr;
    }
    c->g_graph_key = -1;
    return SI_OK;
}

si_status si_describe(const si_ctx *ctx, char *buf, int32_t len) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c || !buf || len <= 0) return SI_ERR_INVALID_ARG;
    const char *prec[] = {"fp32", "fp64", "j_fp8_q_bf16", "j_bf16_q_bf16"};
    if (c->path == Path::TENSOR && c->grp) {
        group_ctx_describe(c, buf, len);
    } else if (c->path == Path::TENSOR) {
        tc_describe(c, buf, len);
    } else if (c->path == Path::PLAIN_PERSISTENT) {
        std::snprintf(buf, len, "plain_persistent prec=%s n=%d R=%d", prec[c->prm.prec], c->n, c->R);
    } else {
        std::snprintf(buf, len, "simt_tiled prec=%s n=%d R=%d tile=64x64", prec[c->prm.prec], c->n, c->R);
    }
    if (c->g_path) {
        const size_t l = std::strlen(buf);
        if ((int)l + 1 < len) {
            if (c->g_path == 2 && adj_tc_run_splits(c->g_tc) > 0)
                std::snprintf(buf + l, len - l, " grad=tcgen05-bf16x3 ksplit=%d sweep=persistent%s",
                              adj_tc_run_splits(c->g_tc), adj_tc_run_pair(c->g_tc) ? "-side-by-side" : "");
            else if (c->g_path == 2)
                std::snprintf(buf + l, len - l, " grad=tcgen05-bf16x3 ksplit=%d sweep=per-step",
                              adj_tc_splits(c->g_tc));
            else
                std::snprintf(buf + l, len - l, " grad=cuda-core");
        }
    }
    return SI_OK;
}

si_status si_enable_timing(si_ctx *ctx, int32_t on) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return SI_ERR_INVALID_ARG;
    if (on && !c->ev0) {
        SI_CUDA_TRY(cudaEventCreate(&c->ev0));
        SI_CUDA_TRY(cudaEventCreate(&c->ev1));
    }
    c->timing = on != 0;
    c->ev_valid = false;
    return SI_OK;
}

si_status si_synchronize(si_ctx *ctx) {
    NvtxRange nvtx_range("si_synchronize");
    set_error("");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) {
        set_error("si_synchronize: ctx is required");
        return SI_ERR_INVALID_ARG;
    }
    if (c->derr) return check_device_error(c);
    SI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SI_OK;
}

si_status si_last_kernel_time(const si_ctx *ctx, float *ms) {
    Ctx *c = const_cast<Ctx *>(reinterpret_cast<const Ctx *>(ctx));
    if (!c || !ms) return SI_ERR_INVALID_ARG;
    if (!c->ev_valid) {
        set_error("no timed run (enable timing before si_run)");
        return SI_ERR_INVALID_ARG;
    }
    SI_CUDA_TRY(cudaEventSynchronize(c->ev1));
    if (c->derr && c->have_run) {
        // a run that returned early may have ended on a timed-out wait: its
        // events then bracket an aborted kernel, so report the error instead
        const si_status e = check_device_error(c);
        if (e != SI_OK) {
            c->ev_valid = false;
            return e;
        }
    }
    SI_CUDA_TRY(cudaEventElapsedTime(ms, c->ev0, c->ev1));
    return SI_OK;
}

int32_t si_last_launch_count(const si_ctx *ctx) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    return c ? c->launches : 0;
}

const char *si_last_error(void) { return g_last_error.c_str(); }

void si_destroy(si_ctx *ctx) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

}  // extern "C"
