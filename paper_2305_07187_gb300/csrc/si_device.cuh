// Device-side helpers shared by the CUDA translation units: bounded waits,
// the inter-CTA step barrier and the integrator of one time step.
#pragma once

#include "si_internal.cuh"

namespace si {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int *p) {
    return *(const volatile int *)p;
}

// Spin until *ctr >= target (wrap-around safe).  Gives up when another CTA
// has raised the error word or when limit_ns has passed; in the latter case
// it raises DEV_TIMEOUT_BARRIER itself.  Returns true on success.
__device__ __forceinline__ bool wait_counter_geq(const unsigned *ctr, unsigned target,
                                                 int *err, long long limit_ns) {
    unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        unsigned v = ld_acquire_gpu(ctr);
        if ((int)(v - target) >= 0) return true;
        if ((it & 31u) == 0) {
            if (err && ld_volatile_int(err) != 0) return false;
            if ((long long)(globaltimer_ns() - t0) > limit_ns) {
                if (err) atomicCAS(err, 0, DEV_TIMEOUT_BARRIER);
                return false;
            }
        }
    }
}

// Barrier over all CTAs of the grid for step t (counter starts at 0 each
// launch).  Every thread of the CTA must call it; returns false for all of
// them if the wait failed.
__device__ __forceinline__ bool grid_barrier(unsigned *ctr, unsigned target, int *err,
                                             long long limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_gpu_add(ctr, 1u);
        ok = wait_counter_geq(ctr, target, err, limit_ns) ? 1 : 0;
    }
    __syncthreads();
    return ok != 0;
}

// One time step for one (spin, replica) pair.  F already includes h.
// order 0 (Eq. 8): p from q(t_n), then q from the new p.
// order 1 (Eq. 5): both from the old state.
// Walls (Eq. 6): clamp q to [-q_max, q_max], p to [-p_max, p_max]; with
// wall_zero_p the momentum of a clipped spin is set to zero.
// MODE 1 is the same arithmetic with order 0 and wall_zero_p off fixed at
// compile time (for loops that test those parameters once, outside).
// The roundings are pinned (no contraction left to the compiler), in this
// order: d = q - q0, u = (-k) d, w = zeta F + u (fused), a = dt w + p
// (fused), b = dtm x + q (fused), so that the two-wide form below and every
// kernel compute the same values.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T, int MODE = 0>
__device__ __forceinline__ void integrate(T q, T p, T F, T zeta, T dt, T dtm,
                                          const StepParams &sp, T &q_out, T &p_out) {
    const T k = (T)sp.k, q0 = (T)sp.q0, qmax = (T)sp.q_max, pmax = (T)sp.p_max;
    const int order = MODE == 1 ? 0 : sp.order;
    const bool wall_zero_p = MODE == 1 ? false : sp.wall_zero_p != 0;
    const T d = rn_add(q, -q0);
    const T u = rn_mul(-k, d);
    const T w = rn_fma(zeta, F, u);
    const T a = rn_fma(dt, w, p);
    const T pn0 = fmin(fmax(a, -pmax), pmax);
    const T b = rn_fma(dtm, order == 0 ? pn0 : p, q);
    T pn = pn0;
    const T qn = fmin(fmax(b, -qmax), qmax);
    if (wall_zero_p && qn != b) pn = (T)0;
    q_out = qn;
    p_out = pn;
}

// Two (spin, replica) pairs of the default update (kick-drift, walls without
// momentum zeroing) with Blackwell's two-wide FP32 instructions: the same
// roundings as integrate<float, 1> element by element.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ void integrate2_kd(float q_lo, float q_hi, float p_lo, float p_hi, float F_lo, float F_hi,
                                              float zeta, float dt, float dtm, const StepParams &sp,
                                              float &qo_lo, float &qo_hi, float &po_lo, float &po_hi) {
    const float qmax = sp.q_max, pmax = sp.p_max;
    const unsigned long long Q = f2_pack(q_lo, q_hi);
    const unsigned long long d = f2_add(Q, f2_pack(-sp.q0, -sp.q0));
    const unsigned long long u = f2_mul(f2_pack(-sp.k, -sp.k), d);
    const unsigned long long w = f2_fma(f2_pack(zeta, zeta), f2_pack(F_lo, F_hi), u);
    const unsigned long long av = f2_fma(f2_pack(dt, dt), w, f2_pack(p_lo, p_hi));
    float a0, a1;
    f2_unpack(av, a0, a1);
    const float pn0 = fminf(fmaxf(a0, -pmax), pmax), pn1 = fminf(fmaxf(a1, -pmax), pmax);
    const unsigned long long bv = f2_fma(f2_pack(dtm, dtm), f2_pack(pn0, pn1), Q);
    float b0, b1;
    f2_unpack(bv, b0, b1);
    qo_lo = fminf(fmaxf(b0, -qmax), qmax);
    qo_hi = fminf(fmaxf(b1, -qmax), qmax);
    po_lo = pn0;
    po_hi = pn1;
}

// One reverse step of the kick-drift iteration (the adjoint of Eq. 8 with
// the walls of Eq. 6), with pinned roundings so that every adjoint kernel
// computes the same values.  Through the clamps, with the interior
// indicators of the stored next state (|q'| < q_max, |p'| < p_max):
//   lb = D_q lq',  la = D_p (lp' + (dt/m) lb).
template <typename T>
__device__ __forceinline__ void adj_clamps(T lq, T lp, T qn, T pn, T qmax, T pmax, T dtm, T &la, T &lb) {
    lb = (fabs(qn) < qmax) ? lq : (T)0;
    la = (fabs(pn) < pmax) ? rn_fma(dtm, lb, lp) : (T)0;
}
// lq = lb + dt (-k la + zeta G) with G = J la (and lp = la).
template <typename T>
__device__ __forceinline__ T adj_lq(T lb, T la, T G, T dtt, T zt, T k) {
    return rn_fma(dtt, rn_fma(-k, la, rn_mul(zt, G)), lb);
}
// One element's terms of g_dt, g_zeta and g_k at step t (q, F of step t,
// p' of step t+1):
//   lb p'/m + la (-k (q - q0) + zeta F),   dt la F,   -dt la (q - q0).
template <typename T>
__device__ __forceinline__ void adj_terms(T la, T lb, T q, T F, T pn, T q0, T k, T m, T zt, T dtt, T &g_dt,
                                          T &g_zeta, T &g_k) {
    const T dq = rn_add(q, -q0);
    const T force = rn_fma(-k, dq, rn_mul(zt, F));
    g_dt = rn_fma(la, force, rn_mul(lb, pn) / m);
    const T dla = rn_mul(dtt, la);
    g_zeta = rn_mul(dla, F);
    g_k = -rn_mul(dla, dq);
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = a + b;
    const T z = s - a;
    e = (a - (s - z)) + (b - z);
}

// Compensated accumulator: (hi, lo) carries a running sum whose rounding
// errors are kept in lo; chunk partial sums are added with two_sum.
template <typename T>
struct CompSum {
    T hi, lo;
    __device__ __forceinline__ void init() { hi = (T)0; lo = (T)0; }
    __device__ __forceinline__ void add(T x) {
        T s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ void merge(T ohi, T olo) {
        T s, e;
        two_sum(hi, ohi, s, e);
        hi = s;
        lo += olo + e;
    }
    __device__ __forceinline__ T value() const { return hi + lo; }
};

// Three-piece bf16 split of an FP32 value: x = p0 + p1 + p2 up to the last
// bits of the significand, each piece the round-to-nearest bf16 of the
// residual left by the previous ones (the residuals are exact in FP32).
__device__ __forceinline__ void bf16_split3(float x, __nv_bfloat16 &p0, __nv_bfloat16 &p1, __nv_bfloat16 &p2) {
    p0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(p0);
    p1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(p1);
    p2 = __float2bfloat16_rn(r2);
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their writes are visible (returns at once when the
// launch had no programmatic dependency), and let the next grid in the
// stream start its prologue.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ int8_t spin_of(T q) {
    return q >= (T)0 ? (int8_t)1 : (int8_t)-1;
}

}  // namespace si
