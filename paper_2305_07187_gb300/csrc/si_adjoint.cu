// Adjoint sweep of the Spring-Ising iteration (FP32 / FP64 on CUDA cores).
//
// Objective: the relaxed Ising energy at the final step,
//   L = sum_r ( -1/2 q_r^T J q_r - h^T q_r ),   q_r = positions after T steps,
// differentiated with respect to the schedules zeta[T], dt[T] and the spring
// constant k.  One kick-drift step (Eq. 8 with the walls of Eq. 6) maps
//   a  = p + dt (-k (q - q0) + zeta F),   F = J q + h,
//   p' = clip(a),  b = q + (dt/m) p',  q' = clip(b),
// and its adjoint, with D_p, D_q the interior indicators of the clamps, is
//   lb = D_q lq',  la = D_p (lp' + (dt/m) lb),
//   lq = lb + dt (-k la + zeta J la),  lp = la,
//   g_dt   += sum lb p'/m + la (-k (q - q0) + zeta F)
//   g_zeta += dt sum la F,   g_k += -dt sum la (q - q0),
// started from lq_T = -(J q_T + h), lp_T = 0.
//
// A clamp is active exactly when the clamped value sits on the wall, so the
// indicators are read from the stored next state: D_p = |p'| < p_max and
// D_q = |q'| < q_max (strict, the derivative at the kink is taken as 0).
//
// Memory: checkpoints of (q, p) every K steps; a segment of K steps is
// recomputed from its checkpoint with the same kernels (bit-identical
// states), keeping q_t, p_t and F_t of every step of the segment, then swept
// backwards.  Gradient sums are per-block partials reduced in a fixed order
// (deterministic).
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <type_traits>

#include "si_device.cuh"

namespace si {

constexpr int AG_M = 64, AG_R = 64, AG_K = 16, AG_THREADS = 256;
constexpr int AE_BLOCKS = 256, AE_THREADS = 256;

enum GemmMode { GM_FORWARD = 0, GM_TERMINAL = 1, GM_ADJOINT = 2 };

template <typename T>
struct AdjGemmArgs {
    const T *J;
    int ldj;
    const T *h;
    int n, R;
    const T *X;          // operand [R][ldj]
    // forward: X = q_t;  P = p_t;  outputs q_{t+1}, p_{t+1}, F_t
    const T *P;
    T *Qn, *Pn, *Fo;
    // adjoint: X = la;  reads lb;  writes lq, lp
    const T *LB;
    T *LQ, *LP;
    // terminal: objective partials per block (-1/2 x.G - h.x)
    T *obj_part;
    StepParams sp;
    const float *zeta, *dt;
    int t;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(AG_THREADS) k_adj_gemm(AdjGemmArgs<T> a) {
    __shared__ T As[AG_K][AG_M + 1];
    __shared__ T Bs[AG_K][AG_R + 1];
    __shared__ T red[AG_THREADS];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int i0 = blockIdx.x * AG_M, r0 = blockIdx.y * AG_R;
    CompSum<T> acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v].init();
    const int lrow = tid / 4, lk = (tid % 4) * 4;
    for (int k0 = 0; k0 < a.ldj; k0 += AG_K) {
        const int i = i0 + lrow;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            As[lk + v][lrow] = (i < a.n) ? a.J[(size_t)i * a.ldj + k0 + lk + v] : (T)0;
        const int r = r0 + lrow;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            Bs[lk + v][lrow] = (r < a.R) ? a.X[(size_t)r * a.ldj + k0 + lk + v] : (T)0;
        __syncthreads();
        T part[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) part[u][v] = (T)0;
#pragma unroll
        for (int kk = 0; kk < AG_K; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = Bs[kk][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) part[u][v] = fma(av[u], bv[v], part[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v].add(part[u][v]);
        __syncthreads();
    }
    T objp = (T)0;
    const T k = (T)a.sp.k, q0 = (T)a.sp.q0;
    T zt = 0, dtt = 0, dtm = 0;
    if (MODE != GM_TERMINAL) {
        zt = (T)a.zeta[a.t];
        dtt = (T)a.dt[a.t];
        dtm = dtt / (T)a.sp.m;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty * 4 + u;
        if (i >= a.n) continue;
        const T hi = a.h ? a.h[i] : (T)0;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = r0 + tx * 4 + v;
            if (r >= a.R) continue;
            const size_t e = (size_t)r * a.ldj + i;
            const T G = acc[u][v].value();
            if (MODE == GM_FORWARD) {
                const T F = G + hi;
                T qo, po;
                integrate<T>(a.X[e], a.P[e], F, zt, dtt, dtm, a.sp, qo, po);
                a.Qn[e] = qo;
                a.Pn[e] = po;
                a.Fo[e] = F;
            } else if (MODE == GM_TERMINAL) {
                const T x = a.X[e];
                a.LQ[e] = -(G + hi);
                a.LP[e] = (T)0;
                objp += (T)-0.5 * x * G - hi * x;
            } else {
                const T la = a.X[e];
                a.LQ[e] = adj_lq(a.LB[e], la, G, dtt, zt, k);
                a.LP[e] = la;
            }
        }
    }
    (void)q0;
    if (MODE == GM_TERMINAL) {
        red[tid] = objp;
        __syncthreads();
        if (tid == 0) {
            CompSum<T> s;
            s.init();
            for (int w = 0; w < AG_THREADS; ++w) s.add(red[w]);
            a.obj_part[blockIdx.y * gridDim.x + blockIdx.x] = s.value();
        }
    }
}

// Elementwise part of one reverse step: indicators, la, lb and the per-block
// partial sums of the three gradient contributions.
template <typename T>
__global__ void __launch_bounds__(AE_THREADS) k_adj_elem(
    int n, int R, int ld, const T *q, const T *p, const T *F, const T *qn, const T *pn,
    const T *lq, const T *lp, T *la_out, T *lb_out, StepParams sp, const float *zeta,
    const float *dt, int t, T *part /* [3][AE_BLOCKS] of step t */,
    __nv_bfloat16 *xs_la /* tensor-core operand pieces of la, or null */, int ldk) {
    __shared__ T r0s[AE_THREADS], r1s[AE_THREADS], r2s[AE_THREADS];
    grid_dep_wait();
    grid_dep_launch();
    const T k = (T)sp.k, q0 = (T)sp.q0, qmax = (T)sp.q_max, pmax = (T)sp.p_max, m = (T)sp.m;
    const T zt = (T)zeta[t], dtt = (T)dt[t];
    const T dtm = dtt / m;
    CompSum<T> s0, s1, s2;
    s0.init();
    s1.init();
    s2.init();
    const long long total = (long long)R * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), i = (int)(e % n);
        const size_t x = (size_t)r * ld + i;
        T la, lb;
        adj_clamps(lq[x], lp[x], qn[x], pn[x], qmax, pmax, dtm, la, lb);
        la_out[x] = la;
        lb_out[x] = lb;
        if (xs_la) {
            __nv_bfloat16 p0, p1, p2;
            bf16_split3((float)la, p0, p1, p2);
            __nv_bfloat16 *xb = xs_la + ((size_t)(r / ADJ_TC_RB) * ADJ_TC_BN + (r % ADJ_TC_RB)) * ldk + i;
            xb[0] = p0;
            xb[(size_t)ADJ_TC_RB * ldk] = p1;
            xb[(size_t)2 * ADJ_TC_RB * ldk] = p2;
        }
        T g0, g1, g2;
        adj_terms(la, lb, q[x], F[x], pn[x], q0, k, m, zt, dtt, g0, g1, g2);
        s0.add(g0);
        s1.add(g1);
        s2.add(g2);
    }
    (void)p;
    // fixed-shape reduction: warp shuffle trees of the compensated sums,
    // then the warps' results in warp order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T h0 = __shfl_down_sync(0xffffffffu, s0.hi, off), l0 = __shfl_down_sync(0xffffffffu, s0.lo, off);
        const T h1 = __shfl_down_sync(0xffffffffu, s1.hi, off), l1 = __shfl_down_sync(0xffffffffu, s1.lo, off);
        const T h2 = __shfl_down_sync(0xffffffffu, s2.hi, off), l2 = __shfl_down_sync(0xffffffffu, s2.lo, off);
        s0.merge(h0, l0);
        s1.merge(h1, l1);
        s2.merge(h2, l2);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        r0s[warp] = s0.value();
        r1s[warp] = s1.value();
        r2s[warp] = s2.value();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        CompSum<T> a0, a1, a2;
        a0.init();
        a1.init();
        a2.init();
        for (int w = 0; w < AE_THREADS / 32; ++w) {
            a0.add(r0s[w]);
            a1.add(r1s[w]);
            a2.add(r2s[w]);
        }
        part[blockIdx.x] = a0.value();
        part[AE_BLOCKS + blockIdx.x] = a1.value();
        part[2 * AE_BLOCKS + blockIdx.x] = a2.value();
    }
}

// Final fixed-order reductions: g_dt[t], g_zeta[t], g_k and the objective.
// One thread per step for g_dt / g_zeta; block 0 also reduces g_k (thread u
// sums steps u, u+128, ... and thread 0 adds the 128 results in order) and
// the objective.  Launched with 128 threads per block.
template <typename T>
__global__ void k_adj_finish(int T_steps, const T *part, int nb, int nobj, const T *obj_part, float *g_zeta,
                             float *g_dt, float *g_k, float *objective) {
    __shared__ T gks[128];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T_steps) {
        const T *pp = part + (size_t)t * 3 * nb;
        CompSum<T> a0, a1;
        a0.init();
        a1.init();
        for (int b = 0; b < nb; ++b) {
            a0.add(pp[b]);
            a1.add(pp[nb + b]);
        }
        if (g_dt) g_dt[t] = (float)a0.value();
        if (g_zeta) g_zeta[t] = (float)a1.value();
    }
    if (blockIdx.x == 0) {
        CompSum<T> gk;
        gk.init();
        for (int s = threadIdx.x; s < T_steps; s += blockDim.x) {
            const T *pp = part + (size_t)s * 3 * nb + 2 * nb;
            for (int b = 0; b < nb; ++b) gk.add(pp[b]);
        }
        gks[threadIdx.x] = gk.value();
        __syncthreads();
        if (threadIdx.x == 0) {
            CompSum<T> g2, ob;
            g2.init();
            ob.init();
            for (int u = 0; u < (int)blockDim.x; ++u) g2.add(gks[u]);
            for (int b = 0; b < nobj; ++b) ob.add(obj_part[b]);
            if (g_k) *g_k = (float)g2.value();
            if (objective) *objective = (float)ob.value();
        }
    }
}

template <typename T>
__global__ void k_adj_load_state(const float *q_init, const float *p_init, int n, int R, int ld,
                                 T *q, T *p) {
    const long long total = (long long)R * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / ld), i = (int)(e % ld);
        q[e] = i < n ? (T)q_init[(size_t)r * n + i] : (T)0;
        p[e] = (i < n && p_init) ? (T)p_init[(size_t)r * n + i] : (T)0;
    }
}

template <typename T>
static si_status adjoint_impl(Ctx *c, int steps, float *g_zeta, float *g_dt, float *g_k,
                              float *objective, const float *q_init, const float *p_init, AdjTc *tc) {
    const int n = c->n, R = c->R, ld = c->ldj;
    const int K = c->prm.ckpt_every > 0 ? c->prm.ckpt_every : 50;
    const int nseg = steps > 0 ? cdiv(steps, K) : 0;
    const size_t plane = (size_t)R * ld;
    const dim3 ggrid(cdiv(n, AG_M), cdiv(R, AG_R));
    const int nobj = tc ? adj_tc_nobj(tc) : (int)(ggrid.x * ggrid.y);
    // The persistent sweep (tensor cores) keeps two sets of slots, so that a
    // segment can be recomputed while the next one is swept back, and writes
    // one gradient partial per CTA and step.
    const bool persistent = tc && adj_tc_run_splits(tc) > 0;
    const int nb = persistent ? adj_tc_run_nparts(tc) : AE_BLOCKS;
    const int nsets = persistent ? 2 : 1;
    // workspace: ckpt (nseg+1) x {q,p}; nsets x slots (K+1) x {q,p}, F K;
    // lq, lp, la, lb; partials 3 * nb * steps; objective partials.
    const size_t n_planes =
        2 * (size_t)(nseg + 1) + (size_t)nsets * (2 * (size_t)(K + 1) + (size_t)K) + 4;
    // + the outputs g_zeta[T], g_dt[T], g_k, objective (float) at the end
    const size_t out_floats = 2 * (size_t)std::max(steps, 1) + 2;
    const size_t bytes = sizeof(T) * (n_planes * plane + 3 * (size_t)nb * std::max(steps, 1) +
                                      (size_t)nobj) + sizeof(float) * out_floats;
    if (c->g_ws_bytes < bytes) {
        if (c->g_ws) cudaFree(c->g_ws);
        c->g_ws = nullptr;
        c->g_ws_bytes = 0;
        SI_CUDA_TRY(si_dev_malloc(&c->g_ws, bytes));
        c->g_ws_bytes = bytes;
        // Zero once: the padding columns of every plane are never written
        // afterwards and must stay zero for the CUDA-core products.
        SI_CUDA_TRY(cudaMemsetAsync(c->g_ws, 0, bytes, c->stream));
    }
    T *w = (T *)c->g_ws;
    T *ckq = w;                            w += (size_t)(nseg + 1) * plane;
    T *ckp = w;                            w += (size_t)(nseg + 1) * plane;
    T *sq = w;                             w += (size_t)(K + 1) * plane;
    T *sp = w;                             w += (size_t)(K + 1) * plane;
    T *sF = w;                             w += (size_t)K * plane;
    T *sq1 = sq, *sp1 = sp, *sF1 = sF;     // second slot set (persistent sweep)
    if (persistent) {
        sq1 = w;                           w += (size_t)(K + 1) * plane;
        sp1 = w;                           w += (size_t)(K + 1) * plane;
        sF1 = w;                           w += (size_t)K * plane;
    }
    T *lq = w;                             w += plane;
    T *lp = w;                             w += plane;
    T *la = w;                             w += plane;
    T *lb = w;                             w += plane;
    T *part = w;                           w += 3 * (size_t)nb * std::max(steps, 1);
    T *objp = w;                           w += nobj;
    float *gout = reinterpret_cast<float *>(w);   // g_zeta[T], g_dt[T], g_k, objective
    const StepParams spar{c->prm.k, c->prm.m, c->prm.q0, c->prm.q_max, c->prm.p_max, 0, 0};
    const int lg = std::min(4096, cdiv((long long)plane, 256));
    k_adj_load_state<T><<<lg, 256, 0, c->stream>>>(q_init, p_init, n, R, ld, ckq, ckp);
    SI_CUDA_TRY(cudaGetLastError());
    c->launches += 1;

    // The sweep after the initial state is the same sequence of launches on
    // every call of a context: it is captured once into a CUDA graph (on a
    // private stream) and replayed, so the ~7 launches per step do not wait
    // on the host.
    auto sweep = [&]() -> si_status {
        AdjGemmArgs<T> g{};
        g.J = (const T *)c->dJ;
        g.ldj = ld;
        g.h = (const T *)c->dh;
        g.n = n;
        g.R = R;
        g.sp = spar;
        g.zeta = c->dzeta;
        g.dt = c->ddt;

        // The three products of the sweep: on the tensor cores (three-piece bf16
        // split of the operand, FP32 accumulation) when the context has one, else
        // the CUDA-core tiles.  On the tensor cores the operand pieces of a
        // segment's forward chain alternate between buffers 0 and 1 (each
        // forward product writes the pieces of q_{t+1} for the next one; only a
        // segment's first product splits its checkpoint), and lambda_a's pieces,
        // written by the elementwise adjoint kernel, sit in buffer 2.
        auto gemm_forward = [&](const T *X, const T *P, T *Qn, T *Pn, T *Fo, int t, int j) -> si_status {
            if (tc) {
                return adj_tc_gemm(c, tc, 0, (const float *)X, (const float *)P, (float *)Qn, (float *)Pn,
                                   (float *)Fo, nullptr, nullptr, nullptr, nullptr, t, j & 1, j == 0, (j + 1) & 1);
            }
            g.X = X;
            g.P = P;
            g.Qn = Qn;
            g.Pn = Pn;
            g.Fo = Fo;
            g.t = t;
            k_adj_gemm<T, GM_FORWARD><<<ggrid, AG_THREADS, 0, c->stream>>>(g);
            SI_CUDA_TRY(cudaGetLastError());
            c->launches += 1;
            return SI_OK;
        };
        auto gemm_terminal = [&](const T *X) -> si_status {
            if (tc) {
                return adj_tc_gemm(c, tc, 1, (const float *)X, nullptr, nullptr, nullptr, nullptr, nullptr,
                                   (float *)lq, (float *)lp, (float *)objp, 0, 2, true, -1);
            }
            g.X = X;
            g.LQ = lq;
            g.LP = lp;
            g.obj_part = objp;
            k_adj_gemm<T, GM_TERMINAL><<<ggrid, AG_THREADS, 0, c->stream>>>(g);
            SI_CUDA_TRY(cudaGetLastError());
            c->launches += 1;
            return SI_OK;
        };
        auto gemm_adjoint = [&](int t) -> si_status {
            if (tc) {
                return adj_tc_gemm(c, tc, 2, (const float *)la, nullptr, nullptr, nullptr, nullptr, (const float *)lb,
                                   (float *)lq, (float *)lp, nullptr, t, 2, false, -1);
            }
            g.X = la;
            g.LB = lb;
            g.LQ = lq;
            g.LP = lp;
            g.t = t;
            k_adj_gemm<T, GM_ADJOINT><<<ggrid, AG_THREADS, 0, c->stream>>>(g);
            SI_CUDA_TRY(cudaGetLastError());
            c->launches += 1;
            return SI_OK;
        };

        // Recompute segment s from its checkpoint into the slots (q_t, p_t, F_t).
        si_status st;
        auto recompute = [&](int s) -> si_status {
            const int t0 = s * K, len = std::min(K, steps - t0);
            SI_CUDA_TRY(cudaMemcpyAsync(sq, ckq + (size_t)s * plane, sizeof(T) * plane, cudaMemcpyDeviceToDevice, c->stream));
            SI_CUDA_TRY(cudaMemcpyAsync(sp, ckp + (size_t)s * plane, sizeof(T) * plane, cudaMemcpyDeviceToDevice, c->stream));
            for (int j = 0; j < len; ++j) {
                si_status e = gemm_forward(sq + (size_t)j * plane, sp + (size_t)j * plane, sq + (size_t)(j + 1) * plane,
                                           sp + (size_t)(j + 1) * plane, sF + (size_t)j * plane, t0 + j, j);
                if (e != SI_OK) return e;
            }
            return SI_OK;
        };

        if (persistent) {
            // Persistent sweep: the forward pass is one launch (checkpoints at
            // segment ends, segment s's slots in set s & 1); each later
            // launch sweeps segment s back while segment s - 1 is recomputed
            // into the other set (side by side when both chains fit, else
            // one after the other).
            if constexpr (std::is_same<T, float>::value) {
                AdjChain f{};
                f.reverse = 0;
                f.buf0 = 0;
                f.flags = adj_tc_run_flags(tc, 0);
                f.sq[0] = sq; f.sp[0] = sp; f.sF[0] = sF;
                f.sq[1] = sq1; f.sp[1] = sp1; f.sF[1] = sF1;
                AdjChain r = f;
                r.reverse = 1;
                r.buf0 = 2;
                r.flags = adj_tc_run_flags(tc, 1);
                r.lq = lq;
                r.lp = lp;
                r.part = part;
                f.t_start = 0;
                f.len = steps;
                f.q_in = ckq;
                f.p_in = ckp;
                f.ckq = ckq;
                f.ckp = ckp;
                if (steps > 0 && (st = adj_tc_run(c, tc, &f, 1, K)) != SI_OK) return st;
                SI_CUDA_TRY(cudaMemcpyAsync(c->dqbuf, ckq + (size_t)nseg * plane, sizeof(T) * plane,
                                            cudaMemcpyDeviceToDevice, c->stream));
                SI_CUDA_TRY(cudaMemcpy2DAsync(c->dp, sizeof(T) * n, ckp + (size_t)nseg * plane, sizeof(T) * ld,
                                              sizeof(T) * n, R, cudaMemcpyDeviceToDevice, c->stream));
                if ((st = gemm_terminal(ckq + (size_t)nseg * plane)) != SI_OK) return st;
                const bool pair = adj_tc_run_pair(tc);
                for (int s = nseg - 1; s >= 0; --s) {
                    r.t_start = s * K;
                    r.len = std::min(K, steps - s * K);
                    AdjChain ch2[2] = {r, f};
                    int nch = 1;
                    if (s > 0) {
                        ch2[1].t_start = (s - 1) * K;
                        ch2[1].len = K;
                        ch2[1].q_in = ckq + (size_t)(s - 1) * plane;
                        ch2[1].p_in = ckp + (size_t)(s - 1) * plane;
                        ch2[1].ckq = nullptr;
                        ch2[1].ckp = nullptr;
                        nch = 2;
                    }
                    if (nch == 2 && !pair) {
                        if ((st = adj_tc_run(c, tc, &ch2[0], 1, K)) != SI_OK) return st;
                        if ((st = adj_tc_run(c, tc, &ch2[1], 1, K)) != SI_OK) return st;
                    } else if ((st = adj_tc_run(c, tc, ch2, nch, K)) != SI_OK) {
                        return st;
                    }
                }
                const int T1 = std::max(steps, 1);
                k_adj_finish<T><<<cdiv(T1, 128), 128, 0, c->stream>>>(steps, part, nb, nobj, objp, gout, gout + T1,
                                                                      gout + 2 * T1, gout + 2 * T1 + 1);
                SI_CUDA_TRY(cudaGetLastError());
                c->launches += 1;
                return SI_OK;
            }
        }
        // Forward pass: checkpoints at the start of every segment and at T.
        for (int s = 0; s < nseg; ++s) {
            if ((st = recompute(s)) != SI_OK) return st;
            const int len = std::min(K, steps - s * K);
            SI_CUDA_TRY(cudaMemcpyAsync(ckq + (size_t)(s + 1) * plane, sq + (size_t)len * plane, sizeof(T) * plane,
                                        cudaMemcpyDeviceToDevice, c->stream));
            SI_CUDA_TRY(cudaMemcpyAsync(ckp + (size_t)(s + 1) * plane, sp + (size_t)len * plane, sizeof(T) * plane,
                                        cudaMemcpyDeviceToDevice, c->stream));
        }
        // The final state of the forward sweep becomes the context's state
        // (si_get_state reads it): q into exchange buffer 0, p into [R][n].
        SI_CUDA_TRY(cudaMemcpyAsync(c->dqbuf, ckq + (size_t)nseg * plane, sizeof(T) * plane, cudaMemcpyDeviceToDevice,
                                    c->stream));
        SI_CUDA_TRY(cudaMemcpy2DAsync(c->dp, sizeof(T) * n, ckp + (size_t)nseg * plane, sizeof(T) * ld, sizeof(T) * n, R,
                                      cudaMemcpyDeviceToDevice, c->stream));
        // Terminal adjoint and objective at q_T.
        if ((st = gemm_terminal(ckq + (size_t)nseg * plane)) != SI_OK) return st;
        // Reverse sweep.  The slots still hold the last segment from the
        // forward pass, so only the earlier segments are recomputed.
        for (int s = nseg - 1; s >= 0; --s) {
            if (s != nseg - 1 && (st = recompute(s)) != SI_OK) return st;
            const int t0 = s * K, len = std::min(K, steps - t0);
            for (int j = len - 1; j >= 0; --j) {
                const int t = t0 + j;
                {
                    // programmatic dependent launch: the prologue overlaps the
                    // previous product; the kernel waits before reading it
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3(AE_BLOCKS);
                    cfg.blockDim = dim3(AE_THREADS);
                    cfg.stream = c->stream;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    SI_CUDA_TRY(cudaLaunchKernelEx(
                        &cfg, k_adj_elem<T>, n, R, ld, (const T *)(sq + (size_t)j * plane),
                        (const T *)(sp + (size_t)j * plane), (const T *)(sF + (size_t)j * plane),
                        (const T *)(sq + (size_t)(j + 1) * plane), (const T *)(sp + (size_t)(j + 1) * plane),
                        (const T *)lq, (const T *)lp, la, lb, spar, (const float *)c->dzeta, (const float *)c->ddt, t,
                        part + (size_t)t * 3 * AE_BLOCKS, tc ? adj_tc_xs(tc, 2) : (__nv_bfloat16 *)nullptr,
                        tc ? adj_tc_ldk(tc) : 0));
                }
                c->launches += 1;
                if ((st = gemm_adjoint(t)) != SI_OK) return st;
            }
        }
        const int T1 = std::max(steps, 1);
        k_adj_finish<T><<<cdiv(T1, 128), 128, 0, c->stream>>>(steps, part, nb, nobj, objp, gout, gout + T1,
                                                              gout + 2 * T1, gout + 2 * T1 + 1);
        SI_CUDA_TRY(cudaGetLastError());
        c->launches += 1;
        return SI_OK;
    };
    const int key = steps * 4 + (tc ? 1 : 0) + (sizeof(T) == 8 ? 2 : 0);
    if (!c->g_graph || c->g_graph_key != key || c->g_graph_ws != c->g_ws) {
        if (c->g_graph) cudaGraphExecDestroy(c->g_graph);
        c->g_graph = nullptr;
        cudaStream_t cs;
        SI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaStream_t saved = c->stream;
        const int launches0 = c->launches;
        c->stream = cs;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        si_status s = SI_OK;
        if (e == cudaSuccess) {
            s = sweep();
            e = cudaStreamEndCapture(cs, &graph);
        }
        c->stream = saved;
        cudaStreamDestroy(cs);
        c->g_graph_launches = c->launches - launches0;
        c->launches = launches0;
        if (s != SI_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        SI_CUDA_TRY(e);
        e = cudaGraphInstantiate(&c->g_graph, graph, 0);
        cudaGraphDestroy(graph);
        SI_CUDA_TRY(e);
        c->g_graph_key = key;
        c->g_graph_ws = c->g_ws;
    }
    SI_CUDA_TRY(cudaGraphLaunch(c->g_graph, c->stream));
    c->launches += c->g_graph_launches;
    c->cur_parity = 0;
    c->have_run = true;
    const int T1 = std::max(steps, 1);
    if (g_zeta && steps > 0)
        SI_CUDA_TRY(cudaMemcpyAsync(g_zeta, gout, sizeof(float) * steps, cudaMemcpyDeviceToDevice, c->stream));
    if (g_dt && steps > 0)
        SI_CUDA_TRY(cudaMemcpyAsync(g_dt, gout + T1, sizeof(float) * steps, cudaMemcpyDeviceToDevice, c->stream));
    if (g_k) SI_CUDA_TRY(cudaMemcpyAsync(g_k, gout + 2 * T1, sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    if (objective)
        SI_CUDA_TRY(cudaMemcpyAsync(objective, gout + 2 * T1 + 1, sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    return SI_OK;
}

si_status adjoint_grad(Ctx *c, int steps, float *g_zeta, float *g_dt, float *g_k, float *objective,
                       const float *q_init, const float *p_init) {
    if (c->prm.prec == SI_PREC_FP64) {
        c->g_path = 1;
        return adjoint_impl<double>(c, steps, g_zeta, g_dt, g_k, objective, q_init, p_init, nullptr);
    }
    // FP32: the tensor cores take the products when J is exact in bf16
    // (SI_ADJOINT_SIMT=1 keeps them on the CUDA cores).
    AdjTc *tc = nullptr;
    const char *env = std::getenv("SI_ADJOINT_SIMT");
    if (c->bf16_j && !(env && std::atoi(env) == 1)) {
        si_status s = adj_tc_prepare(c, &tc);
        if (s != SI_OK) return s;
    }
    c->g_path = tc ? 2 : 1;
    return adjoint_impl<float>(c, steps, g_zeta, g_dt, g_k, objective, q_init, p_init, tc);
}

}  // namespace si
