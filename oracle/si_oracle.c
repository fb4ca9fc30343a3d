/*
 * Spring-Ising Algorithm -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the paper's equations that the CUDA path is checked
 * against.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product library never links or calls it.
 * It shares no code, header, table or helper with the CUDA sources.
 *
 * Paper: "Point convolutional neural network algorithm for Ising model ground
 * state research based on spring vibration" (arXiv 2305.07187).
 *
 * Every loop below is written in the order the equations state it: no
 * blocking, no fusion, no reordering.  All arithmetic is double precision,
 * round-to-nearest (the paper fixes no precision).
 *
 * Readings of the paper that this file relies on (the paper is silent or
 * inconsistent on these points):
 *   - The coupling force includes the field:  F_i = sum_j J_ij q_j + h_i,
 *     i.e. minus the gradient of the relaxed Ising energy of Eq. 1
 *     (Eq. 4, 5 and 8 print the force without h).
 *   - Default update order is kick-then-drift symplectic Euler: the momentum
 *     line of Eq. 8 is taken literally (it uses q(t_n)), and the position
 *     line then uses the new momentum, which is what makes the scheme
 *     symplectic as Section "Symplectic method" claims.  order == 1 gives
 *     the literal explicit form of Eq. 5 (both lines read the old state).
 *   - Position update uses Delta/m (Eq. 5); Eq. 8 drops m (m = 1 there).
 *   - Walls (Eq. 6 and the constraints after Eq. 8): q is clamped to
 *     [-q_max, q_max] and p to [-p_max, p_max] after each update; with
 *     wall_zero_p != 0 the momentum of a spin whose position was clipped is
 *     set to zero (the "perfectly inelastic wall" reading).
 *   - Spin readout: sigma_i = +1 when q_i >= 0 (including -0.0), else -1.
 *   - MAX-CUT weights are w_ij = -J_ij.
 *
 * Layout: J is n x n row-major; per-replica vectors are replica-major,
 * x[r*n + i].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2

static double clampd(double x, double lo, double hi) {
    if (x < lo) return lo;
    if (x > hi) return hi;
    return x;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * One time step of Eq. 8 (order 0) or Eq. 5 (order 1) for one replica.
 * q, p: length-n state of this replica, updated in place.
 * F: caller-provided length-n work array.
 */
static void or_step_one(int n, const double *J, const double *h, double zeta_n,
                        double dt_n, double k, double m, double q0c,
                        double qmax, double pmax, int order, int wall_zero_p,
                        double *q, double *p, double *F, double *qold) {
    int i, j;
    /* Coupling force, Eq. 4: F_i = sum_j J_ij q_j (+ h_i). */
    for (i = 0; i < n; i++) {
        double s = 0.0;
        for (j = 0; j < n; j++) s += J[(size_t)i * n + j] * q[j];
        F[i] = s + (h ? h[i] : 0.0);
    }
    if (order == 0) {
        /* Momentum line of Eq. 8, then the wall on p. */
        for (i = 0; i < n; i++) {
            double pn = p[i] + dt_n * (-k * (q[i] - q0c) + zeta_n * F[i]);
            p[i] = clampd(pn, -pmax, pmax);
        }
        /* Position line with the new momentum (Eq. 5 with Delta/m), wall of
         * Eq. 6 on q. */
        for (i = 0; i < n; i++) {
            double qn = q[i] + (dt_n / m) * p[i];
            double qc = clampd(qn, -qmax, qmax);
            if (wall_zero_p && qc != qn) p[i] = 0.0;
            q[i] = qc;
        }
    } else {
        /* Literal Eq. 5: both lines read the state at t_n. */
        for (i = 0; i < n; i++) qold[i] = q[i];
        for (i = 0; i < n; i++) {
            double qn = qold[i] + (dt_n / m) * p[i];
            double pn = p[i] + dt_n * (-k * (qold[i] - q0c) + zeta_n * F[i]);
            double qc = clampd(qn, -qmax, qmax);
            p[i] = clampd(pn, -pmax, pmax);
            if (wall_zero_p && qc != qn) p[i] = 0.0;
            q[i] = qc;
        }
    }
}

/*
 * Run T steps of the Spring-Ising iteration (Eq. 8 with the walls of Eq. 6)
 * for R independent replicas (the "parallel tests" of Fig. 3).
 * zeta[T], dt[T]: per-step coupling coefficient zeta(t_step) and time step.
 * q, p: [R][n] in/out.  h may be NULL (zero field).
 */
int or_run(int n, int R, int T, const double *J, const double *h,
           const double *zeta, const double *dt, double k, double m,
           double q0c, double qmax, double pmax, int order, int wall_zero_p,
           double *q, double *p) {
    int r, failed = 0;
    if (n < 1 || R < 0 || T < 0 || !J || !zeta || !dt || !q || !p || m == 0.0)
        return OR_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (r = 0; r < R; r++) {
        double *F = (double *)malloc(sizeof(double) * (size_t)n);
        double *qold = (double *)malloc(sizeof(double) * (size_t)n);
        int t;
        if (!F || !qold) {
            failed = 1;
        } else {
            for (t = 0; t < T; t++)
                or_step_one(n, J, h, zeta[t], dt[t], k, m, q0c, qmax, pmax,
                            order, wall_zero_p, q + (size_t)r * n,
                            p + (size_t)r * n, F, qold);
        }
        free(F);
        free(qold);
    }
    return failed ? OR_ERR_OOM : OR_OK;
}

/* Spin readout: sigma_i = sign(q_i), with sign(0) = +1. */
void or_sign(int count, const double *q, int8_t *sigma) {
    int i;
    for (i = 0; i < count; i++) sigma[i] = (q[i] >= 0.0) ? 1 : -1;
}

/*
 * Ising energy, Eq. 1, written as printed:
 *   H = - sum_{i<j} J_ij s_i s_j - sum_i h_i s_i.
 * s: [R][n] spins in {-1,+1}; E: [R].
 */
void or_energy(int n, int R, const double *J, const double *h,
               const int8_t *s, double *E) {
    int r, i, j;
    for (r = 0; r < R; r++) {
        const int8_t *sr = s + (size_t)r * n;
        double pair = 0.0, field = 0.0;
        for (i = 0; i < n; i++)
            for (j = i + 1; j < n; j++)
                pair += J[(size_t)i * n + j] * (double)sr[i] * (double)sr[j];
        if (h)
            for (i = 0; i < n; i++) field += h[i] * (double)sr[i];
        E[r] = -pair - field;
    }
}

/*
 * Cut value of the MAX-CUT instance with weights w_ij = -J_ij:
 *   cut = sum_{i<j} w_ij * [s_i != s_j].
 */
void or_cut(int n, int R, const double *J, const int8_t *s, double *cut) {
    int r, i, j;
    for (r = 0; r < R; r++) {
        const int8_t *sr = s + (size_t)r * n;
        double c = 0.0;
        for (i = 0; i < n; i++)
            for (j = i + 1; j < n; j++)
                if (sr[i] != sr[j]) c += -J[(size_t)i * n + j];
        cut[r] = c;
    }
}

/*
 * Continuous Ising energy (the relaxation sigma -> q of the spring model):
 *   H(q) = - sum_{i<j} J_ij q_i q_j - sum_i h_i q_i.
 */
void or_relaxed_energy(int n, int R, const double *J, const double *h,
                       const double *q, double *E) {
    int r, i, j;
    for (r = 0; r < R; r++) {
        const double *x = q + (size_t)r * n;
        double pair = 0.0, field = 0.0;
        for (i = 0; i < n; i++)
            for (j = i + 1; j < n; j++) pair += J[(size_t)i * n + j] * x[i] * x[j];
        if (h)
            for (i = 0; i < n; i++) field += h[i] * x[i];
        E[r] = -pair - field;
    }
}

/*
 * Hamiltonian of Eq. 3 / Eq. 7 with qdot = p/m:
 *   H = sum_i 1/2 qdot_i p_i + sum_i 1/2 k (q_i - q0)^2 + zeta * H_Ising(q).
 */
void or_hamiltonian(int n, int R, const double *J, const double *h,
                    double zeta, double k, double m, double q0c,
                    const double *q, const double *p, double *Hout) {
    int r, i;
    double *Ei = (double *)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
    or_relaxed_energy(n, R, J, h, q, Ei);
    for (r = 0; r < R; r++) {
        double kin = 0.0, spring = 0.0;
        for (i = 0; i < n; i++) {
            double pi = p[(size_t)r * n + i], qi = q[(size_t)r * n + i];
            kin += 0.5 * (pi / m) * pi;
            spring += 0.5 * k * (qi - q0c) * (qi - q0c);
        }
        Hout[r] = kin + spring + zeta * Ei[r];
    }
    free(Ei);
}

/*
 * Exhaustive ground state of Eq. 1 for n <= 24: tries all 2^n spin vectors
 * (bit b of the counter set means spin b is -1).  Writes the minimum energy
 * and one minimiser.
 */
int or_bruteforce(int n, const double *J, const double *h, double *Emin,
                  int8_t *argmin) {
    uint64_t c, total;
    int8_t *s;
    double best = 0.0;
    int have = 0, i;
    if (n < 1 || n > 24) return OR_ERR_ARG;
    s = (int8_t *)malloc((size_t)n);
    if (!s) return OR_ERR_OOM;
    total = (uint64_t)1 << n;
    for (c = 0; c < total; c++) {
        double E;
        for (i = 0; i < n; i++) s[i] = ((c >> i) & 1u) ? -1 : 1;
        or_energy(n, 1, J, h, s, &E);
        if (!have || E < best) {
            best = E;
            have = 1;
            memcpy(argmin, s, (size_t)n);
        }
    }
    *Emin = best;
    free(s);
    return OR_OK;
}

/*
 * Reverse-mode gradient of the relaxed energy at the final step,
 *   L = sum_r ( -1/2 q_r^T J q_r - h^T q_r ),  q_r = position after T steps,
 * with respect to zeta[T], dt[T] and k.  The forward pass stores every state;
 * the reverse pass applies the hand-derived adjoint of one step of Eq. 8
 * (order 0) or Eq. 5 (order 1), taking the derivative of each clamp of
 * Eq. 6 as 1 strictly inside the wall and 0 on or beyond it.
 *
 * Adjoint of one kick-drift step (a = pre-clamp momentum, b = pre-clamp
 * position, F = J q + h, D_p / D_q the interior indicators):
 *   lb   = D_q * lq'
 *   mu   = lp' + (dt/m) lb
 *   la   = D_p * mu
 *   lq   = lb + dt (-k la + zeta J la)
 *   lp   = la
 *   g_dt   += sum lb p'/m + sum la (-k (q - q0) + zeta F)
 *   g_zeta += dt sum la F
 *   g_k    += -dt sum la (q - q0)
 * Terminal adjoint: lq_T = -(J q_T + h), lp_T = 0.
 * wall_zero_p is not differentiated (returns OR_ERR_ARG).
 */
int or_grad(int n, int R, int T, const double *J, const double *h,
            const double *zeta, const double *dt, double k, double m,
            double q0c, double qmax, double pmax, int order,
            const double *q_init, const double *p_init, double *g_zeta,
            double *g_dt, double *g_k, double *objective) {
    size_t nn = (size_t)n, st = (size_t)R * nn;
    double *Q, *P, *F, *lq, *lp, *lqn, *lpn, *la, *lb, *Jla, *tmp, *tmp2;
    int t, r, i, j;
    double obj = 0.0, gk = 0.0;
    if (n < 1 || R < 1 || T < 0 || order < 0 || order > 1) return OR_ERR_ARG;
    Q = (double *)malloc(sizeof(double) * st * (size_t)(T + 1));
    P = (double *)malloc(sizeof(double) * st * (size_t)(T + 1));
    F = (double *)malloc(sizeof(double) * nn);
    lq = (double *)malloc(sizeof(double) * st);
    lp = (double *)malloc(sizeof(double) * st);
    lqn = (double *)malloc(sizeof(double) * nn);
    lpn = (double *)malloc(sizeof(double) * nn);
    la = (double *)malloc(sizeof(double) * nn);
    lb = (double *)malloc(sizeof(double) * nn);
    Jla = (double *)malloc(sizeof(double) * nn);
    tmp = (double *)malloc(sizeof(double) * nn);
    tmp2 = (double *)malloc(sizeof(double) * nn);
    if (!Q || !P || !F || !lq || !lp || !lqn || !lpn || !la || !lb || !Jla ||
        !tmp || !tmp2) {
        free(Q); free(P); free(F); free(lq); free(lp); free(lqn); free(lpn);
        free(la); free(lb); free(Jla); free(tmp); free(tmp2);
        return OR_ERR_OOM;
    }
    /* Forward pass, storing every state. */
    memcpy(Q, q_init, sizeof(double) * st);
    if (p_init) memcpy(P, p_init, sizeof(double) * st);
    else memset(P, 0, sizeof(double) * st);
    for (t = 0; t < T; t++) {
        memcpy(Q + st * (size_t)(t + 1), Q + st * (size_t)t, sizeof(double) * st);
        memcpy(P + st * (size_t)(t + 1), P + st * (size_t)t, sizeof(double) * st);
        for (r = 0; r < R; r++)
            or_step_one(n, J, h, zeta[t], dt[t], k, m, q0c, qmax, pmax, order,
                        0, Q + st * (size_t)(t + 1) + (size_t)r * nn,
                        P + st * (size_t)(t + 1) + (size_t)r * nn, F, tmp);
    }
    /* Objective and terminal adjoint. */
    {
        double *Er = (double *)malloc(sizeof(double) * (size_t)R);
        or_relaxed_energy(n, R, J, h, Q + st * (size_t)T, Er);
        for (r = 0; r < R; r++) obj += Er[r];
        free(Er);
    }
    for (r = 0; r < R; r++) {
        const double *x = Q + st * (size_t)T + (size_t)r * nn;
        for (i = 0; i < n; i++) {
            double s = 0.0;
            for (j = 0; j < n; j++) s += J[(size_t)i * n + j] * x[j];
            lq[(size_t)r * nn + i] = -(s + (h ? h[i] : 0.0));
            lp[(size_t)r * nn + i] = 0.0;
        }
    }
    for (t = 0; t < T; t++) { g_zeta[t] = 0.0; g_dt[t] = 0.0; }
    /* Reverse pass. */
    for (t = T - 1; t >= 0; t--) {
        double z = zeta[t], d = dt[t];
        double gz = 0.0, gd = 0.0;
        for (r = 0; r < R; r++) {
            const double *q = Q + st * (size_t)t + (size_t)r * nn;
            const double *p = P + st * (size_t)t + (size_t)r * nn;
            const double *pn = P + st * (size_t)(t + 1) + (size_t)r * nn;
            double *lqr = lq + (size_t)r * nn, *lpr = lp + (size_t)r * nn;
            /* Recompute the force and the pre-clamp values of this step. */
            for (i = 0; i < n; i++) {
                double s = 0.0;
                for (j = 0; j < n; j++) s += J[(size_t)i * n + j] * q[j];
                F[i] = s + (h ? h[i] : 0.0);
            }
            for (i = 0; i < n; i++) {
                double a = p[i] + d * (-k * (q[i] - q0c) + z * F[i]);
                double Dp = (a > -pmax && a < pmax) ? 1.0 : 0.0;
                double b, Dq;
                if (order == 0) b = q[i] + (d / m) * pn[i];
                else b = q[i] + (d / m) * p[i];
                Dq = (b > -qmax && b < qmax) ? 1.0 : 0.0;
                lb[i] = Dq * lqr[i];
                if (order == 0) la[i] = Dp * (lpr[i] + (d / m) * lb[i]);
                else la[i] = Dp * lpr[i];
            }
            for (i = 0; i < n; i++) {
                double s = 0.0;
                for (j = 0; j < n; j++) s += J[(size_t)i * n + j] * la[j];
                Jla[i] = s;
            }
            for (i = 0; i < n; i++) {
                double force = -k * (q[i] - q0c) + z * F[i];
                double pused = (order == 0) ? pn[i] : p[i];
                gd += lb[i] * pused / m + la[i] * force;
                gz += d * la[i] * F[i];
                gk += -d * la[i] * (q[i] - q0c);
                lqn[i] = lb[i] + d * (-k * la[i] + z * Jla[i]);
                lpn[i] = (order == 0) ? la[i] : la[i] + (d / m) * lb[i];
            }
            for (i = 0; i < n; i++) { lqr[i] = lqn[i]; lpr[i] = lpn[i]; }
        }
        g_zeta[t] = gz;
        g_dt[t] = gd;
    }
    *g_k = gk;
    *objective = obj;
    free(Q); free(P); free(F); free(lq); free(lp); free(lqn); free(lpn);
    free(la); free(lb); free(Jla); free(tmp); free(tmp2);
    return OR_OK;
}
