/*
 * FP64 CPU oracle for the Bloch-simulation hot path.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's
 * CPU-baseline / reference leg are the only users. The CUDA library shares
 * no code, header, table or helper with this file, and this file includes
 * nothing from it.
 *
 * What it computes (KomaMRI.jl paper, Section "Physical and Mathematical
 * Background" and "Simulation blocks, Regime Switching, and Sequence-Aware
 * Time Stepping"), for every spin j independently (spin independence, same
 * section), one discretised step at a time, in the paper's order:
 *
 *   B_z = Gbar_n . x_j(t_mid) + dw_j / gamma     (Eq. "B definition"; Gbar_n is
 *                                                 the trapezoid mean of the
 *                                                 step's two gradient vertices,
 *                                                 x_j(t_mid) the position at the
 *                                                 step's midpoint)
 *   if B1_n != 0  (excitation regime):
 *       |B| = sqrt(|B1|^2 + B_z^2), phi = -gamma |B| dt          (Eq. angle_precession)
 *       n_xy = B1/|B|, n_z = B_z/|B|
 *       alpha = cos(phi/2) - i n_z sin(phi/2), beta = -i n_xy sin(phi/2)   (spinor eqs.)
 *       Mxy+ = 2 conj(alpha) beta Mz + conj(alpha)^2 Mxy - beta^2 conj(Mxy)
 *       Mz+  = (|alpha|^2 - |beta|^2) Mz - 2 Re(alpha beta conj(Mxy))     (Eq. Rot_exc)
 *   else (precession regime):
 *       phi = -gamma * integral of B_z(t) over the step; for a static spin this is
 *       -gamma B_z dt (trapezoid rule, exact for piecewise-linear G),
 *       Mxy+ = Mxy e^{i phi}                                      (Eq. Rotation_precession)
 *   then relaxation (the relaxation update following Eq. relax_Bloch):
 *       Mxy+ = e^{-dt/T2} Mxy, Mz+ = Mz e^{-dt/T1} + M0 (1 - e^{-dt/T1})
 *   and if the ADC samples time point t_{n+1}, Mxy is added to sig[k].
 *
 * The signal is the plain sum of Mxy over spins (Section "GPU/CPU
 * Parallelization": per-thread signal matrices added at the end; here each
 * thread owns a contiguous spin range and the per-thread arrays are added in
 * thread order, so the result does not depend on scheduling).
 *
 * Motion (the phantom's u(x, t), Section "Overview" and Eq. "B definition"):
 * constant velocity per spin, x(t) = x + v t with t from t_0. In precession
 * the phase integral of G(t).x(t) is evaluated exactly (Simpson's rule on
 * the quadratic integrand; for static spins this is the trapezoid rule); an
 * RF step uses the position at its midpoint (its field is held constant).
 *
 * Readings where the paper is silent: initial state Mxy = 0, Mz = M0; the
 * sample at t_i is the state after step i-1; the precession phase uses the
 * signed B_z (the integral form), which is also what the spinor formula
 * gives for a field along z; T1 or T2 = +inf means no relaxation.
 *
 * oracle_rk4 integrates the Bloch equation (Eq. Bloch) directly with
 * classical fourth-order Runge-Kutta, with B1 constant over each step, G
 * linear between its vertices and the spin at x + v t; it is the
 * brute-force check of the oracle. The *_moving entry points take the
 * velocities; the plain ones are the static case.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* proton gyromagnetic ratio, rad/s/T: 2 pi x 42.577478518 MHz/T (CODATA 2018) */
static const double ORACLE_GAMMA = 2.0 * M_PI * 42.577478518e6;

typedef struct {
    /* phantom */
    const double *x, *y, *z, *pd, *t1, *t2, *dw;
    const double *vx, *vy, *vz; /* NULL: static spins; else x(t) = x + v t */
    const int64_t *group_offsets; /* NULL => one group */
    int64_t n_groups;
    /* sequence */
    int64_t n_steps;
    const double *dt, *gx, *gy, *gz, *b1re, *b1im;
    const uint8_t *adc;
    int64_t n_adc;
    /* outputs */
    double *m_final; /* NULL or [n][3] */
    /* work split */
    int64_t spin_lo, spin_hi;   /* spins owned by this worker (group == 1)    */
    int64_t group_lo, group_hi; /* groups owned by this worker (groups > 1)   */
    double *sig;                /* [n_adc][2] private (one group) or shared  */
} oracle_job;

/* Step one spin through the whole sequence; its Mxy at every ADC time point
 * is added to out[k] (interleaved re, im). */
static void oracle_spin(const oracle_job *J, int64_t j, double *out)
{
    const double xj = J->x[j], yj = J->y[j], zj = J->z[j];
    const double vxj = J->vx ? J->vx[j] : 0.0, vyj = J->vy ? J->vy[j] : 0.0, vzj = J->vz ? J->vz[j] : 0.0;
    const double m0 = J->pd[j], T1 = J->t1[j], T2 = J->t2[j], dwj = J->dw[j];
    double complex mxy = 0.0;
    double mz = m0;
    double t = 0.0; /* time of the current time point */
    int64_t k = 0;
    if (J->adc[0]) {
        out[0] += creal(mxy);
        out[1] += cimag(mxy);
        k = 1;
    }
    for (int64_t n = 0; n < J->n_steps; ++n) {
        const double dt = J->dt[n];
        const double gxm = 0.5 * (J->gx[n] + J->gx[n + 1]);
        const double gym = 0.5 * (J->gy[n] + J->gy[n + 1]);
        const double gzm = 0.5 * (J->gz[n] + J->gz[n + 1]);
        /* spin position at the step's midpoint (motion: x(t) = x + v t) */
        const double tm = t + 0.5 * dt;
        const double xm = xj + vxj * tm, ym = yj + vyj * tm, zm = zj + vzj * tm;
        const double bz = gxm * xm + gym * ym + gzm * zm + dwj / ORACLE_GAMMA;
        const double complex b1 = J->b1re[n] + I * J->b1im[n];
        if (J->b1re[n] != 0.0 || J->b1im[n] != 0.0) {
            /* excitation regime: Cayley-Klein spinor rotation */
            const double bnorm = sqrt(creal(b1) * creal(b1) + cimag(b1) * cimag(b1) + bz * bz);
            const double phi = -ORACLE_GAMMA * bnorm * dt;
            const double complex nxy = b1 / bnorm;
            const double nz = bz / bnorm;
            const double complex alpha = cos(phi / 2.0) - I * nz * sin(phi / 2.0);
            const double complex beta = -I * nxy * sin(phi / 2.0);
            const double complex mxy_new = 2.0 * conj(alpha) * beta * mz
                                         + conj(alpha) * conj(alpha) * mxy
                                         - beta * beta * conj(mxy);
            const double mz_new = (creal(alpha * conj(alpha)) - creal(beta * conj(beta))) * mz
                                - 2.0 * creal(alpha * beta * conj(mxy));
            mxy = mxy_new;
            mz = mz_new;
        } else {
            /* precession regime: rotation about z by the integrated phase
             * -gamma * integral of (G(t).x(t) + dw/gamma) dt. G and x are linear
             * over the step, so G.x is quadratic and Simpson's rule is exact
             * (for a static spin it reduces to the trapezoid rule). */
            const double t1s = t + dt;
            const double f0 = J->gx[n] * (xj + vxj * t) + J->gy[n] * (yj + vyj * t) + J->gz[n] * (zj + vzj * t);
            const double f1 = J->gx[n + 1] * (xj + vxj * t1s) + J->gy[n + 1] * (yj + vyj * t1s)
                            + J->gz[n + 1] * (zj + vzj * t1s);
            const double fm = gxm * xm + gym * ym + gzm * zm;
            const double integral = dt / 6.0 * (f0 + 4.0 * fm + f1);
            const double phi = -ORACLE_GAMMA * integral - dwj * dt;
            mxy = mxy * cexp(I * phi);
        }
        /* relaxation */
        const double e2 = exp(-dt / T2);
        const double e1 = exp(-dt / T1);
        mxy = mxy * e2;
        mz = mz * e1 + m0 * (1.0 - e1);
        t += dt;
        if (J->adc[n + 1]) {
            out[2 * k] += creal(mxy);
            out[2 * k + 1] += cimag(mxy);
            ++k;
        }
    }
    if (J->m_final) {
        J->m_final[3 * j + 0] = creal(mxy);
        J->m_final[3 * j + 1] = cimag(mxy);
        J->m_final[3 * j + 2] = mz;
    }
}

static void *oracle_worker(void *arg)
{
    oracle_job *J = (oracle_job *)arg;
    if (J->group_offsets == NULL) {
        for (int64_t j = J->spin_lo; j < J->spin_hi; ++j) oracle_spin(J, j, J->sig);
    } else {
        for (int64_t g = J->group_lo; g < J->group_hi; ++g) {
            double *row = J->sig + 2 * J->n_adc * g;
            for (int64_t j = J->group_offsets[g]; j < J->group_offsets[g + 1]; ++j)
                oracle_spin(J, j, row);
        }
    }
    return NULL;
}

static int64_t oracle_count_adc(int64_t n_steps, const uint8_t *adc)
{
    int64_t c = 0;
    for (int64_t i = 0; i <= n_steps; ++i) c += adc[i] != 0;
    return c;
}

/* sig: [n_groups][n_adc][2] (re, im), overwritten. m_final: NULL or [n][3].
 * Returns 0 on success, -1 on bad arguments or allocation failure. */
int oracle_simulate_moving(int64_t n_spins, const double *x, const double *y, const double *z,
                           const double *pd, const double *t1, const double *t2, const double *dw,
                           const double *vx, const double *vy, const double *vz,
                           const int64_t *group_offsets, int64_t n_groups,
                           int64_t n_steps, const double *dt, const double *gx, const double *gy,
                           const double *gz, const double *b1re, const double *b1im,
                           const uint8_t *adc, int n_threads, double *sig, double *m_final)
{
    if (n_spins < 0 || n_steps < 0 || n_groups < 1) return -1;
    if (group_offsets == NULL && n_groups != 1) return -1;
    const int64_t n_adc = oracle_count_adc(n_steps, adc);
    memset(sig, 0, sizeof(double) * 2 * (size_t)(n_adc * n_groups));
    if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (n_threads < 1) n_threads = 1;
    const int64_t units = group_offsets ? n_groups : n_spins;
    if (n_threads > units) n_threads = units > 0 ? (int)units : 1;

    oracle_job base = {x, y, z, pd, t1, t2, dw, vx, vy, vz, group_offsets, n_groups,
                       n_steps, dt, gx, gy, gz, b1re, b1im, adc, n_adc, m_final,
                       0, 0, 0, 0, NULL};
    oracle_job *jobs = (oracle_job *)calloc((size_t)n_threads, sizeof(oracle_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    double *priv = NULL;
    if (!jobs || !tid) { free(jobs); free(tid); return -1; }
    if (!group_offsets) {
        priv = (double *)calloc((size_t)n_threads * 2 * (size_t)(n_adc > 0 ? n_adc : 1), sizeof(double));
        if (!priv) { free(jobs); free(tid); return -1; }
    }
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = base;
        const int64_t lo = units * t / n_threads, hi = units * (t + 1) / n_threads;
        if (group_offsets) {
            jobs[t].group_lo = lo; jobs[t].group_hi = hi; jobs[t].sig = sig;
        } else {
            jobs[t].spin_lo = lo; jobs[t].spin_hi = hi; jobs[t].sig = priv + (size_t)t * 2 * n_adc;
        }
    }
    int started = 0;
    for (int t = 1; t < n_threads; ++t) {
        if (pthread_create(&tid[t], NULL, oracle_worker, &jobs[t]) != 0) break;
        started = t;
    }
    oracle_worker(&jobs[0]);
    for (int t = started + 1; t < n_threads; ++t) oracle_worker(&jobs[t]); /* not started */
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    if (!group_offsets) {
        /* per-thread signal arrays added in thread order */
        for (int t = 0; t < n_threads; ++t)
            for (int64_t k = 0; k < 2 * n_adc; ++k) sig[k] += priv[(size_t)t * 2 * n_adc + k];
    }
    free(priv);
    free(jobs);
    free(tid);
    return 0;
}

int oracle_simulate(int64_t n_spins, const double *x, const double *y, const double *z,
                    const double *pd, const double *t1, const double *t2, const double *dw,
                    const int64_t *group_offsets, int64_t n_groups,
                    int64_t n_steps, const double *dt, const double *gx, const double *gy,
                    const double *gz, const double *b1re, const double *b1im,
                    const uint8_t *adc, int n_threads, double *sig, double *m_final)
{
    return oracle_simulate_moving(n_spins, x, y, z, pd, t1, t2, dw, NULL, NULL, NULL, group_offsets,
                                  n_groups, n_steps, dt, gx, gy, gz, b1re, b1im, adc, n_threads, sig,
                                  m_final);
}

/* ---------------- brute force: RK4 on the Bloch equation ---------------- */

typedef struct {
    double b1x, b1y;  /* constant over the step */
    double g0[3], g1[3];
    double t_len;
    double t_start;   /* absolute time of the step's start */
    double x[3], v[3], dw, T1, T2, m0;
} rk4_step;

/* dM/dt = gamma M x B + ((M0 - Mz)/T1) z - (Mx x + My y)/T2, at time s into the step */
static void bloch_rhs(const rk4_step *S, double s, const double *M, double *dM)
{
    const double f = s / S->t_len;
    double bz = S->dw / ORACLE_GAMMA;
    for (int a = 0; a < 3; ++a)
        bz += ((1.0 - f) * S->g0[a] + f * S->g1[a]) * (S->x[a] + S->v[a] * (S->t_start + s));
    const double bx = S->b1x, by = S->b1y;
    /* M x B */
    const double cx = M[1] * bz - M[2] * by;
    const double cy = M[2] * bx - M[0] * bz;
    const double cz = M[0] * by - M[1] * bx;
    dM[0] = ORACLE_GAMMA * cx - M[0] / S->T2;
    dM[1] = ORACLE_GAMMA * cy - M[1] / S->T2;
    dM[2] = ORACLE_GAMMA * cz + (S->m0 - M[2]) / S->T1;
}

/* One spin per call. sig: [n_adc][2] overwritten; m_final: [3]. */
int oracle_rk4_moving(double x, double y, double z, double pd, double t1, double t2, double dw,
                      double vx, double vy, double vz,
                      int64_t n_steps, const double *dt, const double *gx, const double *gy,
                      const double *gz, const double *b1re, const double *b1im, const uint8_t *adc,
                      int64_t substeps, double *sig, double *m_final)
{
    if (substeps < 1 || n_steps < 0) return -1;
    double M[3] = {0.0, 0.0, pd};
    int64_t k = 0;
    if (adc[0]) { sig[0] = 0.0; sig[1] = 0.0; k = 1; }
    rk4_step S;
    S.x[0] = x; S.x[1] = y; S.x[2] = z;
    S.v[0] = vx; S.v[1] = vy; S.v[2] = vz;
    S.dw = dw; S.T1 = t1; S.T2 = t2; S.m0 = pd;
    double t_abs = 0.0;
    for (int64_t n = 0; n < n_steps; ++n) {
        S.t_start = t_abs;
        t_abs += dt[n];
        S.b1x = b1re[n]; S.b1y = b1im[n];
        S.g0[0] = gx[n]; S.g0[1] = gy[n]; S.g0[2] = gz[n];
        S.g1[0] = gx[n + 1]; S.g1[1] = gy[n + 1]; S.g1[2] = gz[n + 1];
        S.t_len = dt[n];
        const double h = dt[n] / (double)substeps;
        for (int64_t q = 0; q < substeps; ++q) {
            const double s = q * h;
            double k1[3], k2[3], k3[3], k4[3], T[3];
            bloch_rhs(&S, s, M, k1);
            for (int a = 0; a < 3; ++a) T[a] = M[a] + 0.5 * h * k1[a];
            bloch_rhs(&S, s + 0.5 * h, T, k2);
            for (int a = 0; a < 3; ++a) T[a] = M[a] + 0.5 * h * k2[a];
            bloch_rhs(&S, s + 0.5 * h, T, k3);
            for (int a = 0; a < 3; ++a) T[a] = M[a] + h * k3[a];
            bloch_rhs(&S, s + h, T, k4);
            for (int a = 0; a < 3; ++a) M[a] += h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        }
        if (adc[n + 1]) { sig[2 * k] = M[0]; sig[2 * k + 1] = M[1]; ++k; }
    }
    m_final[0] = M[0]; m_final[1] = M[1]; m_final[2] = M[2];
    return 0;
}

int oracle_rk4(double x, double y, double z, double pd, double t1, double t2, double dw,
               int64_t n_steps, const double *dt, const double *gx, const double *gy,
               const double *gz, const double *b1re, const double *b1im, const uint8_t *adc,
               int64_t substeps, double *sig, double *m_final)
{
    return oracle_rk4_moving(x, y, z, pd, t1, t2, dw, 0.0, 0.0, 0.0, n_steps, dt, gx, gy, gz, b1re,
                             b1im, adc, substeps, sig, m_final);
}
