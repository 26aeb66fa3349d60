/*
 * mrsim_oracle.c -- plain, slow, FP64 CPU oracle of the spin-based Bloch simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * What it computes (Kürsch, §5.1.1 "Ablauf einer spinbasierten Simulation"):
 *   every spin starts in thermal equilibrium M = (0, 0, M0) and is propagated
 *   through the elementary sequences in order, each one applied as Eq. 4.1
 *       M <- T_Relax * T_grad * T'_HF * M + T_Relax,z
 *   i.e. (1) the hard RF pulse at the start of the event (Eq. 3.19),
 *        (2) the clockwise precession about z by the accumulated angle
 *            θ = (γ G·x + Δω) Δt            (Eqs. 3.5, 3.11, 3.14),
 *        (3) T2 decay of Mx, My and T1 recovery of Mz over Δt (Eq. 3.5).
 *   An event with an ADC flag stores the magnetisation after its step and
 *   adds it, demodulated by exp(-j*adc_phase), into its sample of the complex
 *   signal (§5.1.1; quadrature signal of Eqs. 3.30-3.32: the signal is the sum
 *   of the rotating-frame transverse magnetisations, constant factors dropped).
 *
 * Readings where the paper is silent or inconsistent (they are listed with
 * reasons in the design notes of the repository):
 *   - γ is a parameter (γ/2π in Hz/T); angles use γ = 2π·gamma_hz_per_t.
 *   - precession is clockwise, Mxy <- Mxy·exp(-jθ), with the positive angle
 *     of Eqs. 3.5/3.14 and Δω added to γ G·x as in Eq. 3.11.
 *   - within an event: RF first (instantaneous), then precession and
 *     relaxation over Δt, then the ADC sample (taken at the event's end).
 *
 * Every spin is computed with nothing but libm sin/cos/exp in double; there is
 * no caching, no reordering and no blocking beyond the per-thread partial sums
 * that OpenMP needs (summed in thread order afterwards).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One event record as the caller lays it out: 7 doubles, int32 adc flag, int32 reserved. */
typedef struct {
    double dt, gx, gy, gz, rf_flip, rf_phase, adc_phase;
    int32_t adc;
    int32_t reserved;
} oracle_event;

static const double ORACLE_TWO_PI = 6.283185307179586476925286766559;

/* Eq. 3.19: hard RF pulse with flip α about the axis in the x'y' plane at phase φ. */
static void rf_rotation(double alpha, double phi, double R[3][3])
{
    const double ca = cos(alpha), sa = sin(alpha);
    const double cp = cos(phi), sp = sin(phi);
    R[0][0] = cp * cp + sp * sp * ca;
    R[0][1] = sp * cp * (1.0 - ca);
    R[0][2] = -sp * sa;
    R[1][0] = sp * cp * (1.0 - ca);
    R[1][1] = sp * sp + cp * cp * ca;
    R[1][2] = cp * sa;
    R[2][0] = sp * sa;
    R[2][1] = -cp * sa;
    R[2][2] = ca;
}

/* One elementary sequence (Eq. 4.1) applied to one spin; returns 1 if it samples. */
static int apply_event(const oracle_event *e, double gamma, double x, double y, double z,
                       double rho, double t1, double t2, double dw, double M[3])
{
    if (e->rf_flip != 0.0) {
        double R[3][3];
        rf_rotation(e->rf_flip, e->rf_phase, R);
        const double mx = R[0][0] * M[0] + R[0][1] * M[1] + R[0][2] * M[2];
        const double my = R[1][0] * M[0] + R[1][1] * M[1] + R[1][2] * M[2];
        const double mz = R[2][0] * M[0] + R[2][1] * M[1] + R[2][2] * M[2];
        M[0] = mx; M[1] = my; M[2] = mz;
    }
    /* Eq. 3.14 with the off-resonance term of Eq. 3.11: angle over Δt. */
    const double theta = (gamma * (e->gx * x + e->gy * y + e->gz * z) + dw) * e->dt;
    const double c = cos(theta), s = sin(theta);
    /* Eq. 3.5: T_Relax * T0 * M + T_Relax,z */
    const double e2 = exp(-e->dt / t2);
    const double e1 = exp(-e->dt / t1);
    const double mx = (M[0] * c + M[1] * s) * e2;
    const double my = (-M[0] * s + M[1] * c) * e2;
    const double mz = M[2] * e1 + rho * (1.0 - e1);
    M[0] = mx; M[1] = my; M[2] = mz;
    return e->adc != 0;
}

static int64_t count_adc(const oracle_event *ev, int64_t n)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) k += ev[i].adc != 0;
    return k;
}

/*
 * Forward simulation.
 *   spins: SoA x, y, z [m], rho = M0, t1, t2 [s] (INFINITY allowed), dw [rad/s]
 *   m_init:  NULL (thermal equilibrium) or 3*n_spins doubles (Mx, My, Mz per spin)
 *   events:  n_events records (see oracle_event)
 *   signal:  NULL or 2*n_adc doubles, interleaved (re, im), overwritten
 *   m_final: NULL or 3*n_spins doubles, overwritten with the state after the last event
 * Returns 0, or -1 if n_adc differs from the number of ADC events, -2 on allocation failure.
 */
int oracle_simulate(int64_t n_spins, const double *x, const double *y, const double *z,
                    const double *rho, const double *t1, const double *t2, const double *dw,
                    const double *m_init, int64_t n_events, const void *events,
                    double gamma_hz_per_t, double *signal, int64_t n_adc, double *m_final,
                    int n_threads)
{
    const oracle_event *ev = (const oracle_event *)events;
    if (count_adc(ev, n_events) != n_adc) return -1;
    const double gamma = ORACLE_TWO_PI * gamma_hz_per_t;
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
#endif
    double *partial = NULL;
    if (signal) {
        partial = (double *)calloc((size_t)nt * (size_t)(2 * n_adc + 1), sizeof(double));
        if (!partial) return -2;
    }
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = partial ? partial + (size_t)tid * (size_t)(2 * n_adc + 1) : NULL;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t s = 0; s < n_spins; ++s) {
            double M[3];
            if (m_init) {
                M[0] = m_init[3 * s]; M[1] = m_init[3 * s + 1]; M[2] = m_init[3 * s + 2];
            } else {
                M[0] = 0.0; M[1] = 0.0; M[2] = rho[s];
            }
            int64_t j = 0;
            for (int64_t e = 0; e < n_events; ++e) {
                if (apply_event(&ev[e], gamma, x[s], y[s], z[s], rho[s], t1[s], t2[s], dw[s], M)) {
                    if (mine) {
                        const double cph = cos(ev[e].adc_phase), sph = sin(ev[e].adc_phase);
                        /* (Mx + j My) * exp(-j adc_phase) */
                        mine[2 * j] += M[0] * cph + M[1] * sph;
                        mine[2 * j + 1] += M[1] * cph - M[0] * sph;
                    }
                    ++j;
                }
            }
            if (m_final) {
                m_final[3 * s] = M[0]; m_final[3 * s + 1] = M[1]; m_final[3 * s + 2] = M[2];
            }
        }
    }
    if (signal) {
        memset(signal, 0, sizeof(double) * (size_t)(2 * n_adc));
        for (int t = 0; t < nt; ++t) {
            const double *p = partial + (size_t)t * (size_t)(2 * n_adc + 1);
            for (int64_t i = 0; i < 2 * n_adc; ++i) signal[i] += p[i];
        }
        free(partial);
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
