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

/*
 * Forward simulation with receive-coil weighting (Eq. 3.25; §6.1 "Inhomogenitäten der
 * Empfangssensitivität"): before the superposition of a sample, each spin's magnetisation is
 * weighted with its coil's receive sensitivity, the scalar product of Eq. 3.25 taken as the
 * complex product C·(Mx + jMy) of a transverse sensitivity C with the transverse magnetisation.
 *   sens:   n_coils*n_spins complex values, interleaved (re, im), coil-major: C[c][s]
 *   signal: n_coils*2*n_adc doubles, coil-major, overwritten:
 *           signal_c[j] = exp(-j adc_phase_j) * sum_s C[c][s] * (Mx + jMy)_s
 * Every spin starts in thermal equilibrium.  Returns as oracle_simulate.
 */
int oracle_simulate_coils(int64_t n_spins, const double *x, const double *y, const double *z,
                          const double *rho, const double *t1, const double *t2, const double *dw,
                          int64_t n_events, const void *events, double gamma_hz_per_t,
                          int32_t n_coils, const double *sens, double *signal, int64_t n_adc,
                          int n_threads)
{
    const oracle_event *ev = (const oracle_event *)events;
    if (count_adc(ev, n_events) != n_adc || n_coils < 1) return -1;
    const double gamma = ORACLE_TWO_PI * gamma_hz_per_t;
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
#endif
    const size_t per = (size_t)n_coils * (size_t)(2 * n_adc) + 1;
    double *partial = (double *)calloc((size_t)nt * per, sizeof(double));
    if (!partial) return -2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = partial + (size_t)tid * per;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t s = 0; s < n_spins; ++s) {
            double M[3] = {0.0, 0.0, rho[s]};
            int64_t j = 0;
            for (int64_t e = 0; e < n_events; ++e) {
                if (apply_event(&ev[e], gamma, x[s], y[s], z[s], rho[s], t1[s], t2[s], dw[s], M)) {
                    const double cph = cos(ev[e].adc_phase), sph = sin(ev[e].adc_phase);
                    const double wr = M[0] * cph + M[1] * sph, wi = M[1] * cph - M[0] * sph;
                    for (int32_t c = 0; c < n_coils; ++c) {
                        const double cr = sens[2 * ((size_t)c * (size_t)n_spins + (size_t)s)];
                        const double ci = sens[2 * ((size_t)c * (size_t)n_spins + (size_t)s) + 1];
                        double *sig = mine + (size_t)c * (size_t)(2 * n_adc);
                        sig[2 * j] += cr * wr - ci * wi;
                        sig[2 * j + 1] += cr * wi + ci * wr;
                    }
                    ++j;
                }
            }
        }
    }
    memset(signal, 0, sizeof(double) * (per - 1));
    for (int t = 0; t < nt; ++t) {
        const double *p = partial + (size_t)t * per;
        for (size_t i = 0; i + 1 < per; ++i) signal[i] += p[i];
    }
    free(partial);
    return 0;
}

/* Forward simulation with learnable flip angles: as oracle_simulate, but event e's flip angle is
 * rf_values[rf_param[e]] wherever rf_param[e] >= 0. */
int oracle_simulate_rf(int64_t n_spins, const double *x, const double *y, const double *z,
                       const double *rho, const double *t1, const double *t2, const double *dw,
                       int64_t n_events, const void *events, double gamma_hz_per_t,
                       const int32_t *rf_param, const double *rf_values, double *signal, int64_t n_adc,
                       int n_threads)
{
    const oracle_event *ev = (const oracle_event *)events;
    oracle_event *copy = (oracle_event *)malloc(sizeof(oracle_event) * (size_t)(n_events > 0 ? n_events : 1));
    if (!copy) return -2;
    for (int64_t e = 0; e < n_events; ++e) {
        copy[e] = ev[e];
        if (rf_param && rf_param[e] >= 0) copy[e].rf_flip = rf_values[rf_param[e]];
    }
    int rc = oracle_simulate(n_spins, x, y, z, rho, t1, t2, dw, NULL, n_events, copy, gamma_hz_per_t, signal,
                             n_adc, NULL, n_threads);
    free(copy);
    return rc;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Gradient of a real loss L of the signal, by forward-mode differentiation of the same
 * step-by-step simulation (tangent propagation; every step differentiated by hand from
 * Eqs. 3.5 and 3.19).
 *   h:        2*n_adc doubles, h_j = dL/dRe(s_j) + j dL/dIm(s_j) (gradient of L w.r.t. the signal)
 *   rf_param: NULL or n_events ints; event e's flip angle is rf_values[rf_param[e]] when >= 0
 *   rf_values:NULL or the learnable flip angles
 *   d_rho, d_t1, d_t2: NULL or n_spins doubles, receive dL/dM0, dL/dT1, dL/dT2 per spin
 *   sel, n_sel, d_sel: directional derivatives dL/d rf_values[sel[i]] into d_sel[i]
 * dL/dp = sum_j Re(conj(h_j) ds_j/dp), s_j = sum_spins (Mx + jMy) exp(-j adc_phase_j).
 */
static double event_flip(const oracle_event *e, int64_t idx, const int32_t *rf_param, const double *rf_values)
{
    if (rf_param && rf_param[idx] >= 0) return rf_values[rf_param[idx]];
    return e->rf_flip;
}

/* derivative of the Eq. 3.19 matrix with respect to the flip angle α */
static void rf_rotation_dalpha(double alpha, double phi, double D[3][3])
{
    const double ca = cos(alpha), sa = sin(alpha);
    const double cp = cos(phi), sp = sin(phi);
    D[0][0] = -sp * sp * sa;
    D[0][1] = sp * cp * sa;
    D[0][2] = -sp * ca;
    D[1][0] = sp * cp * sa;
    D[1][1] = -cp * cp * sa;
    D[1][2] = cp * ca;
    D[2][0] = sp * ca;
    D[2][1] = -cp * ca;
    D[2][2] = -sa;
}

int oracle_gradient(int64_t n_spins, const double *x, const double *y, const double *z,
                    const double *rho, const double *t1, const double *t2, const double *dw,
                    int64_t n_events, const void *events, double gamma_hz_per_t,
                    const int32_t *rf_param, const double *rf_values,
                    const double *h, int64_t n_adc,
                    double *d_rho, double *d_t1, double *d_t2,
                    const int32_t *sel, int32_t n_sel, double *d_sel, int n_threads)
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
    const int nd = 3 + n_sel; /* tangent directions per spin: M0, T1, T2, selected RF parameters */
    double *part = (double *)calloc((size_t)nt * (size_t)(n_sel + 1), sizeof(double));
    if (!part) return -2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = part + (size_t)tid * (size_t)(n_sel + 1);
        double *T = (double *)malloc(sizeof(double) * 3 * (size_t)nd);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t s = 0; s < n_spins; ++s) {
            double M[3] = {0.0, 0.0, rho[s]};
            for (int d = 0; d < 3 * nd; ++d) T[d] = 0.0;
            T[0 * 3 + 2] = 1.0; /* dM/dM0 at equilibrium */
            double g[3] = {0.0, 0.0, 0.0};
            int64_t j = 0;
            for (int64_t e = 0; e < n_events; ++e) {
                const oracle_event *E = &ev[e];
                const double alpha = event_flip(E, e, rf_param, rf_values);
                if (alpha != 0.0) {
                    double R[3][3], D[3][3];
                    rf_rotation(alpha, E->rf_phase, R);
                    rf_rotation_dalpha(alpha, E->rf_phase, D);
                    const int p = rf_param ? rf_param[e] : -1;
                    for (int d = 0; d < nd; ++d) {
                        double *t = T + 3 * d;
                        double u[3];
                        for (int r = 0; r < 3; ++r) u[r] = R[r][0] * t[0] + R[r][1] * t[1] + R[r][2] * t[2];
                        if (d >= 3 && p >= 0 && p == sel[d - 3])
                            for (int r = 0; r < 3; ++r) u[r] += D[r][0] * M[0] + D[r][1] * M[1] + D[r][2] * M[2];
                        t[0] = u[0]; t[1] = u[1]; t[2] = u[2];
                    }
                    double mx = R[0][0] * M[0] + R[0][1] * M[1] + R[0][2] * M[2];
                    double my = R[1][0] * M[0] + R[1][1] * M[1] + R[1][2] * M[2];
                    double mz = R[2][0] * M[0] + R[2][1] * M[1] + R[2][2] * M[2];
                    M[0] = mx; M[1] = my; M[2] = mz;
                }
                const double theta = (gamma * (E->gx * x[s] + E->gy * y[s] + E->gz * z[s]) + dw[s]) * E->dt;
                const double c = cos(theta), sn = sin(theta);
                const double e2 = exp(-E->dt / t2[s]), e1 = exp(-E->dt / t1[s]);
                /* d e2 / d T2 = e2 dt / T2^2, d e1 / d T1 = e1 dt / T1^2 (0 for T = inf) */
                const double de2 = isinf(t2[s]) ? 0.0 : e2 * E->dt / (t2[s] * t2[s]);
                const double de1 = isinf(t1[s]) ? 0.0 : e1 * E->dt / (t1[s] * t1[s]);
                const double px = M[0] * c + M[1] * sn, py = -M[0] * sn + M[1] * c;
                for (int d = 0; d < nd; ++d) {
                    double *t = T + 3 * d;
                    const double qx = t[0] * c + t[1] * sn, qy = -t[0] * sn + t[1] * c;
                    double nx = e2 * qx, ny = e2 * qy, nz = e1 * t[2];
                    if (d == 0) nz += 1.0 - e1;                 /* M0 */
                    if (d == 1) nz += de1 * (M[2] - rho[s]);    /* T1 */
                    if (d == 2) { nx += de2 * px; ny += de2 * py; } /* T2 */
                    t[0] = nx; t[1] = ny; t[2] = nz;
                }
                M[0] = e2 * px;
                M[1] = e2 * py;
                M[2] = M[2] * e1 + rho[s] * (1.0 - e1);
                if (E->adc) {
                    const double cph = cos(E->adc_phase), sph = sin(E->adc_phase);
                    const double hr = h[2 * j], hi = h[2 * j + 1];
                    for (int d = 0; d < nd; ++d) {
                        const double *t = T + 3 * d;
                        /* ds = (tx + j ty) exp(-j phase); dL = Re(conj(h) ds) */
                        const double dsr = t[0] * cph + t[1] * sph, dsi = t[1] * cph - t[0] * sph;
                        const double dl = hr * dsr + hi * dsi;
                        if (d < 3) g[d] += dl; else mine[d - 3] += dl;
                    }
                    ++j;
                }
            }
            if (d_rho) d_rho[s] = g[0];
            if (d_t1) d_t1[s] = g[1];
            if (d_t2) d_t2[s] = g[2];
        }
        free(T);
    }
    for (int i = 0; i < n_sel; ++i) {
        double acc = 0.0;
        for (int t = 0; t < nt; ++t) acc += part[(size_t)t * (size_t)(n_sel + 1) + i];
        if (d_sel) d_sel[i] = acc;
    }
    free(part);
    return 0;
}

/*
 * Non-parallel fields (§3.2, §3.4.3.2): forward simulation where the static field at each spin
 * points along its own unit vector n_s, and an elementary sequence's gradient field may have
 * components transverse to z.
 *
 * §3.2: where the static field is not along z, the frame is turned locally so that one axis lies
 * along the field, the Bloch equation (3.4) is applied in that frame, and the result is turned
 * back.  §3.4.3.2: a constant gradient field with transverse components changes the direction of
 * the total field; T1 relaxation follows the resulting direction and Eqs. 3.14/3.15 hold in the
 * frame turned to it.  Written out for one spin and one event:
 *   b = (gtx.x, gty.x, G.x)              gradient field at the spin [T]
 *   u = B0*n + b,  u_hat = u/|u|         total field and its direction
 *   theta = (gamma*(|u| - B0) + dw)*dt   precession angle in the frame rotating at gamma*B0
 * and, with M_par = M.u_hat and M_perp = M - M_par*u_hat,
 *   M <- E2*(cos(theta)*M_perp - sin(theta)*(u_hat x M_perp)) + (E1*M_par + M0*(1 - E1))*u_hat,
 * the clockwise turn of Eq. 3.5 about u_hat (for u_hat = z it is Eq. 3.5 itself) with T2 decay of
 * the part across the field and T1 recovery along it.  |u| - B0 is evaluated as
 * (2*B0*(n.b) + |b|^2)/(|u| + B0), the same number without the cancellation of two nearly equal
 * terms.  The RF pulse acts first, as Eq. 3.19 in the rotating frame; the sample is
 * (Mx + jMy)*exp(-j*adc_phase) after the step.  Every spin starts in equilibrium along its static
 * field, M = M0*n.
 *   ndir: 3*n_spins doubles (nx, ny, nz) per spin, unit vectors
 *   gt:   NULL or 6*n_events doubles per event: gtx (3), gty (3) [T/m]
 *   b0:   |B0| [T] > 0
 * Returns as oracle_simulate.
 */
static int apply_event_fields(const oracle_event *e, const double *gt, double gamma, double b0,
                              double x, double y, double z, const double n[3], double rho, double t1,
                              double t2, double dw, double M[3])
{
    if (e->rf_flip != 0.0) {
        double R[3][3];
        rf_rotation(e->rf_flip, e->rf_phase, R);
        const double mx = R[0][0] * M[0] + R[0][1] * M[1] + R[0][2] * M[2];
        const double my = R[1][0] * M[0] + R[1][1] * M[1] + R[1][2] * M[2];
        const double mz = R[2][0] * M[0] + R[2][1] * M[1] + R[2][2] * M[2];
        M[0] = mx; M[1] = my; M[2] = mz;
    }
    double b[3] = {0.0, 0.0, e->gx * x + e->gy * y + e->gz * z};
    if (gt) {
        b[0] = gt[0] * x + gt[1] * y + gt[2] * z;
        b[1] = gt[3] * x + gt[4] * y + gt[5] * z;
    }
    const double u[3] = {b0 * n[0] + b[0], b0 * n[1] + b[1], b0 * n[2] + b[2]};
    const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double h[3] = {u[0] / un, u[1] / un, u[2] / un};
    const double nb = n[0] * b[0] + n[1] * b[1] + n[2] * b[2];
    const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const double excess = (2.0 * b0 * nb + bb) / (un + b0); /* |u| - B0 */
    const double theta = (gamma * excess + dw) * e->dt;
    const double c = cos(theta), s = sin(theta);
    const double e2 = exp(-e->dt / t2);
    const double e1 = exp(-e->dt / t1);
    const double par = M[0] * h[0] + M[1] * h[1] + M[2] * h[2];
    const double p[3] = {M[0] - par * h[0], M[1] - par * h[1], M[2] - par * h[2]};
    const double hxp[3] = {h[1] * p[2] - h[2] * p[1], h[2] * p[0] - h[0] * p[2], h[0] * p[1] - h[1] * p[0]};
    const double along = par * e1 + rho * (1.0 - e1);
    for (int i = 0; i < 3; ++i) M[i] = e2 * (c * p[i] - s * hxp[i]) + along * h[i];
    return e->adc != 0;
}

int oracle_simulate_fields(int64_t n_spins, const double *x, const double *y, const double *z,
                           const double *rho, const double *t1, const double *t2, const double *dw,
                           const double *ndir, int64_t n_events, const void *events, const double *gt,
                           double gamma_hz_per_t, double b0, double *signal, int64_t n_adc, double *m_final,
                           int n_threads)
{
    const oracle_event *ev = (const oracle_event *)events;
    if (count_adc(ev, n_events) != n_adc || !(b0 > 0.0)) return -1;
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
            const double *n = ndir + 3 * s;
            double M[3] = {rho[s] * n[0], rho[s] * n[1], rho[s] * n[2]};
            int64_t j = 0;
            for (int64_t e = 0; e < n_events; ++e) {
                if (apply_event_fields(&ev[e], gt ? gt + 6 * e : NULL, gamma, b0, x[s], y[s], z[s], n, rho[s],
                                       t1[s], t2[s], dw[s], M)) {
                    if (mine) {
                        const double cph = cos(ev[e].adc_phase), sph = sin(ev[e].adc_phase);
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
