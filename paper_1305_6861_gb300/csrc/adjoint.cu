// adjoint.cu -- reverse-mode (adjoint, backward-in-time) gradient of a loss of the signal with
// respect to every spin's M0, T1, T2 and to learnable RF flip angles.
//
// Every event is an affine map of a spin's magnetisation (Eq. 4.1): M' = P·R·M + (0, 0, M0(1−E1))
// with R the hard pulse (Eq. 3.19) and P = diag(E2·rot(−θ), E1) (Eq. 3.5).  For a loss L whose
// gradient with respect to the signal is h_j = ∂L/∂Re s_j + j ∂L/∂Im s_j, the adjoint λ of a spin's
// state runs backward through the events: λ ← Rᵀ·Pᵀ·λ, plus conj(d_j)·h_j at the end of every
// event that takes sample j (d_j = exp(−j·adc_phase_j), since s_j = Σ_spins (Mx + jMy)·d_j), and
// the parameter gradients collect λ'ᵀ·∂M'/∂p along the way.  The backward pass needs the states
// in reverse order: the forward pass stores every spin's state at the start of each segment of C
// events (checkpoints); the backward pass restores a checkpoint, recomputes the segment's states
// into a per-thread buffer and sweeps the segment backward.  Everything here is float64.
// The forward pass is the library's float64 forward kernel on a program compiled once with the
// learnable flips as parametric pulses (their rotations read from a table written before each
// launch) and snapshots at the segment starts, which are the checkpoints; with more learnable
// flips than that table holds, a one-thread-per-spin forward kernel of its own does the same.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mrsim.h"
#include "handles.h"
#include "internal.h"
#include "dfloat.cuh"

using namespace mrsim;

namespace {

constexpr int ADJ_MAX_CLASSES = 16;
constexpr int ADJ_MAX_SEG = 128;  // events per checkpoint segment (per-thread state buffer size)
constexpr int ADJ_THREADS = 128;
constexpr int ADJ_LOCAL_PARAMS = 256;  // RF parameters summed per thread in local memory

enum AdjFlags : int32_t { A_RF = 1, A_ADC = 2, A_CLS = 4, A_INL = 8 };

// One event of the differentiation program (64 bytes).
struct AdjEvent {
    int32_t flags;
    int32_t rf;     // RF table entry (A_RF)
    int32_t cls;    // precession/relaxation class (A_CLS)
    int32_t adc;    // sample index (A_ADC)
    double k[3];    // inline moment [cycles/m] (A_INL)
    double dt;      // interval [s]
    float dth, dtl; // the interval as a float pair (hi, lo), for the compensated precision
    double pad;
};
static_assert(sizeof(AdjEvent) == 64, "AdjEvent must be 64 bytes");

// The RF pulse of one RF event: its rotation R (Eq. 3.19) and dR/dα, rebuilt each launch from the
// learnable flips; plus what they are built from.
struct RfSpec {
    double alpha, phi;
    int32_t param, pad;
};
template <typename T>
struct RfE {
    T R[9];
    T G[9];              // (dR/dα)·Rᵀ: the derivative applied to the state after the pulse
    int32_t param, pad;  // learnable parameter index or -1
};
using RfEntry = RfE<double>;  // the compensated precision's table has the same size (8-byte values)
static_assert(sizeof(RfE<double>) == sizeof(RfE<dev::dfl>), "RF table entries of both precisions");

}  // namespace

struct mrsim_adjoint {
    mrsim_ctx *ctx = nullptr;
    int64_t n_events = 0, n_adc = 0;
    int32_t n_params = 0, seg = 64, n_rf = 0, n_cls = 0;
    AdjEvent *d_ev = nullptr;
    RfSpec *d_spec = nullptr;
    RfEntry *d_rf = nullptr;
    double *d_cls = nullptr;    // 4 per class: kx, ky, kz, dt
    double *d_demod = nullptr;  // 2 per sample: cos(adc_phase), -sin(adc_phase)
    double *d_ckpt = nullptr;   // checkpoints: (n_seg - 1) x n_spins x 3 (forward kernel), else n_seg x 3 x n_spins
    mrsim_sequence *fwd = nullptr;  // the forward program (parametric pulses, snapshots at segment starts)
    mrsim_precision prec = MRSIM_FP64;  // MRSIM_FP64, or MRSIM_FP32_KAHAN (double-float recursion)
    void *d_lam = nullptr;              // 2 values per sample: conj(demod)·dL/ds (float64 or double-float)
    size_t ckpt_cap = 0;
    const mrsim_phantom *last_ph = nullptr;
    int64_t last_n = -1;
};

namespace {

// Eq. 3.19 as the rotation by −α about n = (cos φ, sin φ, 0), and its derivative in α.
template <typename T>
__global__ void rf_table_kernel(const RfSpec *spec, int n, const double *values, RfE<T> *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const RfSpec s = spec[i];
        const double a = s.param >= 0 ? values[s.param] : s.alpha;
        double sa, ca, sp, cp;
        sincos(a, &sa, &ca);
        sincos(s.phi, &sp, &cp);
        const double n0 = cp, n1 = sp;
        const double omc = 1.0 - ca;
        RfEntry e;  // built in float64, stored in T
        // R = cos α·I + (1 − cos α)·n nᵀ − sin α·[n]x
        e.R[0] = ca + omc * n0 * n0;
        e.R[1] = omc * n0 * n1;
        e.R[2] = -sa * n1;
        e.R[3] = omc * n0 * n1;
        e.R[4] = ca + omc * n1 * n1;
        e.R[5] = sa * n0;
        e.R[6] = sa * n1;
        e.R[7] = -sa * n0;
        e.R[8] = ca;
        // dR/dα = −sin α·I + sin α·n nᵀ − cos α·[n]x, then G = (dR/dα)·Rᵀ (R is orthogonal, so the
        // state before the pulse is Rᵀ times the state after it)
        double D[9];
        D[0] = -sa + sa * n0 * n0;
        D[1] = sa * n0 * n1;
        D[2] = -ca * n1;
        D[3] = sa * n0 * n1;
        D[4] = -sa + sa * n1 * n1;
        D[5] = ca * n0;
        D[6] = ca * n1;
        D[7] = -ca * n0;
        D[8] = -sa;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                e.G[3 * r + c] = D[3 * r] * e.R[3 * c] + D[3 * r + 1] * e.R[3 * c + 1] + D[3 * r + 2] * e.R[3 * c + 2];
        RfE<T> o;
        for (int q = 0; q < 9; ++q) {
            o.R[q] = T(e.R[q]);
            o.G[q] = T(e.G[q]);
        }
        o.param = s.param;
        o.pad = 0;
        out[i] = o;
    }
}

// the learnable flips into the forward program's sub-pulse table, in both precisions
__global__ void rf_param_table_kernel(const double *values, int n, double *t64, float *t32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double sa, ca;
        sincos(values[i], &sa, &ca);
        t64[2 * i] = ca;
        t64[2 * i + 1] = sa;
        t32[2 * i] = (float)ca;
        t32[2 * i + 1] = (float)sa;
    }
}

// the backward's sample source: conj(demod_j)·h_j per sample, formed in float64 and stored in T
template <typename T>
__global__ void lam_kernel(const double *demod, const double *h, int64_t n, T *out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double cr = demod[2 * j], ci = -demod[2 * j + 1];
        const double hr = h[2 * j], hi = h[2 * j + 1];
        out[2 * j] = T(cr * hr - ci * hi);
        out[2 * j + 1] = T(cr * hi + ci * hr);
    }
}

struct AdjArgs {
    const AdjEvent *ev;
    int64_t n_events;
    const void *rf;          // RfE<T> entries
    const double *cls;
    int32_t n_cls;
    int32_t seg;
    const double *demod;     // forward: 2 per sample
    const double *params;
    int64_t n_spins, n_pad;
    double *ckpt;     // see mrsim_adjoint::d_ckpt
    int32_t ckpt_snap;  // checkpoints written as snapshots by the forward kernel
    double *signal;   // forward
    const void *lam;  // backward: conj(demod)·dL/ds per sample, 2 T values each (the adjoint's sample source)
    double *d_rho, *d_t1, *d_t2, *d_rf;
    int32_t n_params;
};

// Spin parameters: coordinates, Δf and rates in float64 (the phases are formed in float64), and
// M0 and the rates again in the arithmetic type T of the recursion.
template <typename T>
struct SpinP {
    double x, y, z, df, r1d, r2d;
    T rho, r1, r2;
};

template <typename T>
__device__ __forceinline__ SpinP<T> load_spin(const AdjArgs &a, int64_t s) {
    SpinP<T> p{};
    double rho = 0.0, r1 = 0.0, r2 = 0.0;
    p.x = p.y = p.z = p.df = 0.0;
    if (s < a.n_spins) {
        const int64_t np = a.n_pad;
        p.x = a.params[P_X * np + s];
        p.y = a.params[P_Y * np + s];
        p.z = a.params[P_Z * np + s];
        p.df = a.params[P_DF * np + s];
        rho = a.params[P_RHO * np + s];
        r1 = a.params[P_R1 * np + s];
        r2 = a.params[P_R2 * np + s];
    }
    p.r1d = r1;
    p.r2d = r2;
    p.rho = T(rho);
    p.r1 = T(r1);
    p.r2 = T(r2);
    return p;
}

// the event's interval in T
__device__ __forceinline__ double dt_of(const AdjEvent &e, double) { return e.dt; }
__device__ __forceinline__ dev::dfl dt_of(const AdjEvent &e, dev::dfl) { return dev::dfl(e.dth, e.dtl); }

// per-spin class table in shared memory: w (complex, with E2) and E1, per class (float64 math)
template <typename T>
__device__ __forceinline__ void fill_classes(const AdjArgs &a, const SpinP<T> &p, T *tab) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int c = 0; c < a.n_cls; ++c) {
        const double kx = a.cls[4 * c], ky = a.cls[4 * c + 1], kz = a.cls[4 * c + 2], dt = a.cls[4 * c + 3];
        double th = kx * p.x + ky * p.y + kz * p.z + p.df * dt;
        th -= rint(th);
        double sn, cs;
        sincospi(2.0 * th, &sn, &cs);
        const double e2 = exp(-dt * p.r2d);
        tab[(3 * c + 0) * nt + t] = T(e2 * cs);
        tab[(3 * c + 1) * nt + t] = T(-e2 * sn);
        tab[(3 * c + 2) * nt + t] = T(exp(-dt * p.r1d));
    }
}

// precession + relaxation factors of one event for this spin: w = E2·exp(−j2πφ), E1
template <typename T>
__device__ __forceinline__ void factors(const AdjEvent &e, const SpinP<T> &p, const T *tab, T &wr, T &wi, T &e1) {
    const int t = threadIdx.x, nt = blockDim.x;
    if (e.flags & A_CLS) {
        wr = tab[(3 * e.cls + 0) * nt + t];
        wi = tab[(3 * e.cls + 1) * nt + t];
        e1 = tab[(3 * e.cls + 2) * nt + t];
    } else if (e.flags & A_INL) {
        double th = e.k[0] * p.x + e.k[1] * p.y + e.k[2] * p.z + p.df * e.dt;
        th -= rint(th);
        double sn, cs;
        sincospi(2.0 * th, &sn, &cs);
        const double e2 = exp(-e.dt * p.r2d);
        wr = T(e2 * cs);
        wi = T(-e2 * sn);
        e1 = T(exp(-e.dt * p.r1d));
    } else {
        wr = T(1);
        wi = T(0);
        e1 = T(1);
    }
}

// a·b + c·d, a·b − c·d and a·b + c·d + e·f: float64 as written (the compiler forms the same
// multiply-adds as from the expressions inline); double-float in one step each (the products'
// residuals summed once, one renormalisation) instead of a renormalised value per operation
template <typename T>
__device__ __forceinline__ T dot2(T a, T b, T c, T d) { return a * b + c * d; }
template <typename T>
__device__ __forceinline__ T dot2m(T a, T b, T c, T d) { return a * b - c * d; }
template <typename T>
__device__ __forceinline__ T dot3(T a, T b, T c, T d, T e, T f) { return a * b + c * d + e * f; }
__device__ __forceinline__ dev::dfl dot2(dev::dfl a, dev::dfl b, dev::dfl c, dev::dfl d) { return dev::vdot2(a, b, c, d); }
__device__ __forceinline__ dev::dfl dot2m(dev::dfl a, dev::dfl b, dev::dfl c, dev::dfl d) { return dev::vdot2(a, b, c, -d); }
__device__ __forceinline__ dev::dfl dot3(dev::dfl a, dev::dfl b, dev::dfl c, dev::dfl d, dev::dfl e, dev::dfl f) {
    return dev::vdot3(a, b, c, d, e, f);
}

template <typename T>
__device__ __forceinline__ void apply_rf(const T *R, T M[3]) {
    const T x = dot3(R[0], M[0], R[1], M[1], R[2], M[2]);
    const T y = dot3(R[3], M[0], R[4], M[1], R[5], M[2]);
    const T z = dot3(R[6], M[0], R[7], M[1], R[8], M[2]);
    M[0] = x;
    M[1] = y;
    M[2] = z;
}

// the part of an event after its pulse: precession, T2 and T1 over the interval
template <typename T>
__device__ __forceinline__ void after_pulse(const AdjEvent &e, const SpinP<T> &p, const T *tab, T M[3]) {
    T wr, wi, e1;
    factors(e, p, tab, wr, wi, e1);
    const T x = dot2m(M[0], wr, M[1], wi);
    const T y = dot2(M[0], wi, M[1], wr);
    M[0] = x;
    M[1] = y;
    M[2] = dot2(e1, M[2], p.rho, T(1) - e1);
}

template <typename T>
__device__ __forceinline__ const RfE<T> &rf_at(const AdjArgs &a, int i) {
    return static_cast<const RfE<T> *>(a.rf)[i];
}

// forward step of one event (Eq. 4.1)
template <typename T>
__device__ __forceinline__ void step(const AdjArgs &a, const AdjEvent &e, const SpinP<T> &p, const T *tab, T M[3]) {
    if (e.flags & A_RF) apply_rf(rf_at<T>(a, e.rf).R, M);
    after_pulse(e, p, tab, M);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = v + dev::shfl_x(v, off);
    return v;
}

// stage events [e0, e0 + m) of the program into shared memory (all threads)
__device__ __forceinline__ void stage(const AdjArgs &a, int64_t e0, int m, AdjEvent *sev) {
    __syncthreads();
    const int4 *src = reinterpret_cast<const int4 *>(a.ev + e0);
    int4 *dst = reinterpret_cast<int4 *>(sev);
    for (int q = threadIdx.x; q < m * 4; q += blockDim.x) dst[q] = src[q];
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(ADJ_THREADS) adj_forward_kernel(const AdjArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    AdjEvent *sev = reinterpret_cast<AdjEvent *>(smem);
    T *tab = reinterpret_cast<T *>(smem + sizeof(AdjEvent) * a.seg);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const SpinP<T> p = load_spin<T>(a, s);
    fill_classes(a, p, tab);
    T M[3] = {T(0), T(0), p.rho};
    const int lane = threadIdx.x & 31;
    for (int64_t e0 = 0, sg = 0; e0 < a.n_events; e0 += a.seg, ++sg) {
        const int m = (int)min((int64_t)a.seg, a.n_events - e0);
        stage(a, e0, m, sev);
        if (s < a.n_spins) {
            double *ck = a.ckpt + sg * 3 * a.n_spins;
            ck[s] = (double)M[0];
            ck[a.n_spins + s] = (double)M[1];
            ck[2 * a.n_spins + s] = (double)M[2];
        }
        for (int i = 0; i < m; ++i) {
            const AdjEvent &e = sev[i];
            step(a, e, p, tab, M);
            if (e.flags & A_ADC) {
                const double sx = (double)warp_sum(M[0]), sy = (double)warp_sum(M[1]);
                if (lane == 0) {
                    const double cr = a.demod[2 * e.adc], ci = a.demod[2 * e.adc + 1];
                    atomicAdd(a.signal + 2 * e.adc, sx * cr - sy * ci);
                    atomicAdd(a.signal + 2 * e.adc + 1, sx * ci + sy * cr);
                }
            }
        }
    }
}

// LOCAL: each thread sums its RF-parameter gradients in a local array (n_params <= ADJ_LOCAL_PARAMS)
// and the block reduces them once at the end; otherwise every pulse reduces over the warp.
template <typename T, bool LOCAL>
__global__ void __launch_bounds__(ADJ_THREADS) adj_backward_kernel(const AdjArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    AdjEvent *sev = reinterpret_cast<AdjEvent *>(smem);
    T *tab = reinterpret_cast<T *>(smem + sizeof(AdjEvent) * a.seg);
    double *grf = reinterpret_cast<double *>(tab + 3 * a.n_cls * blockDim.x);  // block's RF-parameter gradient
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const SpinP<T> p = load_spin<T>(a, s);
    fill_classes(a, p, tab);
    for (int q = threadIdx.x; q < a.n_params; q += blockDim.x) grf[q] = 0.0;
    const int lane = threadIdx.x & 31;
    const bool valid = s < a.n_spins;
    const T *lam = static_cast<const T *>(a.lam);
    T buf[ADJ_MAX_SEG][5];  // per event of the segment: state after its pulse, then the transverse state after it
    T gl[LOCAL ? ADJ_LOCAL_PARAMS : 1];
    if constexpr (LOCAL)
        for (int q = 0; q < a.n_params; ++q) gl[q] = T(0);
    T L[3] = {T(0), T(0), T(0)};
    T g_rho = T(0), g_r1 = T(0), g_r2 = T(0);
    const int64_t n_seg = (a.n_events + a.seg - 1) / a.seg;
    for (int64_t sg = n_seg - 1; sg >= 0; --sg) {
        const int64_t e0 = sg * a.seg;
        const int m = (int)min((int64_t)a.seg, a.n_events - e0);
        stage(a, e0, m, sev);
        T M[3] = {T(0), T(0), T(0)};
        if (valid && a.ckpt_snap) {  // state after event sg·C − 1; the first segment starts at rest
            if (sg == 0) {
                M[2] = p.rho;
            } else {
                const double *ck = a.ckpt + ((sg - 1) * a.n_spins + s) * 3;
                M[0] = T(ck[0]);
                M[1] = T(ck[1]);
                M[2] = T(ck[2]);
            }
        } else if (valid) {
            const double *ck = a.ckpt + sg * 3 * a.n_spins;
            M[0] = T(ck[s]);
            M[1] = T(ck[a.n_spins + s]);
            M[2] = T(ck[2 * a.n_spins + s]);
        }
        for (int i = 0; i < m; ++i) {
            const AdjEvent &e = sev[i];
            if (e.flags & A_RF) apply_rf(rf_at<T>(a, e.rf).R, M);
            buf[i][0] = M[0];
            buf[i][1] = M[1];
            buf[i][2] = M[2];
            after_pulse(e, p, tab, M);
            buf[i][3] = M[0];
            buf[i][4] = M[1];
        }
        for (int i = m - 1; i >= 0; --i) {
            const AdjEvent &e = sev[i];
            if (e.flags & A_ADC) {  // λ += conj(d_j)·h_j
                L[0] += lam[2 * e.adc];
                L[1] += lam[2 * e.adc + 1];
            }
            const T Ma[3] = {buf[i][0], buf[i][1], buf[i][2]};  // state after the event's pulse
            T wr, wi, e1;
            factors(e, p, tab, wr, wi, e1);
            // parameter gradients through P (λ is the adjoint after the event)
            const T mx = buf[i][3], my = buf[i][4];  // P·M_a, transverse part
            const T ndt = -dt_of(e, T(0));
            g_r2 += ndt * dot2(L[0], mx, L[1], my);
            g_r1 += ndt * e1 * (Ma[2] - p.rho) * L[2];
            g_rho += (T(1) - e1) * L[2];
            // λ_a = Pᵀ λ: conj(w)·λ on the transverse part, E1 on z
            const T lax = dot2(L[0], wr, L[1], wi), lay = dot2m(L[1], wr, L[0], wi), laz = e1 * L[2];
            if (e.flags & A_RF) {
                const RfE<T> &rf = rf_at<T>(a, e.rf);
                if (rf.param >= 0) {
                    // dL/dα = λ_aᵀ·(dR/dα)·M_n = λ_aᵀ·G·M_a
                    const T *G = rf.G;
                    const T dx = dot3(G[0], Ma[0], G[1], Ma[1], G[2], Ma[2]);
                    const T dy = dot3(G[3], Ma[0], G[4], Ma[1], G[5], Ma[2]);
                    const T dz = dot3(G[6], Ma[0], G[7], Ma[1], G[8], Ma[2]);
                    const T g = dot3(lax, dx, lay, dy, laz, dz);
                    if constexpr (LOCAL) {
                        gl[rf.param] += g;
                    } else {  // reduced over the warp, then the block (shared atomics)
                        const double gw = (double)warp_sum(g);
                        if (lane == 0) atomicAdd(&grf[rf.param], gw);
                    }
                }
                // λ_n = Rᵀ λ_a
                L[0] = dot3(rf.R[0], lax, rf.R[3], lay, rf.R[6], laz);
                L[1] = dot3(rf.R[1], lax, rf.R[4], lay, rf.R[7], laz);
                L[2] = dot3(rf.R[2], lax, rf.R[5], lay, rf.R[8], laz);
            } else {
                L[0] = lax;
                L[1] = lay;
                L[2] = laz;
            }
        }
    }
    g_rho += L[2];  // initial state (0, 0, M0)
    if constexpr (LOCAL) {
        for (int q = 0; q < a.n_params; ++q) {
            const double gw = (double)warp_sum(gl[q]);
            if (lane == 0 && gw != 0.0) atomicAdd(&grf[q], gw);
        }
    }
    __syncthreads();
    if (a.d_rf)
        for (int q = threadIdx.x; q < a.n_params; q += blockDim.x)
            if (grf[q] != 0.0) atomicAdd(a.d_rf + q, grf[q]);
    if (valid) {
        // dL/dT = dL/dR · dR/dT = −dL/dR / T², i.e. −dL/dR · R²; T = ∞ (R = 0) gives 0
        if (a.d_rho) a.d_rho[s] = (double)g_rho;
        if (a.d_t1) a.d_t1[s] = -(double)g_r1 * p.r1d * p.r1d;
        if (a.d_t2) a.d_t2[s] = -(double)g_r2 * p.r2d * p.r2d;
    }
}

}  // namespace

namespace {

mrsim_status afail(mrsim_ctx *ctx, mrsim_status st, const std::string &m) {
    if (ctx) ctx->err = m;
    log_failure(st, m);
    return st;
}

bool dev_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t adj_smem(const mrsim_adjoint *adj, bool backward) {
    return sizeof(AdjEvent) * adj->seg + sizeof(double) * 3 * adj->n_cls * ADJ_THREADS +
           (backward ? sizeof(double) * (size_t)adj->n_params : 0);
}

AdjArgs adj_args(const mrsim_adjoint *adj, const mrsim_phantom *ph) {
    AdjArgs a{};
    a.ev = adj->d_ev;
    a.n_events = adj->n_events;
    a.rf = adj->d_rf;
    a.cls = adj->d_cls;
    a.n_cls = adj->n_cls;
    a.seg = adj->seg;
    a.demod = adj->d_demod;
    a.params = ph->params;
    a.n_spins = ph->n;
    a.n_pad = ph->n_pad;
    a.ckpt = adj->d_ckpt;
    a.ckpt_snap = adj->fwd != nullptr;
    a.n_params = adj->n_params;
    return a;
}

mrsim_status prepare_rf(mrsim_adjoint *adj, const double *rf_values, cudaStream_t st) {
    mrsim_ctx *ctx = adj->ctx;
    if (adj->n_params > 0 && !dev_ptr(rf_values)) return afail(ctx, MRSIM_EINVAL, "rf_values must be device memory");
    if (adj->n_rf == 0) return MRSIM_OK;
    if (adj->prec == MRSIM_FP32_KAHAN)
        rf_table_kernel<dev::dfl><<<(adj->n_rf + 127) / 128, 128, 0, st>>>(
            adj->d_spec, adj->n_rf, rf_values, reinterpret_cast<RfE<dev::dfl> *>(adj->d_rf));
    else
        rf_table_kernel<double><<<(adj->n_rf + 127) / 128, 128, 0, st>>>(adj->d_spec, adj->n_rf, rf_values, adj->d_rf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, std::string("rf table: ") + cudaGetErrorString(e));
    return MRSIM_OK;
}

template <class T>
cudaError_t put(mrsim_ctx *ctx, T **d, const std::vector<T> &v) {
    *d = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = ctx_malloc(ctx, d, v.size() * sizeof(T));
    if (e == cudaSuccess) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

extern "C" {

mrsim_status mrsim_adjoint_create(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events, double gamma,
                                  const int32_t *rf_param, int32_t n_params, int32_t ckpt_every,
                                  mrsim_adjoint **out) {
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    // the forward compiler validates the event list with the same rules
    {
        Compiled c;
        std::string err;
        int rc = compile_sequence(events, n_events, gamma, c, err);
        if (rc != MRSIM_OK) return afail(ctx, (mrsim_status)rc, err);
    }
    if (n_params < 0 || (n_params > 0 && !rf_param)) return afail(ctx, MRSIM_EINVAL, "invalid rf_param / n_params");
    if (ckpt_every == 0) ckpt_every = 64;
    if (ckpt_every < 1 || ckpt_every > ADJ_MAX_SEG)
        return afail(ctx, MRSIM_EINVAL, "ckpt_every must be in [1, " + std::to_string(ADJ_MAX_SEG) + "]");
    std::vector<AdjEvent> ev((size_t)n_events);
    std::vector<RfSpec> spec;
    std::vector<double> demod;
    std::map<std::array<double, 4>, std::pair<int64_t, int64_t>> uses;
    for (int64_t i = 0; i < n_events; ++i) {
        const mrsim_event &e = events[i];
        const std::array<double, 4> key = {gamma * e.gx * e.dt, gamma * e.gy * e.dt, gamma * e.gz * e.dt, e.dt};
        if (e.dt > 0.0) {
            auto it = uses.find(key);
            if (it == uses.end())
                uses[key] = {1, i};
            else
                ++it->second.first;
        }
    }
    // up to 16 recurring intervals become per-spin classes (most frequent first)
    std::vector<std::pair<std::array<double, 4>, std::pair<int64_t, int64_t>>> v(uses.begin(), uses.end());
    std::sort(v.begin(), v.end(), [](const auto &a, const auto &b) {
        return a.second.first != b.second.first ? a.second.first > b.second.first : a.second.second < b.second.second;
    });
    std::map<std::array<double, 4>, int> cls;
    std::vector<double> ctab;
    for (auto &kv : v) {
        if ((int)cls.size() >= ADJ_MAX_CLASSES || kv.second.first < 2) break;
        cls[kv.first] = (int)cls.size();
        for (double x : kv.first) ctab.push_back(x);
    }
    int64_t j = 0;
    for (int64_t i = 0; i < n_events; ++i) {
        const mrsim_event &e = events[i];
        AdjEvent a{};
        const int32_t prm = rf_param ? rf_param[i] : -1;
        if (prm >= n_params) return afail(ctx, MRSIM_EINVAL, "rf_param index out of range at event " + std::to_string(i));
        if (e.rf_flip != 0.0 || prm >= 0) {
            a.flags |= A_RF;
            a.rf = (int32_t)spec.size();
            spec.push_back(RfSpec{e.rf_flip, e.rf_phase, prm, 0});
        }
        const std::array<double, 4> key = {gamma * e.gx * e.dt, gamma * e.gy * e.dt, gamma * e.gz * e.dt, e.dt};
        a.dt = e.dt;
        a.dth = (float)e.dt;
        a.dtl = (float)(e.dt - (double)a.dth);
        if (e.dt > 0.0) {
            auto c = cls.find(key);
            if (c != cls.end()) {
                a.flags |= A_CLS;
                a.cls = c->second;
            } else {
                a.flags |= A_INL;
                a.k[0] = key[0];
                a.k[1] = key[1];
                a.k[2] = key[2];
            }
        }
        if (e.adc) {
            a.flags |= A_ADC;
            a.adc = (int32_t)j++;
            demod.push_back(std::cos(e.adc_phase));
            demod.push_back(-std::sin(e.adc_phase));
        }
        ev[(size_t)i] = a;
    }
    cudaSetDevice(ctx->device);
    mrsim_adjoint *adj = new (std::nothrow) mrsim_adjoint();
    if (!adj) return afail(ctx, MRSIM_ENOMEM, "host allocation failed");
    adj->ctx = ctx;
    adj->n_events = n_events;
    adj->n_adc = j;
    adj->n_params = n_params;
    adj->seg = ckpt_every;
    adj->n_rf = (int32_t)spec.size();
    adj->n_cls = (int32_t)cls.size();
    cudaError_t e = put(ctx, &adj->d_ev, ev);
    if (e == cudaSuccess) e = put(ctx, &adj->d_spec, spec);
    if (e == cudaSuccess && !spec.empty()) e = ctx_malloc(ctx, &adj->d_rf, spec.size() * sizeof(RfEntry));
    if (e == cudaSuccess) e = put(ctx, &adj->d_cls, ctab);
    if (e == cudaSuccess) e = put(ctx, &adj->d_demod, demod);
    if (e != cudaSuccess) {
        mrsim_adjoint_destroy(adj);
        cudaGetLastError();
        return afail(ctx, e == cudaErrorMemoryAllocation ? MRSIM_ENOMEM : MRSIM_ECUDA,
                     std::string("adjoint program: ") + cudaGetErrorString(e));
    }
    if (adj_smem(adj, true) > (size_t)ctx->max_smem_optin) {
        mrsim_adjoint_destroy(adj);
        return afail(ctx, MRSIM_EUNSUPPORTED, "adjoint program needs more shared memory than the device has");
    }
    if (n_params <= TRAIN_TABLE_MAX / 2) {  // the forward program: parametric pulses, a snapshot per segment start
        std::vector<int64_t> snaps;
        for (int64_t e0 = ckpt_every; e0 < n_events; e0 += ckpt_every) snaps.push_back(e0 - 1);
        mrsim_compiled c;
        std::shared_ptr<HostProgram> prog;
        std::string err;
        mrsim_status rc = compile_host(n_events, events, gamma, (int64_t)snaps.size(), snaps.data(), prog, err,
                                       n_params > 0 ? rf_param : nullptr, n_params);
        c.prog = std::move(prog);
        if (rc == MRSIM_OK) {
            rc = mrsim_sequence_create(ctx, &c, &adj->fwd);
            if (rc == MRSIM_OK && fwd_smem_bytes(true, adj->fwd->p64, 1, ADJ_THREADS) > (size_t)ctx->max_smem_optin) {
                mrsim_sequence_destroy(adj->fwd);
                adj->fwd = nullptr;
            }
        }
        if (rc != MRSIM_OK) {
            mrsim_adjoint_destroy(adj);
            return afail(ctx, rc, "adjoint forward program: " + (err.empty() ? std::string(mrsim_last_error(ctx)) : err));
        }
    }
    *out = adj;
    return MRSIM_OK;
}

int64_t mrsim_adjoint_num_adc(const mrsim_adjoint *adj) { return adj ? adj->n_adc : -1; }

mrsim_status mrsim_adjoint_forward(mrsim_adjoint *adj, const mrsim_phantom *ph, const double *rf_values,
                                   void *stream, double *signal_out) {
    if (!adj) return MRSIM_EINVAL;
    mrsim_ctx *ctx = adj->ctx;
    if (!ph || ph->ctx != ctx) return afail(ctx, MRSIM_EINVAL, "NULL phantom or another context");
    if (adj->n_adc > 0 && !dev_ptr(signal_out)) return afail(ctx, MRSIM_EINVAL, "signal_out must be device memory");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n_seg = (adj->n_events + adj->seg - 1) / adj->seg;
    const size_t need = (size_t)std::max<int64_t>(n_seg, 1) * 3 * (size_t)std::max<int64_t>(ph->n, 1);
    if (need > adj->ckpt_cap) {
        cudaFree(adj->d_ckpt);
        adj->d_ckpt = nullptr;
        adj->ckpt_cap = 0;
        cudaError_t e = ctx_malloc(ctx, &adj->d_ckpt, need * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return afail(ctx, MRSIM_ENOMEM, "checkpoint storage: " + std::to_string(need * 8) + " bytes");
        }
        adj->ckpt_cap = need;
    }
    mrsim_status rs = prepare_rf(adj, rf_values, st);
    if (rs != MRSIM_OK) return rs;
    if (adj->n_adc > 0) {
        cudaError_t e = cudaMemsetAsync(signal_out, 0, 16 * (size_t)adj->n_adc, st);
        if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, "clear signal");
    }
    adj->last_ph = ph;
    adj->last_n = ph->n;
    if (ph->n == 0) return MRSIM_OK;
    if (adj->fwd) {  // the float64 forward kernel on the parametric program; snapshots = checkpoints
        if (adj->n_params > 0) {
            rf_param_table_kernel<<<(adj->n_params + 127) / 128, 128, 0, st>>>(rf_values, adj->n_params,
                                                                              adj->fwd->d_train64, adj->fwd->d_train32);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, std::string("flip table: ") + cudaGetErrorString(e));
        }
        FwdArgs f{};
        f.prog = adj->fwd->p64;
        f.params = ph->params;
        f.n_spins = ph->n;
        f.n_pad = ph->n_pad;
        f.signal = signal_out;
        f.status = ctx->d_status;
        f.snap = adj->d_ckpt;
        const int rc = adj->prec == MRSIM_FP32_KAHAN ? launch_fwd_df(f, 1, ADJ_THREADS, st)
                                                      : launch_fwd_f64(f, 1, ADJ_THREADS, st);
        if (rc != 0) return afail(ctx, MRSIM_ECUDA, std::string("adjoint forward: ") + cudaGetErrorString((cudaError_t)rc));
        return MRSIM_OK;
    }
    AdjArgs a = adj_args(adj, ph);
    a.signal = signal_out;
    const size_t smem = adj_smem(adj, false);
    const int64_t grid = (ph->n + ADJ_THREADS - 1) / ADJ_THREADS;
    if (adj->prec == MRSIM_FP32_KAHAN) {
        cudaFuncSetAttribute(adj_forward_kernel<dev::dfl>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        adj_forward_kernel<dev::dfl><<<(unsigned)grid, ADJ_THREADS, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(adj_forward_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        adj_forward_kernel<double><<<(unsigned)grid, ADJ_THREADS, smem, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, std::string("adjoint forward: ") + cudaGetErrorString(e));
    return MRSIM_OK;
}

mrsim_status mrsim_adjoint_backward(mrsim_adjoint *adj, const mrsim_phantom *ph, const double *rf_values,
                                    const double *dl_dsignal, void *stream, double *d_rho, double *d_t1,
                                    double *d_t2, double *d_rf) {
    if (!adj) return MRSIM_EINVAL;
    mrsim_ctx *ctx = adj->ctx;
    if (!ph || ph != adj->last_ph || ph->n != adj->last_n)
        return afail(ctx, MRSIM_EINVAL, "backward needs the phantom of the last forward call");
    if (adj->n_adc > 0 && !dev_ptr(dl_dsignal)) return afail(ctx, MRSIM_EINVAL, "dl_dsignal must be device memory");
    for (const double *q : {(const double *)d_rho, (const double *)d_t1, (const double *)d_t2, (const double *)d_rf})
        if (q && !dev_ptr(q)) return afail(ctx, MRSIM_EINVAL, "gradient outputs must be device memory");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    mrsim_status rs = prepare_rf(adj, rf_values, st);
    if (rs != MRSIM_OK) return rs;
    if (d_rf && adj->n_params > 0) {
        cudaError_t e = cudaMemsetAsync(d_rf, 0, sizeof(double) * (size_t)adj->n_params, st);
        if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, "clear d_rf");
    }
    if (ph->n == 0) return MRSIM_OK;
    AdjArgs a = adj_args(adj, ph);
    if (adj->n_adc > 0) {  // the sample source conj(demod)·dL/ds in the recursion's arithmetic
        if (!adj->d_lam) {
            cudaError_t e = ctx_malloc(ctx, &adj->d_lam, 16 * (size_t)adj->n_adc);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return afail(ctx, MRSIM_ENOMEM, "adjoint sample sources");
            }
        }
        const int blocks = (int)std::min<int64_t>((adj->n_adc + 255) / 256, 1024);
        if (adj->prec == MRSIM_FP32_KAHAN)
            lam_kernel<dev::dfl><<<blocks, 256, 0, st>>>(adj->d_demod, dl_dsignal, adj->n_adc,
                                                        static_cast<dev::dfl *>(adj->d_lam));
        else
            lam_kernel<double><<<blocks, 256, 0, st>>>(adj->d_demod, dl_dsignal, adj->n_adc,
                                                      static_cast<double *>(adj->d_lam));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, std::string("adjoint sample sources: ") + cudaGetErrorString(e));
    }
    a.lam = adj->d_lam;
    a.d_rho = d_rho;
    a.d_t1 = d_t1;
    a.d_t2 = d_t2;
    a.d_rf = d_rf;
    const size_t smem = adj_smem(adj, true);
    const int64_t grid = (ph->n + ADJ_THREADS - 1) / ADJ_THREADS;
    auto run = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<(unsigned)grid, ADJ_THREADS, smem, st>>>(a);
    };
    const bool local = adj->n_params <= ADJ_LOCAL_PARAMS;
    if (adj->prec == MRSIM_FP32_KAHAN) {
        if (local) run(adj_backward_kernel<dev::dfl, true>);
        else run(adj_backward_kernel<dev::dfl, false>);
    } else {
        if (local) run(adj_backward_kernel<double, true>);
        else run(adj_backward_kernel<double, false>);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(ctx, MRSIM_ECUDA, std::string("adjoint backward: ") + cudaGetErrorString(e));
    return MRSIM_OK;
}

mrsim_status mrsim_adjoint_set_precision(mrsim_adjoint *adj, mrsim_precision prec) {
    if (!adj) return MRSIM_EINVAL;
    if (prec == MRSIM_FP32) return afail(adj->ctx, MRSIM_EUNSUPPORTED, "the adjoint has no plain float32 recursion");
    if (prec != MRSIM_FP64 && prec != MRSIM_FP32_KAHAN) return afail(adj->ctx, MRSIM_EINVAL, "unknown precision");
    adj->prec = prec;
    adj->last_ph = nullptr;  // checkpoints of the other arithmetic are not reused
    adj->last_n = -1;
    return MRSIM_OK;
}

mrsim_status mrsim_simulate_adjoint(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                                    mrsim_precision prec, int32_t ckpt_every, const double *dl_dsignal, void *stream,
                                    double *d_rho, double *d_t1, double *d_t2, double *d_rf_flip) {
    if (!ctx) return MRSIM_EINVAL;
    if (!ph || !seq || ph->ctx != ctx || seq->ctx != ctx)
        return afail(ctx, MRSIM_EINVAL, "NULL phantom / sequence or another context");
    if (!normalize_precision(prec)) return afail(ctx, MRSIM_EINVAL, "unknown precision");
    if (prec == MRSIM_FP32)
        return afail(ctx, MRSIM_EUNSUPPORTED, "the adjoint runs in float64 or the compensated precision, not float32");
    const HostProgram &hp = *seq->prog;
    const int64_t n_ev = hp.n_events, n_adc = hp.host.n_adc, n = ph->n;
    if (n_adc > 0 && !dl_dsignal) return afail(ctx, MRSIM_EINVAL, "dl_dsignal is NULL");
    // with d_rf_flip every pulse (event with rf_flip != 0) is a learnable flip, in event order
    std::vector<int32_t> rp;
    std::vector<double> flips;
    if (d_rf_flip) {
        rp.assign((size_t)n_ev, -1);
        for (int64_t e = 0; e < n_ev; ++e)
            if (hp.events[(size_t)e].rf_flip != 0.0) {
                rp[(size_t)e] = (int32_t)flips.size();
                flips.push_back(hp.events[(size_t)e].rf_flip);
            }
    }
    const int32_t n_params = (int32_t)flips.size();
    mrsim_adjoint *adj = nullptr;
    mrsim_status rs = mrsim_adjoint_create(ctx, n_ev, hp.events.data(), hp.gamma, d_rf_flip ? rp.data() : nullptr,
                                           n_params, ckpt_every, &adj);
    if (rs != MRSIM_OK) return rs;
    if (prec == MRSIM_FP32_KAHAN) mrsim_adjoint_set_precision(adj, prec);
    // one device block for the flips, the signal and every host-side input or output:
    // [flips | signal | dL/ds | d_rho | d_t1 | d_t2 | d_rf]
    const bool h_dl = n_adc > 0 && !dev_ptr(dl_dsignal);
    double *outs[4] = {d_rho, d_t1, d_t2, d_rf_flip};
    const int64_t out_n[4] = {n, n, n, n_params};
    bool h_out[4];
    size_t need = (size_t)n_params + 2 * (size_t)n_adc + (h_dl ? 2 * (size_t)n_adc : 0);
    for (int i = 0; i < 4; ++i) {
        h_out[i] = outs[i] && out_n[i] > 0 && !dev_ptr(outs[i]);
        if (h_out[i]) need += (size_t)out_n[i];
    }
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    double *blk = nullptr;
    if (need > 0) {
        cudaError_t e = ctx_malloc(ctx, &blk, need * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            mrsim_adjoint_destroy(adj);
            return afail(ctx, MRSIM_ENOMEM, "adjoint buffers: " + std::to_string(need * 8) + " bytes");
        }
    }
    double *q = blk;
    double *rfv = n_params ? q : nullptr;
    q += n_params;
    double *sig = q;
    q += 2 * n_adc;
    const double *dl = dl_dsignal;
    if (h_dl) {
        dl = q;
        q += 2 * n_adc;
    }
    double *dout[4];
    for (int i = 0; i < 4; ++i) {
        dout[i] = outs[i];
        if (h_out[i]) {
            dout[i] = q;
            q += out_n[i];
        }
    }
    cudaError_t e = cudaSuccess;
    if (n_params) e = cudaMemcpyAsync(rfv, flips.data(), flips.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && h_dl)
        e = cudaMemcpyAsync((double *)dl, dl_dsignal, 16 * (size_t)n_adc, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rs = afail(ctx, MRSIM_ECUDA, std::string("adjoint inputs: ") + cudaGetErrorString(e));
    if (rs == MRSIM_OK) rs = mrsim_adjoint_forward(adj, ph, rfv, stream, sig);
    if (rs == MRSIM_OK) rs = mrsim_adjoint_backward(adj, ph, rfv, dl, stream, dout[0], dout[1], dout[2], dout[3]);
    for (int i = 0; i < 4 && rs == MRSIM_OK; ++i)
        if (h_out[i]) {
            e = cudaMemcpyAsync(outs[i], dout[i], sizeof(double) * (size_t)out_n[i], cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) rs = afail(ctx, MRSIM_ECUDA, std::string("adjoint outputs: ") + cudaGetErrorString(e));
        }
    // the adjoint's tables and checkpoints are freed below: wait for the work that reads them
    e = cudaStreamSynchronize(st);
    if (rs == MRSIM_OK && e != cudaSuccess) rs = afail(ctx, MRSIM_ECUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    cudaFree(blk);
    mrsim_adjoint_destroy(adj);
    if (rs == MRSIM_OK) rs = mrsim_stream_status(ctx, stream);
    return rs;
}

void mrsim_adjoint_destroy(mrsim_adjoint *adj) {
    if (!adj) return;
    cudaSetDevice(adj->ctx->device);
    cudaFree(adj->d_ev);
    cudaFree(adj->d_spec);
    cudaFree(adj->d_rf);
    cudaFree(adj->d_cls);
    cudaFree(adj->d_demod);
    cudaFree(adj->d_ckpt);
    cudaFree(adj->d_lam);
    mrsim_sequence_destroy(adj->fwd);
    delete adj;
}

}  // extern "C"
