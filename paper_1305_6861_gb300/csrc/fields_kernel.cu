// fields_kernel.cu -- simulation with non-parallel fields (§3.2, §3.4.3.2): a static field whose
// direction n differs from z at each spin, and gradient fields with components transverse to z.
//
// §3.2 turns the frame locally so that one axis lies along the static field, applies the Bloch
// equation there and turns the result back; §3.4.3.2 lets a constant gradient field with
// transverse components change the direction of the total field, with T1 relaxation following
// that direction.  Per spin and elementary sequence, after the RF pulse (Eq. 3.19, rotating
// frame):
//   b = (gtx.x, gty.x, G.x),  u = B0 n + b,  h = u/|u|
//   θ = γ (|u| - B0) Δt + Δω Δt,      |u| - B0 = p + r²/(|u| + B0 + p),  p = n.b,  r = |b - p n|
//   M <- E2 (cos θ M⊥ - sin θ h × M⊥) + (E1 (M.h) + M0 (1 - E1)) h,      M⊥ = M - (M.h) h
// i.e. Eqs. 3.5/3.14 in the frame turned to h.  Every spin starts at M0 n.
//
// The turn of one interval is an affine map M <- A M + c with
//   A = E2 cos θ (I - h hᵀ) - E2 sin θ [h]x + E1 h hᵀ,   c = M0 (1 - E1) h,
// which depends on the event only through its free interval (Δt, G, transverse components).  Each
// spin keeps the map of the last interval it computed, and an event whose interval equals that one
// (every sub-pulse of a shaped pulse after the first, every step of a readout) applies it with nine
// FMAs instead of recomputing the field, its direction, the phase and the exponentials.
//
// Layout: one spin per thread (float64) or two (float32), state, direction and position in
// registers; the event records are staged through shared memory in chunks of FIELD_CHUNK by the
// whole block; each thread writes its spins' value of each sample to its own column of a shared
// window, the block sums the window's rows after the chunk, and float64 atomics add them across
// blocks.
//
// float32 path: the large part of the phase, γ/2π Δt p = Σ_j n_j (k_j . x) with the moments
// k_j = γ/2π g_j Δt in cycles/m, is summed from float-float products (hi, lo pairs of the
// float64 values) whose integer parts drop out exactly; the small remainder γ/2π Δt r²/(...) and
// everything else are float32.  Its error grows like the square root of the number of events
// (about 1e-7 rad per event).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/mrsim.h"
#include "dfloat.cuh"
#include "handles.h"
#include "internal.h"

using namespace mrsim;

namespace {

constexpr int FIELD_THREADS = 128;
constexpr int FIELD_CHUNK = 32;
constexpr int FIELD_K32 = 2;  // spins per thread of the float32 kernel
constexpr double TWO_PI = 6.283185307179586476925286766559;

// FF_RUN_START: the first event of a run of identical free intervals (same Δt, G, transverse
// components, no pulse): its state before the step is kept.  FF_RUN: an anchored later event of
// the run, whose record holds the run's interval so far (j·Δt and its moments), applied to the kept
// state.  The turn and the relaxation of j equal intervals are one turn by jθ with E^j (the axis h
// is the same for all of them), so an anchored step is computed from the run's start and the
// rounding of one interval's turn does not repeat j times.  Every FIELD_ANCHOR-th step of a run and
// its last step are anchored; the steps between apply the cached one-interval map (FF_SAME), so
// the repeated rounding reaches at most FIELD_ANCHOR - 1 steps and never the state a run hands on.
// FF_SAME: the free interval equals the one whose map the spin holds; apply it.
enum FieldFlags : int32_t {
    FF_RF = 1, FF_TRANSVERSE = 2, FF_ADC = 4, FF_FREE = 8, FF_RUN_START = 16, FF_RUN = 32, FF_SAME = 64,
    FF_TMAP = 128  // the first event of a mapped train: apply train map (flags >> 16) & 0xff; the train's
                   // other events carry no flags
};
// Train maps: a train (two or more consecutive pulsed events without samples that share one free
// interval) that recurs at least TRAIN_MAP_MIN times with the same pulses and interval runs, per
// spin, as one affine map composed at set-up (pulse, then the interval's turn, event by event).
constexpr int FIELD_TRAIN_MAX = 256;  // longest mapped train (its pulses are staged in shared memory)
constexpr int64_t FIELD_ANCHOR = 32;

// The two kinds of event that make up most sequences, which the float32 kernel runs in loops of
// their own: a sample step of a readout (the held map, then the sample) and a sub-pulse of a
// shaped pulse (the pulse, then the held map).  Any other event takes the general path.
constexpr int32_t KIND_MASK = FF_RF | FF_ADC | FF_FREE | FF_RUN_START | FF_RUN | FF_SAME;
constexpr int32_t KIND_READ = FF_ADC | FF_FREE | FF_SAME;
constexpr int32_t KIND_TRAIN = FF_RF | FF_FREE | FF_SAME;

// float64 record: 22 doubles + 4 ints = 192 bytes
struct alignas(16) FieldEv64 {
    double R[9];        // Eq. 3.19 rotation (row-major) when FF_RF
    double g[3];        // G [T/m]: field along z, G.x
    double gt[6];       // transverse components [T/m]: Bx = gt[0..2].x, By = gt[3..5].x
    double gdt;         // γ Δt [rad/(T)]  (in a run: of the run's interval so far)
    double dt;          // Δt [s]          (likewise)
    double dem[2];      // cos, sin of the receiver phase
    int32_t flags;
    int32_t adc;        // index of the event's sample, or of the next sample if it takes none
    int32_t slot;       // position of the sample within the chunk of FIELD_CHUNK events
    int32_t nslot;      // samples in the event's chunk
};
static_assert(sizeof(FieldEv64) == 192, "FieldEv64 layout");

// float32 record: 48 floats/ints = 192 bytes
struct alignas(16) FieldEv32 {
    float R[9];
    float g[3];
    float gt[6];
    float kh[9], kl[9];  // k_j[d] = γ/2π g_j[d] Δt [cycles/m] as (hi, lo): j = z (G), x, y (transverse)
    float dth, dtl;      // Δt as (hi, lo)
    float gdt2pi;        // γ/2π Δt [cycles/T] (for the small remainder)
    float dt;
    float dem[2];
    int32_t flags, adc, slot, nslot;  // as in FieldEv64
    int32_t seg;                      // events from this one on, within the chunk, of the same kind
    int32_t pad;
};
static_assert(sizeof(FieldEv32) == 192, "FieldEv32 layout");

struct FieldArgs {
    const void *ev;
    int64_t n_events;
    const double *params;  // NPARAM x n_pad
    int64_t n_spins, n_pad;
    const double *ndir;    // 3 per spin, or NULL: every spin's field along z
    double b0;
    double *signal;        // 2 per sample
    const void *maps;      // train maps: kind x TRAIN_MAP_ROWS rows of n_pad values (float or double)
};

// The map kinds of an event list: the first occurrence (event, length) of each.
struct FieldKinds {
    int32_t n;
    int32_t len[TRAIN_MAP_MAX];
    int64_t first[TRAIN_MAP_MAX];
};

// train map kind t of spin s applied to (M0, M1, M2): M <- A M + c
template <typename R, typename T>
__device__ __forceinline__ void apply_train_map(const R *maps, int t, int64_t np, int64_t s, T &M0, T &M1, T &M2) {
    const R *m = maps + (int64_t)t * TRAIN_MAP_ROWS * np + s;
    T A[TRAIN_MAP_ROWS];
#pragma unroll
    for (int j = 0; j < TRAIN_MAP_ROWS; ++j) A[j] = (T)m[j * np];
    const T t0 = A[2] * M2 + (A[1] * M1 + (A[0] * M0 + A[9]));
    const T t1 = A[5] * M2 + (A[4] * M1 + (A[3] * M0 + A[10]));
    const T t2 = A[8] * M2 + (A[7] * M1 + (A[6] * M0 + A[11]));
    M0 = t0;
    M1 = t1;
    M2 = t2;
}

// Phase accumulator in cycles for products of (hi, lo) pairs: per product the integer part of
// the leading product is removed exactly (|ah bh| < 2^22, the fractional part is exact), its
// rounding error (an FMA) and the cross terms go to a small part; value() adds the fractional
// parts and the small part and reduces the sum to [-1/2, 1/2].  The sum of a few fractional
// parts rounds at ulp(2) = 2^-22 cycles at most, below the float32 rounding of the turn itself.
struct PhaseAcc {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add_product(float ah, float al, float bh, float bl) {
        const float p = ah * bh;
        c += fmaf(ah, bh, -p) + fmaf(ah, bl, al * bh);
        s += p - rintf(p);
    }
    __device__ __forceinline__ float value() const {
        const float t = (s - rintf(s)) + c;
        return t - rintf(t);
    }
};

__host__ __device__ __forceinline__ void split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// The map of one turn about h by θ with E2 = e2 across and E1 = 1 + e1m along h, in A and c.
template <typename T>
__device__ __forceinline__ void turn_map(T hx, T hy, T hz, T cs, T sn, T e1m, T e2, T m0, T (&A)[9], T (&c)[3]) {
    const T a = e2 * cs, d = e2 * sn;
    const T b = (T(1) + e1m) - a;  // E1 - E2 cos θ: the coefficient of h hᵀ
    const T bx = b * hx, by = b * hy, bz = b * hz;
    const T xy = bx * hy, xz = bx * hz, yz = by * hz;
    A[0] = bx * hx + a;
    A[1] = xy + d * hz;
    A[2] = xz - d * hy;
    A[3] = xy - d * hz;
    A[4] = by * hy + a;
    A[5] = yz + d * hx;
    A[6] = xz + d * hy;
    A[7] = yz - d * hx;
    A[8] = bz * hz + a;
    const T w = -e1m * m0;  // M0 (1 - E1)
    c[0] = w * hx;
    c[1] = w * hy;
    c[2] = w * hz;
}

template <typename T>
__device__ __forceinline__ void apply_map(const T (&A)[9], const T (&c)[3], T &M0, T &M1, T &M2) {
    const T t0 = A[2] * M2 + (A[1] * M1 + (A[0] * M0 + c[0]));  // three multiply-adds per row
    const T t1 = A[5] * M2 + (A[4] * M1 + (A[3] * M0 + c[1]));
    const T t2 = A[8] * M2 + (A[7] * M1 + (A[6] * M0 + c[2]));
    M0 = t0;
    M1 = t1;
    M2 = t2;
}

// float64 sample window: one column per thread, rows of FIELD_THREADS + 2 doubles (row r is
// sample r/2 of the chunk, real or imaginary part)
constexpr int F64_WIN_STRIDE = FIELD_THREADS + 2;
constexpr size_t F64_WIN_BYTES = (size_t)2 * FIELD_CHUNK * F64_WIN_STRIDE * sizeof(double);

// One spin per thread.  Samples: each thread writes its spin's value of each sample of the chunk to
// its own column of a shared window; after the chunk each row is summed over the columns by two
// threads (64 entries each, four partial sums) and added to the signal, so a sample costs a thread
// two stores instead of a ten-add warp butterfly on the float64 pipe.
__global__ void __launch_bounds__(FIELD_THREADS) fields_kernel_f64(FieldArgs a) {
    static_assert(FIELD_THREADS == 128, "two threads per window row");
    __shared__ FieldEv64 evs[FIELD_CHUNK];
    extern __shared__ __align__(16) double wind[];  // 2 * FIELD_CHUNK rows of F64_WIN_STRIDE
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < a.n_spins;
    const int64_t si = live ? s : 0;
    const int64_t np = a.n_pad;
    const double x = a.params[P_X * np + si], y = a.params[P_Y * np + si], z = a.params[P_Z * np + si];
    const double dw = TWO_PI * a.params[P_DF * np + si];
    const double m0 = live ? a.params[P_RHO * np + si] : 0.0;
    const double r1 = a.params[P_R1 * np + si], r2 = a.params[P_R2 * np + si];
    const double n0 = a.ndir ? a.ndir[3 * si] : 0.0, n1 = a.ndir ? a.ndir[3 * si + 1] : 0.0;
    const double n2 = a.ndir ? a.ndir[3 * si + 2] : 1.0;
    const double b0 = a.b0;
    double M0 = m0 * n0, M1 = m0 * n1, M2 = m0 * n2;
    double S0 = M0, S1 = M1, S2 = M2;  // state at the start of the current run
    double A[9] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0}, cv[3] = {0.0, 0.0, 0.0};  // cached map
    const FieldEv64 *src = static_cast<const FieldEv64 *>(a.ev);
    const int t = threadIdx.x, row = t / 2, part = t % 2;
    for (int64_t c0 = 0; c0 < a.n_events; c0 += FIELD_CHUNK) {
        __syncthreads();
        const int nc = (int)min((int64_t)FIELD_CHUNK, a.n_events - c0);
        {
            const int4 *s4 = reinterpret_cast<const int4 *>(src + c0);
            int4 *d4 = reinterpret_cast<int4 *>(evs);
            const int words = nc * (int)(sizeof(FieldEv64) / sizeof(int4));
            for (int i = t; i < words; i += FIELD_THREADS) d4[i] = s4[i];
        }
        __syncthreads();
        for (int i = 0; i < nc; ++i) {
            const FieldEv64 &e = evs[i];
            if ((e.flags & FF_TMAP) && s < np)
                apply_train_map(static_cast<const double *>(a.maps), (e.flags >> 16) & 0xff, np, s, M0, M1, M2);
            if (e.flags & FF_RF) {
                const double t0 = e.R[0] * M0 + e.R[1] * M1 + e.R[2] * M2;
                const double t1 = e.R[3] * M0 + e.R[4] * M1 + e.R[5] * M2;
                const double t2 = e.R[6] * M0 + e.R[7] * M1 + e.R[8] * M2;
                M0 = t0;
                M1 = t1;
                M2 = t2;
            }
            if (e.flags & FF_RUN_START) {
                S0 = M0;
                S1 = M1;
                S2 = M2;
            } else if (e.flags & FF_RUN) {
                M0 = S0;
                M1 = S1;
                M2 = S2;
            }
            if ((e.flags & FF_FREE) && (e.flags & FF_SAME)) {
                apply_map(A, cv, M0, M1, M2);
            } else if (e.flags & FF_FREE) {
                double bx = 0.0, by = 0.0;
                const double bz = e.g[0] * x + e.g[1] * y + e.g[2] * z;
                if (e.flags & FF_TRANSVERSE) {
                    bx = e.gt[0] * x + e.gt[1] * y + e.gt[2] * z;
                    by = e.gt[3] * x + e.gt[4] * y + e.gt[5] * z;
                }
                const double p = n0 * bx + n1 * by + n2 * bz;
                const double qx = bx - p * n0, qy = by - p * n1, qz = bz - p * n2;
                const double ux = b0 * n0 + bx, uy = b0 * n1 + by, uz = b0 * n2 + bz;
                const double un = sqrt(ux * ux + uy * uy + uz * uz);
                const double excess = p + (qx * qx + qy * qy + qz * qz) / (un + b0 + p);
                const double inv = 1.0 / un;
                const double hx = ux * inv, hy = uy * inv, hz = uz * inv;
                double sn, cs;
                sincos(e.gdt * excess + dw * e.dt, &sn, &cs);
                const double e1m = expm1(-e.dt * r1), e2 = exp(-e.dt * r2);
                double B[9], cb[3];
                turn_map(hx, hy, hz, cs, sn, e1m, e2, m0, B, cb);
                apply_map(B, cb, M0, M1, M2);
                if (!(e.flags & FF_RUN)) {  // an anchored step's map spans j intervals: not cached
#pragma unroll
                    for (int q = 0; q < 9; ++q) A[q] = B[q];
#pragma unroll
                    for (int q = 0; q < 3; ++q) cv[q] = cb[q];
                }
            }
            if (e.flags & FF_ADC) {  // a spin past the phantom's end has M = 0
                double *w = wind + (2 * e.slot) * F64_WIN_STRIDE + t;
                w[0] = M0 * e.dem[0] + M1 * e.dem[1];
                w[F64_WIN_STRIDE] = M1 * e.dem[0] - M0 * e.dem[1];
            }
        }
        __syncthreads();
        const int nslot = evs[0].nslot, adc0 = evs[0].adc;
        double v = 0.0;
        if (row < 2 * nslot) {
            const double *w = wind + row * F64_WIN_STRIDE + part;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int q = 0; q < FIELD_THREADS / 2; ++q) acc[q & 3] += w[2 * q];
            v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (part == 0 && row < 2 * nslot) atomicAdd(&a.signal[2 * (int64_t)adc0 + row], v);
    }
}

// One spin of the float32 kernel: its constants (set up in float64), its state and the map of the
// last interval it computed.  A spin past the end of the phantom has M0 = 0: its state stays zero
// (every map is linear with c = M0 (1 - E1) h = 0), so it needs no test.
struct FSpin32 {
    float wh[9], wl[9];  // n_j x_d as (hi, lo): j = z, x, y (the order of the moments k_j), d = x, y, z
    float dfh, dfl;      // Δf as (hi, lo)
    float x, y, z, n0, n1, n2, m0, r1, r2;
    float M0, M1, M2, S0, S1, S2;  // state, and the state at the start of the current run
    float A[9], cv[3];             // the map of the last computed interval

    __device__ __forceinline__ void setup(const FieldArgs &a, int64_t s) {
        const bool live = s < a.n_spins;
        const int64_t si = live ? s : 0;
        const int64_t np = a.n_pad;
        const double xd[3] = {a.params[P_X * np + si], a.params[P_Y * np + si], a.params[P_Z * np + si]};
        const double nd[3] = {a.ndir ? a.ndir[3 * si] : 0.0, a.ndir ? a.ndir[3 * si + 1] : 0.0,
                              a.ndir ? a.ndir[3 * si + 2] : 1.0};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            split(nd[2] * xd[d], wh[d], wl[d]);
            split(nd[0] * xd[d], wh[3 + d], wl[3 + d]);
            split(nd[1] * xd[d], wh[6 + d], wl[6 + d]);
        }
        split(a.params[P_DF * np + si], dfh, dfl);
        x = (float)xd[0];
        y = (float)xd[1];
        z = (float)xd[2];
        n0 = (float)nd[0];
        n1 = (float)nd[1];
        n2 = (float)nd[2];
        m0 = live ? (float)a.params[P_RHO * np + si] : 0.0f;
        r1 = (float)a.params[P_R1 * np + si];
        r2 = (float)a.params[P_R2 * np + si];
        M0 = S0 = m0 * n0;
        M1 = S1 = m0 * n1;
        M2 = S2 = m0 * n2;
#pragma unroll
        for (int q = 0; q < 9; ++q) A[q] = (q % 4 == 0) ? 1.0f : 0.0f;
        cv[0] = cv[1] = cv[2] = 0.0f;
    }

    __device__ __forceinline__ void rf(const float (&R)[9]) {
        const float t0 = R[2] * M2 + (R[1] * M1 + R[0] * M0);
        const float t1 = R[5] * M2 + (R[4] * M1 + R[3] * M0);
        const float t2 = R[8] * M2 + (R[7] * M1 + R[6] * M0);
        M0 = t0;
        M1 = t1;
        M2 = t2;
    }

    // the held map applied to (u0, u1, u2), written to (o0, o1, o2)
    __device__ __forceinline__ void map(float u0, float u1, float u2, float &o0, float &o1, float &o2) const {
        o0 = A[2] * u2 + (A[1] * u1 + (A[0] * u0 + cv[0]));
        o1 = A[5] * u2 + (A[4] * u1 + (A[3] * u0 + cv[1]));
        o2 = A[8] * u2 + (A[7] * u1 + (A[6] * u0 + cv[2]));
    }

    // An interval computed from its record: the field, its direction, the phase and the
    // exponentials; the map is applied and, unless the step is anchored (its record spans j
    // intervals of a run), kept for the events that repeat the interval.
    __device__ __forceinline__ void full(const FieldEv32 &e, float b0, int flags) {
        float bx = 0.0f, by = 0.0f;
        const float bz = e.g[0] * x + e.g[1] * y + e.g[2] * z;
        // phase in cycles: n_z (k_z . x) [+ n_x (k_x . x) + n_y (k_y . x)] + Δf Δt + remainder
        PhaseAcc acc;
#pragma unroll
        for (int q = 0; q < 3; ++q) acc.add_product(e.kh[q], e.kl[q], wh[q], wl[q]);
        acc.add_product(dfh, dfl, e.dth, e.dtl);
        if (flags & FF_TRANSVERSE) {
            bx = e.gt[0] * x + e.gt[1] * y + e.gt[2] * z;
            by = e.gt[3] * x + e.gt[4] * y + e.gt[5] * z;
#pragma unroll
            for (int q = 3; q < 9; ++q) acc.add_product(e.kh[q], e.kl[q], wh[q], wl[q]);
        }
        const float p = n0 * bx + n1 * by + n2 * bz;
        const float qx = bx - p * n0, qy = by - p * n1, qz = bz - p * n2;
        const float ux = b0 * n0 + bx, uy = b0 * n1 + by, uz = b0 * n2 + bz;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float inv = rsqrtf(uu);  // 1/|u|
        const float un = uu * inv;
        // the remainder r²/(|u| + B0 + n.b) is a second-order correction: a fast quotient suffices
        acc.c += e.gdt2pi * __fdividef(qx * qx + qy * qy + qz * qz, un + b0 + p);
        const float t = acc.value();
        float sn, cs;
        sincospif(2.0f * t, &sn, &cs);
        const float e1m = expm1f(-e.dt * r1), e2 = expf(-e.dt * r2);
        float B[9], cb[3];
        turn_map(ux * inv, uy * inv, uz * inv, cs, sn, e1m, e2, m0, B, cb);
        apply_map(B, cb, M0, M1, M2);
        if (!(flags & FF_RUN)) {
#pragma unroll
            for (int q = 0; q < 9; ++q) A[q] = B[q];
#pragma unroll
            for (int q = 0; q < 3; ++q) cv[q] = cb[q];
        }
    }
};

template <int K>
__device__ __forceinline__ void write_sample(float *win, int stride, int slot, float d0, float d1, const float (&u0)[K],
                                             const float (&u1)[K]) {
    float sr = u0[0] * d0 + u1[0] * d1, sim = u1[0] * d0 - u0[0] * d1;
#pragma unroll
    for (int k = 1; k < K; ++k) {
        sr = u1[k] * d1 + (u0[k] * d0 + sr);
        sim = u1[k] * d0 + (sim - u0[k] * d1);
    }
    float *w = win + (2 * slot) * stride;
    w[0] = sr;
    w[stride] = sim;
}

// K spins per thread, T threads per block: spin k of thread t in block b is (b·K + k)·T + t
// (coalesced per k).  The events of a chunk run as segments: a run of readout samples (the host
// marks its length) applies the held map in a loop unrolled by two, whose halves alternate between
// the state and a second set of registers; a run of sub-pulses turns and maps each spin with no
// copy; a run of events without effect (the events of a mapped train after its first) is passed
// over in one step; any other event (a mapped train's first applies its train map) takes the
// general path, its flags tested once for all K spins.  Samples:
// each thread writes the sum over its spins of each sample of the chunk to its own column of a
// shared window (no exchange between threads while the events run); after the chunk, each of the
// 2·nslot rows (a sample's real or imaginary part) is summed over the T columns (64 entries per
// thread, in four partial sums) and added to the signal in float64.  The rows are padded to
// T + T/64 floats so that the threads summing different rows at the same time read different banks.
template <int K, int T>
__global__ void __launch_bounds__(T, 512 / T) fields_kernel_f32(FieldArgs a) {
    static_assert(T == 64 || T == 128, "one or two threads per window row");
    constexpr int PER_ROW = T / 64, STRIDE = T + PER_ROW;
    __shared__ FieldEv32 evs[FIELD_CHUNK];
    __shared__ float win[2 * FIELD_CHUNK * STRIDE];
    const int t = threadIdx.x;
    FSpin32 sp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) sp[k].setup(a, ((int64_t)blockIdx.x * K + k) * T + t);
    const float b0 = (float)a.b0;
    const FieldEv32 *src = static_cast<const FieldEv32 *>(a.ev);
    const int row = t / PER_ROW, part = t % PER_ROW;
    float *wcol = win + t;
    for (int64_t c0 = 0; c0 < a.n_events; c0 += FIELD_CHUNK) {
        __syncthreads();
        const int nc = (int)min((int64_t)FIELD_CHUNK, a.n_events - c0);
        {
            const int4 *s4 = reinterpret_cast<const int4 *>(src + c0);
            int4 *d4 = reinterpret_cast<int4 *>(evs);
            const int words = nc * (int)(sizeof(FieldEv32) / sizeof(int4));
            for (int i = t; i < words; i += T) d4[i] = s4[i];
        }
        __syncthreads();
        int i = 0;
        while (i < nc) {
            const FieldEv32 &e = evs[i];
            const int flags = e.flags;
            const int kind = flags & KIND_MASK;
            if (flags == 0) {  // a run of events without effect (inside a mapped train, or empty)
                i += e.seg;
                continue;
            }
            if (kind == KIND_READ) {
                const int n = e.seg;
                int slot = e.slot;
                int j = 0;
                for (; j + 1 < n; j += 2, slot += 2) {
                    float u0[K], u1[K], u2[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) sp[k].map(sp[k].M0, sp[k].M1, sp[k].M2, u0[k], u1[k], u2[k]);
                    write_sample<K>(wcol, STRIDE, slot, evs[i + j].dem[0], evs[i + j].dem[1], u0, u1);
                    float m0[K], m1[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        sp[k].map(u0[k], u1[k], u2[k], sp[k].M0, sp[k].M1, sp[k].M2);
                        m0[k] = sp[k].M0;
                        m1[k] = sp[k].M1;
                    }
                    write_sample<K>(wcol, STRIDE, slot + 1, evs[i + j + 1].dem[0], evs[i + j + 1].dem[1], m0, m1);
                }
                if (j < n) {
                    float m0[K], m1[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float u0, u1, u2;
                        sp[k].map(sp[k].M0, sp[k].M1, sp[k].M2, u0, u1, u2);
                        sp[k].M0 = m0[k] = u0;
                        sp[k].M1 = m1[k] = u1;
                        sp[k].M2 = u2;
                    }
                    write_sample<K>(wcol, STRIDE, slot, evs[i + j].dem[0], evs[i + j].dem[1], m0, m1);
                }
                i += n;
            } else if (kind == KIND_TRAIN) {
                const int n = e.seg;
                for (int j = 0; j < n; ++j) {
                    const float4 ra = *reinterpret_cast<const float4 *>(&evs[i + j].R[0]);
                    const float4 rb = *reinterpret_cast<const float4 *>(&evs[i + j].R[4]);
                    const float r8 = evs[i + j].R[8];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float M0 = sp[k].M0, M1 = sp[k].M1, M2 = sp[k].M2;
                        const float u0 = ra.z * M2 + (ra.y * M1 + ra.x * M0);
                        const float u1 = rb.y * M2 + (rb.x * M1 + ra.w * M0);
                        const float u2 = r8 * M2 + (rb.w * M1 + rb.z * M0);
                        sp[k].map(u0, u1, u2, sp[k].M0, sp[k].M1, sp[k].M2);
                    }
                }
                i += n;
            } else {
                if (flags & FF_TMAP) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int64_t si = ((int64_t)blockIdx.x * K + k) * T + t;
                        if (si < a.n_pad)
                            apply_train_map(static_cast<const float *>(a.maps), (flags >> 16) & 0xff, a.n_pad, si,
                                            sp[k].M0, sp[k].M1, sp[k].M2);
                    }
                }
                if (flags & FF_RF) {
                    float R[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) R[q] = e.R[q];
#pragma unroll
                    for (int k = 0; k < K; ++k) sp[k].rf(R);
                }
                if (flags & FF_RUN_START) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        sp[k].S0 = sp[k].M0;
                        sp[k].S1 = sp[k].M1;
                        sp[k].S2 = sp[k].M2;
                    }
                } else if (flags & FF_RUN) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        sp[k].M0 = sp[k].S0;
                        sp[k].M1 = sp[k].S1;
                        sp[k].M2 = sp[k].S2;
                    }
                }
                if (flags & FF_SAME) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float u0, u1, u2;
                        sp[k].map(sp[k].M0, sp[k].M1, sp[k].M2, u0, u1, u2);
                        sp[k].M0 = u0;
                        sp[k].M1 = u1;
                        sp[k].M2 = u2;
                    }
                } else if (flags & FF_FREE) {
#pragma unroll
                    for (int k = 0; k < K; ++k) sp[k].full(e, b0, flags);
                }
                if (flags & FF_ADC) {
                    float m0[K], m1[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        m0[k] = sp[k].M0;
                        m1[k] = sp[k].M1;
                    }
                    write_sample<K>(wcol, STRIDE, e.slot, e.dem[0], e.dem[1], m0, m1);
                }
                i += 1;
            }
        }
        __syncthreads();
        const int nslot = evs[0].nslot, adc0 = evs[0].adc;
        float v = 0.0f;
        if (row < 2 * nslot) {
            const float *w = win + row * STRIDE + part;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < 64; ++q) acc[q & 3] += w[PER_ROW * q];
            v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        }
        if (PER_ROW == 2) v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (part == 0 && row < 2 * nslot) atomicAdd(&a.signal[2 * (int64_t)adc0 + row], (double)v);
    }
}

__device__ __forceinline__ double fdot3(double a, double b, double c, double d, double e, double f) {
    return a * b + c * d + e * f;
}
__device__ __forceinline__ dev::dfl fdot3(dev::dfl a, dev::dfl b, dev::dfl c, dev::dfl d, dev::dfl e, dev::dfl f) {
    return dev::vdot3(a, b, c, d, e, f);
}

// Train maps (set-up): thread (s, t) forms, in float64, spin s's turn for the free interval of map
// kind t (the same in every event of the train: the field, its direction, the phase, the
// exponentials, as the float64 kernel forms them), then steps the three unit states (the columns
// of A) and the zero state (c) through the train's events, pulse then turn, in C arithmetic
// (double-float, or float64 for the float64 kernel); the pulses are staged per block in shared
// memory.  Stored rounded to R.
template <typename C, typename R>
__global__ void __launch_bounds__(128) fields_map_kernel(FieldArgs a, const FieldEv64 *ev, FieldKinds k, R *maps) {
    __shared__ C rp[FIELD_TRAIN_MAX * 9];
    const int t = blockIdx.y;
    const int64_t i0 = k.first[t];
    const int n = k.len[t];
    for (int q = threadIdx.x; q < 9 * n; q += blockDim.x) rp[q] = C(ev[i0 + q / 9].R[q % 9]);
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_pad) return;
    const bool live = s < a.n_spins;
    const int64_t si = live ? s : 0;
    const int64_t np = a.n_pad;
    const double x = a.params[P_X * np + si], y = a.params[P_Y * np + si], z = a.params[P_Z * np + si];
    const double dw = TWO_PI * a.params[P_DF * np + si];
    const double m0 = live ? a.params[P_RHO * np + si] : 0.0;
    const double r1 = a.params[P_R1 * np + si], r2 = a.params[P_R2 * np + si];
    const double n0 = a.ndir ? a.ndir[3 * si] : 0.0, n1 = a.ndir ? a.ndir[3 * si + 1] : 0.0;
    const double n2 = a.ndir ? a.ndir[3 * si + 2] : 1.0;
    const FieldEv64 &e = ev[i0];
    const double bz = e.g[0] * x + e.g[1] * y + e.g[2] * z;
    const double bx = e.gt[0] * x + e.gt[1] * y + e.gt[2] * z;
    const double by = e.gt[3] * x + e.gt[4] * y + e.gt[5] * z;
    const double p = n0 * bx + n1 * by + n2 * bz;
    const double qx = bx - p * n0, qy = by - p * n1, qz = bz - p * n2;
    const double ux = a.b0 * n0 + bx, uy = a.b0 * n1 + by, uz = a.b0 * n2 + bz;
    const double un = sqrt(ux * ux + uy * uy + uz * uz);
    const double excess = p + (qx * qx + qy * qy + qz * qz) / (un + a.b0 + p);
    const double inv = 1.0 / un;
    double sn, cs;
    sincos(e.gdt * excess + dw * e.dt, &sn, &cs);
    double Ad[9], cd[3];
    turn_map(ux * inv, uy * inv, uz * inv, cs, sn, expm1(-e.dt * r1), exp(-e.dt * r2), m0, Ad, cd);
    C A[9], cc[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = C(Ad[q]);
#pragma unroll
    for (int q = 0; q < 3; ++q) cc[q] = C(cd[q]);
    C V[4][3] = {{C(1.0), C(0.0), C(0.0)}, {C(0.0), C(1.0), C(0.0)}, {C(0.0), C(0.0), C(1.0)}, {C(0.0), C(0.0), C(0.0)}};
    for (int i = 0; i < n; ++i) {
        const C *Rm = rp + 9 * i;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const C w0 = fdot3(Rm[0], V[v][0], Rm[1], V[v][1], Rm[2], V[v][2]);  // the pulse
            const C w1 = fdot3(Rm[3], V[v][0], Rm[4], V[v][1], Rm[5], V[v][2]);
            const C w2 = fdot3(Rm[6], V[v][0], Rm[7], V[v][1], Rm[8], V[v][2]);
            V[v][0] = fdot3(A[0], w0, A[1], w1, A[2], w2);  // the interval's turn
            V[v][1] = fdot3(A[3], w0, A[4], w1, A[5], w2);
            V[v][2] = fdot3(A[6], w0, A[7], w1, A[8], w2);
            if (v == 3) {
                V[v][0] = V[v][0] + cc[0];
                V[v][1] = V[v][1] + cc[1];
                V[v][2] = V[v][2] + cc[2];
            }
        }
    }
    R *m = maps + (int64_t)t * TRAIN_MAP_ROWS * np + s;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int v = 0; v < 3; ++v) m[(3 * j + v) * np] = R(double(V[v][j]));
        m[(9 + j) * np] = R(double(V[3][j]));
    }
}

// lowest index of a direction that is not a finite unit vector (|n| - 1 beyond 1e-9)
__global__ void check_dirs_kernel(int64_t n, const double *nd, int *bad) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const double a = nd[3 * s], b = nd[3 * s + 1], c = nd[3 * s + 2];
        const double l = a * a + b * b + c * c;
        if (!(isfinite(a) && isfinite(b) && isfinite(c)) || !(fabs(l - 1.0) <= 2e-9))
            atomicMin(bad, (int)min(s, (int64_t)0x7ffffffe));
    }
}

// Eq. 3.19: the hard pulse as the rotation by -α about (cos φ, sin φ, 0), written as
// R = cos α I + (1 - cos α) a aᵀ - sin α [a]x.
void rf_matrix(double alpha, double phi, double R[9]) {
    const double ca = std::cos(alpha), sa = std::sin(alpha), ax = std::cos(phi), ay = std::sin(phi);
    const double o = 1.0 - ca;
    R[0] = ca + o * ax * ax;
    R[1] = o * ax * ay;
    R[2] = -sa * ay;
    R[3] = o * ax * ay;
    R[4] = ca + o * ay * ay;
    R[5] = sa * ax;
    R[6] = sa * ay;
    R[7] = -sa * ax;
    R[8] = ca;
}

bool finite_event(const mrsim_event &e) {
    for (double v : {e.dt, e.gx, e.gy, e.gz, e.rf_flip, e.rf_phase, e.adc_phase})
        if (!std::isfinite(v)) return false;
    return e.dt >= 0.0 && (e.adc == 0 || e.adc == 1) && e.reserved == 0;
}

mrsim_status ffail(mrsim_ctx *ctx, mrsim_status st, const std::string &m) {
    if (ctx) ctx->err = m;
    log_failure(st, m);
    return st;
}

bool on_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct mrsim_fields {
    mrsim_ctx *ctx = nullptr;
    int64_t n_events = 0, n_adc = 0;
    double b0 = 0.0;
    FieldKinds kinds{};  // train-map kinds (none when the context's train maps were off at creation)
    unsigned char *d_rec = nullptr;  // [float64 records | float32 records]
    size_t off32 = 0;
};

extern "C" {

mrsim_status mrsim_phantom_set_b0_direction(mrsim_phantom *ph, const double *b0_dir, void *stream) {
    if (!ph) return MRSIM_EINVAL;
    mrsim_ctx *ctx = ph->ctx;
    if (ph->n > 0 && !b0_dir) return ffail(ctx, MRSIM_EINVAL, "b0_dir is NULL");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 24 * (size_t)ph->n;
    double *d = nullptr;
    if (bytes) {
        cudaError_t e = ctx_malloc(ctx, &d, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ffail(ctx, MRSIM_ENOMEM, "field directions: " + std::to_string(bytes) + " bytes");
        }
        e = cudaMemcpyAsync(d, b0_dir, bytes, on_device(b0_dir) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bad, 0x7f, sizeof(int), st);
        if (e == cudaSuccess) {
            check_dirs_kernel<<<(int)std::min<int64_t>((ph->n + 255) / 256, 4096), 256, 0, st>>>(ph->n, d, ctx->d_bad);
            e = cudaGetLastError();
        }
        int bad = 0x7f7f7f7f;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || bad != 0x7f7f7f7f) {
            cudaFree(d);
            if (e != cudaSuccess) return ffail(ctx, MRSIM_ECUDA, std::string("field directions: ") + cudaGetErrorString(e));
            return ffail(ctx, MRSIM_EINVAL, "b0_dir of spin " + std::to_string(bad) + " is not a finite unit vector");
        }
    }
    cudaFree(ph->d_dir);
    ph->d_dir = d;
    return MRSIM_OK;
}

mrsim_status mrsim_fields_create(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events,
                                 const double *g_transverse, double gamma_hz_per_t, double b0_tesla,
                                 mrsim_fields **out) {
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (n_events < 0 || (n_events > 0 && !events)) return ffail(ctx, MRSIM_EINVAL, "invalid event list");
    if (n_events > 0 && on_device(events)) return ffail(ctx, MRSIM_EINVAL, "events must be in host memory");
    if (g_transverse && on_device(g_transverse)) return ffail(ctx, MRSIM_EINVAL, "g_transverse must be in host memory");
    if (!(gamma_hz_per_t > 0.0) || !std::isfinite(gamma_hz_per_t)) return ffail(ctx, MRSIM_EINVAL, "gamma must be > 0");
    if (!(b0_tesla > 0.0) || !std::isfinite(b0_tesla)) return ffail(ctx, MRSIM_EINVAL, "b0_tesla must be > 0");
    for (int64_t i = 0; i < n_events; ++i) {
        if (!finite_event(events[i])) return ffail(ctx, MRSIM_EINVAL, "invalid event " + std::to_string(i));
        if (g_transverse)
            for (int q = 0; q < 6; ++q)
                if (!std::isfinite(g_transverse[6 * i + q]))
                    return ffail(ctx, MRSIM_EINVAL, "non-finite transverse gradient at event " + std::to_string(i));
    }
    const double gamma = TWO_PI * gamma_hz_per_t;
    std::vector<FieldEv64> e64;
    std::vector<FieldEv32> e32;
    try {
        e64.resize((size_t)n_events);
        e32.resize((size_t)n_events);
    } catch (const std::bad_alloc &) {
        return ffail(ctx, MRSIM_ENOMEM, "host allocation failed");
    }
    static const double zero6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    auto same_interval = [&](int64_t i, int64_t k) {  // equal Δt, G and transverse components
        const mrsim_event &u = events[i], &v = events[k];
        const double *gi = g_transverse ? g_transverse + 6 * i : zero6, *gk = g_transverse ? g_transverse + 6 * k : zero6;
        bool same = u.dt == v.dt && u.gx == v.gx && u.gy == v.gy && u.gz == v.gz;
        for (int q = 0; q < 6 && same; ++q) same = gi[q] == gk[q];
        return same;
    };
    // run[i]: position of event i in its run of identical free intervals without pulses (1 = the
    // first, 0 = none); len[i]: the length of that run
    std::vector<int64_t> run, len;
    try {
        run.assign((size_t)n_events, 0);
        len.assign((size_t)n_events, 0);
    } catch (const std::bad_alloc &) {
        return ffail(ctx, MRSIM_ENOMEM, "host allocation failed");
    }
    for (int64_t i = 0; i < n_events; ++i) {
        const mrsim_event &v = events[i];
        if (v.rf_flip == 0.0 && v.dt > 0.0) run[i] = (i > 0 && run[i - 1] > 0 && same_interval(i - 1, i)) ? run[i - 1] + 1 : 1;
    }
    for (int64_t i = n_events - 1; i >= 0; --i)
        if (run[i] > 0) len[i] = (i + 1 < n_events && run[i + 1] == run[i] + 1) ? len[i + 1] : run[i];
    // Train maps: trains (>= 2 consecutive pulsed events without samples sharing one free interval,
    // at most FIELD_TRAIN_MAX) keyed by their interval and pulses; a key that occurs
    // TRAIN_MAP_MIN times or more becomes a map kind (in order of first occurrence, at most
    // TRAIN_MAP_MAX).  tkind[i]: the kind of the mapped train that starts at event i (-1: none);
    // inside[i]: event i belongs to a mapped train and is not its first.
    std::vector<int32_t> tkind;
    std::vector<char> inside;
    FieldKinds kinds{};
    try {
        tkind.assign((size_t)n_events, -1);
        inside.assign((size_t)n_events, 0);
        if (ctx->train_maps) {
            auto pulsed = [&](int64_t k) { return events[k].rf_flip != 0.0 && events[k].dt > 0.0 && !events[k].adc; };
            auto bits = [](double d) {
                uint64_t u;
                std::memcpy(&u, &d, 8);
                return u;
            };
            std::map<std::vector<uint64_t>, std::vector<int64_t>> starts;
            std::vector<std::pair<int64_t, const std::vector<uint64_t> *>> order;
            std::vector<int64_t> lens((size_t)n_events, 0);
            for (int64_t i = 0; i < n_events;) {
                if (!pulsed(i)) {
                    ++i;
                    continue;
                }
                int64_t k = i + 1;
                while (k < n_events && k - i < FIELD_TRAIN_MAX && pulsed(k) && same_interval(i, k)) ++k;
                if (k - i >= 2) {
                    const mrsim_event &v = events[i];
                    const double *gt = g_transverse ? g_transverse + 6 * i : zero6;
                    std::vector<uint64_t> key = {bits(v.dt), bits(v.gx), bits(v.gy), bits(v.gz)};
                    for (int q = 0; q < 6; ++q) key.push_back(bits(gt[q]));
                    for (int64_t q = i; q < k; ++q) {
                        key.push_back(bits(events[q].rf_flip));
                        key.push_back(bits(events[q].rf_phase));
                    }
                    auto it = starts.emplace(std::move(key), std::vector<int64_t>()).first;
                    if (it->second.empty()) order.emplace_back(i, &it->first);
                    it->second.push_back(i);
                    lens[(size_t)i] = k - i;
                }
                i = k;
            }
            for (const auto &o : order) {
                if (kinds.n == TRAIN_MAP_MAX) break;
                const std::vector<int64_t> &st = starts[*o.second];
                if ((int)st.size() < TRAIN_MAP_MIN) continue;
                const int t = kinds.n++;
                kinds.first[t] = st[0];
                kinds.len[t] = (int32_t)lens[(size_t)st[0]];
                for (int64_t i0 : st) {
                    tkind[(size_t)i0] = t;
                    for (int64_t q = i0 + 1; q < i0 + kinds.len[t]; ++q) inside[(size_t)q] = 1;
                }
            }
        }
    } catch (const std::bad_alloc &) {
        return ffail(ctx, MRSIM_ENOMEM, "host allocation failed");
    }
    int64_t j = 0, cached = -1;  // cached: the event whose one-interval map the spins hold
    int slot = 0;
    for (int64_t i = 0; i < n_events; ++i) {
        if (i % FIELD_CHUNK == 0) slot = 0;
        const mrsim_event &v = events[i];
        const double *gt = g_transverse ? g_transverse + 6 * i : nullptr;
        const bool tr = gt && (gt[0] != 0.0 || gt[1] != 0.0 || gt[2] != 0.0 || gt[3] != 0.0 || gt[4] != 0.0 || gt[5] != 0.0);
        const bool free = v.dt > 0.0;
        const int64_t pos = run[(size_t)i];
        const bool anchor = pos > 1 && (pos % FIELD_ANCHOR == 0 || pos == len[(size_t)i]);
        const bool mapped = tkind[(size_t)i] >= 0 || inside[(size_t)i];  // a mapped train leaves the held map alone
        const bool same = !mapped && free && !anchor && cached >= 0 && same_interval(cached, i);
        if (!mapped && free && !anchor && !same) cached = i;
        const double span = anchor ? v.dt * (double)pos : v.dt;  // an anchored step: the run's interval so far
        int32_t flags = (v.rf_flip != 0.0 ? FF_RF : 0) | (tr ? FF_TRANSVERSE : 0) | (v.adc ? FF_ADC : 0) |
                        (free ? FF_FREE : 0) | (pos == 1 ? FF_RUN_START : 0) | (anchor ? FF_RUN : 0) |
                        (same ? FF_SAME : 0);
        if (tkind[(size_t)i] >= 0) flags = FF_TMAP | (tkind[(size_t)i] << 16);
        else if (inside[(size_t)i]) flags = 0;
        double R[9];
        rf_matrix(v.rf_flip, v.rf_phase, R);
        const double g[3] = {v.gx, v.gy, v.gz};
        const double dem[2] = {std::cos(v.adc_phase), std::sin(v.adc_phase)};
        const int32_t adc = (int32_t)j, sl = v.adc ? slot : 0;
        FieldEv64 &r = e64[(size_t)i];
        FieldEv32 &f = e32[(size_t)i];
        for (int q = 0; q < 9; ++q) {
            r.R[q] = R[q];
            f.R[q] = (float)R[q];
        }
        for (int q = 0; q < 3; ++q) {
            r.g[q] = g[q];
            f.g[q] = (float)g[q];
        }
        for (int q = 0; q < 6; ++q) {
            r.gt[q] = tr ? gt[q] : 0.0;
            f.gt[q] = (float)r.gt[q];
        }
        for (int d = 0; d < 3; ++d) {
            split(gamma_hz_per_t * g[d] * span, f.kh[d], f.kl[d]);
            split(gamma_hz_per_t * r.gt[d] * span, f.kh[3 + d], f.kl[3 + d]);
            split(gamma_hz_per_t * r.gt[3 + d] * span, f.kh[6 + d], f.kl[6 + d]);
        }
        r.gdt = gamma * span;
        r.dt = span;
        split(span, f.dth, f.dtl);
        f.gdt2pi = (float)(gamma_hz_per_t * span);
        f.dt = (float)span;
        r.dem[0] = dem[0];
        r.dem[1] = dem[1];
        f.dem[0] = (float)dem[0];
        f.dem[1] = (float)dem[1];
        r.flags = f.flags = flags;
        f.seg = 1;
        f.pad = 0;
        r.adc = f.adc = adc;
        r.slot = f.slot = sl;
        if (v.adc) {
            ++j;
            ++slot;
        }
        if ((i + 1) % FIELD_CHUNK == 0 || i + 1 == n_events)  // the chunk is complete: its sample count
            for (int64_t k = i / FIELD_CHUNK * FIELD_CHUNK; k <= i; ++k) e64[(size_t)k].nslot = e32[(size_t)k].nslot = slot;
        // segment lengths, once the chunk is complete: events of kind READ or TRAIN followed by
        // events of the same kind within the chunk
        if ((i + 1) % FIELD_CHUNK == 0 || i + 1 == n_events) {
            const int64_t k0 = i / FIELD_CHUNK * FIELD_CHUNK;
            for (int64_t k = i; k >= k0; --k) {
                FieldEv32 &f = e32[(size_t)k];
                const int32_t kind = f.flags & KIND_MASK;
                f.seg = 1;
                if ((kind == KIND_READ || kind == KIND_TRAIN) && k < i && (e32[(size_t)k + 1].flags & KIND_MASK) == kind)
                    f.seg = e32[(size_t)k + 1].seg + 1;
                if (f.flags == 0 && k < i && e32[(size_t)k + 1].flags == 0) f.seg = e32[(size_t)k + 1].seg + 1;
            }
        }
    }
    cudaSetDevice(ctx->device);
    mrsim_fields *fh = new (std::nothrow) mrsim_fields();
    if (!fh) return ffail(ctx, MRSIM_ENOMEM, "host allocation failed");
    fh->ctx = ctx;
    fh->n_events = n_events;
    fh->n_adc = j;
    fh->b0 = b0_tesla;
    fh->kinds = kinds;
    const size_t b64 = (size_t)n_events * sizeof(FieldEv64), b32 = (size_t)n_events * sizeof(FieldEv32);
    fh->off32 = (b64 + 255) / 256 * 256;
    if (n_events > 0) {
        cudaError_t e = ctx_malloc(ctx, &fh->d_rec, fh->off32 + b32);
        if (e == cudaSuccess) e = cudaMemcpy(fh->d_rec, e64.data(), b64, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(fh->d_rec + fh->off32, e32.data(), b32, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(fh->d_rec);
            delete fh;
            return ffail(ctx, e == cudaErrorMemoryAllocation ? MRSIM_ENOMEM : MRSIM_ECUDA,
                         std::string("field records: ") + cudaGetErrorString(e));
        }
    }
    *out = fh;
    return MRSIM_OK;
}

int64_t mrsim_fields_num_adc(const mrsim_fields *f) { return f ? f->n_adc : -1; }

int32_t mrsim_fields_num_train_maps(const mrsim_fields *f) { return f ? f->kinds.n : -1; }

void mrsim_fields_destroy(mrsim_fields *f) {
    if (!f) return;
    cudaSetDevice(f->ctx->device);
    cudaFree(f->d_rec);
    delete f;
}

mrsim_status mrsim_simulate_fields(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_fields *f,
                                   mrsim_precision prec, void *stream, double *signal_out, int64_t n_adc) {
    if (!ctx) return MRSIM_EINVAL;
    if (!ph || !f || ph->ctx != ctx || f->ctx != ctx) return ffail(ctx, MRSIM_EINVAL, "NULL handle or another context");
    if (!normalize_precision(prec, true)) return ffail(ctx, MRSIM_EINVAL, "unknown precision");
    if (n_adc != f->n_adc) return ffail(ctx, MRSIM_EINVAL, "n_adc does not match the sample events");
    if (n_adc > 0 && !signal_out) return ffail(ctx, MRSIM_EINVAL, "signal_out is NULL");
    const bool f64 = prec == MRSIM_FP64;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t sig_bytes = 16 * (size_t)n_adc;
    const bool host_sig = n_adc > 0 && !on_device(signal_out);
    double *sig = signal_out;
    if (host_sig) {  // the context's signal scratch
        if (sig_bytes > ctx->sig_cap * sizeof(double)) {
            cudaFree(ctx->d_sig);
            ctx->d_sig = nullptr;
            ctx->sig_cap = 0;
            cudaError_t e = ctx_malloc(ctx, &ctx->d_sig, sig_bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return ffail(ctx, MRSIM_ENOMEM, "signal scratch");
            }
            ctx->sig_cap = 2 * (size_t)n_adc;
        }
        sig = ctx->d_sig;
    }
    cudaError_t e = cudaSuccess;
    void *maps = nullptr;
    if (n_adc > 0) e = cudaMemsetAsync(sig, 0, sig_bytes, st);
    if (e == cudaSuccess && ph->n > 0 && f->n_events > 0) {
        FieldArgs a{};
        a.ev = f64 ? (const void *)f->d_rec : (const void *)(f->d_rec + f->off32);
        a.n_events = f->n_events;
        a.params = ph->params;
        a.n_spins = ph->n;
        a.n_pad = ph->n_pad;
        a.ndir = ph->d_dir;
        a.b0 = f->b0;
        a.signal = sig;
        if (f->kinds.n > 0) {  // the train maps of this phantom, from the context's pool
            const size_t mb = (size_t)f->kinds.n * TRAIN_MAP_ROWS * (size_t)ph->n_pad * (f64 ? sizeof(double) : sizeof(float));
            e = ctx_malloc_maps(ctx, &maps, mb, st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return ffail(ctx, MRSIM_ENOMEM, "fields train maps");
            }
            const dim3 mg((unsigned)((ph->n_pad + 127) / 128), (unsigned)f->kinds.n);
            const FieldEv64 *ev64 = reinterpret_cast<const FieldEv64 *>(f->d_rec);
            if (f64)
                fields_map_kernel<double, double><<<mg, 128, 0, st>>>(a, ev64, f->kinds, static_cast<double *>(maps));
            else
                fields_map_kernel<dev::dfl, float><<<mg, 128, 0, st>>>(a, ev64, f->kinds, static_cast<float *>(maps));
            a.maps = maps;
        }
        if (f64) {
            const unsigned grid = (unsigned)((ph->n + FIELD_THREADS - 1) / FIELD_THREADS);
            cudaFuncSetAttribute(fields_kernel_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F64_WIN_BYTES);
            fields_kernel_f64<<<grid, FIELD_THREADS, F64_WIN_BYTES, st>>>(a);
        } else {
            // 64 or 128 threads per block, whichever fills the last wave of resident blocks better
            const int64_t blocks128 = (ph->n + FIELD_K32 * 128 - 1) / (FIELD_K32 * 128);
            const int64_t blocks64 = (ph->n + FIELD_K32 * 64 - 1) / (FIELD_K32 * 64);
            int r128 = 0, r64 = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r128, fields_kernel_f32<FIELD_K32, 128>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r64, fields_kernel_f32<FIELD_K32, 64>, 64, 0);
            auto waves = [&](int64_t blocks, int per_sm) {  // time in units of one full wave of 64-thread work
                const int64_t cap = std::max<int64_t>(1, (int64_t)per_sm * ctx->num_sms);
                return (double)((blocks + cap - 1) / cap);
            };
            // a wave of 128-thread blocks holds r128 blocks per SM, each twice the spins of a 64-thread block
            const double w128 = waves(blocks128, r128) * 2.0 * r128, w64 = waves(blocks64, r64) * r64;
            if (r64 > 0 && (r128 <= 0 || w64 < w128))
                fields_kernel_f32<FIELD_K32, 64><<<(unsigned)blocks64, 64, 0, st>>>(a);
            else
                fields_kernel_f32<FIELD_K32, 128><<<(unsigned)blocks128, 128, 0, st>>>(a);
        }
        e = cudaGetLastError();
        if (maps) cudaFreeAsync(maps, st);
    }
    if (e == cudaSuccess && host_sig) {
        e = cudaMemcpyAsync(signal_out, sig, sig_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return ffail(ctx, MRSIM_ECUDA, std::string("fields simulation: ") + cudaGetErrorString(e));
    return MRSIM_OK;
}

}  // extern "C"
