// kt_kernel.cu -- K-t formalism (§4.2): configuration populations of many spin ensembles.
//
// An ensemble (a voxel's isochromats, or one entry of a (T1, T2, B1, Δf) dictionary) is the set
// of populations a_i (transverse configurations E_i, i = -K..K) and b_i (longitudinal Z_i) of
// §4.2.1, M0 = 1, starting at b_0 = 1.  Per elementary sequence (Eq. 4.1): the hard pulse mixes
// (a_i, a*_-i, b_i) with T'_HF of Eq. 4.2 for every order (Eq. 4.14); over the interval the
// gradient moves every transverse order by q (Eq. 4.17; orders beyond ±K are dropped),
// relaxation scales the populations (Eq. 4.15) and refills b_0 (Eq. 4.16), and the ensemble's
// off-resonance turns the transverse populations; a sampled step records a_0·exp(-j adc_phase).
// b_-i = conj(b_i), so M_z = Z_0 stays real.
//
// GPU layout: one warp per ensemble.  Lane l holds the orders i = l + 32·m (m < M) as a_i,
// a_-i and b_i: the pulse is lane-local (order i couples with -i only); a one-order shift moves
// a_i one lane up (and a_-i one lane down), with the wrap between slots m and the exchange
// a_0 <-> a_∓1 done by shuffles.  Every lane computes the step's scalars (sin/cos of the scaled
// flip, E1, E2, off-resonance phasor) for one step of every 32 and the warp broadcasts them; no
// warp waits on another.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace mrsim {
namespace {

constexpr unsigned FULLW = 0xffffffffu;

template <typename R>
struct Cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) {
    return {a.re + b.re, a.im + b.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> cconj(Cx<R> a) {
    return {a.re, -a.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> shfl(Cx<R> v, int src) {
    return {__shfl_sync(FULLW, v.re, src), __shfl_sync(FULLW, v.im, src)};
}
template <typename R>
__device__ __forceinline__ Cx<R> shfl_up1(Cx<R> v) {
    return {__shfl_up_sync(FULLW, v.re, 1), __shfl_up_sync(FULLW, v.im, 1)};
}
template <typename R>
__device__ __forceinline__ Cx<R> shfl_down1(Cx<R> v) {
    return {__shfl_down_sync(FULLW, v.re, 1), __shfl_down_sync(FULLW, v.im, 1)};
}

__device__ __forceinline__ void sc(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void scpi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void scpi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float em1(float x) { return expm1f(x); }
__device__ __forceinline__ double em1(double x) { return expm1(x); }
__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }

template <typename R, int M>
struct Ensemble {
    Cx<R> ap[M], an[M], bz[M];  // a_i, a_-i, b_i for i = lane + 32 m
    int lane, K;

    __device__ __forceinline__ bool has(int m) const { return lane + 32 * m <= K; }

    // Eq. 4.14 with T'_HF of Eq. 4.2: c2 = cos²(α/2), ca = cos α, t01 = sin²(α/2) e^{2jφ},
    // t02 = sin α e^{j(φ+π/2)}, t20 = (sin α / 2) e^{-j(φ-π/2)}; the other entries are conjugates
    __device__ __forceinline__ void pulse(R c2, R ca, Cx<R> t01, Cx<R> t02, Cx<R> t20) {
        const Cx<R> t10 = cconj(t01), t12 = cconj(t02), t21 = cconj(t20);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const Cx<R> x = ap[m], y = cconj(an[m]), z = bz[m];
            const Cx<R> nx = cadd(cadd(Cx<R>{c2 * x.re, c2 * x.im}, cmul(t01, y)), cmul(t02, z));
            const Cx<R> ny = cadd(cadd(cmul(t10, x), Cx<R>{c2 * y.re, c2 * y.im}), cmul(t12, z));
            const Cx<R> nz = cadd(cadd(cmul(t20, x), cmul(t21, y)), Cx<R>{ca * z.re, ca * z.im});
            ap[m] = nx;
            an[m] = cconj(ny);
            bz[m] = nz;
        }
        if (lane == 0) an[0] = ap[0];  // order 0: a_-0 is a_0
    }

    // Eq. 4.17 with q = +1: a_i <- a_{i-1} (i >= 1), a_0 <- a_-1, a_-i <- a_-(i+1)
    __device__ __forceinline__ void shift_up() {
        const Cx<R> a_m1 = shfl(an[0], 1);  // a_-1 from lane 1
        Cx<R> nap[M], nan[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            Cx<R> up = shfl_up1(ap[m]);                               // a_{i-1} within the slot
            const Cx<R> wrap = shfl(m > 0 ? ap[m - 1] : ap[0], 31);   // a_{32m-1} from lane 31
            if (lane == 0) up = m > 0 ? wrap : a_m1;
            nap[m] = has(m) ? up : Cx<R>{0, 0};                       // orders beyond K are dropped
            Cx<R> dn = shfl_down1(an[m]);                             // a_-(i+1) within the slot
            const Cx<R> wrap2 = shfl(m + 1 < M ? an[m + 1] : an[0], 0);
            if (lane == 31) dn = m + 1 < M ? wrap2 : Cx<R>{0, 0};
            nan[m] = has(m) ? dn : Cx<R>{0, 0};
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            ap[m] = nap[m];
            an[m] = nan[m];
        }
        if (lane == 0) an[0] = ap[0];
    }

    // Eq. 4.17 with q = -1: a_i <- a_{i+1} (i >= 0), a_-1 <- a_0, a_-i <- a_-(i-1)
    __device__ __forceinline__ void shift_down() {
        const Cx<R> a_0 = shfl(ap[0], 0);
        Cx<R> nap[M], nan[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            Cx<R> dn = shfl_down1(ap[m]);
            const Cx<R> wrap = shfl(m + 1 < M ? ap[m + 1] : ap[0], 0);
            if (lane == 31) dn = m + 1 < M ? wrap : Cx<R>{0, 0};
            nap[m] = has(m) ? dn : Cx<R>{0, 0};
            Cx<R> up = shfl_up1(an[m]);
            const Cx<R> wrap2 = shfl(m > 0 ? an[m - 1] : an[0], 31);
            if (lane == 0) up = m > 0 ? wrap2 : an[0];
            if (lane == 1 && m == 0) up = a_0;
            nan[m] = has(m) ? up : Cx<R>{0, 0};
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            ap[m] = nap[m];
            an[m] = nan[m];
        }
        if (lane == 0) an[0] = ap[0];
    }

    // Eqs. 4.15, 4.16 and the ensemble's precession: a *= E2·exp(-jθ), b *= E1, b_0 += 1 - E1
    __device__ __forceinline__ void relax(R e1m1, Cx<R> w) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            ap[m] = cmul(ap[m], w);
            an[m] = cmul(an[m], w);
            bz[m] = {bz[m].re + e1m1 * bz[m].re, bz[m].im + e1m1 * bz[m].im};
        }
        if (lane == 0) bz[0].re -= e1m1;  // b_0 + (E1 - 1)(b_0 - 1)
    }
};

// The per-step scalars of one ensemble: pulse entries, relaxation, demodulation, flags.  Lane l
// of a warp computes them for step base + l of a 32-step chunk; the warp then walks the chunk
// and broadcasts each step's values with shuffles (the transcendentals are spread over the lanes).
template <typename R>
struct StepScalars {
    R c2, ca, t01r, t01i, t02r, t02i, t20r, t20i;  // pulse (Eq. 4.2)
    R e1m1, wr, wi;                                // E1 - 1; E2·exp(-j2πΔfτ)
    R cadc, sadc;                                  // demodulation
    int flags;                                     // shift + 128 (8 bits) | sample << 8 | pulse << 9
};

template <typename R, typename StepT>
__device__ __forceinline__ StepScalars<R> step_scalars(const StepT &s, R b1, R r1, R r2, R df) {
    StepScalars<R> o;
    const R alpha = b1 * (R)s.alpha;
    R sh, ch;
    sc((R)0.5 * alpha, &sh, &ch);
    const R cp = (R)s.cphi, sp = (R)s.sphi, s2 = sh * sh, sa = (R)2 * sh * ch, hs = sh * ch;
    o.c2 = ch * ch;
    o.ca = o.c2 - s2;
    o.t01r = s2 * (R)s.c2phi;
    o.t01i = s2 * (R)s.s2phi;
    o.t02r = -sa * sp;  // j sin α e^{jφ}
    o.t02i = sa * cp;
    o.t20r = hs * sp;  // j (sin α / 2) e^{-jφ}
    o.t20i = hs * cp;
    const R tau = (R)s.tau;
    o.e1m1 = em1(-tau * r1);
    const R e2 = ex(-tau * r2);
    R sn, cs;
    scpi((R)2 * df * tau, &sn, &cs);
    o.wr = e2 * cs;
    o.wi = -e2 * sn;
    o.cadc = (R)s.cadc;
    o.sadc = (R)s.sadc;
    o.flags = (s.shift + 128) | (s.sample << 8) | ((s.alpha != 0) << 9);
    return o;
}

template <typename R, int M, typename StepT>
__global__ void __launch_bounds__(128) kt_kernel(const KtArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t set = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (set >= a.n_sets) return;  // uniform over the warp
    const StepT *steps = reinterpret_cast<const StepT *>(a.steps);
    const double t1 = a.t1[set], t2 = a.t2[set];
    const R r1 = isinf(t1) ? (R)0 : (R)(1.0 / t1), r2 = isinf(t2) ? (R)0 : (R)(1.0 / t2);
    const R b1 = a.b1 ? (R)a.b1[set] : (R)1;
    const R df = a.df ? (R)a.df[set] : (R)0;
    Ensemble<R, M> e;
    e.lane = lane;
    e.K = a.max_order;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        e.ap[m] = {0, 0};
        e.an[m] = {0, 0};
        e.bz[m] = {0, 0};
    }
    if (lane == 0) e.bz[0].re = (R)1;
    double *out = a.signal + 2 * set * a.n_samples;
    int64_t j = 0;  // samples written before this chunk
    for (int64_t base = 0; base < a.n_steps; base += 32) {
        const int cnt = (int)min((int64_t)32, a.n_steps - base);
        StepScalars<R> my{};
        if (lane < cnt) my = step_scalars<R>(steps[base + lane], b1, r1, r2, df);
        // lane k keeps the sample of step base + k and stores it after the chunk (one conversion
        // to float64 per lane instead of one per sample for the whole warp)
        const unsigned smask = __ballot_sync(FULLW, lane < cnt && (my.flags & 256));
        Cx<R> mine{0, 0};
        for (int k = 0; k < cnt; ++k) {
            const int fl = __shfl_sync(FULLW, my.flags, k);
            if (fl & 512)
                e.pulse(__shfl_sync(FULLW, my.c2, k), __shfl_sync(FULLW, my.ca, k),
                        Cx<R>{__shfl_sync(FULLW, my.t01r, k), __shfl_sync(FULLW, my.t01i, k)},
                        Cx<R>{__shfl_sync(FULLW, my.t02r, k), __shfl_sync(FULLW, my.t02i, k)},
                        Cx<R>{__shfl_sync(FULLW, my.t20r, k), __shfl_sync(FULLW, my.t20i, k)});
            const int q = (fl & 255) - 128;
            for (int i = 0; i < q; ++i) e.shift_up();
            for (int i = 0; i > q; --i) e.shift_down();
            e.relax(__shfl_sync(FULLW, my.e1m1, k), Cx<R>{__shfl_sync(FULLW, my.wr, k), __shfl_sync(FULLW, my.wi, k)});
            if (fl & 256) {
                const Cx<R> a0 = shfl(e.ap[0], 0);
                if (lane == k) mine = a0;
            }
        }
        if (smask & (1u << lane)) {  // demodulated with this lane's own step
            const Cx<R> v = cmul(mine, Cx<R>{my.cadc, -my.sadc});
            const int64_t jj = j + __popc(smask & ((1u << lane) - 1u));
            out[2 * jj] = (double)v.re;
            out[2 * jj + 1] = (double)v.im;
        }
        j += __popc(smask);
    }
}

template <typename R, typename StepT>
int launch_kt_t(const KtArgs &a, void *stream) {
    const int threads = 128;
    const int64_t blocks = (a.n_sets + 3) / 4;
    if (blocks <= 0) return 0;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    const int M = (a.max_order + 32) / 32;  // slots per lane
    cudaStream_t st = (cudaStream_t)stream;
    if (M <= 1)
        kt_kernel<R, 1, StepT><<<(unsigned)blocks, threads, 0, st>>>(a);
    else if (M <= 2)
        kt_kernel<R, 2, StepT><<<(unsigned)blocks, threads, 0, st>>>(a);
    else if (M <= 4)
        kt_kernel<R, 4, StepT><<<(unsigned)blocks, threads, 0, st>>>(a);
    else if (M <= 8)
        kt_kernel<R, 8, StepT><<<(unsigned)blocks, threads, 0, st>>>(a);
    else
        return (int)cudaErrorInvalidValue;
    return (int)cudaGetLastError();
}

__global__ void kt_check_kernel(int64_t n, const double *t1, const double *t2, const double *b1, const double *df,
                                int *bad) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = t1[s] > 0.0 && t2[s] > 0.0 && !isnan(t1[s]) && !isnan(t2[s]) && (!b1 || isfinite(b1[s])) &&
                        (!df || isfinite(df[s]));
        if (!ok) atomicMin(bad, (int)min(s, (int64_t)0x7ffffffe));
    }
}

}  // namespace

int check_kt_params(int64_t n, const double *t1, const double *t2, const double *b1, const double *df, int *bad,
                    void *stream) {
    if (n <= 0) return 0;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    kt_check_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, t1, t2, b1, df, bad);
    return (int)cudaGetLastError();
}

int launch_kt(const KtArgs &a, bool fp64, void *stream) {
    return fp64 ? launch_kt_t<double, KtStepDev>(a, stream) : launch_kt_t<float, KtStepF>(a, stream);
}

}  // namespace mrsim
