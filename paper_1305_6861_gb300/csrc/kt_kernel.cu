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
// GPU layout: one warp per ensemble.  Lane l holds the M consecutive orders i = M·l + m (m < M)
// as a_i, a_-i and b_i: the pulse is lane-local (order i couples with -i only) and runs on slot
// pairs with f32x2 arithmetic in float32; a one-order shift moves the slots within each lane and
// takes one value per quantity from the neighbouring lane (one shuffle).  Every lane computes the coefficients of one step of every 32 (sin/cos of the scaled
// flip, E1, E2, off-resonance phasor) into shared memory, replicated for the packed arithmetic,
// and the warp reads each step's set with broadcast loads; no warp waits on another.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "packed.cuh"

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

__device__ __forceinline__ void sc(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void scpi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void scpi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float em1(float x) { return expm1f(x); }
__device__ __forceinline__ double em1(double x) { return expm1(x); }
__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }

// Coefficient values: float32 with M >= 2 order slots per lane works on slot pairs (2p, 2p + 1)
// with f32x2 arithmetic, so each coefficient is replicated into a pair; otherwise one slot per
// operation.
template <typename R, int M>
struct KtPack {
    using P = R;
    static constexpr int L = 1, NP = M;
};
template <int M>
struct KtPack<float, M> {
    using P = typename std::conditional<(M >= 2), dev::f2, float>::type;
    static constexpr int L = M >= 2 ? 2 : 1, NP = M >= 2 ? M / 2 : 1;
};

__device__ __forceinline__ float lo(float v) { return v; }
__device__ __forceinline__ double lo(double v) { return v; }
__device__ __forceinline__ float lo(dev::f2 v) { return dev::lane_of(v, 0); }

// The per-step coefficients of Eqs. 4.2 (T'_HF entries and their negatives), 4.15/4.16 and the
// ensemble's precession, each replicated to a register value P.  Lane k of a warp computes the
// set of step base + k of a 32-step chunk into shared memory; every lane then reads each step's
// set with broadcast loads.
template <typename P>
struct alignas(16) Coef {
    P c2, ca, t01r, t01i, nt01r, t02r, t02i, nt02r, nt02i, t20r, t20i, nt20r, nt20i;  // pulse
    P e1m1, wr, wi, nwi;  // E1 - 1; E2·exp(-j2πΔfτ) and its negated imaginary part
    int flags;            // shift + 128 (8 bits) | sample << 8 | pulse << 9
};

// The populations of one ensemble in a warp: one register per order slot and quantity (the
// shifts move single slots between lanes); the pulse and the relaxation pack slot pairs.
template <typename R, int M>
struct Ensemble {
    using KP = KtPack<R, M>;
    using P = typename KP::P;
    static constexpr int L = KP::L, NP = KP::NP;
    R apr[M], api[M], anr[M], ani[M], bzr[M], bzi[M];  // a_i, a_-i, b_i for i = M·lane + slot
    int lane, K;
    bool full;  // K = 32·M - 1: every stored order exists

    __device__ __forceinline__ P ld(const R (&v)[M], int p) const {
        if constexpr (L == 2)
            return dev::pk2(v[2 * p], v[2 * p + 1]);
        else
            return v[p];
    }
    __device__ __forceinline__ void st(R (&v)[M], int p, P x) {
        if constexpr (L == 2)
            dev::unpk2(x, v[2 * p], v[2 * p + 1]);
        else
            v[p] = x;
    }

    // order 0: a_-0 is a_0 (kept bit-identical)
    __device__ __forceinline__ void tie_zero() {
        if (lane == 0) {
            anr[0] = apr[0];
            ani[0] = api[0];
        }
    }

    // Eq. 4.14 with T'_HF of Eq. 4.2 acting on (a_i, conj(a_-i), b_i), written out in real
    // arithmetic for (a_i, a_-i, b_i)
    __device__ __forceinline__ void pulse(const Coef<P> &c) {
        using namespace dev;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const P xr = ld(apr, p), xi = ld(api, p), ar = ld(anr, p), ai = ld(ani, p), zr = ld(bzr, p),
                    zi = ld(bzi, p);
            st(apr, p, vfma(c.nt02i, zi, vfma(c.t02r, zr, vfma(c.t01i, ai, vfma(c.t01r, ar, vmul(c.c2, xr))))));
            st(api, p, vfma(c.t02i, zr, vfma(c.t02r, zi, vfma(c.t01i, ar, vfma(c.nt01r, ai, vmul(c.c2, xi))))));
            st(anr, p, vfma(c.t02i, zi, vfma(c.t02r, zr, vfma(c.c2, ar, vfma(c.t01i, xi, vmul(c.t01r, xr))))));
            st(ani, p, vfma(c.t02i, zr, vfma(c.nt02r, zi, vfma(c.c2, ai, vfma(c.t01i, xr, vmul(c.nt01r, xi))))));
            st(bzr, p, vfma(c.ca, zr, vfma(c.nt20i, ai, vfma(c.t20r, ar, vfma(c.nt20i, xi, vmul(c.t20r, xr))))));
            st(bzi, p, vfma(c.ca, zi, vfma(c.nt20i, ar, vfma(c.nt20r, ai, vfma(c.t20i, xr, vmul(c.t20r, xi))))));
        }
        tie_zero();
    }

    // Eq. 4.17 with q = +1: a_i <- a_{i-1} (i >= 1), a_0 <- a_-1, a_-i <- a_-(i+1).  Within a lane
    // the slots move by one; the slot that crosses a lane boundary comes from the neighbour (one
    // shuffle per quantity).  At lane 0, a_-1 is its own slot 1 (with one slot per lane, lane 1's
    // slot 0).  The new a_-0 is the old a_-1 as well, so the order-0 pair stays tied.
    __device__ __forceinline__ void shift_up() {
        const int up = (lane + 31) & 31, dn = (lane + 1) & 31;
        const R rr = __shfl_sync(FULLW, apr[M - 1], up), ri = __shfl_sync(FULLW, api[M - 1], up);
        const R sr = __shfl_sync(FULLW, anr[0], dn), si = __shfl_sync(FULLW, ani[0], dn);
        R m1r = sr, m1i = si;
        if constexpr (M > 1) {
            m1r = anr[1];
            m1i = ani[1];
        }
#pragma unroll
        for (int s = M - 1; s > 0; --s) {
            apr[s] = apr[s - 1];
            api[s] = api[s - 1];
        }
        apr[0] = lane == 0 ? m1r : rr;
        api[0] = lane == 0 ? m1i : ri;
#pragma unroll
        for (int s = 0; s + 1 < M; ++s) {
            anr[s] = anr[s + 1];
            ani[s] = ani[s + 1];
        }
        anr[M - 1] = lane == 31 ? (R)0 : sr;  // order -(32M) does not exist
        ani[M - 1] = lane == 31 ? (R)0 : si;
        if (!full) drop(apr, api);
    }

    // Eq. 4.17 with q = -1: a_i <- a_{i+1} (i >= 0), a_-1 <- a_0, a_-i <- a_-(i-1).  a_-1 <- a_0
    // comes from the old a_-0 (tied to a_0); the new a_-0 is tied to the new a_0 at the end.
    __device__ __forceinline__ void shift_down() {
        const int up = (lane + 31) & 31, dn = (lane + 1) & 31;
        const R rr = __shfl_sync(FULLW, apr[0], dn), ri = __shfl_sync(FULLW, api[0], dn);
        const R sr = __shfl_sync(FULLW, anr[M - 1], up), si = __shfl_sync(FULLW, ani[M - 1], up);
#pragma unroll
        for (int s = 0; s + 1 < M; ++s) {
            apr[s] = apr[s + 1];
            api[s] = api[s + 1];
        }
        apr[M - 1] = lane == 31 ? (R)0 : rr;  // order 32M does not exist
        api[M - 1] = lane == 31 ? (R)0 : ri;
#pragma unroll
        for (int s = M - 1; s > 0; --s) {
            anr[s] = anr[s - 1];
            ani[s] = ani[s - 1];
        }
        anr[0] = sr;  // at lane 0 replaced by the tie below
        ani[0] = si;
        if (!full) drop(anr, ani);
        tie_zero();  // a_0 <- a_1, and a_-0 with it
    }

    // populations pushed past order K are dropped (only needed when the top slot is partial)
    __device__ __forceinline__ void drop(R (&re)[M], R (&im)[M]) {
#pragma unroll
        for (int s = 0; s < M; ++s)
            if (M * lane + s > K) {
                re[s] = (R)0;
                im[s] = (R)0;
            }
    }

    // Eqs. 4.15, 4.16 and the ensemble's precession: a *= E2·exp(-jθ), b *= E1, b_0 += 1 - E1
    __device__ __forceinline__ void relax(const Coef<P> &c) {
        using namespace dev;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const P xr = ld(apr, p), xi = ld(api, p), yr = ld(anr, p), yi = ld(ani, p), br = ld(bzr, p),
                    bi = ld(bzi, p);
            st(apr, p, vfma(xi, c.nwi, vmul(xr, c.wr)));
            st(api, p, vfma(xi, c.wr, vmul(xr, c.wi)));
            st(anr, p, vfma(yi, c.nwi, vmul(yr, c.wr)));
            st(ani, p, vfma(yi, c.wr, vmul(yr, c.wi)));
            st(bzr, p, vfma(br, c.e1m1, br));
            st(bzi, p, vfma(bi, c.e1m1, bi));
        }
        if (lane == 0) bzr[0] -= lo(c.e1m1);  // b_0 + (E1 - 1)(b_0 - 1)
    }
};

template <typename P, typename R>
__device__ __forceinline__ P rep(R x) {
    P o;
    dev::splat(o, x);
    return o;
}

// The coefficient set of one step for one ensemble (Eq. 4.2 entries from the B1-scaled flip)
template <typename P, typename R, typename StepT>
__device__ __forceinline__ void step_coef(Coef<P> &o, const StepT &s, R b1, R r1, R r2, R df) {
    const R alpha = b1 * (R)s.alpha;
    R sh, ch;
    sc((R)0.5 * alpha, &sh, &ch);
    const R cp = (R)s.cphi, sp = (R)s.sphi, s2 = sh * sh, sa = (R)2 * sh * ch, hs = sh * ch;
    const R c2 = ch * ch;
    const R t01r = s2 * (R)s.c2phi, t01i = s2 * (R)s.s2phi;
    const R t02r = -sa * sp, t02i = sa * cp;  // j sin α e^{jφ}
    const R t20r = hs * sp, t20i = hs * cp;   // j (sin α / 2) e^{-jφ}
    o.c2 = rep<P>(c2);
    o.ca = rep<P>(c2 - s2);
    o.t01r = rep<P>(t01r);
    o.t01i = rep<P>(t01i);
    o.nt01r = rep<P>(-t01r);
    o.t02r = rep<P>(t02r);
    o.t02i = rep<P>(t02i);
    o.nt02r = rep<P>(-t02r);
    o.nt02i = rep<P>(-t02i);
    o.t20r = rep<P>(t20r);
    o.t20i = rep<P>(t20i);
    o.nt20r = rep<P>(-t20r);
    o.nt20i = rep<P>(-t20i);
    const R tau = (R)s.tau;
    o.e1m1 = rep<P>(em1(-tau * r1));
    const R e2 = ex(-tau * r2);
    R sn, cs;
    scpi((R)2 * df * tau, &sn, &cs);
    o.wr = rep<P>(e2 * cs);
    o.wi = rep<P>(-e2 * sn);
    o.nwi = rep<P>(e2 * sn);
    o.flags = (s.shift + 128) | (s.sample << 8) | ((s.alpha != 0) << 9);
}

constexpr int KT_WARPS = 4;  // warps (ensembles) per block

// FULL: every stored order exists (K = 32·M − 1), so shifts never drop a population
template <typename R, int M, typename StepT, bool FULL>
__global__ void __launch_bounds__(32 * KT_WARPS) kt_kernel(const KtArgs a) {
    using E = Ensemble<R, M>;
    using P = typename E::P;
    __shared__ Coef<P> coef[KT_WARPS][32];
    __shared__ Cx<R> smp[KT_WARPS][32];  // a_0 after the chunk's sampled steps (written by lane 0)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t set = (int64_t)blockIdx.x * KT_WARPS + w;
    if (set >= a.n_sets) return;  // uniform over the warp; no block-wide barrier follows
    const StepT *steps = reinterpret_cast<const StepT *>(a.steps);
    const double t1 = a.t1[set], t2 = a.t2[set];
    const R r1 = isinf(t1) ? (R)0 : (R)(1.0 / t1), r2 = isinf(t2) ? (R)0 : (R)(1.0 / t2);
    const R b1 = a.b1 ? (R)a.b1[set] : (R)1;
    const R df = a.df ? (R)a.df[set] : (R)0;
    E e;
    e.lane = lane;
    e.K = a.max_order;
    e.full = FULL;
#pragma unroll
    for (int s = 0; s < M; ++s) e.apr[s] = e.api[s] = e.anr[s] = e.ani[s] = e.bzr[s] = e.bzi[s] = (R)0;
    if (lane == 0) e.bzr[0] = (R)1;
    double *out = a.signal + 2 * set * a.n_samples;
    Coef<P> *cw = coef[w];
    int64_t j = 0;  // samples written before this chunk
    for (int64_t base = 0; base < a.n_steps; base += 32) {
        const int cnt = (int)min((int64_t)32, a.n_steps - base);
        __syncwarp();  // the previous chunk's reads are done
        R cadc = 0, sadc = 0;
        int myflags = 0;
        if (lane < cnt) {
            const StepT st = steps[base + lane];
            step_coef<P, R>(cw[lane], st, b1, r1, r2, df);
            cadc = (R)st.cadc;
            sadc = (R)st.sadc;
            myflags = cw[lane].flags;
        }
        __syncwarp();
        // lane k keeps the sample of step base + k and stores it after the chunk (one conversion
        // to float64 per lane instead of one per sample for the whole warp)
        const unsigned smask = __ballot_sync(FULLW, lane < cnt && (myflags & 256));
        Cx<R> *sw = smp[w];
        for (int k = 0; k < cnt; ++k) {
            const Coef<P> &c = cw[k];
            const int fl = c.flags;
            if (FULL && fl == (512 | 256 | 129)) {  // the common step: pulse, one order up, sample
                e.pulse(c);
                e.shift_up();
                e.relax(c);
                if (lane == 0) sw[k] = Cx<R>{e.apr[0], e.api[0]};
                continue;
            }
            if (fl & 512) e.pulse(c);
            const int q = (fl & 255) - 128;
            for (int i = 0; i < q; ++i) e.shift_up();
            for (int i = 0; i > q; --i) e.shift_down();
            e.relax(c);
            if ((fl & 256) && lane == 0) sw[k] = Cx<R>{e.apr[0], e.api[0]};
        }
        __syncwarp();  // lane 0's samples are visible to the warp
        if (smask & (1u << lane)) {  // demodulated with this lane's own step
            const Cx<R> mine = sw[lane];
            const Cx<R> v = cmul(mine, Cx<R>{cadc, -sadc});
            const int64_t jj = j + __popc(smask & ((1u << lane) - 1u));
            out[2 * jj] = (double)v.re;
            out[2 * jj + 1] = (double)v.im;
        }
        j += __popc(smask);
    }
}

template <typename R, typename StepT>
int launch_kt_t(const KtArgs &a, void *stream) {
    const int threads = 32 * KT_WARPS;
    const int64_t blocks = (a.n_sets + KT_WARPS - 1) / KT_WARPS;
    if (blocks <= 0) return 0;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    const int M = (a.max_order + 32) / 32;  // slots per lane
    cudaStream_t st = (cudaStream_t)stream;
    // FULL: K = 32·M − 1 for the slot count the kernel is built for, so no order is ever dropped
    const bool full = a.max_order + 1 == 32 * (M <= 1 ? 1 : M <= 2 ? 2 : M <= 4 ? 4 : 8);
#define KTL(MM) (full ? kt_kernel<R, MM, StepT, true><<<(unsigned)blocks, threads, 0, st>>>(a)                       : kt_kernel<R, MM, StepT, false><<<(unsigned)blocks, threads, 0, st>>>(a))
    if (M <= 1)
        KTL(1);
    else if (M <= 2)
        KTL(2);
    else if (M <= 4)
        KTL(4);
    else if (M <= 8)
        KTL(8);
    else
        return (int)cudaErrorInvalidValue;
#undef KTL
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
