// fwd_kernel.cuh -- forward kernel: per-isochromat Bloch propagation + per-sample signal sum.
//
// One thread owns K spins (§5.3.2 domain decomposition: spins are independent) and keeps
// their magnetisation in registers for the whole sequence.  A thread block owns S = K·threads
// spins.  Every thread walks the same compiled operation stream (see internal.h), which thread
// 0 stages into shared memory in chunks with bulk asynchronous copies (cp.async.bulk, completed
// on an mbarrier) while the block computes on the previous chunk.
//
// Per operation (Eq. 4.1: M <- T_Relax·T_grad·T'_HF·M + T_Relax,z), with the transverse part
// carried as u + jv = (Mx + jMy)·exp(-jψ) in the frame of the latest pulse phase ψ:
//   RF   : lazy T1 recovery Mz <- Mz − ε1·(Mz − M0) over the time since the previous pulse
//          (ε1 = 1 − exp(−τ/T1) evaluated accurately, never 1 − E1 in float32), then the
//          Eq. 3.19 rotation, which in the pulse frame is a turn about the frame's x axis;
//   PREC : u + jv <- (u + jv)·E2·exp(-j2πφ) with φ = k·x + Δf·Δt in cycles (Eqs. 3.5/3.11/3.14);
//   RUN  : n samples of one constant-gradient readout, each (u + jv) <- (u + jv)·w, optionally
//          preceded by an inline precession (a folded phase encoding) and ended by an anchor
//          that sets the state from the one before the run times an exact class phasor;
//   samples: Σ_spins (u + jv) (§5.1.1, Eq. 3.32) reduced in-thread over the K spins (tree),
//            across the warp by a transposed butterfly (16 samples per pass: lane l ends up
//            with the warp total of value l), across warps in shared memory and across blocks
//            with float64 atomics after multiplying by exp(-j(adc_phase − ψ)).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "../../include/mrsim.h"
#include "internal.h"
#include "dfloat.cuh"
#include "packed.cuh"

namespace mrsim {
namespace dev {

__device__ __forceinline__ uint32_t su32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(b))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase; false once `limit_ns` of wall time has passed.
static __device__ __noinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test(b, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_test(b, parity))
        if (gtimer() - t0 > limit_ns) return false;
    return true;
}

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s for one 4 KB chunk: only a fault takes that long

constexpr unsigned FULL = 0xffffffffu;
constexpr int RED_STRIDE = SAMPLE_WINDOW_F64 + 16;  // float64: per-warp, per-component window row
constexpr int WIN_STRIDE = SAMPLE_WINDOW_F32 + 16;  // float32: block-wide window, per component

__device__ __forceinline__ void red_shared_add(float *p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(su32(p)), "f"(v) : "memory");
}

// Rounding constant 1.5·2^23: for |p| < 2^22, (p + c) − c is p rounded to the nearest integer
// (round-to-nearest-even), so p − ((p + c) − c) is the exact fractional part in [−1/2, 1/2].
constexpr float RINT_MAGIC = 12582912.0f;
// The packed fractional-part step on spin pairs needs |k_hi·x_hi| < 2^22 cycles; blocks whose
// coordinates and program could reach PHASE_SAFE take the one-spin-at-a-time path instead.
constexpr float PHASE_SAFE = 2097152.0f;  // 2^21
// Taylor coefficients of sin(πt) = Σ (−1)^k π^(2k+1) t^(2k+1)/(2k+1)! and
// cos(πt) = Σ (−1)^k π^(2k) t^(2k)/(2k)!, truncated for |t| <= 1/2: the first omitted terms are
// below 7e-10 (sine, t^15) and 7e-9 (cosine, t^14).
constexpr double PI_D = 3.14159265358979323846;
constexpr double taylor_pi(int n) {  // π^n / n!
    double c = 1.0;
    for (int i = 1; i <= n; ++i) c *= PI_D / i;
    return c;
}
constexpr float SIN_C0 = (float)taylor_pi(1), SIN_C1 = (float)-taylor_pi(3), SIN_C2 = (float)taylor_pi(5),
                SIN_C3 = (float)-taylor_pi(7), SIN_C4 = (float)taylor_pi(9), SIN_C5 = (float)-taylor_pi(11),
                SIN_C6 = (float)taylor_pi(13);
constexpr float COS_C1 = (float)-taylor_pi(2), COS_C2 = (float)taylor_pi(4), COS_C3 = (float)-taylor_pi(6),
                COS_C4 = (float)taylor_pi(8), COS_C5 = (float)-taylor_pi(10), COS_C6 = (float)taylor_pi(12);
template <typename R, int K>
struct Packing {  // float64: one spin per value
    using P = R;
    static constexpr int L = 1;
};
template <int K>
struct Packing<float, K> {  // float32: pairs when the thread has two spins or more
    using P = typename std::conditional<(K >= 2), f2, float>::type;
    static constexpr int L = K >= 2 ? 2 : 1;
};

// per-spin phasor class entry (w = wr + j·wi) of one packed value
template <typename P>
struct alignas(2 * sizeof(P)) Cw {
    P re, im;
};

// Shared-memory transpose that leaves lane l with the warp-wide sum of value l of a 16-sample
// tile (sample l/2, component l%2).  Lane k stores its (x, y) pair of sample m with one 8-byte
// store into row m, half k/16 of the tile (conflict-free: each half-warp fills 128 contiguous
// bytes); lane l then reads row l/2, half l%2 (the pairs of 16 lanes, 8 conflict-free 16-byte
// loads), adds the 16 pairs with packed adds and takes the other half-warp's share from its
// neighbour lane: 16 stores, 8 loads, 16 adds and one shuffle per tile.
constexpr int TILE_HALF = 36;  // floats per half row: 16 (x, y) pairs + 4 floats of padding
constexpr int TILE_ROW = 2 * TILE_HALF;
constexpr int TILE_FLOATS = 16 * TILE_ROW;  // one warp's tile
__device__ __forceinline__ float tile_reduce_pairs(const f2 (&v)[16], int lane, float *tile) {
    f2 *dst = reinterpret_cast<f2 *>(tile + (lane >> 4) * TILE_HALF) + (lane & 15);
#pragma unroll
    for (int m = 0; m < 16; ++m) dst[m * (TILE_ROW / 2)] = v[m];
    __syncwarp();
    const float4 *row = reinterpret_cast<const float4 *>(tile + (lane >> 1) * TILE_ROW + (lane & 1) * TILE_HALF);
    f2 a[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 t = row[q];
        a[2 * q] = pk2(t.x, t.y);
        a[2 * q + 1] = pk2(t.z, t.w);
    }
    __syncwarp();
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
#pragma unroll
        for (int i = 0; i < w; ++i) a[i] = vadd(a[i], a[i + w]);
    }
    float x, y;
    unpk2(a[0], x, y);
    const bool odd = (lane & 1) != 0;
    const float mine = odd ? y : x, theirs = odd ? x : y;
    return mine + __shfl_xor_sync(FULL, theirs, 1);
}

// Butterfly that leaves lane l with the warp-wide sum of v[l] (32 values per lane in, 1 out);
// used by the float64 path.
template <typename R>
__device__ __forceinline__ R transpose_reduce32(R (&v)[32], int lane) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const R a = v[i], b = v[i + off];
            const R send = up ? a : b;
            const R keep = up ? b : a;
            v[i] = keep + shfl_x(send, off);
        }
    }
    return v[0];
}

// Pairwise (tree) sum of N values: log2(N) dependent adds instead of N − 1.
template <typename P, int N>
__device__ __forceinline__ P tree_sum(const P (&a)[N]) {
    if constexpr (N == 1) {
        return a[0];
    } else if constexpr (N == 2) {
        return vadd(a[0], a[1]);
    } else if constexpr (N == 4) {
        return vadd(vadd(a[0], a[1]), vadd(a[2], a[3]));
    } else {
        static_assert(N == 8, "N must be 1, 2, 4 or 8");
        return vadd(vadd(vadd(a[0], a[1]), vadd(a[2], a[3])), vadd(vadd(a[4], a[5]), vadd(a[6], a[7])));
    }
}

// Float-float product k·x reduced modulo 1 (cycles): returns frac(kh·xh) and accumulates the
// small remainder kh·xh − fl(kh·xh) + kh·xl + kl·xh into `err`.
__device__ __forceinline__ float ff_term(float kh, float kl, float xh, float xl, float &err) {
    const float p = kh * xh;
    float e = fmaf(kh, xh, -p);
    e = fmaf(kh, xl, e);
    e = fmaf(kl, xh, e);
    err += e;
    return p - rintf(p);
}
__device__ __forceinline__ float wrap1(float t) { return t - rintf(t); }

// Sum the sample window over warps (float64), multiply by the sample's demodulation factor and
// add the block's partial sums to the global signal.  Every thread of the block must call it.
template <typename R>
__device__ __noinline__ void flush_window(const R *red, const double *demod, double *signal, int win_base,
                                          int win_end, int tid, int nthr, int nwarp) {
    __syncthreads();
    const int cnt = win_end - win_base;
    for (int s = tid; s < cnt; s += nthr) {
        double re = 0.0, im = 0.0;
        for (int w = 0; w < nwarp; ++w) {
            re += (double)red[w * 2 * RED_STRIDE + s];
            im += (double)red[w * 2 * RED_STRIDE + RED_STRIDE + s];
        }
        const int64_t j = (int64_t)win_base + s;
        const double cr = demod[2 * j], ci = demod[2 * j + 1];
        atomicAdd(signal + 2 * j, re * cr - im * ci);
        atomicAdd(signal + 2 * j + 1, re * ci + im * cr);
    }
    __syncthreads();
}

// float32: multiply the block-wide window by the float32 demodulation factors, add it to the
// global signal with float64 atomics and clear it.  Every thread of the block must call it.
static __device__ __noinline__ void flush_window_f32(float *win, const float *demod32, double *signal, int win_base,
                                             int win_end, int tid, int nthr) {
    __syncthreads();
    const int cnt = win_end - win_base;
    for (int s = tid; s < cnt; s += nthr) {
        const float re = win[s], im = win[WIN_STRIDE + s];
        win[s] = 0.0f;
        win[WIN_STRIDE + s] = 0.0f;
        const int64_t j = (int64_t)win_base + s;
        const float2 d = reinterpret_cast<const float2 *>(demod32)[j];
        atomicAdd(signal + 2 * j, (double)(re * d.x - im * d.y));
        atomicAdd(signal + 2 * j + 1, (double)(re * d.y + im * d.x));
    }
    __syncthreads();
}

// With receive coils the window holds NCR slots per sample (one per coil row): slot v
// is sample win_base + v / NCR of coil v % NCR, whose signal starts at signal + coil * coil_stride.
// Padding coils (coil >= n_coils) are not written.

// Receive coils, float64: as flush_window with coil-major slots.
template <typename R, int NCR>
__device__ __noinline__ void flush_window_coils(const R *red, const double *demod, double *signal, int win_base,
                                          int win_end, int tid, int nthr, int nwarp, int n_coils,
                                          int64_t coil_stride) {
    __syncthreads();
    const int cnt = (win_end - win_base) * NCR;
    for (int s = tid; s < cnt; s += nthr) {
        const int coil = s % NCR;
        if (coil >= n_coils) continue;
        double re = 0.0, im = 0.0;
        for (int w = 0; w < nwarp; ++w) {
            re += (double)red[w * 2 * RED_STRIDE + s];
            im += (double)red[w * 2 * RED_STRIDE + RED_STRIDE + s];
        }
        const int64_t j = (int64_t)win_base + s / NCR;
        const double cr = demod[2 * j], ci = demod[2 * j + 1];
        double *sig = signal + coil * coil_stride;
        atomicAdd(sig + 2 * j, re * cr - im * ci);
        atomicAdd(sig + 2 * j + 1, re * ci + im * cr);
    }
    __syncthreads();
}

// Receive coils, float32: as flush_window_f32 with coil-major slots.
template <int NCR>
static __device__ __noinline__ void flush_window_coils_f32(float *win, const float *demod32, double *signal, int win_base,
                                                     int win_end, int tid, int nthr, int n_coils,
                                                     int64_t coil_stride) {
    __syncthreads();
    const int cnt = (win_end - win_base) * NCR;
    for (int s = tid; s < cnt; s += nthr) {
        const float re = win[s], im = win[WIN_STRIDE + s];
        win[s] = 0.0f;
        win[WIN_STRIDE + s] = 0.0f;
        const int coil = s % NCR;
        if (coil >= n_coils) continue;
        const int64_t j = (int64_t)win_base + s / NCR;
        const float2 d = reinterpret_cast<const float2 *>(demod32)[j];
        double *sig = signal + coil * coil_stride;
        atomicAdd(sig + 2 * j, (double)(re * d.x - im * d.y));
        atomicAdd(sig + 2 * j + 1, (double)(re * d.y + im * d.x));
    }
    __syncthreads();
}

// NC > 0: receive coils (Eq. 3.25 with per-spin sensitivities): each sample yields NC weighted
// sums (NC = 1, 2, 4 or 8; the caller's coils beyond n_coils have zero weight and are not stored).
template <typename R, int K, int NC = 0>
struct Spins {
    using Op = typename std::conditional<std::is_same<R, float>::value, OpF32, OpF64>::type;
    using P = typename Packing<R, K>::P;
    using CwT = Cw<P>;
    static constexpr int L = Packing<R, K>::L;  // spins per packed value
    static constexpr int NP = K / L;            // packed values per quantity
    // float64 and double-float (the compensated precision) share the float64 program, layouts and
    // code paths; float32 has its own
    static constexpr bool F64 = is_wide<R>::value;
    static constexpr int WIN = F64 ? SAMPLE_WINDOW_F64 : SAMPLE_WINDOW_F32;  // window slots
    static constexpr int NCR = NC > 0 ? NC : 1;                                // slots per sample
    static constexpr int WINS = WIN / NCR;                                     // samples per window
    static_assert(NCR == 1 || NCR == 2 || NCR == 4 || NCR == 8, "coil rows per sample: 1, 2, 4 or 8");

    // spin i = q + h·NP of the thread is lane h of packed value q
    P u[NP], v[NP], mz[NP], rho[NP];  // transverse part in the pulse frame, longitudinal, M0
    P wr[NP], wi[NP], nwi[NP];        // cached phasor class (nwi = −wi, kept for the pairs only)
    P e1v[NP];                        // cached T1 class ε1
    P cre[NCR][NP], cim[NCR][NP];  // coils: sensitivities C = cre + j·cim (−cim formed on the integer pipe)
    int win_base, win_end;
    int n_coils;          // receive coils stored (<= NCR)
    int64_t coil_stride;  // doubles between two coils' signals (2·n_adc)

    // shared-memory views and block geometry
    const CwT *cw;
    const void *train;  // sub-pulse table: float32 (cos, cos, sin, sin), float64 (cos, sin)
    const P *ce1, *ce2;
    const P *prm;      // spin coordinates for inline precessions (float32: hi/lo rows), pair-major
    bool big_phase;    // some |k_hi·x_hi| of this block may reach PHASE_SAFE: scalar phase path
    bool zero_df;      // every spin of this block has Δf = 0: no Δf·Δt phase term
    R *red;       // float64: per-warp window rows
    float *tile;  // float32: this warp's transpose tile
    float *win;   // float32: block-wide window
    int S, SP, nthr, tid, lane, warp, nwarp;
    int64_t base, np, n_spins;
    const double *params;
    const R *maps;  // NULL or the train maps (kind x TRAIN_MAP_ROWS rows of np values)
    double *snap;   // NULL or the snapshot buffer (n_snap x n_spins x 3)
    const double *demod;
    const float *demod32;
    double *signal;

    __device__ __forceinline__ int li(int i) const { return i * nthr + tid; }  // spin i in the block
    __device__ __forceinline__ int pi(int q) const { return q * nthr + tid; }  // packed value q
    __device__ __forceinline__ P nwi_of(int q) const {
        if constexpr (L == 2)
            return nwi[q];
        else
            return vneg(wi[q]);
    }

    __device__ __forceinline__ void load_w(int c) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const CwT w = cw[c * SP + pi(q)];
            wr[q] = w.re;
            wi[q] = w.im;
            if constexpr (L == 2) nwi[q] = vneg(w.im);
        }
    }
    __device__ __forceinline__ void rot_w() {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const P nu = vdot2(v[q], nwi_of(q), u[q], wr[q]);
            const P nv = vdot2(v[q], wr[q], u[q], wi[q]);
            u[q] = nu;
            v[q] = nv;
        }
    }
    __device__ __forceinline__ void t1_cached() {
#pragma unroll
        for (int q = 0; q < NP; ++q) mz[q] = vfma(e1v[q], vsub(rho[q], mz[q]), mz[q]);
    }
    // lazy T1 recovery over the interval since the previous pulse
    __device__ __forceinline__ void t1_relax(const Op &op) {
        if (op.flags & F_E1CLS) {
            if (op.flags & F_E1LOAD) {
#pragma unroll
                for (int q = 0; q < NP; ++q) e1v[q] = ce1[op.ecls * SP + pi(q)];
            }
            t1_cached();
        } else if (op.flags & F_E1INL) {
            const double tau = (double)op.f[10];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                R eps[L];
#pragma unroll
                for (int h = 0; h < L; ++h) {
                    const int64_t s = base + li(q + h * NP);
                    const double r1 = s < n_spins ? params[P_R1 * np + s] : 0.0;
                    eps[h] = (R)(-expm1(-tau * r1));
                }
                P e;
                set_lanes(e, eps);
                mz[q] = vfma(e, vsub(rho[q], mz[q]), mz[q]);
            }
        }
    }
    // hard pulse about the frame's x axis (Eq. 3.19 in the pulse frame); nsa = −sin α
    __device__ __forceinline__ void rf_turn(P ca, P sa, P nsa) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const P nv = vdot2(v[q], ca, mz[q], sa);
            const P nz = vdot2(v[q], nsa, mz[q], ca);
            v[q] = nv;
            mz[q] = nz;
        }
    }
    // the op's own rotation, or for a parametric pulse the one in sub-pulse table entry op.tab
    // (parametric programs drive the float64 adjoint forward only; the float32 kernels skip the test)
    __device__ __forceinline__ void rf_turn_op(const Op &op) {
        if constexpr (F64) {
            if (op.flags & F_RFTAB) {
                P ca, sa, nsa;
                load_train(op.tab, ca, sa, nsa);
                rf_turn(ca, sa, nsa);
                return;
            }
        }
        rf_turn_s((R)op.f[0], (R)op.f[1]);
    }
    __device__ __forceinline__ void rf_turn_s(R ca, R sa) {
        P c, s, ns;
        splat(c, ca);
        splat(s, sa);
        splat(ns, -sa);
        rf_turn(c, s, ns);
    }
    // turn the frame by exp(-jδ) (uniform over spins); float32 uses (hi, lo) constants
    __device__ __forceinline__ void frame_turn(const Op &op) {
        if constexpr (F64) {
            P c, s, ns;
            splat(c, (R)op.f[2]);
            splat(s, (R)op.f[3]);
            splat(ns, (R)-op.f[3]);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const P nu = vdot2(u[q], c, v[q], s);
                const P nv = vdot2(v[q], c, u[q], ns);
                u[q] = nu;
                v[q] = nv;
            }
        } else {
            P ch, cl, sh, sl, nsh, nsl;
            splat(ch, op.f[2]);
            splat(cl, op.f[3]);
            splat(sh, op.f[4]);
            splat(sl, op.f[5]);
            splat(nsh, -op.f[4]);
            splat(nsl, -op.f[5]);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const P nu = vfma(u[q], ch, vfma(v[q], sh, vfma(u[q], cl, vmul(v[q], sl))));
                const P nv = vfma(v[q], ch, vfma(u[q], nsh, vfma(u[q], nsl, vmul(v[q], cl))));
                u[q] = nu;
                v[q] = nv;
            }
        }
    }
    __device__ __forceinline__ R prm_at(int row, int q, int h) const { return lane_of(prm[row * SP + pi(q)], h); }

    // precession by the op's own moment and interval (not a cached class)
    __device__ __forceinline__ void prec_inline(const Op &op) {
        if constexpr (L == 2) {
            if (!big_phase) {
                prec_inline_pairs(op);
                return;
            }
        }
        prec_inline_lanes(op);
    }

    // float32 pairs: phase φ = Σ k·x in cycles with k and x as float-float pairs: fractional part
    // of each rounded product k_hi·x_hi (RINT_MAGIC), plus its exact residual and the cross terms,
    // reduced to t ∈ [−1/2, 1/2]; sin and cos of πt
    // from the Taylor polynomials, then of 2πt by the double-angle formulas; u + jv is multiplied
    // by E2·exp(−j2πt) (Eqs. 3.5, 3.14 in the pulse frame)
    __device__ __forceinline__ void prec_inline_pairs(const Op &op) {
        const f2 mg = pk2(RINT_MAGIC, RINT_MAGIC);
        const uint16_t fl = op.flags;
        const bool tx = fl & F_KX, ty = fl & F_KY, tz = fl & F_KZ, tdf = (fl & F_DT) && !zero_df;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            f2 t = pk2(0.0f, 0.0f), er = pk2(0.0f, 0.0f);
            auto term = [&](int a) {
                f2 kh, kl;
                splat(kh, op.f[2 * a]);
                splat(kl, op.f[2 * a + 1]);
                const f2 xh = prm[(2 * a) * SP + pi(q)], xl = prm[(2 * a + 1) * SP + pi(q)];
                const f2 p = vmul(kh, xh);
                t = vadd(t, vsub(p, vsub(vadd(p, mg), mg)));  // frac(p), exact
                er = vadd(er, vfma(kh, xh, vneg(p)));          // kh·xh − p, exact
                er = vfma(kl, xh, vfma(kh, xl, er));
            };
            if (tx) term(0);
            if (ty) term(1);
            if (tz) term(2);
            if (tdf) term(3);
            t = vadd(t, er);
            t = vsub(t, vsub(vadd(t, mg), mg));
            const f2 s2 = vmul(t, t);
            auto horner = [&](f2 acc, float c) { return vfma(acc, s2, pk2(c, c)); };
            f2 sp = pk2(SIN_C6, SIN_C6), cp = pk2(COS_C6, COS_C6);
            sp = horner(horner(horner(horner(horner(horner(sp, SIN_C5), SIN_C4), SIN_C3), SIN_C2), SIN_C1), SIN_C0);
            cp = horner(horner(horner(horner(horner(horner(cp, COS_C5), COS_C4), COS_C3), COS_C2), COS_C1), 1.0f);
            const f2 sn = vmul(sp, t);  // sin πt
            const f2 twos = vadd(sn, sn);
            f2 one;
            splat(one, 1.0f);
            f2 ar = vfma(twos, vneg(sn), one);  // cos 2πt = 1 − 2 sin²πt
            f2 as = vmul(twos, cp);             // sin 2πt
            if (fl & (F_E2CLS | F_DT)) {
                f2 e2;
                if (fl & F_E2CLS) {
                    e2 = ce2[op.ecls * SP + pi(q)];
                } else {
                    float ev[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int64_t s = base + li(q + h * NP);
                        const double r2 = s < n_spins ? params[P_R2 * np + s] : 0.0;
                        ev[h] = (float)exp(-(double)op.f[8] * r2);
                    }
                    set_lanes(e2, ev);
                }
                ar = vmul(e2, ar);
                as = vmul(e2, as);
            }
            // (u + jv)·(ar − j·as)
            const f2 nu = vfma(v[q], as, vmul(u[q], ar));
            const f2 nv = vfma(u[q], vneg(as), vmul(v[q], ar));
            u[q] = nu;
            v[q] = nv;
        }
    }

    // one spin at a time (float64; float32 with one spin per thread or large phases)
    __device__ __forceinline__ void prec_inline_lanes(const Op &op) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            R ar[L], ai[L], nai[L];
#pragma unroll
            for (int h = 0; h < L; ++h) {
                const int l = li(q + h * NP);
                R e2;
                if (op.flags & F_E2CLS) {
                    e2 = lane_of(ce2[op.ecls * SP + pi(q)], h);
                } else if (op.flags & F_DT) {
                    const int64_t s = base + l;
                    const double r2 = s < n_spins ? params[P_R2 * np + s] : 0.0;
                    e2 = (R)exp(-(double)op.f[F64 ? 3 : 8] * r2);
                } else {
                    e2 = (R)1;
                }
                R sn, cs;
                if constexpr (F64) {
                    double th = 0.0;
                    if (op.flags & F_KX) th += op.f[0] * (double)prm_at(0, q, h);
                    if (op.flags & F_KY) th += op.f[1] * (double)prm_at(1, q, h);
                    if (op.flags & F_KZ) th += op.f[2] * (double)prm_at(2, q, h);
                    if (op.flags & F_DT) th += op.f[3] * (double)prm_at(3, q, h);
                    th -= rint(th);
                    double snd, csd;
                    sincospi(2.0 * th, &snd, &csd);
                    sn = (R)snd;
                    cs = (R)csd;
                } else {
                    float err = 0.0f, t = 0.0f;
                    if (op.flags & F_KX) t = wrap1(t + ff_term(op.f[0], op.f[1], prm_at(0, q, h), prm_at(1, q, h), err));
                    if (op.flags & F_KY) t = wrap1(t + ff_term(op.f[2], op.f[3], prm_at(2, q, h), prm_at(3, q, h), err));
                    if (op.flags & F_KZ) t = wrap1(t + ff_term(op.f[4], op.f[5], prm_at(4, q, h), prm_at(5, q, h), err));
                    if (op.flags & F_DT) t = wrap1(t + ff_term(op.f[6], op.f[7], prm_at(6, q, h), prm_at(7, q, h), err));
                    t = wrap1(t + err);
                    // accurate sin/cos of the reduced angle (the hardware approximation's 2^-21 absolute
                    // error would accumulate over many inline intervals)
                    sincospif(2.0f * t, &sn, &cs);
                }
                ar[h] = e2 * cs;
                ai[h] = -e2 * sn;
                nai[h] = e2 * sn;
            }
            P AR, AI, NAI;
            set_lanes(AR, ar);
            set_lanes(AI, ai);
            set_lanes(NAI, nai);
            const P nu = vdot2(v[q], NAI, u[q], AR);
            const P nv = vdot2(v[q], AR, u[q], AI);
            u[q] = nu;
            v[q] = nv;
        }
    }

    __device__ __forceinline__ R *red_row(int comp) { return red + warp * 2 * RED_STRIDE + comp * RED_STRIDE; }

    __device__ __forceinline__ void flush() {
        if constexpr (NC > 0) {
            if constexpr (F64)
                flush_window_coils<R, NCR>(red, demod, signal, win_base, win_end, tid, nthr, nwarp, n_coils,
                                           coil_stride);
            else
                flush_window_coils_f32<NCR>(win, demod32, signal, win_base, win_end, tid, nthr, n_coils, coil_stride);
        } else if constexpr (F64) {
            flush_window(red, demod, signal, win_base, win_end, tid, nthr, nwarp);
        } else {
            flush_window_f32(win, demod32, signal, win_base, win_end, tid, nthr);
        }
        win_base = win_end;
    }

    // ---- receive coils ----------------------------------------------------------------------
    // the thread's spins weighted with coil c's sensitivities: Σ_k C_ck·(u_k + j v_k)
    __device__ __forceinline__ void coil_sum(int c, R &sx, R &sy) {
        P re = vfma(v[0], vneg(cim[c][0]), vmul(u[0], cre[c][0]));
        P im = vfma(u[0], cim[c][0], vmul(v[0], cre[c][0]));
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            re = vfma(v[q], vneg(cim[c][q]), vfma(u[q], cre[c][q], re));
            im = vfma(u[q], cim[c][q], vfma(v[q], cre[c][q], im));
        }
        sx = hsum(re);
        sy = hsum(im);
    }
    // tt (<= 16 / NCR) sample steps of a run; row s·NCR + c of the tile is sample s, coil c; the
    // warp total of value l (row l/2, component l%2) ends up in lane l
    template <bool FULL_TILE>
    __device__ __forceinline__ R coil_tile(int tt) {
        constexpr int TS = 16 / NCR;
        if constexpr (F64) {
            R vv[32];
#pragma unroll
            for (int t = 0; t < TS; ++t) {
                if (FULL_TILE || t < tt) rot_w();
#pragma unroll
                for (int c = 0; c < NCR; ++c) {
                    const int r = t * NCR + c;
                    if (FULL_TILE || t < tt) {
                        coil_sum(c, vv[2 * r], vv[2 * r + 1]);
                    } else {
                        vv[2 * r] = (R)0;
                        vv[2 * r + 1] = (R)0;
                    }
                }
            }
            return transpose_reduce32(vv, lane);
        } else {
            f2 vt[16];
#pragma unroll
            for (int t = 0; t < TS; ++t) {
                if (FULL_TILE || t < tt) rot_w();
#pragma unroll
                for (int c = 0; c < NCR; ++c) {
                    R sx = 0.0f, sy = 0.0f;
                    if (FULL_TILE || t < tt) coil_sum(c, sx, sy);
                    vt[t * NCR + c] = pk2(sx, sy);
                }
            }
            return tile_reduce_pairs(vt, lane, tile);
        }
    }
    // a sample run with coils: the window holds WINS samples, so long runs go in window-sized
    // chunks with a flush in between (every thread of the block takes the same path)
    __device__ __forceinline__ void run_coils(const Op &op) {
        constexpr int TS = 16 / NCR;
        const int n = op.n, j0 = op.adc0;
        if (op.flags & F_PLOAD) load_w(op.pcls);
        P au[NP], av[NP];
        const bool anchor = (op.flags & F_ANCHOR) != 0;
        if (anchor) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                au[q] = u[q];
                av[q] = v[q];
            }
        }
        if (op.flags & F_INLINE) prec_inline(op);  // the run's leading precession (the anchor restores from before it)
        for (int t0 = 0; t0 < n;) {
            if (j0 + t0 - win_base >= WINS) flush();
            const int m = min(n - t0, WINS - (j0 + t0 - win_base));
            const int slot0 = (j0 + t0 - win_base) * NCR;
            int s0 = 0;
            for (; s0 + TS <= m; s0 += TS) store_tile(slot0 + s0 * NCR, coil_tile<true>(TS));
            if (s0 < m) {
                const int tt = m - s0;
                const R tot = coil_tile<false>(tt);
                if (lane < 2 * tt * NCR) store_tile(slot0 + s0 * NCR, tot);
            }
            t0 += m;
            win_end = j0 + t0;
        }
        if (anchor) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const CwT w = cw[op.acls * SP + pi(q)];
                u[q] = vdot2(av[q], vneg(w.im), au[q], w.re);
                v[q] = vdot2(av[q], w.re, au[q], w.im);
            }
        }
    }
    __device__ __forceinline__ void sample_coils(int j) {
        if (j + 1 - win_base > WINS) flush();
#pragma unroll
        for (int c = 0; c < NCR; ++c) {
            R sx, sy;
            coil_sum(c, sx, sy);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                sx += shfl_x(sx, off);
                sy += shfl_x(sy, off);
            }
            const int slot = (j - win_base) * NCR + c;
            if (lane == 0) {
                if constexpr (F64) {
                    red_row(0)[slot] = sx;
                    red_row(1)[slot] = sy;
                } else {
                    red_shared_add(win + slot, sx);
                    red_shared_add(win + WIN_STRIDE + slot, sy);
                }
            }
        }
        win_end = j + 1;
    }
    __device__ __forceinline__ void sample_any(int j) {
        if constexpr (NC > 0)
            sample_coils(j);
        else
            sample1(j);
    }

    __device__ __forceinline__ void sample1(int j) {
        if (j + 1 - win_base > WIN) flush();
        R sx = hsum(tree_sum<P, NP>(u)), sy = hsum(tree_sum<P, NP>(v));
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            sx += shfl_x(sx, off);
            sy += shfl_x(sy, off);
        }
        if (lane == 0) {
            if constexpr (F64) {
                red_row(0)[j - win_base] = sx;
                red_row(1)[j - win_base] = sy;
            } else {
                red_shared_add(win + (j - win_base), sx);
                red_shared_add(win + WIN_STRIDE + (j - win_base), sy);
            }
        }
        win_end = j + 1;
    }

    // lane l holds the warp total of value l (sample l/2, component l%2) of a 16-sample tile
    __device__ __forceinline__ void store_tile(int slot, R tot) {
        if constexpr (F64)
            red_row(lane & 1)[slot + (lane >> 1)] = tot;
        else
            red_shared_add(win + (lane & 1) * WIN_STRIDE + slot + (lane >> 1), tot);
    }

    // one sample step of a run: rotate by the cached class, return the thread's sums
    __device__ __forceinline__ void run_step(R &sx, R &sy) {
        rot_w();
        sx = hsum(tree_sum<P, NP>(u));
        sy = hsum(tree_sum<P, NP>(v));
    }

    // tt (<= 16) sample steps; the warp total of value l of the tile ends up in lane l
    template <bool FULL_TILE>
    __device__ __forceinline__ R tile_steps(int tt) {
        if constexpr (F64) {
            R vv[32];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                if (FULL_TILE || t < tt) {
                    run_step(vv[2 * t], vv[2 * t + 1]);
                } else {
                    vv[2 * t] = (R)0;
                    vv[2 * t + 1] = (R)0;
                }
            }
            return transpose_reduce32(vv, lane);
        } else {
            f2 vt[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                R sx = 0.0f, sy = 0.0f;
                if (FULL_TILE || t < tt) run_step(sx, sy);
                vt[t] = pk2(sx, sy);
            }
            return tile_reduce_pairs(vt, lane, tile);
        }
    }

    __device__ __forceinline__ void run(const Op &op) {
        const int n = op.n, j0 = op.adc0;
        if (op.flags & F_PLOAD) load_w(op.pcls);
        P au[NP], av[NP];
        const bool anchor = (op.flags & F_ANCHOR) != 0;
        if (anchor) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                au[q] = u[q];
                av[q] = v[q];
            }
        }
        if (op.flags & F_INLINE) prec_inline(op);  // the run's leading precession (the anchor restores from before it)
        if (j0 + n - win_base > WIN) flush();
        const int slot0 = j0 - win_base;
        int t0 = 0;
        for (; t0 + 16 <= n; t0 += 16) store_tile(slot0 + t0, tile_steps<true>(16));  // full tiles
        if (t0 < n) {  // ragged tail
            const int tt = n - t0;
            const R tot = tile_steps<false>(tt);
            if (lane < 2 * tt) store_tile(slot0 + t0, tot);
        }
        win_end = j0 + n;
        if (anchor) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const CwT w = cw[op.acls * SP + pi(q)];
                u[q] = vdot2(av[q], vneg(w.im), au[q], w.re);
                v[q] = vdot2(av[q], w.re, au[q], w.im);
            }
        }
    }

    __device__ __forceinline__ void load_train(int k, P &ca, P &sa, P &nsa) const {
        if constexpr (std::is_same<R, dfl>::value) {  // converted once at set-up: (cos, sin) as pairs
            const dfl *t = reinterpret_cast<const dfl *>(train) + 2 * k;
            ca = t[0];
            sa = t[1];
            nsa = -t[1];
        } else if constexpr (F64) {
            const double2 t = reinterpret_cast<const double2 *>(train)[k];
            ca = t.x;
            sa = t.y;
            nsa = -t.y;
        } else {
            const float4 t = reinterpret_cast<const float4 *>(train)[k];
            if constexpr (L == 2) {
                ca = pk2(t.x, t.y);
                sa = pk2(t.z, t.w);
                nsa = vneg(sa);
            } else {
                ca = t.x;
                sa = t.z;
                nsa = -t.z;
            }
        }
    }

    // n sub-pulses of a shaped pulse (Eq. 3.23): lazy T1 with the cached class, the pulse-frame
    // turn with table entry i, precession by the cached class
    __device__ __forceinline__ void train_run(int off, int n) {
#pragma unroll 2
        for (int i = 0; i < n; ++i) {
            P ca, sa, nsa;
            load_train(off + i, ca, sa, nsa);
            t1_cached();
            rf_turn(ca, sa, nsa);
            rot_w();
        }
    }

    // a recurring train as its map of kind t: (u, v, Mz) <- A (u, v, Mz) + c for every spin (the
    // same composition of the train's sub-pulses as train_run, formed once per launch)
    __device__ __forceinline__ void train_map(int t) {
        const R *m = maps + (int64_t)t * TRAIN_MAP_ROWS * np;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            P A[TRAIN_MAP_ROWS];
#pragma unroll
            for (int j = 0; j < TRAIN_MAP_ROWS; ++j) {
                R x[L];
#pragma unroll
                for (int h = 0; h < L; ++h) {
                    const int64_t s = base + li(q + h * NP);
                    x[h] = s < n_spins ? m[j * np + s] : R(0);
                }
                set_lanes(A[j], x);
            }
            const P nu = vfma(A[2], mz[q], vfma(A[1], v[q], vfma(A[0], u[q], A[9])));
            const P nv = vfma(A[5], mz[q], vfma(A[4], v[q], vfma(A[3], u[q], A[10])));
            const P nz = vfma(A[8], mz[q], vfma(A[7], v[q], vfma(A[6], u[q], A[11])));
            u[q] = nu;
            v[q] = nv;
            mz[q] = nz;
        }
    }

    __device__ __forceinline__ void snapshot(const Op &op) {
        const double cps = (double)op.f[0], sps = (double)op.f[1];
        double *dst = snap + (int64_t)op.adc0 * n_spins * 3;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int64_t s = base + li(i);
            const int qi = i % NP, hi = i / NP;
            if (s < n_spins) {
                const double uu = (double)lane_of(u[qi], hi), vv = (double)lane_of(v[qi], hi);
                dst[3 * s] = uu * cps - vv * sps;
                dst[3 * s + 1] = uu * sps + vv * cps;
                dst[3 * s + 2] = (double)lane_of(mz[qi], hi);
            }
        }
    }

    __device__ __forceinline__ void exec(const Op &op) {
        switch (op.kind) {
        case OP_RF_TRAIN:
            if (maps && (op.flags & F_TMAP))
                train_map(op.tab);
            else
                train_run(op.adc0, op.n);
            break;
        case OP_RF_FAST:  // sub-pulse of a shaped pulse: every cache already holds the right class
            t1_cached();
            rf_turn_op(op);
            rot_w();
            break;
        case OP_RF:
            if (op.flags & F_FRAME) frame_turn(op);
            t1_relax(op);
            rf_turn_op(op);
            if (op.flags & F_PCLS) {
                if (op.flags & F_PLOAD) load_w(op.pcls);
                rot_w();
            }
            if (op.flags & F_ADC) sample_any(op.adc0);
            break;
        case OP_PREC:
            if (op.flags & F_PCLS) {
                if (op.flags & F_PLOAD) load_w(op.pcls);
                rot_w();
            } else if (op.flags & F_INLINE) {
                prec_inline(op);
            }
            if (op.flags & F_ADC) sample_any(op.adc0);
            break;
        case OP_RUN:
            if constexpr (NC > 0)
                run_coils(op);
            else
                run(op);
            break;
        case OP_SNAP:  // bring Mz up to date, then record (Mx, My, Mz) in the laboratory frame
            t1_relax(op);
            if (snap) snapshot(op);
            break;
        default:  // OP_END
            t1_relax(op);
            break;
        }
    }
};

// Shared-memory layout (bytes) of one block; identical on host and device.
struct SmemLayout {
    size_t ops, bars, flag, cw, ce1, ce2, prm, train, red, total;
};
__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
__host__ __device__ inline SmemLayout smem_layout(bool f64, int n_pcls, int n_e1, int n_e2, int n_train, int S,
                                                  int nwarp) {
    SmemLayout L;
    const size_t rs = f64 ? 8 : 4;
    const size_t opb = f64 ? sizeof(OpF64) * 2 * CHUNK_F64 : sizeof(OpF32) * 2 * CHUNK_F32;
    const int nprm = f64 ? 4 : 8;
    size_t o = 0;
    L.ops = o;
    o += opb;
    L.bars = o;
    o += 16;
    L.flag = o;  // abort flag, then 4 words of per-axis coordinate maxima (float bits)
    o += 32;
    L.cw = o;
    o = align_up(o + (size_t)n_pcls * S * 2 * rs, 16);
    L.ce1 = o;
    o = align_up(o + (size_t)n_e1 * S * rs, 16);
    L.ce2 = o;
    o = align_up(o + (size_t)n_e2 * S * rs, 16);
    L.prm = o;
    o = align_up(o + (size_t)nprm * S * rs, 16);
    L.train = o;
    o = align_up(o + (size_t)n_train * 16, 16);  // float32 (c, c, s, s), float64 (c, s)
    L.red = o;
    if (f64)
        o = align_up(o + (size_t)nwarp * 2 * RED_STRIDE * rs, 16);
    else  // transpose tiles, then the block-wide window
        o = align_up(o + (size_t)nwarp * TILE_FLOATS * 4 + (size_t)2 * WIN_STRIDE * 4, 16);
    L.total = o;
    return L;
}

// Barriers of the two op buffers; initialised once per block (thread 0).
__device__ __forceinline__ void init_op_barriers(unsigned char *smem, bool f64) {
    const SmemLayout L = smem_layout(f64, 0, 0, 0, 0, 0, 0);  // ops, bars and flag do not depend on the program
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
}

// One tile of S = K·blockDim spins (spins tile·S ... tile·S + S − 1 of the phantom in `a`) through
// the whole program.  `seq` counts the op chunks this block has staged so far (it selects the
// buffer and the mbarrier phase, so consecutive tiles of a persistent block can reuse the
// barriers).  Returns false if a bounded wait ran out (status recorded, block must stop).
template <typename R, int K, int NC = 0>
__device__ __forceinline__ bool run_tile(const FwdArgs &a, int64_t tile, unsigned char *smem, uint32_t &seq) {
    using SP = Spins<R, K, NC>;
    using Op = typename SP::Op;
    using PV = typename SP::P;
    using CwT = typename SP::CwT;
    constexpr bool F64 = SP::F64;
    constexpr int CH = F64 ? CHUNK_F64 : CHUNK_F32;
    constexpr int LN = SP::L, NP = SP::NP;

    SP sp;
    sp.nthr = blockDim.x;
    sp.tid = threadIdx.x;
    sp.lane = sp.tid & 31;
    sp.warp = sp.tid >> 5;
    sp.nwarp = sp.nthr >> 5;
    sp.S = K * sp.nthr;
    sp.SP = NP * sp.nthr;
    const int S = sp.S, SPK = sp.SP;
    const Program &P = a.prog;
    const SmemLayout L = smem_layout(F64, P.n_pcls, P.n_e1, P.n_e2, P.n_train, S, sp.nwarp);
    Op *opbuf = reinterpret_cast<Op *>(smem + L.ops);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.flag);
    CwT *cw = reinterpret_cast<CwT *>(smem + L.cw);
    PV *ce1 = reinterpret_cast<PV *>(smem + L.ce1);
    PV *ce2 = reinterpret_cast<PV *>(smem + L.ce2);
    PV *prm = reinterpret_cast<PV *>(smem + L.prm);
    unsigned *bmax = reinterpret_cast<unsigned *>(smem + L.flag + 16);
    sp.cw = cw;
    if constexpr (std::is_same<R, dfl>::value) {  // double-float: the table as pairs, converted once here
        dfl *tr = reinterpret_cast<dfl *>(smem + L.train);
        const double2 *gtr = reinterpret_cast<const double2 *>(P.train);
        for (int q = sp.tid; q < P.n_train; q += sp.nthr) {
            const double2 t = gtr[q];
            tr[2 * q] = dfl(t.x);
            tr[2 * q + 1] = dfl(t.y);
        }
        sp.train = tr;
    } else if constexpr (F64) {
        double2 *tr = reinterpret_cast<double2 *>(smem + L.train);
        const double2 *gtr = reinterpret_cast<const double2 *>(P.train);
        for (int q = sp.tid; q < P.n_train; q += sp.nthr) tr[q] = gtr[q];
        sp.train = tr;
    } else {
        float4 *tr = reinterpret_cast<float4 *>(smem + L.train);
        const float2 *gtr = reinterpret_cast<const float2 *>(P.train);
        for (int q = sp.tid; q < P.n_train; q += sp.nthr) {
            const float2 t = gtr[q];
            tr[q] = make_float4(t.x, t.x, t.y, t.y);
        }
        sp.train = tr;
    }
    sp.ce1 = ce1;
    sp.ce2 = ce2;
    sp.prm = prm;
    sp.red = reinterpret_cast<R *>(smem + L.red);
    sp.tile = reinterpret_cast<float *>(smem + L.red) + sp.warp * TILE_FLOATS;
    sp.win = reinterpret_cast<float *>(smem + L.red) + sp.nwarp * TILE_FLOATS;
    if constexpr (!F64)
        for (int q = sp.tid; q < 2 * WIN_STRIDE; q += sp.nthr) sp.win[q] = 0.0f;
    sp.demod = P.demod;
    sp.demod32 = P.demod32;
    sp.signal = a.signal;
    sp.params = a.params;
    sp.maps = static_cast<const R *>(a.maps);
    sp.snap = a.snap;
    sp.win_base = 0;
    sp.win_end = 0;
    if constexpr (NC > 0) {
        sp.n_coils = a.n_coils;
        sp.coil_stride = 2 * P.n_adc;
    }
    sp.base = tile * S;
    sp.np = a.n_pad;
    sp.n_spins = a.n_spins;

    const Op *gops = reinterpret_cast<const Op *>(P.ops);
    const int n_ops = P.n_ops;
    const int n_chunks = (n_ops + CH - 1) / CH;
    // chunk c of this tile is the block's chunk number seq + c: buffer (seq + c) & 1,
    // mbarrier phase ((seq + c) >> 1) & 1
    auto issue = [&](int c) {
        const uint32_t g = seq + (uint32_t)c;
        const int m = min(CH, n_ops - c * CH);
        const uint32_t bytes = (uint32_t)(m * (int)sizeof(Op));
        fence_proxy_async();
        mbar_expect_tx(&bars[g & 1], bytes);
        bulk_g2s(opbuf + (g & 1) * CH, gops + (size_t)c * CH, bytes, &bars[g & 1]);
    };
    if (sp.tid == 0) {
        *abort_flag = 0;
        for (int q = 0; q < 4; ++q) bmax[q] = 0u;
        if (n_chunks > 0) issue(0);
        if (n_chunks > 1) issue(1);
    }

    // ---- per-spin set-up: parameters, class tables (float64 math), initial state -------------
    // Spin i of the thread is lane i / NP of packed value i % NP; a packed table entry holds its
    // lanes' real parts first, then (phasor classes) their imaginary parts.
    const int64_t np = a.n_pad;
    R su[K], sv[K], smz[K], srho[K];
    float amax[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // this thread's max |x_hi|, |y_hi|, |z_hi|, |Δf_hi|
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int l = sp.li(i);
        const int qi = i % NP, hi = i / NP;
        const int64_t s = sp.base + l;
        const bool valid = s < a.n_spins;
        const double x = valid ? a.params[P_X * np + s] : 0.0;
        const double y = valid ? a.params[P_Y * np + s] : 0.0;
        const double z = valid ? a.params[P_Z * np + s] : 0.0;
        const double df = valid ? a.params[P_DF * np + s] : 0.0;
        const double m0 = valid ? a.params[P_RHO * np + s] : 0.0;
        const double r1 = valid ? a.params[P_R1 * np + s] : 0.0;
        const double r2 = valid ? a.params[P_R2 * np + s] : 0.0;
        srho[i] = (R)m0;
        if constexpr (F64) {
            const double vals[4] = {x, y, z, df};
#pragma unroll
            for (int q = 0; q < 4; ++q) reinterpret_cast<R *>(prm + q * SPK + sp.pi(qi))[hi] = vals[q];
        } else {
            const double vals[4] = {x, y, z, df};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float h = (float)vals[q];
                reinterpret_cast<R *>(prm + (2 * q) * SPK + sp.pi(qi))[hi] = h;
                reinterpret_cast<R *>(prm + (2 * q + 1) * SPK + sp.pi(qi))[hi] = (float)(vals[q] - (double)h);
                amax[q] = fmaxf(amax[q], fabsf(h));
            }
        }
        for (int c = 0; c < P.n_pcls; ++c) {
            const double kx = __ldg(P.pcls + 4 * c), ky = __ldg(P.pcls + 4 * c + 1);
            const double kz = __ldg(P.pcls + 4 * c + 2), dt = __ldg(P.pcls + 4 * c + 3);
            double th = kx * x + ky * y + kz * z + df * dt;
            th -= rint(th);
            double sn, cs;
            sincospi(2.0 * th, &sn, &cs);
            const double e2 = exp(-dt * r2);
            R *w = reinterpret_cast<R *>(cw + c * SPK + sp.pi(qi));
            w[hi] = (R)(e2 * cs);
            w[LN + hi] = (R)(-e2 * sn);
        }
        for (int c = 0; c < P.n_e1; ++c)
            reinterpret_cast<R *>(ce1 + c * SPK + sp.pi(qi))[hi] = (R)(-expm1(-__ldg(P.e1 + c) * r1));
        for (int c = 0; c < P.n_e2; ++c)
            reinterpret_cast<R *>(ce2 + c * SPK + sp.pi(qi))[hi] = (R)exp(-__ldg(P.e2 + c) * r2);
        if (a.state_in && valid) {  // laboratory frame = pulse frame ψ = 0 at the start
            su[i] = (R)a.state_in[3 * s];
            sv[i] = (R)a.state_in[3 * s + 1];
            smz[i] = (R)a.state_in[3 * s + 2];
        } else {
            su[i] = (R)0;
            sv[i] = (R)0;
            smz[i] = (R)m0;
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        R lu[LN], lv[LN], lz[LN], lr[LN], one[LN], zero[LN];
#pragma unroll
        for (int h = 0; h < LN; ++h) {
            lu[h] = su[q + h * NP];
            lv[h] = sv[q + h * NP];
            lz[h] = smz[q + h * NP];
            lr[h] = srho[q + h * NP];
            one[h] = (R)1;
            zero[h] = (R)0;
        }
        set_lanes(sp.u[q], lu);
        set_lanes(sp.v[q], lv);
        set_lanes(sp.mz[q], lz);
        set_lanes(sp.rho[q], lr);
        set_lanes(sp.wr[q], one);
        set_lanes(sp.wi[q], zero);
        set_lanes(sp.nwi[q], zero);
        set_lanes(sp.e1v[q], zero);
    }
    if constexpr (NC > 0) {  // sensitivities: [coil][n_pad] (re, im), zero for padding coils/spins
        using V2T = typename std::conditional<F64, double2, float2>::type;
        const V2T *sens = reinterpret_cast<const V2T *>(a.sens);
#pragma unroll
        for (int c = 0; c < SP::NCR; ++c) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                R re[LN], im[LN];
#pragma unroll
                for (int h = 0; h < LN; ++h) {
                    const int64_t s = sp.base + sp.li(q + h * NP);
                    V2T w;
                    w.x = (R)0;
                    w.y = (R)0;
                    if (c < a.n_coils && s < a.n_spins) w = sens[(int64_t)c * np + s];
                    re[h] = w.x;
                    im[h] = w.y;
                }
                set_lanes(sp.cre[c][q], re);
                set_lanes(sp.cim[c][q], im);

            }
        }
    }
    __syncthreads();
    if constexpr (!F64) {
        // block-wide coordinate maxima decide whether the packed phase step is exact for every
        // inline precession of the program (|k_hi|max · |x_hi|max < PHASE_SAFE per axis)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned m = __reduce_max_sync(FULL, __float_as_uint(amax[q]));
            if (sp.lane == 0) atomicMax(bmax + q, m);
        }
        __syncthreads();
        bool big = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) big |= !(P.kmax[q] * __uint_as_float(bmax[q]) < PHASE_SAFE);
        sp.big_phase = big;
        sp.zero_df = bmax[3] == 0u;
    } else {
        sp.big_phase = true;
        sp.zero_df = false;
    }

    // ---- the operation stream ------------------------------------------------------------------
    for (int c = 0; c < n_chunks; ++c) {
        const uint32_t g = seq + (uint32_t)c;
        if (sp.tid == 0) {
            if (!mbar_wait_bounded(&bars[g & 1], (g >> 1) & 1u, WAIT_LIMIT_NS)) {
                atomicCAS(a.status, 0, (int)MRSIM_ETIMEOUT);
                *abort_flag = 1;
            }
        }
        __syncthreads();
        if (*abort_flag) {
            if (sp.tid == 0 && c + 1 < n_chunks)
                mbar_wait_bounded(&bars[(g + 1) & 1], ((g + 1) >> 1) & 1u, WAIT_LIMIT_NS);
            return false;
        }
        const Op *ops = opbuf + (g & 1) * CH;
        const int m = min(CH, n_ops - c * CH);
        for (int o = 0; o < m; ++o) sp.exec(ops[o]);
        __syncthreads();
        if (sp.tid == 0 && c + 2 < n_chunks) issue(c + 2);
    }
    seq += (uint32_t)n_chunks;
    if (sp.win_end > sp.win_base) sp.flush();

    if (a.state_out) {
        // the final OP_END carries the frame angle: (Mx + jMy) = (u + jv)·(cos ψ + j sin ψ)
        const Op &last = gops[n_ops - 1];
        const bool end = last.kind == OP_END;
        const double cps = end ? (double)last.f[0] : 1.0, sps = end ? (double)last.f[1] : 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int64_t s = sp.base + sp.li(i);
            const int qi = i % NP, hi = i / NP;
            if (s < a.n_spins) {
                const double uu = (double)lane_of(sp.u[qi], hi), vv = (double)lane_of(sp.v[qi], hi);
                a.state_out[3 * s] = uu * cps - vv * sps;
                a.state_out[3 * s + 1] = uu * sps + vv * cps;
                a.state_out[3 * s + 2] = (double)lane_of(sp.mz[qi], hi);
            }
        }
    }
    __syncthreads();  // the block's shared memory may be reused by the next tile
    return true;
}

template <typename R, int K, int MAXT, int NC = 0>
__global__ void __launch_bounds__(MAXT, 1) fwd_kernel(const FwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (threadIdx.x == 0) init_op_barriers(smem, is_wide<R>::value);
    uint32_t seq = 0;
    run_tile<R, K, NC>(a, (int64_t)blockIdx.x, smem, seq);
}

// Persistent batch kernel: each block pops (phantom, tile) work items from a global counter
// (dynamic assignment of spin blocks, §5.3.2) until the queue is empty.  Items are ordered
// longest first on the host.  No block waits on another.
template <typename R, int K, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) batch_kernel(const BatchArgs b) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    if (threadIdx.x == 0) init_op_barriers(smem, is_wide<R>::value);
    uint32_t seq = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.head, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= b.n_items) break;
        const BatchItem item = b.items[it];
        const FwdArgs a = b.descs[item.desc];
        if (!run_tile<R, K>(a, (int64_t)item.tile, smem, seq)) return;
    }
}

template <typename R, int K, int MAXT, int NC = 0>
int launch_one(const FwdArgs &a, int threads, void *stream) {
    if (threads <= 0 || threads > MAXT || threads % 32) return (int)cudaErrorInvalidValue;
    if (a.n_spins <= 0) return 0;
    const int S = K * threads;
    const SmemLayout L = smem_layout(is_wide<R>::value, a.prog.n_pcls, a.prog.n_e1, a.prog.n_e2,
                                     a.prog.n_train, S, threads / 32);
    auto kern = fwd_kernel<R, K, MAXT, NC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return (int)e;
    const int64_t grid = (a.n_spins + S - 1) / S;
    if (grid > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    kern<<<(unsigned)grid, threads, L.total, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

template <typename R, int K, int MAXT>
int launch_batch_one(const BatchArgs &b, int threads, size_t smem, int grid, void *stream) {
    if (threads <= 0 || threads > MAXT || threads % 32 || grid <= 0) return (int)cudaErrorInvalidValue;
    auto kern = batch_kernel<R, K, MAXT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    kern<<<grid, threads, smem, (cudaStream_t)stream>>>(b);
    return (int)cudaGetLastError();
}

template <typename R, int K, int MAXT>
int batch_blocks_per_sm(int threads, size_t smem) {
    if (threads <= 0 || threads > MAXT || threads % 32) return 0;
    auto kern = batch_kernel<R, K, MAXT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <typename R, int K, int MAXT>
int blocks_per_sm(int threads, size_t smem) {
    if (threads <= 0 || threads > MAXT || threads % 32) return 0;
    auto kern = fwd_kernel<R, K, MAXT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <typename R, int K, int MAXT>
int regs_of() {
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, fwd_kernel<R, K, MAXT>) != cudaSuccess) return 0;
    return at.numRegs;
}

}  // namespace dev
}  // namespace mrsim
