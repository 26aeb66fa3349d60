// fwd_kernel.cuh -- forward kernel: per-isochromat Bloch propagation + per-sample signal sum.
//
// One thread owns K spins (§5.3.2 domain decomposition: spins are independent) and keeps
// their magnetisation in registers for the whole sequence.  A thread block owns S = K·threads
// spins.  Every thread walks the same compiled operation stream (see internal.h), which thread
// 0 stages into shared memory in chunks with bulk asynchronous copies (cp.async.bulk, completed
// on an mbarrier) while the block computes on the previous chunk.
//
// Per operation (Eq. 4.1: M <- T_Relax·T_grad·T'_HF·M + T_Relax,z):
//   RF   : lazy T1 over the time since the previous pulse, then the Eq. 3.19 rotation;
//   PREC : Mxy <- Mxy·E2·exp(-j2πφ) with φ = k·x + Δf·Δt in cycles (Eqs. 3.5/3.11/3.14);
//   RUN  : n samples of one constant-gradient readout, each Mxy <- Mxy·w (w cached per spin);
//   samples: the sum Σ_spins Mxy (§5.1.1, Eq. 3.32) is reduced in-thread over the K spins,
//            across the warp by a transposed butterfly (16 samples per pass: lane l ends up
//            holding the warp total of value l), across warps in shared memory, and across
//            blocks with float64 atomics after demodulation by exp(-j·adc_phase).
//
// Longitudinal magnetisation is carried as Dz = Mz − M0, so T1 recovery is Dz <- (1 − ε1)·Dz
// with ε1 = 1 − exp(−τ/T1) evaluated accurately (expm1) even for the short sub-pulse spacing of
// shaped pulses, where 1 − E1 would cancel in float32.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "../../include/mrsim.h"
#include "internal.h"

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

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s for one 8 KB chunk: only a fault takes that long
constexpr unsigned FULL = 0xffffffffu;
constexpr int RED_STRIDE = SAMPLE_WINDOW + 16;  // per-component row of the reduction window

// Butterfly that leaves lane l with the warp-wide sum of v[l] (32 values per lane in, 1 out).
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
            v[i] = keep + __shfl_xor_sync(FULL, send, off);
        }
    }
    return v[0];
}

template <typename R>
struct V2;
template <>
struct V2<float> {
    using T = float2;
};
template <>
struct V2<double> {
    using T = double2;
};

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

// Sum the sample window over warps (float64), demodulate by exp(-j·adc_phase) and add the
// block's partial sums to the global signal.  Every thread of the block must call it.
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

template <typename R, int K>
struct Spins {
    using Op = typename std::conditional<std::is_same<R, float>::value, OpF32, OpF64>::type;
    using V = typename V2<R>::T;
    static constexpr bool F64 = std::is_same<R, double>::value;
    static constexpr int NPRM = F64 ? 6 : 10;  // per-spin rows kept in shared memory

    R mx[K], my[K], dz[K], rho[K];
    R wr[K], wi[K];
    R e1v[K];
    int cur_p, cur_e1;
    int win_base, win_end;

    // shared-memory views
    const V *cw;
    const R *ce1, *ce2, *prm;
    R *red;
    int S, nthr, tid, lane, warp, nwarp;
    const double *demod;
    double *signal;

    __device__ __forceinline__ int li(int i) const { return i * nthr + tid; }

    __device__ __forceinline__ void load_w(int c) {
        if (c == cur_p) return;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const V w = cw[c * S + li(i)];
            wr[i] = w.x;
            wi[i] = w.y;
        }
        cur_p = c;
    }
    __device__ __forceinline__ void rot_w() {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const R nx = mx[i] * wr[i] - my[i] * wi[i];
            const R ny = mx[i] * wi[i] + my[i] * wr[i];
            mx[i] = nx;
            my[i] = ny;
        }
    }
    // lazy T1 recovery over the interval since the previous pulse
    __device__ __forceinline__ void t1_relax(const Op &op) {
        if (op.flags & F_E1CLS) {
            if (op.ecls != cur_e1) {
#pragma unroll
                for (int i = 0; i < K; ++i) e1v[i] = ce1[op.ecls * S + li(i)];
                cur_e1 = op.ecls;
            }
#pragma unroll
            for (int i = 0; i < K; ++i) dz[i] = dz[i] - e1v[i] * dz[i];
        } else if (op.flags & F_E1INL) {
            const R tau = (R)op.f[10];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const R r1 = prm[(NPRM - 2) * S + li(i)];
                const R eps = -expm1(-tau * r1);
                dz[i] = dz[i] - eps * dz[i];
            }
        }
    }
    __device__ __forceinline__ void rf(const Op &op) {
        const R r00 = (R)op.f[0], r01 = (R)op.f[1], r02 = (R)op.f[2];
        const R r10 = (R)op.f[3], r11 = (R)op.f[4], r12 = (R)op.f[5];
        const R r20 = (R)op.f[6], r21 = (R)op.f[7], r22 = (R)op.f[8], r22m1 = (R)op.f[9];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            // (Mx, My, Dz + M0) rotated, Dz' = Mz' − M0 = r20 Mx + r21 My + r22 Dz + (r22 − 1) M0
            const R nx = r00 * mx[i] + r01 * my[i] + r02 * dz[i] + r02 * rho[i];
            const R ny = r10 * mx[i] + r11 * my[i] + r12 * dz[i] + r12 * rho[i];
            const R nz = r20 * mx[i] + r21 * my[i] + r22 * dz[i] + r22m1 * rho[i];
            mx[i] = nx;
            my[i] = ny;
            dz[i] = nz;
        }
    }
    // precession by the op's own moment and interval (not a cached class)
    __device__ __forceinline__ void prec_inline(const Op &op) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int l = li(i);
            R e2;
            if (op.flags & F_E2CLS)
                e2 = ce2[op.ecls * S + l];
            else if (op.flags & F_DT)
                e2 = exp(-(R)op.f[F64 ? 3 : 8] * prm[(NPRM - 1) * S + l]);
            else
                e2 = (R)1;
            R sn, cs;
            if constexpr (F64) {
                double th = 0.0;
                if (op.flags & F_KX) th += op.f[0] * prm[0 * S + l];
                if (op.flags & F_KY) th += op.f[1] * prm[1 * S + l];
                if (op.flags & F_KZ) th += op.f[2] * prm[2 * S + l];
                if (op.flags & F_DT) th += op.f[3] * prm[3 * S + l];
                th -= rint(th);
                sincospi(2.0 * th, &sn, &cs);
            } else {
                float err = 0.0f, t = 0.0f;
                if (op.flags & F_KX) t = wrap1(t + ff_term(op.f[0], op.f[1], prm[0 * S + l], prm[1 * S + l], err));
                if (op.flags & F_KY) t = wrap1(t + ff_term(op.f[2], op.f[3], prm[2 * S + l], prm[3 * S + l], err));
                if (op.flags & F_KZ) t = wrap1(t + ff_term(op.f[4], op.f[5], prm[4 * S + l], prm[5 * S + l], err));
                if (op.flags & F_DT) t = wrap1(t + ff_term(op.f[6], op.f[7], prm[6 * S + l], prm[7 * S + l], err));
                t = wrap1(t + err);
                __sincosf(6.283185307179586f * t, &sn, &cs);
            }
            const R ar = e2 * cs, ai = -e2 * sn;
            const R nx = mx[i] * ar - my[i] * ai;
            const R ny = mx[i] * ai + my[i] * ar;
            mx[i] = nx;
            my[i] = ny;
        }
    }

    __device__ __forceinline__ R *red_row(int comp) { return red + warp * 2 * RED_STRIDE + comp * RED_STRIDE; }

    __device__ __forceinline__ void flush() {
        flush_window(red, demod, signal, win_base, win_end, tid, nthr, nwarp);
        win_base = win_end;
    }

    __device__ __forceinline__ void sample1(int j) {
        if (j + 1 - win_base > SAMPLE_WINDOW) flush();
        R sx = mx[0], sy = my[0];
#pragma unroll
        for (int i = 1; i < K; ++i) {
            sx += mx[i];
            sy += my[i];
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            sx += __shfl_xor_sync(FULL, sx, off);
            sy += __shfl_xor_sync(FULL, sy, off);
        }
        if (lane == 0) {
            red_row(0)[j - win_base] = sx;
            red_row(1)[j - win_base] = sy;
        }
        win_end = j + 1;
    }

    __device__ __forceinline__ void run(const Op &op) {
        const int n = op.n, j0 = op.adc0;
        load_w(op.pcls);
        R ax[K], ay[K];
        const bool anchor = (op.flags & F_ANCHOR) != 0;
        if (anchor) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                ax[i] = mx[i];
                ay[i] = my[i];
            }
        }
        if (j0 + n - win_base > SAMPLE_WINDOW) flush();
        R *r0 = red_row(0) + (j0 - win_base);
        R *r1 = red_row(1) + (j0 - win_base);
        for (int t0 = 0; t0 < n; t0 += 16) {
            const int tt = min(16, n - t0);
            R v[32];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                if (t < tt) {
                    rot_w();
                    R sx = mx[0], sy = my[0];
#pragma unroll
                    for (int i = 1; i < K; ++i) {
                        sx += mx[i];
                        sy += my[i];
                    }
                    v[2 * t] = sx;
                    v[2 * t + 1] = sy;
                } else {
                    v[2 * t] = (R)0;
                    v[2 * t + 1] = (R)0;
                }
            }
            const R tot = transpose_reduce32(v, lane);
            if (lane < 2 * tt) ((lane & 1) ? r1 : r0)[t0 + (lane >> 1)] = tot;
        }
        win_end = j0 + n;
        if (anchor) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const V w = cw[op.acls * S + li(i)];
                mx[i] = ax[i] * w.x - ay[i] * w.y;
                my[i] = ax[i] * w.y + ay[i] * w.x;
            }
        }
    }

    __device__ __forceinline__ void exec(const Op &op) {
        switch (op.kind) {
        case OP_RF:
            t1_relax(op);
            rf(op);
            if (op.flags & F_PCLS) {
                load_w(op.pcls);
                rot_w();
            }
            if (op.flags & F_ADC) sample1(op.adc0);
            break;
        case OP_PREC:
            if (op.flags & F_PCLS) {
                load_w(op.pcls);
                for (int r = 0; r < op.n; ++r) rot_w();
            } else if (op.flags & F_INLINE) {
                prec_inline(op);
            }
            if (op.flags & F_ADC) sample1(op.adc0);
            break;
        case OP_RUN:
            run(op);
            break;
        default:  // OP_END
            t1_relax(op);
            break;
        }
    }
};

// Shared-memory layout (bytes) of one block; identical on host and device.
struct SmemLayout {
    size_t ops, bars, flag, cw, ce1, ce2, prm, red, total;
};
__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
__host__ __device__ inline SmemLayout smem_layout(bool f64, int n_pcls, int n_e1, int n_e2, int S, int nwarp) {
    SmemLayout L;
    const size_t rs = f64 ? 8 : 4;
    const size_t opb = f64 ? sizeof(OpF64) * 2 * CHUNK_F64 : sizeof(OpF32) * 2 * CHUNK_F32;
    const int nprm = f64 ? 6 : 10;
    size_t o = 0;
    L.ops = o;
    o += opb;
    L.bars = o;
    o += 16;
    L.flag = o;
    o += 16;
    L.cw = o;
    o = align_up(o + (size_t)n_pcls * S * 2 * rs, 16);
    L.ce1 = o;
    o = align_up(o + (size_t)n_e1 * S * rs, 16);
    L.ce2 = o;
    o = align_up(o + (size_t)n_e2 * S * rs, 16);
    L.prm = o;
    o = align_up(o + (size_t)nprm * S * rs, 16);
    L.red = o;
    o = align_up(o + (size_t)nwarp * 2 * RED_STRIDE * rs, 16);
    L.total = o;
    return L;
}

template <typename R, int K, int MAXT>
__global__ void __launch_bounds__(MAXT) fwd_kernel(const FwdArgs a) {
    using SP = Spins<R, K>;
    using Op = typename SP::Op;
    using V = typename SP::V;
    constexpr bool F64 = SP::F64;
    constexpr int CH = F64 ? CHUNK_F64 : CHUNK_F32;
    extern __shared__ __align__(128) unsigned char smem[];

    SP sp;
    sp.nthr = blockDim.x;
    sp.tid = threadIdx.x;
    sp.lane = sp.tid & 31;
    sp.warp = sp.tid >> 5;
    sp.nwarp = sp.nthr >> 5;
    sp.S = K * sp.nthr;
    const int S = sp.S;
    const Program &P = a.prog;
    const SmemLayout L = smem_layout(F64, P.n_pcls, P.n_e1, P.n_e2, S, sp.nwarp);
    Op *opbuf = reinterpret_cast<Op *>(smem + L.ops);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.flag);
    V *cw = reinterpret_cast<V *>(smem + L.cw);
    R *ce1 = reinterpret_cast<R *>(smem + L.ce1);
    R *ce2 = reinterpret_cast<R *>(smem + L.ce2);
    R *prm = reinterpret_cast<R *>(smem + L.prm);
    sp.cw = cw;
    sp.ce1 = ce1;
    sp.ce2 = ce2;
    sp.prm = prm;
    sp.red = reinterpret_cast<R *>(smem + L.red);
    sp.demod = P.demod;
    sp.signal = a.signal;
    sp.cur_p = -1;
    sp.cur_e1 = -1;
    sp.win_base = 0;
    sp.win_end = 0;

    const Op *gops = reinterpret_cast<const Op *>(P.ops);
    const int n_ops = P.n_ops;
    const int n_chunks = (n_ops + CH - 1) / CH;
    auto issue = [&](int c) {
        const int m = min(CH, n_ops - c * CH);
        const uint32_t bytes = (uint32_t)(m * (int)sizeof(Op));
        fence_proxy_async();
        mbar_expect_tx(&bars[c & 1], bytes);
        bulk_g2s(opbuf + (c & 1) * CH, gops + (size_t)c * CH, bytes, &bars[c & 1]);
    };
    if (sp.tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        *abort_flag = 0;
        if (n_chunks > 0) issue(0);
        if (n_chunks > 1) issue(1);
    }

    // ---- per-spin set-up: parameters, class tables (float64 math), initial state -------------
    const int64_t base = (int64_t)blockIdx.x * S;
    const int64_t np = a.n_pad;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int l = sp.li(i);
        const int64_t s = base + l;
        const bool valid = s < a.n_spins;
        const double x = valid ? a.params[P_X * np + s] : 0.0;
        const double y = valid ? a.params[P_Y * np + s] : 0.0;
        const double z = valid ? a.params[P_Z * np + s] : 0.0;
        const double df = valid ? a.params[P_DF * np + s] : 0.0;
        const double m0 = valid ? a.params[P_RHO * np + s] : 0.0;
        const double r1 = valid ? a.params[P_R1 * np + s] : 0.0;
        const double r2 = valid ? a.params[P_R2 * np + s] : 0.0;
        sp.rho[i] = (R)m0;
        if constexpr (F64) {
            prm[0 * S + l] = x;
            prm[1 * S + l] = y;
            prm[2 * S + l] = z;
            prm[3 * S + l] = df;
            prm[4 * S + l] = r1;
            prm[5 * S + l] = r2;
        } else {
            const double v[4] = {x, y, z, df};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float h = (float)v[q];
                prm[(2 * q) * S + l] = h;
                prm[(2 * q + 1) * S + l] = (float)(v[q] - (double)h);
            }
            prm[8 * S + l] = (float)r1;
            prm[9 * S + l] = (float)r2;
        }
        for (int c = 0; c < P.n_pcls; ++c) {
            const double kx = __ldg(P.pcls + 4 * c), ky = __ldg(P.pcls + 4 * c + 1);
            const double kz = __ldg(P.pcls + 4 * c + 2), dt = __ldg(P.pcls + 4 * c + 3);
            double th = kx * x + ky * y + kz * z + df * dt;
            th -= rint(th);
            double sn, cs;
            sincospi(2.0 * th, &sn, &cs);
            const double e2 = exp(-dt * r2);
            V w;
            w.x = (R)(e2 * cs);
            w.y = (R)(-e2 * sn);
            cw[c * S + l] = w;
        }
        for (int c = 0; c < P.n_e1; ++c) ce1[c * S + l] = (R)(-expm1(-__ldg(P.e1 + c) * r1));
        for (int c = 0; c < P.n_e2; ++c) ce2[c * S + l] = (R)exp(-__ldg(P.e2 + c) * r2);
        if (a.state_in && valid) {
            sp.mx[i] = (R)a.state_in[3 * s];
            sp.my[i] = (R)a.state_in[3 * s + 1];
            sp.dz[i] = (R)(a.state_in[3 * s + 2] - m0);
        } else {
            sp.mx[i] = (R)0;
            sp.my[i] = (R)0;
            sp.dz[i] = (R)0;
        }
    }
    __syncthreads();

    // ---- the operation stream ------------------------------------------------------------------
    for (int c = 0; c < n_chunks; ++c) {
        if (sp.tid == 0) {
            if (!mbar_wait_bounded(&bars[c & 1], (uint32_t)((c >> 1) & 1), WAIT_LIMIT_NS)) {
                atomicCAS(a.status, 0, (int)MRSIM_ETIMEOUT);
                *abort_flag = 1;
            }
        }
        __syncthreads();
        if (*abort_flag) {
            if (sp.tid == 0 && c + 1 < n_chunks) mbar_wait_bounded(&bars[(c + 1) & 1], (uint32_t)(((c + 1) >> 1) & 1), WAIT_LIMIT_NS);
            return;
        }
        const Op *ops = opbuf + (c & 1) * CH;
        const int m = min(CH, n_ops - c * CH);
        for (int o = 0; o < m; ++o) sp.exec(ops[o]);
        __syncthreads();
        if (sp.tid == 0 && c + 2 < n_chunks) issue(c + 2);
    }
    if (sp.win_end > sp.win_base) sp.flush();

    if (a.state_out) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int64_t s = base + sp.li(i);
            if (s < a.n_spins) {
                a.state_out[3 * s] = (double)sp.mx[i];
                a.state_out[3 * s + 1] = (double)sp.my[i];
                a.state_out[3 * s + 2] = (double)sp.dz[i] + (double)a.params[P_RHO * np + s];
            }
        }
    }
}

template <typename R, int K, int MAXT>
int launch_one(const FwdArgs &a, int threads, void *stream) {
    if (threads <= 0 || threads > MAXT || threads % 32) return (int)cudaErrorInvalidValue;
    if (a.n_spins <= 0) return 0;
    const int S = K * threads;
    const SmemLayout L = smem_layout(std::is_same<R, double>::value, a.prog.n_pcls, a.prog.n_e1, a.prog.n_e2, S, threads / 32);
    auto kern = fwd_kernel<R, K, MAXT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return (int)e;
    const int64_t grid = (a.n_spins + S - 1) / S;
    if (grid > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    kern<<<(unsigned)grid, threads, L.total, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace dev
}  // namespace mrsim
