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
//   RUN  : n samples of one constant-gradient readout, each (u + jv) <- (u + jv)·w;
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
constexpr int TILE_STRIDE = 36;                     // float32: row of a warp's 32x32 transpose tile

__device__ __forceinline__ void red_shared_add(float *p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(su32(p)), "f"(v) : "memory");
}

// Shared-memory transpose that leaves lane l with the warp-wide sum of v[l]: every lane writes
// its 32 values down tile column `lane` (32 conflict-free stores that nothing waits on), reads
// tile row l as 8 conflict-free 16-byte loads and adds the 32 values as a tree: 71 instructions
// instead of the 124 of a shuffle butterfly.
__device__ __forceinline__ float tile_reduce32(float (&v)[32], int lane, float *tile) {
#pragma unroll
    for (int i = 0; i < 32; ++i) tile[i * TILE_STRIDE + lane] = v[i];
    __syncwarp();
    float a[32];
    const float4 *row = reinterpret_cast<const float4 *>(tile + lane * TILE_STRIDE);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 t = row[q];
        a[4 * q] = t.x;
        a[4 * q + 1] = t.y;
        a[4 * q + 2] = t.z;
        a[4 * q + 3] = t.w;
    }
    __syncwarp();
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
#pragma unroll
        for (int i = 0; i < w; ++i) a[i] += a[i + w];
    }
    return a[0];
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
            v[i] = keep + __shfl_xor_sync(FULL, send, off);
        }
    }
    return v[0];
}

// Pairwise (tree) sum of K values: log2(K) dependent adds instead of K − 1.
template <typename R, int K>
__device__ __forceinline__ R tree_sum(const R (&a)[K]) {
    if constexpr (K == 1) {
        return a[0];
    } else if constexpr (K == 2) {
        return a[0] + a[1];
    } else if constexpr (K == 4) {
        return (a[0] + a[1]) + (a[2] + a[3]);
    } else {
        static_assert(K == 8, "K must be 1, 2, 4 or 8");
        return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
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

template <typename R, int K>
struct Spins {
    using Op = typename std::conditional<std::is_same<R, float>::value, OpF32, OpF64>::type;
    using V = typename V2<R>::T;
    static constexpr bool F64 = std::is_same<R, double>::value;
    static constexpr int WIN = F64 ? SAMPLE_WINDOW_F64 : SAMPLE_WINDOW_F32;

    R u[K], v[K], mz[K], rho[K];  // transverse part in the pulse frame, longitudinal, M0
    R wr[K], wi[K];               // cached phasor class
    R e1v[K];                     // cached T1 class ε1
    int win_base, win_end;

    // shared-memory views and block geometry
    const V *cw;
    const V *train;  // sub-pulse table (cos α, sin α)
    const R *ce1, *ce2, *prm;
    R *red;       // float64: per-warp window rows
    float *tile;  // float32: this warp's transpose tile
    float *win;   // float32: block-wide window
    int S, nthr, tid, lane, warp, nwarp;
    int64_t base, np, n_spins;
    const double *params;
    const double *demod;
    const float *demod32;
    double *signal;

    __device__ __forceinline__ int li(int i) const { return i * nthr + tid; }

    __device__ __forceinline__ void load_w(int c) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const V w = cw[c * S + li(i)];
            wr[i] = w.x;
            wi[i] = w.y;
        }
    }
    __device__ __forceinline__ void rot_w() {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const R nu = u[i] * wr[i] - v[i] * wi[i];
            const R nv = u[i] * wi[i] + v[i] * wr[i];
            u[i] = nu;
            v[i] = nv;
        }
    }
    __device__ __forceinline__ void t1_cached() {
#pragma unroll
        for (int i = 0; i < K; ++i) mz[i] = mz[i] - e1v[i] * (mz[i] - rho[i]);
    }
    // lazy T1 recovery over the interval since the previous pulse
    __device__ __forceinline__ void t1_relax(const Op &op) {
        if (op.flags & F_E1CLS) {
            if (op.flags & F_E1LOAD) {
#pragma unroll
                for (int i = 0; i < K; ++i) e1v[i] = ce1[op.ecls * S + li(i)];
            }
            t1_cached();
        } else if (op.flags & F_E1INL) {
            const double tau = (double)op.f[10];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int64_t s = base + li(i);
                const double r1 = s < n_spins ? params[P_R1 * np + s] : 0.0;
                const R eps = (R)(-expm1(-tau * r1));
                mz[i] = mz[i] - eps * (mz[i] - rho[i]);
            }
        }
    }
    // hard pulse about the frame's x axis (Eq. 3.19 in the pulse frame)
    __device__ __forceinline__ void rf_turn(R ca, R sa) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const R nv = ca * v[i] + sa * mz[i];
            const R nz = ca * mz[i] - sa * v[i];
            v[i] = nv;
            mz[i] = nz;
        }
    }
    // turn the frame by exp(-jδ) (uniform over spins); float32 uses (hi, lo) constants
    __device__ __forceinline__ void frame_turn(const Op &op) {
        if constexpr (F64) {
            const double c = op.f[2], s = op.f[3];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const double nu = u[i] * c + v[i] * s;
                const double nv = v[i] * c - u[i] * s;
                u[i] = nu;
                v[i] = nv;
            }
        } else {
            const float ch = op.f[2], cl = op.f[3], sh = op.f[4], sl = op.f[5];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const float nu = fmaf(u[i], ch, fmaf(v[i], sh, fmaf(u[i], cl, v[i] * sl)));
                const float nv = fmaf(v[i], ch, -fmaf(u[i], sh, fmaf(u[i], sl, -v[i] * cl)));
                u[i] = nu;
                v[i] = nv;
            }
        }
    }
    // precession by the op's own moment and interval (not a cached class)
    __device__ __forceinline__ void prec_inline(const Op &op) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int l = li(i);
            R e2;
            if (op.flags & F_E2CLS) {
                e2 = ce2[op.ecls * S + l];
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
                // accurate sin/cos of the reduced angle (the hardware approximation's 2^-21 absolute
                // error would accumulate over many inline intervals)
                sincospif(2.0f * t, &sn, &cs);
            }
            const R ar = e2 * cs, ai = -e2 * sn;
            const R nu = u[i] * ar - v[i] * ai;
            const R nv = u[i] * ai + v[i] * ar;
            u[i] = nu;
            v[i] = nv;
        }
    }

    __device__ __forceinline__ R *red_row(int comp) { return red + warp * 2 * RED_STRIDE + comp * RED_STRIDE; }

    __device__ __forceinline__ void flush() {
        if constexpr (F64)
            flush_window(red, demod, signal, win_base, win_end, tid, nthr, nwarp);
        else
            flush_window_f32(win, demod32, signal, win_base, win_end, tid, nthr);
        win_base = win_end;
    }

    __device__ __forceinline__ void sample1(int j) {
        if (j + 1 - win_base > WIN) flush();
        R sx = tree_sum<R, K>(u), sy = tree_sum<R, K>(v);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            sx += __shfl_xor_sync(FULL, sx, off);
            sy += __shfl_xor_sync(FULL, sy, off);
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
    __device__ __forceinline__ R warp_tile_total(R (&vv)[32]) {
        if constexpr (F64)
            return transpose_reduce32(vv, lane);
        else
            return tile_reduce32(vv, lane, tile);
    }
    __device__ __forceinline__ void store_tile(int slot, R tot) {
        if constexpr (F64)
            red_row(lane & 1)[slot + (lane >> 1)] = tot;
        else
            red_shared_add(win + (lane & 1) * WIN_STRIDE + slot + (lane >> 1), tot);
    }

    // one sample step of a run: rotate by the cached class, return the thread's sums
    __device__ __forceinline__ void run_step(R &sx, R &sy) {
        rot_w();
        sx = tree_sum<R, K>(u);
        sy = tree_sum<R, K>(v);
    }

    __device__ __forceinline__ void run(const Op &op) {
        const int n = op.n, j0 = op.adc0;
        if (op.flags & F_PLOAD) load_w(op.pcls);
        R au[K], av[K];
        const bool anchor = (op.flags & F_ANCHOR) != 0;
        if (anchor) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                au[i] = u[i];
                av[i] = v[i];
            }
        }
        if (j0 + n - win_base > WIN) flush();
        const int slot0 = j0 - win_base;
        int t0 = 0;
        for (; t0 + 16 <= n; t0 += 16) {  // full tiles: no guards
            R vv[32];
#pragma unroll
            for (int t = 0; t < 16; ++t) run_step(vv[2 * t], vv[2 * t + 1]);
            store_tile(slot0 + t0, warp_tile_total(vv));
        }
        if (t0 < n) {  // ragged tail
            const int tt = n - t0;
            R vv[32];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                if (t < tt) {
                    run_step(vv[2 * t], vv[2 * t + 1]);
                } else {
                    vv[2 * t] = (R)0;
                    vv[2 * t + 1] = (R)0;
                }
            }
            const R tot = warp_tile_total(vv);
            if (lane < 2 * tt) store_tile(slot0 + t0, tot);
        }
        win_end = j0 + n;
        if (anchor) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const V w = cw[op.acls * S + li(i)];
                u[i] = au[i] * w.x - av[i] * w.y;
                v[i] = au[i] * w.y + av[i] * w.x;
            }
        }
    }

    // n sub-pulses of a shaped pulse (Eq. 3.23): lazy T1 with the cached class, the pulse-frame
    // turn with table entry i, precession by the cached class
    __device__ __forceinline__ void train_run(int off, int n) {
#pragma unroll 2
        for (int i = 0; i < n; ++i) {
            const V cs = train[off + i];
            t1_cached();
            rf_turn(cs.x, cs.y);
            rot_w();
        }
    }

    __device__ __forceinline__ void exec(const Op &op) {
        switch (op.kind) {
        case OP_RF_TRAIN:
            train_run(op.adc0, op.n);
            break;
        case OP_RF_FAST:  // sub-pulse of a shaped pulse: every cache already holds the right class
            t1_cached();
            rf_turn((R)op.f[0], (R)op.f[1]);
            rot_w();
            break;
        case OP_RF:
            if (op.flags & F_FRAME) frame_turn(op);
            t1_relax(op);
            rf_turn((R)op.f[0], (R)op.f[1]);
            if (op.flags & F_PCLS) {
                if (op.flags & F_PLOAD) load_w(op.pcls);
                rot_w();
            }
            if (op.flags & F_ADC) sample1(op.adc0);
            break;
        case OP_PREC:
            if (op.flags & F_PCLS) {
                if (op.flags & F_PLOAD) load_w(op.pcls);
                rot_w();
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
    L.train = o;
    o = align_up(o + (size_t)n_train * 2 * rs, 16);
    L.red = o;
    if (f64)
        o = align_up(o + (size_t)nwarp * 2 * RED_STRIDE * rs, 16);
    else  // transpose tiles, then the block-wide window
        o = align_up(o + (size_t)nwarp * 32 * TILE_STRIDE * 4 + (size_t)2 * WIN_STRIDE * 4, 16);
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
template <typename R, int K>
__device__ __forceinline__ bool run_tile(const FwdArgs &a, int64_t tile, unsigned char *smem, uint32_t &seq) {
    using SP = Spins<R, K>;
    using Op = typename SP::Op;
    using V = typename SP::V;
    constexpr bool F64 = SP::F64;
    constexpr int CH = F64 ? CHUNK_F64 : CHUNK_F32;

    SP sp;
    sp.nthr = blockDim.x;
    sp.tid = threadIdx.x;
    sp.lane = sp.tid & 31;
    sp.warp = sp.tid >> 5;
    sp.nwarp = sp.nthr >> 5;
    sp.S = K * sp.nthr;
    const int S = sp.S;
    const Program &P = a.prog;
    const SmemLayout L = smem_layout(F64, P.n_pcls, P.n_e1, P.n_e2, P.n_train, S, sp.nwarp);
    Op *opbuf = reinterpret_cast<Op *>(smem + L.ops);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.flag);
    V *cw = reinterpret_cast<V *>(smem + L.cw);
    R *ce1 = reinterpret_cast<R *>(smem + L.ce1);
    R *ce2 = reinterpret_cast<R *>(smem + L.ce2);
    R *prm = reinterpret_cast<R *>(smem + L.prm);
    sp.cw = cw;
    {
        V *tr = reinterpret_cast<V *>(smem + L.train);
        const V *gtr = reinterpret_cast<const V *>(P.train);
        for (int q = sp.tid; q < P.n_train; q += sp.nthr) tr[q] = gtr[q];
        sp.train = tr;
    }
    sp.ce1 = ce1;
    sp.ce2 = ce2;
    sp.prm = prm;
    sp.red = reinterpret_cast<R *>(smem + L.red);
    sp.tile = reinterpret_cast<float *>(smem + L.red) + sp.warp * 32 * TILE_STRIDE;
    sp.win = reinterpret_cast<float *>(smem + L.red) + sp.nwarp * 32 * TILE_STRIDE;
    if constexpr (!F64)
        for (int q = sp.tid; q < 2 * WIN_STRIDE; q += sp.nthr) sp.win[q] = 0.0f;
    sp.demod = P.demod;
    sp.demod32 = P.demod32;
    sp.signal = a.signal;
    sp.params = a.params;
    sp.win_base = 0;
    sp.win_end = 0;
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
        if (n_chunks > 0) issue(0);
        if (n_chunks > 1) issue(1);
    }

    // ---- per-spin set-up: parameters, class tables (float64 math), initial state -------------
    const int64_t np = a.n_pad;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int l = sp.li(i);
        const int64_t s = sp.base + l;
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
        } else {
            const double vals[4] = {x, y, z, df};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float h = (float)vals[q];
                prm[(2 * q) * S + l] = h;
                prm[(2 * q + 1) * S + l] = (float)(vals[q] - (double)h);
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
            V w;
            w.x = (R)(e2 * cs);
            w.y = (R)(-e2 * sn);
            cw[c * S + l] = w;
        }
        for (int c = 0; c < P.n_e1; ++c) ce1[c * S + l] = (R)(-expm1(-__ldg(P.e1 + c) * r1));
        for (int c = 0; c < P.n_e2; ++c) ce2[c * S + l] = (R)exp(-__ldg(P.e2 + c) * r2);
        if (a.state_in && valid) {  // laboratory frame = pulse frame ψ = 0 at the start
            sp.u[i] = (R)a.state_in[3 * s];
            sp.v[i] = (R)a.state_in[3 * s + 1];
            sp.mz[i] = (R)a.state_in[3 * s + 2];
        } else {
            sp.u[i] = (R)0;
            sp.v[i] = (R)0;
            sp.mz[i] = (R)m0;
        }
        sp.wr[i] = (R)1;
        sp.wi[i] = (R)0;
        sp.e1v[i] = (R)0;
    }
    __syncthreads();

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
            if (s < a.n_spins) {
                const double uu = (double)sp.u[i], vv = (double)sp.v[i];
                a.state_out[3 * s] = uu * cps - vv * sps;
                a.state_out[3 * s + 1] = uu * sps + vv * cps;
                a.state_out[3 * s + 2] = (double)sp.mz[i];
            }
        }
    }
    __syncthreads();  // the block's shared memory may be reused by the next tile
    return true;
}

template <typename R, int K, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) fwd_kernel(const FwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (threadIdx.x == 0) init_op_barriers(smem, std::is_same<R, double>::value);
    uint32_t seq = 0;
    run_tile<R, K>(a, (int64_t)blockIdx.x, smem, seq);
}

// Persistent batch kernel: each block pops (phantom, tile) work items from a global counter
// (dynamic assignment of spin blocks, §5.3.2) until the queue is empty.  Items are ordered
// longest first on the host.  No block waits on another.
template <typename R, int K, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) batch_kernel(const BatchArgs b) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    if (threadIdx.x == 0) init_op_barriers(smem, std::is_same<R, double>::value);
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

template <typename R, int K, int MAXT>
int launch_one(const FwdArgs &a, int threads, void *stream) {
    if (threads <= 0 || threads > MAXT || threads % 32) return (int)cudaErrorInvalidValue;
    if (a.n_spins <= 0) return 0;
    const int S = K * threads;
    const SmemLayout L = smem_layout(std::is_same<R, double>::value, a.prog.n_pcls, a.prog.n_e1, a.prog.n_e2,
                                     a.prog.n_train, S, threads / 32);
    auto kern = fwd_kernel<R, K, MAXT>;
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
