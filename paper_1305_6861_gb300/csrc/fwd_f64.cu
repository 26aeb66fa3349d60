// fwd_f64.cu -- float64 instantiations of the forward kernel (K = spins per thread).
#include "fwd_kernel.cuh"

namespace mrsim {
namespace dev {
// Diagnostic: the op-stream pipeline's bounded wait on an mbarrier that nothing completes (no copy
// is issued and nobody arrives), so that the timeout path (status word, no fault, the context
// stays usable) can be exercised on purpose.
__global__ void wait_probe_kernel(int *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns)) atomicCAS(status, 0, (int)MRSIM_ETIMEOUT);
}
}  // namespace dev

int launch_wait_probe(int *status, uint64_t limit_ns, void *stream) {
    dev::wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(status, limit_ns);
    return (int)cudaGetLastError();
}

int launch_fwd_f64(const FwdArgs &a, int k, int threads, void *stream) {
    switch (k) {
    case 1: return dev::launch_one<double, 1, 256>(a, threads, stream);
    case 2: return dev::launch_one<double, 2, 256>(a, threads, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

int fwd_regs_f32(int k);
int launch_batch_f32(const BatchArgs &b, int k, int threads, size_t smem, int grid, void *stream);
int batch_blocks_per_sm_f32(int k, int threads, size_t smem);
int launch_batch_df(const BatchArgs &b, int k, int threads, size_t smem, int grid, void *stream);
int batch_blocks_per_sm_df(int k, int threads, size_t smem);
int fwd_blocks_per_sm_df(int k, int threads, size_t smem);
int fwd_regs_df(int k);

int launch_batch(int mode, const BatchArgs &b, int k, int threads, size_t smem, int grid, void *stream) {
    if (mode == MODE_F32) return launch_batch_f32(b, k, threads, smem, grid, stream);
    if (mode == MODE_DF) return launch_batch_df(b, k, threads, smem, grid, stream);
    switch (k) {
    case 1: return dev::launch_batch_one<double, 1, 256>(b, threads, smem, grid, stream);
    case 2: return dev::launch_batch_one<double, 2, 256>(b, threads, smem, grid, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

int batch_blocks_per_sm(int mode, int k, int threads, size_t smem) {
    if (mode == MODE_F32) return batch_blocks_per_sm_f32(k, threads, smem);
    if (mode == MODE_DF) return batch_blocks_per_sm_df(k, threads, smem);
    switch (k) {
    case 1: return dev::batch_blocks_per_sm<double, 1, 256>(threads, smem);
    case 2: return dev::batch_blocks_per_sm<double, 2, 256>(threads, smem);
    default: return 0;
    }
}
int fwd_blocks_per_sm_f32(int k, int threads, size_t smem);
int fwd_blocks_per_sm(int mode, int k, int threads, size_t smem) {
    if (mode == MODE_F32) return fwd_blocks_per_sm_f32(k, threads, smem);
    if (mode == MODE_DF) return fwd_blocks_per_sm_df(k, threads, smem);
    switch (k) {
    case 1: return dev::blocks_per_sm<double, 1, 256>(threads, smem);
    case 2: return dev::blocks_per_sm<double, 2, 256>(threads, smem);
    default: return 0;
    }
}

int fwd_regs(int mode, int k) {
    if (mode == MODE_F32) return fwd_regs_f32(k);
    if (mode == MODE_DF) return fwd_regs_df(k);
    switch (k) {
    case 1: return dev::regs_of<double, 1, 256>();
    case 2: return dev::regs_of<double, 2, 256>();
    default: return 0;
    }
}

size_t fwd_smem_bytes(bool fp64, const Program &p, int k, int threads) {
    return dev::smem_layout(fp64, p.n_pcls, p.n_e1, p.n_e2, p.n_train, k * threads, threads / 32).total;
}

// Validate and pack the seven float64 spin arrays into the parameter block (see internal.h).
__global__ void pack_kernel(int64_t n, int64_t np, const double *x, const double *y, const double *z,
                            const double *rho, const double *t1, const double *t2, const double *dw,
                            double *params, int *bad) {
    const double INV_TWO_PI = 0.15915494309189533577;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const double vx = x[s], vy = y[s], vz = z[s], vr = rho[s], v1 = t1[s], v2 = t2[s], vw = dw[s];
        const bool ok = isfinite(vx) && isfinite(vy) && isfinite(vz) && isfinite(vr) && isfinite(vw) &&
                        v1 > 0.0 && v2 > 0.0 && !isnan(v1) && !isnan(v2);
        if (!ok) atomicMin(bad, (int)min(s, (int64_t)0x7ffffffe));
        params[P_X * np + s] = vx;
        params[P_Y * np + s] = vy;
        params[P_Z * np + s] = vz;
        params[P_DF * np + s] = vw * INV_TWO_PI;
        params[P_RHO * np + s] = vr;
        params[P_R1 * np + s] = isinf(v1) ? 0.0 : 1.0 / v1;
        params[P_R2 * np + s] = isinf(v2) ? 0.0 : 1.0 / v2;
    }
}

__global__ void pack_sens_kernel(int32_t n_coils, int64_t n, int64_t n_pad, const double *src, void *dst, bool f32,
                                 int *bad) {
    const int64_t total = (int64_t)n_coils * n_pad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / n_pad, s = i % n_pad;
        double re = 0.0, im = 0.0;
        if (s < n) {
            re = src[2 * (c * n + s)];
            im = src[2 * (c * n + s) + 1];
            if (!isfinite(re) || !isfinite(im)) atomicMin(bad, (int)min(c * n + s, (int64_t)0x7ffffffe));
        }
        if (f32)
            reinterpret_cast<float2 *>(dst)[i] = make_float2((float)re, (float)im);
        else
            reinterpret_cast<double2 *>(dst)[i] = make_double2(re, im);
    }
}

int pack_sens(int32_t n_coils, int64_t n, int64_t n_pad, const double *src, void *dst, bool f32, int *bad,
              void *stream) {
    const int64_t total = (int64_t)n_coils * n_pad;
    if (total <= 0) return 0;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pack_sens_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n_coils, n, n_pad, src, dst, f32, bad);
    return (int)cudaGetLastError();
}

// Zero the signal buffers of a batch (one launch instead of one memset per phantom).
__global__ void zero_signals_kernel(const FwdArgs *descs, int n) {
    for (int d = 0; d < n; ++d) {
        double *sig = descs[d].signal;
        const int64_t m = 2 * descs[d].prog.n_adc;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
            sig[i] = 0.0;
    }
}

int zero_signals(const FwdArgs *descs, int n, void *stream) {
    if (n <= 0) return 0;
    zero_signals_kernel<<<152, 256, 0, (cudaStream_t)stream>>>(descs, n);
    return (int)cudaGetLastError();
}

int pack_params(int64_t n, int64_t n_pad, const double *x, const double *y, const double *z, const double *rho,
                const double *t1, const double *t2, const double *dw, double *params, int *bad, void *stream) {
    if (n <= 0) return 0;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pack_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, n_pad, x, y, z, rho, t1, t2, dw, params, bad);
    return (int)cudaGetLastError();
}

int launch_fwd_coils_f64(const FwdArgs &a, int threads, void *stream) {
    if (a.n_coils <= 1) return dev::launch_one<double, 1, 256, 1>(a, threads, stream);
    if (a.n_coils <= 2) return dev::launch_one<double, 1, 256, 2>(a, threads, stream);
    if (a.n_coils <= 4) return dev::launch_one<double, 1, 256, 4>(a, threads, stream);
    if (a.n_coils <= MAX_COILS) return dev::launch_one<double, 1, 256, 8>(a, threads, stream);
    return (int)cudaErrorInvalidValue;
}

}  // namespace mrsim
