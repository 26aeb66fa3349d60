// batch_static.cu -- batched simulation for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they want to simulate: a plug-in whose
// host application owns every device allocation, or a real-time loop that runs under a fixed
// memory budget.  mrsim_simulate_batch_static serves them: it runs the same persistent batch
// kernel as mrsim_batch_launch, but its scratch memory (the work-queue counter, the per-phantom
// descriptors and the work items) lives in one file-scope device array of fixed size that every
// GPU which loads the library holds until the process exits.  Nothing is allocated per call: no
// cudaMalloc, no cudaFree, no allocating library routine; the work list is staged through a
// file-scope host buffer of the same size.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mrsim.h"
#include "handles.h"
#include "internal.h"

using namespace mrsim;

namespace {

constexpr size_t SCRATCH_BYTES = MRSIM_STATIC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;
constexpr size_t HEAD_BYTES = 256;  // work-queue counter, padded so the descriptors stay aligned

// The device scratch: [queue counter | descriptors | work items].
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];
// Host staging of the same layout, and the per-device address of g_scratch.
static unsigned char h_stage[SCRATCH_BYTES];
static void *g_scratch_dev[MAX_DEVICES];
static std::mutex g_mu;

mrsim_status bad(mrsim_ctx *ctx, mrsim_status st, const std::string &m) {
    ctx->err = m;
    return st;
}

// Makes the context's device current for the call and gives the caller's current device back on
// every way out of it.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// The work list of one launch shape in the host staging area, after the descriptors: every
// phantom's tiles, longest sequences first.  Returns MRSIM_OK and the sizes, or the status and a
// message saying which limit was hit.
struct Layout {
    size_t items_off = 0, n_items = 0, smem = 0;
    int per_sm = 0;
};

mrsim_status lay_out(mrsim_ctx *ctx, int n, const mrsim_sequence *const *seqs, const FwdArgs *hd, int mode,
                     const Launch &L, Layout *out, std::string *msg) {
    const bool fp64 = mode != MODE_F32;
    Layout y;
    y.items_off = (HEAD_BYTES + (size_t)n * sizeof(FwdArgs) + 255) / 256 * 256;
    BatchItem *hi = reinterpret_cast<BatchItem *>(h_stage + y.items_off);
    const size_t max_items = (SCRATCH_BYTES - y.items_off) / sizeof(BatchItem);
    const int64_t S = (int64_t)L.k * L.threads;
    // order phantoms by sequence length without allocating: repeated selection of the next longest
    int64_t prev = INT64_MAX;
    int prev_idx = -1;
    for (int done = 0; done < n; ++done) {
        int pick = -1;
        for (int i = 0; i < n; ++i) {
            const int64_t e = seqs[i]->n_events;
            const bool after_prev = e < prev || (e == prev && i > prev_idx);
            if (after_prev && (pick < 0 || e > seqs[pick]->n_events)) pick = i;
        }
        prev = seqs[pick]->n_events;
        prev_idx = pick;
        const int64_t tiles = (hd[pick].n_spins + S - 1) / S;
        if ((int64_t)y.n_items + tiles > (int64_t)max_items) {
            *msg = "batch needs more work items than the static scratch holds (" + std::to_string(max_items) +
                   " with this launch shape)";
            return MRSIM_EINVAL;
        }
        for (int64_t t = 0; t < tiles; ++t) hi[y.n_items++] = BatchItem{pick, (int32_t)t};
        y.smem = std::max(y.smem, fwd_smem_bytes(fp64, hd[pick].prog, L.k, L.threads));
    }
    if (y.smem > (size_t)ctx->max_smem_optin) {
        *msg = "launch shape exceeds shared memory";
        return MRSIM_EUNSUPPORTED;
    }
    y.per_sm = batch_blocks_per_sm(mode, L.k, L.threads, y.smem);
    if (y.per_sm <= 0) {
        *msg = "launch shape cannot be resident";
        return MRSIM_EUNSUPPORTED;
    }
    *out = y;
    return MRSIM_OK;
}

}  // namespace

extern "C" mrsim_status mrsim_simulate_batch_static(mrsim_ctx *ctx, int32_t n, const mrsim_phantom *const *phantoms,
                                                    const mrsim_sequence *const *seqs, mrsim_precision prec,
                                                    void *stream, double *const *signals_out, int32_t spins_per_thread,
                                                    int32_t threads_per_block) {
    if (!ctx) return MRSIM_EINVAL;
    if (n < 0 || (n > 0 && (!phantoms || !seqs || !signals_out))) return bad(ctx, MRSIM_EINVAL, "invalid batch arrays");
    if (!normalize_precision(prec)) return bad(ctx, MRSIM_EINVAL, "unknown precision");
    if (ctx->device < 0 || ctx->device >= MAX_DEVICES) return bad(ctx, MRSIM_EUNSUPPORTED, "device ordinal too large");
    const int mode = launch_mode(prec);
    const bool fp64 = mode != MODE_F32;  // float64 program and layouts (float64, double-float)
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScope scope(ctx->device);
    // set-up, once per device, with that device current: the device address of g_scratch
    if (!g_scratch_dev[ctx->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return bad(ctx, MRSIM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_dev[ctx->device] = p;
    }
    unsigned char *dev = static_cast<unsigned char *>(g_scratch_dev[ctx->device]);
    if (n == 0) return MRSIM_OK;

    // descriptors, written straight into the host staging area
    const size_t desc_bytes = (size_t)n * sizeof(FwdArgs);
    if (HEAD_BYTES + desc_bytes > SCRATCH_BYTES)
        return bad(ctx, MRSIM_EINVAL, "batch of " + std::to_string(n) + " phantoms exceeds the static scratch of " +
                                          std::to_string(SCRATCH_BYTES) + " bytes");
    FwdArgs *hd = reinterpret_cast<FwdArgs *>(h_stage + HEAD_BYTES);
    int64_t max_n = 0;
    for (int i = 0; i < n; ++i) {
        const mrsim_phantom *p = phantoms[i];
        const mrsim_sequence *q = seqs[i];
        if (!p || !q || p->ctx != ctx || q->ctx != ctx)
            return bad(ctx, MRSIM_EINVAL, "batch entry " + std::to_string(i) + ": NULL handle or another context");
        cudaPointerAttributes at;
        if (q->prog->host.n_adc > 0 && (!signals_out[i] || cudaPointerGetAttributes(&at, signals_out[i]) != cudaSuccess ||
                                  (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged))) {
            cudaGetLastError();
            return bad(ctx, MRSIM_EINVAL, "batch entry " + std::to_string(i) + ": signal buffer must be device memory");
        }
        FwdArgs a{};
        a.prog = fp64 ? q->p64 : q->p32;
        a.params = p->params;
        a.n_spins = p->n;
        a.n_pad = p->n_pad;
        a.signal = signals_out[i];
        a.status = ctx->d_status;
        hd[i] = a;
        max_n = std::max(max_n, p->n);
    }
    Launch L = choose_launch(ctx, fp64, max_n);
    const bool library_shape = !spins_per_thread && !threads_per_block;
    if (spins_per_thread) L.k = spins_per_thread;
    if (threads_per_block) L.threads = threads_per_block;
    const bool k_ok = fp64 ? (L.k == 1 || L.k == 2) : (L.k == 1 || L.k == 2 || L.k == 4 || L.k == 8);
    if (!k_ok || L.threads < 32 || L.threads % 32 || L.threads > (fp64 || L.k == 8 ? 256 : 512))
        return bad(ctx, MRSIM_EINVAL, "unsupported spins_per_thread / threads_per_block");

    // work items after the descriptors; the library's own shape falls back to smaller blocks
    // (1 x 64, then 1 x 32) when it does not fit, as mrsim_batch_create does
    Layout y;
    std::string msg;
    mrsim_status ls = lay_out(ctx, n, seqs, hd, mode, L, &y, &msg);
    if (ls == MRSIM_EUNSUPPORTED && library_shape) {
        for (const Launch f : {Launch{1, 64}, Launch{1, 32}}) {
            if ((ls = lay_out(ctx, n, seqs, hd, mode, f, &y, &msg)) != MRSIM_EUNSUPPORTED) {
                L = f;
                break;
            }
        }
    }
    if (ls != MRSIM_OK) return bad(ctx, ls, msg);
    const size_t items_off = y.items_off, n_items = y.n_items, smem = y.smem;
    const int per_sm = y.per_sm;

    cudaStream_t st = (cudaStream_t)stream;
    const size_t used = items_off + n_items * sizeof(BatchItem);
    cudaError_t e = cudaMemcpyAsync(dev + HEAD_BYTES, h_stage + HEAD_BYTES, used - HEAD_BYTES, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, sizeof(int), st);  // the queue counter starts at zero
    if (e != cudaSuccess) return bad(ctx, MRSIM_ECUDA, std::string("stage batch: ") + cudaGetErrorString(e));
    const FwdArgs *dd = reinterpret_cast<const FwdArgs *>(dev + HEAD_BYTES);
    int rc = zero_signals(dd, n, st);
    if (rc != 0 || n_items == 0) return rc ? bad(ctx, MRSIM_ECUDA, "zero signals") : MRSIM_OK;
    BatchArgs a{};
    a.descs = dd;
    a.items = reinterpret_cast<const BatchItem *>(dev + items_off);
    a.n_items = (int32_t)n_items;
    a.head = reinterpret_cast<int *>(dev);
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * ctx->num_sms, (int64_t)n_items);
    rc = launch_batch(mode, a, L.k, L.threads, smem, grid, stream);
    if (rc != 0) return bad(ctx, MRSIM_ECUDA, std::string("launch batch kernel: ") + cudaGetErrorString((cudaError_t)rc));
    return MRSIM_OK;
}
