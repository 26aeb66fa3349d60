// handles.h -- the opaque C-ABI handles (definitions shared by the library's host files).
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mrsim.h"
#include "compiled.h"
#include "internal.h"

using mrsim::BatchItem;
using mrsim::Compiled;
using mrsim::FwdArgs;
using mrsim::Program;

struct TunedShape {
    int k = 0, threads = 0;
    float ms = 0.0f;
};
// Autotuned launch shapes are kept per context, keyed by what determines the kernel's cost:
// precision, spin count and the compiled program's size and class-table sizes.
using TuneKey = std::array<int64_t, 7>;

struct mrsim_ctx {
    std::map<TuneKey, TunedShape> tuned;
    std::string tune_cache;  // MRSIM_AUTOTUNE_CACHE: file that keeps tuned shapes across processes
    int fail_alloc = -1;     // test hook: device allocations left before one fails (-1: off)
    int device = 0;
    int num_sms = 0;
    int max_smem_optin = 0;
    std::string err;
    int *d_status = nullptr;
    // scratch for host-side outputs and inputs, grown on demand
    double *d_sig = nullptr;
    size_t sig_cap = 0;
    double *d_state = nullptr;
    size_t state_cap = 0;
    double *d_stage = nullptr;
    size_t stage_cap = 0;
    double *d_sens = nullptr;  // receive-coil sensitivities in the kernel's layout
    size_t sens_cap = 0;
    double *d_kt = nullptr;    // K-t steps and staged ensemble parameters
    size_t kt_cap = 0;
    double *d_snap = nullptr;  // snapshots for host output
    size_t snap_cap = 0;
    cudaMemPool_t map_pool = nullptr;  // train maps of single-phantom launches: allocated on the call's
                                       // stream and freed after its kernel, so concurrent calls never share
    bool train_maps = true;            // mrsim_context_set_train_maps
    int *d_bad = nullptr;
};

struct mrsim_phantom {
    mrsim_ctx *ctx = nullptr;
    int64_t n = 0, n_pad = 0;
    double *params = nullptr;
    double *d_dir = nullptr;  // static-field direction per spin (3 each), NULL = along z
};

namespace mrsim {
// Device allocation for the library's handles; honours the context's failure-injection hook
// (mrsim_debug_fail_alloc), which makes one chosen allocation report out-of-memory.
inline cudaError_t ctx_malloc(mrsim_ctx *ctx, void **p, size_t bytes) {
    if (ctx && ctx->fail_alloc >= 0 && ctx->fail_alloc-- == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
// Stream-ordered allocation from the context's train-map pool (created on first use; it keeps its
// memory between calls); honours the same failure-injection hook.
inline cudaError_t ctx_malloc_maps(mrsim_ctx *ctx, void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (ctx->fail_alloc >= 0 && ctx->fail_alloc-- == 0) return cudaErrorMemoryAllocation;
    if (!ctx->map_pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        cudaError_t e = cudaMemPoolCreate(&ctx->map_pool, &props);
        if (e != cudaSuccess) {
            ctx->map_pool = nullptr;
            return e;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(ctx->map_pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return cudaMallocFromPoolAsync(p, bytes, ctx->map_pool, st);
}
template <class T>
cudaError_t ctx_malloc(mrsim_ctx *ctx, T **p, size_t bytes) {
    return ctx_malloc(ctx, reinterpret_cast<void **>(p), bytes);
}
// Reports a failed call to the log callback (mrsim_set_log_callback) and, with MRSIM_LOG set, to
// stderr.
void log_failure(mrsim_status st, const std::string &msg);

// A compiled program with the host-side conversions the upload needs (float32 copies of the
// demodulation and sub-pulse tables, the moment bound of the float32 inline phase terms).
struct HostProgram {
    Compiled host;
    std::vector<float> demod32, train32;
    float kmax[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int64_t n_events = 0;
    // the event list and γ/2π it was compiled from (the one-shot adjoint recompiles them with
    // learnable pulses)
    std::vector<mrsim_event> events;
    double gamma = 0.0;
    // every device table in one 256-byte-aligned image, uploaded with a single copy: operations
    // (float32, float64), phasor classes, T1 and T2 classes, demodulation (float64, float32),
    // sub-pulse tables (float32, float64), train-map kinds
    enum Table { OPS32, OPS64, PCLS, E1, E2, DEMOD, DEMOD32, TRAIN32, TRAIN64, TMAP, N_TABLES };
    std::vector<unsigned char> image;
    size_t off[N_TABLES] = {}, len[N_TABLES] = {};
};
}  // namespace mrsim

namespace mrsim {
// mrsim_compile without the handle: compilation plus the host-side conversions of the upload (no
// CUDA call); rf_param / n_params as for compile_sequence.
mrsim_status compile_host(int64_t n_events, const mrsim_event *events, double gamma, int64_t n_snap,
                          const int64_t *snap_after, std::shared_ptr<HostProgram> &out, std::string &err,
                          const int32_t *rf_param = nullptr, int32_t n_params = 0);
}  // namespace mrsim

struct mrsim_compiled {
    std::shared_ptr<const mrsim::HostProgram> prog;
};

struct mrsim_sequence {
    mrsim_ctx *ctx = nullptr;
    int64_t n_events = 0;
    std::shared_ptr<const mrsim::HostProgram> prog;  // shared with the mrsim_compiled it came from
    unsigned char *d_image = nullptr;                 // the program's tables; the pointers below view it
    void *d_ops32 = nullptr, *d_ops64 = nullptr;
    double *d_pcls = nullptr, *d_e1 = nullptr, *d_e2 = nullptr, *d_demod = nullptr;
    float *d_demod32 = nullptr;
    float *d_train32 = nullptr;
    double *d_train64 = nullptr;
    Program p32{}, p64{};
};

struct mrsim_batch {
    mrsim_ctx *ctx = nullptr;
    mrsim_precision prec = MRSIM_FP32;
    std::vector<const mrsim_phantom *> ph;
    std::vector<const mrsim_sequence *> seq;
    std::vector<FwdArgs> descs;
    std::vector<BatchItem> items;
    FwdArgs *d_descs = nullptr;
    BatchItem *d_items = nullptr;
    int *d_head = nullptr;  // work-queue counter
    unsigned char *d_maps = nullptr;  // every phantom's train maps (descs[i].maps points into it)
    int k = 0, threads = 0, grid = 0;
    size_t smem = 0;
    int64_t spin_steps = 0;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t graph = nullptr;
};


namespace mrsim {

// Accepts the three precisions of the C-ABI.  Calls without a compensated kernel (receive
// coils, K-t, non-parallel fields) serve MRSIM_FP32_KAHAN with their float32 kernels: they pass
// fold_kahan = true and get MRSIM_FP32.
inline bool normalize_precision(mrsim_precision &p, bool fold_kahan = false) {
    if (fold_kahan && p == MRSIM_FP32_KAHAN) p = MRSIM_FP32;
    return p == MRSIM_FP64 || p == MRSIM_FP32 || p == MRSIM_FP32_KAHAN;
}

struct Launch {
    int k, threads;
};

// Default launch shape: the largest spins-per-thread that still gives every SM about two blocks.
inline Launch choose_launch(const mrsim_ctx *ctx, bool fp64, int64_t n) {
    static const Launch f32[] = {{4, 128}, {2, 128}, {1, 128}, {1, 64}, {1, 32}};
    static const Launch f64[] = {{1, 128}, {1, 64}, {1, 32}};
    const Launch *c = fp64 ? f64 : f32;
    const int nc = fp64 ? 3 : 5;
    for (int i = 0; i < nc; ++i) {
        const int64_t S = (int64_t)c[i].k * c[i].threads;
        if ((n + S - 1) / S >= 2LL * ctx->num_sms) return c[i];
    }
    return c[nc - 1];
}

}  // namespace mrsim
