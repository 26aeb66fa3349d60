// capi.cu -- the C-ABI of libmrsim (see include/mrsim.h): handles, validation, memory, launches.
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mrsim.h"
#include "compiled.h"
#include "handles.h"
#include "internal.h"

using namespace mrsim;


namespace {

std::atomic<mrsim_log_fn> g_log_fn{nullptr};
std::atomic<void *> g_log_user{nullptr};

bool env_log() {
    static const bool on = [] {
        const char *v = std::getenv("MRSIM_LOG");
        return v && *v && std::strcmp(v, "0") != 0;
    }();
    return on;
}

// One NVTX range per public call, visible in nsys / ncu --nvtx timelines (free without a tool).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

mrsim_status fail(mrsim_ctx *ctx, mrsim_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    log_failure(st, msg);
    return st;
}

mrsim_status cuda_fail(mrsim_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, MRSIM_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return fail(ctx, MRSIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

mrsim_status grow(mrsim_ctx *ctx, double **buf, size_t *cap, size_t need_doubles) {
    if (need_doubles <= *cap) return MRSIM_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    size_t n = std::max<size_t>(need_doubles, 1024);
    CK(ctx_malloc(ctx, buf, n * sizeof(double)), "cudaMalloc scratch");
    *cap = n;
    return MRSIM_OK;
}

// The train maps of a single-phantom launch (the program's recurring trains composed per spin),
// allocated on the stream from the context's pool; the caller frees *own on the stream after its
// kernel.  a.maps stays NULL (trains run sub-pulse by sub-pulse) when the program has no map kinds,
// the phantom no spins, or maps are switched off.
mrsim_status prepare_maps(mrsim_ctx *ctx, const mrsim_sequence *seq, int mode, FwdArgs &a, void *stream, void **own) {
    *own = nullptr;
    if (!ctx->train_maps || a.prog.n_tmap <= 0 || a.n_spins <= 0) return MRSIM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    void *m = nullptr;
    cudaError_t e = ctx_malloc_maps(ctx, &m, train_map_bytes(mode, a.prog, a.n_pad), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "train maps");
    const int rc = launch_train_maps(mode, a, seq->d_train64, m, stream);
    if (rc != 0) {
        cudaFreeAsync(m, st);
        return cuda_fail(ctx, (cudaError_t)rc, "train maps");
    }
    a.maps = m;
    *own = m;
    return MRSIM_OK;
}

mrsim_status pack(mrsim_ctx *ctx, int64_t n, const double *const src[7], cudaStream_t st, mrsim_phantom **out) {
    mrsim_phantom *p = new (std::nothrow) mrsim_phantom();
    if (!p) return fail(ctx, MRSIM_ENOMEM, "host allocation failed");
    p->ctx = ctx;
    p->n = n;
    p->n_pad = (n + 31) / 32 * 32;
    if (n > 0) {
        cudaError_t e = ctx_malloc(ctx, &p->params, (size_t)NPARAM * p->n_pad * sizeof(double));
        if (e != cudaSuccess) {
            delete p;
            return cuda_fail(ctx, e, "cudaMalloc phantom");
        }
        const int big = 0x7fffffff;
        cudaMemsetAsync(p->params, 0, (size_t)NPARAM * p->n_pad * sizeof(double), st);  // padding rows = 0
        cudaMemcpyAsync(ctx->d_bad, &big, sizeof(int), cudaMemcpyHostToDevice, st);
        int rc = pack_params(n, p->n_pad, src[0], src[1], src[2], src[3], src[4], src[5], src[6], p->params,
                             ctx->d_bad, st);
        int bad = big;
        if (rc == 0) rc = (int)cudaMemcpyAsync(&bad, ctx->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (rc == 0) rc = (int)cudaStreamSynchronize(st);
        if (rc != 0) {
            cudaFree(p->params);
            delete p;
            return cuda_fail(ctx, (cudaError_t)rc, "pack phantom");
        }
        if (bad != big) {
            cudaFree(p->params);
            delete p;
            return fail(ctx, MRSIM_EINVAL,
                        "spin " + std::to_string(bad) + ": non-finite position/rho/dw or T1/T2 <= 0");
        }
    }
    *out = p;
    return MRSIM_OK;
}

// MRSIM_AUTOTUNE_CACHE: one line per tuned shape, "mrsim-tune-1 <SMs> <key x 7> <K> <threads> <ms>";
// lines of another SM count or malformed ones are ignored.
void load_tune_cache(mrsim_ctx *ctx) {
    std::ifstream in(ctx->tune_cache);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream is(line);
        std::string tag;
        int sms = 0;
        TuneKey key{};
        TunedShape sh;
        if (!(is >> tag >> sms) || tag != "mrsim-tune-1" || sms != ctx->num_sms) continue;
        bool ok = true;
        for (auto &v : key) ok = ok && static_cast<bool>(is >> v);
        if (ok && (is >> sh.k >> sh.threads >> sh.ms) && sh.k > 0 && sh.threads > 0) ctx->tuned[key] = sh;
    }
}

void save_tune_entry(const mrsim_ctx *ctx, const TuneKey &key, const TunedShape &sh) {
    if (ctx->tune_cache.empty()) return;
    std::ostringstream os;
    os << "mrsim-tune-1 " << ctx->num_sms;
    for (int64_t v : key) os << ' ' << v;
    os << ' ' << sh.k << ' ' << sh.threads << ' ' << sh.ms << '\n';
    std::ofstream out(ctx->tune_cache, std::ios::app);  // one short append per entry
    out << os.str();
}

TuneKey tune_key(mrsim_precision prec, const mrsim_phantom *ph, const mrsim_sequence *seq) {
    const Compiled &c = seq->prog->host;
    return TuneKey{(int64_t)prec, ph->n, (int64_t)c.ops32.size(), c.n_pcls, c.n_e1, c.n_e2,
                   c.n_adc * 4096 + (int64_t)c.train.size()};
}


}  // namespace

void mrsim::log_failure(mrsim_status st, const std::string &msg) {
    if (mrsim_log_fn f = g_log_fn.load()) f(st, msg.c_str(), g_log_user.load());
    if (env_log()) std::fprintf(stderr, "mrsim: %s: %s\n", mrsim_status_string(st), msg.c_str());
}

extern "C" {

const char *mrsim_status_string(mrsim_status s) {
    switch (s) {
    case MRSIM_OK: return "ok";
    case MRSIM_EINVAL: return "invalid argument";
    case MRSIM_ENOMEM: return "out of memory";
    case MRSIM_ECUDA: return "CUDA error";
    case MRSIM_ETIMEOUT: return "device wait timed out";
    case MRSIM_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

void mrsim_set_log_callback(mrsim_log_fn fn, void *user) {
    g_log_user.store(user);
    g_log_fn.store(fn);
}

mrsim_status mrsim_debug_fail_alloc(mrsim_ctx *ctx, int32_t after) {
    if (!ctx) return MRSIM_EINVAL;
    ctx->fail_alloc = after < 0 ? -1 : after;
    return MRSIM_OK;
}

mrsim_status mrsim_context_set_train_maps(mrsim_ctx *ctx, int32_t enable) {
    if (!ctx) return MRSIM_EINVAL;
    ctx->train_maps = enable != 0;
    return MRSIM_OK;
}

mrsim_status mrsim_debug_wait_timeout(mrsim_ctx *ctx, int64_t limit_ns, void *stream) {
    if (!ctx) return MRSIM_EINVAL;
    if (limit_ns < 1000 || limit_ns > 1000000000) return fail(ctx, MRSIM_EINVAL, "limit_ns must be in [1e3, 1e9]");
    cudaSetDevice(ctx->device);
    const int rc = launch_wait_probe(ctx->d_status, (uint64_t)limit_ns, stream);
    if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "wait probe");
    return MRSIM_OK;
}

const char *mrsim_last_error(const mrsim_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mrsim_status mrsim_context_create(int device, mrsim_ctx **out) {
    if (!out) return MRSIM_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return MRSIM_EUNSUPPORTED;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MRSIM_ECUDA;
    if (prop.major != 10 || prop.minor != 3) return MRSIM_EUNSUPPORTED;  // built for sm_103a only
    if (cudaSetDevice(device) != cudaSuccess) return MRSIM_ECUDA;
    mrsim_ctx *ctx = new (std::nothrow) mrsim_ctx();
    if (!ctx) return MRSIM_ENOMEM;
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    if (const char *cache = std::getenv("MRSIM_AUTOTUNE_CACHE")) {
        ctx->tune_cache = cache;
        load_tune_cache(ctx);
    }
    if (const char *f = std::getenv("MRSIM_FAIL_ALLOC")) {  // the allocation-failure hook, armed for every context
        char *end = nullptr;
        const long v = std::strtol(f, &end, 10);
        if (end != f && v >= 0 && v <= INT32_MAX) ctx->fail_alloc = (int32_t)v;
    }
    cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&ctx->d_bad, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(ctx->d_status);
        cudaFree(ctx->d_bad);
        delete ctx;
        return MRSIM_ENOMEM;
    }
    *out = ctx;
    return MRSIM_OK;
}

void mrsim_context_destroy(mrsim_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_bad);
    cudaFree(ctx->d_sig);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_stage);
    cudaFree(ctx->d_sens);
    cudaFree(ctx->d_kt);
    cudaFree(ctx->d_snap);
    if (ctx->map_pool) cudaMemPoolDestroy(ctx->map_pool);  // released once its last allocation is freed
    delete ctx;
}

mrsim_status mrsim_stream_status(mrsim_ctx *ctx, void *stream) {
    if (!ctx) return MRSIM_EINVAL;
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
    int st = 0;
    CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (st != 0) {
        cudaMemset(ctx->d_status, 0, sizeof(int));
        return fail(ctx, (mrsim_status)st, "a kernel reported a device-side failure");
    }
    return MRSIM_OK;
}

mrsim_status mrsim_phantom_create(mrsim_ctx *ctx, int64_t n, const double *x, const double *y, const double *z,
                                  const double *rho, const double *t1, const double *t2, const double *dw,
                                  mrsim_phantom **out) {
    Range nvtx_range("mrsim_phantom_create");
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (n < 0) return fail(ctx, MRSIM_EINVAL, "n_spins < 0");
    const double *src[7] = {x, y, z, rho, t1, t2, dw};
    if (n > 0)
        for (auto p : src)
            if (!p) return fail(ctx, MRSIM_EINVAL, "NULL spin array");
    cudaSetDevice(ctx->device);
    mrsim_status st = grow(ctx, &ctx->d_stage, &ctx->stage_cap, (size_t)7 * (size_t)std::max<int64_t>(n, 1));
    if (st != MRSIM_OK) return st;
    const double *dsrc[7];
    for (int i = 0; i < 7; ++i) {
        double *dst = ctx->d_stage + (size_t)i * (size_t)n;
        if (n > 0) CK(cudaMemcpyAsync(dst, src[i], (size_t)n * sizeof(double), cudaMemcpyDefault, 0), "copy spins");
        dsrc[i] = dst;
    }
    return pack(ctx, n, dsrc, 0, out);
}

mrsim_status mrsim_phantom_create_device(mrsim_ctx *ctx, int64_t n, const double *x, const double *y,
                                         const double *z, const double *rho, const double *t1, const double *t2,
                                         const double *dw, void *stream, mrsim_phantom **out) {
    Range nvtx_range("mrsim_phantom_create_device");
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (n < 0) return fail(ctx, MRSIM_EINVAL, "n_spins < 0");
    const double *src[7] = {x, y, z, rho, t1, t2, dw};
    if (n > 0)
        for (auto p : src)
            if (!p || !is_device_ptr(p)) return fail(ctx, MRSIM_EINVAL, "spin arrays must be device pointers");
    cudaSetDevice(ctx->device);
    return pack(ctx, n, src, (cudaStream_t)stream, out);
}

int64_t mrsim_phantom_num_spins(const mrsim_phantom *p) { return p ? p->n : -1; }

void mrsim_phantom_destroy(mrsim_phantom *p) {
    if (!p) return;
    cudaSetDevice(p->ctx->device);
    cudaFree(p->params);
    cudaFree(p->d_dir);
    delete p;
}

mrsim_status mrsim_sequence_load(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events, double gamma,
                                 mrsim_sequence **out) {
    return mrsim_sequence_load_snapshots(ctx, n_events, events, gamma, 0, nullptr, out);
}

int64_t mrsim_sequence_num_snapshots(const mrsim_sequence *s) { return s ? s->prog->host.n_snap : -1; }

}  // extern "C"

namespace {
thread_local std::string t_compile_err;  // mrsim_compile's message, per calling thread
}  // namespace

// Compilation plus the host-side conversions of the upload; no CUDA call.
mrsim_status mrsim::compile_host(int64_t n_events, const mrsim_event *events, double gamma, int64_t n_snap,
                                 const int64_t *snap_after, std::shared_ptr<HostProgram> &out, std::string &err,
                                 const int32_t *rf_param, int32_t n_params) {
    std::shared_ptr<HostProgram> c;
    try {
        c = std::make_shared<HostProgram>();
        int rc = compile_sequence(events, n_events, gamma, c->host, err, n_snap, snap_after, rf_param, n_params);
        if (rc != MRSIM_OK) return (mrsim_status)rc;
        c->n_events = n_events;
        if (n_events > 0) c->events.assign(events, events + n_events);
        c->gamma = gamma;
        c->demod32.assign(c->host.demod.begin(), c->host.demod.end());
        c->train32.assign(c->host.train.begin(), c->host.train.end());
        for (const OpF32 &o : c->host.ops32)  // magnitude bound of the float32 inline phase terms
            if ((o.kind == OP_PREC || o.kind == OP_RUN) && (o.flags & F_INLINE))
                for (int a = 0; a < 4; ++a) c->kmax[a] = std::max(c->kmax[a], std::fabs(o.f[2 * a]));
        const Compiled &h = c->host;
        const void *src[HostProgram::N_TABLES] = {h.ops32.data(), h.ops64.data(), h.pcls.data(), h.e1.data(),
                                                  h.e2.data(), h.demod.data(), c->demod32.data(),
                                                  c->train32.data(), h.train.data(), h.tmap.data()};
        const size_t bytes[HostProgram::N_TABLES] = {
            h.ops32.size() * sizeof(OpF32), h.ops64.size() * sizeof(OpF64), h.pcls.size() * sizeof(double),
            h.e1.size() * sizeof(double),   h.e2.size() * sizeof(double),    h.demod.size() * sizeof(double),
            c->demod32.size() * sizeof(float), c->train32.size() * sizeof(float), h.train.size() * sizeof(double),
            h.tmap.size() * sizeof(int32_t)};
        size_t o = 0;
        for (int t = 0; t < HostProgram::N_TABLES; ++t) {
            c->off[t] = o;
            c->len[t] = bytes[t];
            o = (o + bytes[t] + 255) / 256 * 256;
        }
        c->image.assign(o, 0);
        for (int t = 0; t < HostProgram::N_TABLES; ++t)
            if (bytes[t]) std::memcpy(c->image.data() + c->off[t], src[t], bytes[t]);
    } catch (const std::bad_alloc &) {
        err = "host allocation failed";
        return MRSIM_ENOMEM;
    }
    out = std::move(c);
    return MRSIM_OK;
}

extern "C" {

mrsim_status mrsim_compile(int64_t n_events, const mrsim_event *events, double gamma, int64_t n_snap,
                           const int64_t *snap_after, mrsim_compiled **out) {
    Range nvtx_range("mrsim_compile");
    t_compile_err.clear();
    if (!out) {
        t_compile_err = "NULL output handle";
        return MRSIM_EINVAL;
    }
    *out = nullptr;
    if (n_events > 0 && is_device_ptr(events)) {
        t_compile_err = "events must be in host memory";
        return MRSIM_EINVAL;
    }
    std::shared_ptr<HostProgram> prog;
    std::string err;
    mrsim_status rc = compile_host(n_events, events, gamma, n_snap, snap_after, prog, err);
    if (rc != MRSIM_OK) {
        t_compile_err = err;
        log_failure(rc, err);
        return rc;
    }
    mrsim_compiled *c = new (std::nothrow) mrsim_compiled();
    if (!c) {
        t_compile_err = "host allocation failed";
        return MRSIM_ENOMEM;
    }
    c->prog = std::move(prog);
    *out = c;
    return MRSIM_OK;
}

const char *mrsim_compile_last_error(void) { return t_compile_err.c_str(); }

int64_t mrsim_compiled_num_adc(const mrsim_compiled *c) { return c ? c->prog->host.n_adc : -1; }

int64_t mrsim_compiled_upload_bytes(const mrsim_compiled *c) { return c ? (int64_t)c->prog->image.size() : -1; }

void mrsim_compiled_destroy(mrsim_compiled *c) { delete c; }

mrsim_status mrsim_sequence_create(mrsim_ctx *ctx, const mrsim_compiled *c, mrsim_sequence **out) {
    Range nvtx_range("mrsim_sequence_create");
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (!c) return fail(ctx, MRSIM_EINVAL, "NULL compiled program");
    mrsim_sequence *s = new (std::nothrow) mrsim_sequence();
    if (!s) return fail(ctx, MRSIM_ENOMEM, "host allocation failed");
    s->ctx = ctx;
    s->prog = c->prog;
    s->n_events = c->prog->n_events;
    const HostProgram &h = *s->prog;
    cudaSetDevice(ctx->device);
    if (!h.image.empty()) {  // one allocation and one copy for every table
        cudaError_t e = ctx_malloc(ctx, &s->d_image, h.image.size());
        if (e == cudaSuccess) e = cudaMemcpy(s->d_image, h.image.data(), h.image.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            mrsim_sequence_destroy(s);
            return cuda_fail(ctx, e, "upload sequence");
        }
    }
    auto at = [&](HostProgram::Table t) -> void * { return h.len[t] ? (void *)(s->d_image + h.off[t]) : nullptr; };
    s->d_ops32 = at(HostProgram::OPS32);
    s->d_ops64 = at(HostProgram::OPS64);
    s->d_pcls = (double *)at(HostProgram::PCLS);
    s->d_e1 = (double *)at(HostProgram::E1);
    s->d_e2 = (double *)at(HostProgram::E2);
    s->d_demod = (double *)at(HostProgram::DEMOD);
    s->d_demod32 = (float *)at(HostProgram::DEMOD32);
    s->d_train32 = (float *)at(HostProgram::TRAIN32);
    s->d_train64 = (double *)at(HostProgram::TRAIN64);
    Program p{};
    p.n_ops = (int32_t)h.host.ops32.size();
    p.n_pcls = h.host.n_pcls;
    p.n_e1 = h.host.n_e1;
    p.n_e2 = h.host.n_e2;
    p.pcls = s->d_pcls;
    p.e1 = s->d_e1;
    p.e2 = s->d_e2;
    p.demod = s->d_demod;
    p.demod32 = s->d_demod32;
    p.n_train = (int32_t)(h.host.train.size() / 2);
    p.n_adc = h.host.n_adc;
    for (int a = 0; a < 4; ++a) p.kmax[a] = h.kmax[a];
    p.tmap = (const int32_t *)at(HostProgram::TMAP);
    p.n_tmap = (int32_t)(h.host.tmap.size() / 4);
    s->p32 = p;
    s->p32.ops = s->d_ops32;
    s->p32.train = s->d_train32;
    s->p64 = p;
    s->p64.ops = s->d_ops64;
    s->p64.train = s->d_train64;
    *out = s;
    return MRSIM_OK;
}

mrsim_status mrsim_sequence_load_snapshots(mrsim_ctx *ctx, int64_t n_events, const mrsim_event *events,
                                           double gamma, int64_t n_snap, const int64_t *snap_after,
                                           mrsim_sequence **out) {
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (n_events > 0 && is_device_ptr(events)) return fail(ctx, MRSIM_EINVAL, "events must be in host memory");
    mrsim_compiled c;
    std::shared_ptr<HostProgram> prog;
    std::string err;
    mrsim_status rc = compile_host(n_events, events, gamma, n_snap, snap_after, prog, err);
    if (rc != MRSIM_OK) return fail(ctx, rc, err);
    c.prog = std::move(prog);
    return mrsim_sequence_create(ctx, &c, out);
}

int64_t mrsim_sequence_num_adc(const mrsim_sequence *s) { return s ? s->prog->host.n_adc : -1; }
int64_t mrsim_sequence_num_events(const mrsim_sequence *s) { return s ? s->n_events : -1; }
int64_t mrsim_sequence_num_ops(const mrsim_sequence *s) { return s ? (int64_t)s->prog->host.ops32.size() : -1; }

int64_t mrsim_sequence_num_pulses(const mrsim_sequence *s) {
    if (!s) return -1;
    int64_t n = 0;
    for (const mrsim_event &e : s->prog->events) n += e.rf_flip != 0.0;
    return n;
}

void mrsim_sequence_destroy(mrsim_sequence *s) {
    if (!s) return;
    cudaSetDevice(s->ctx->device);
    cudaFree(s->d_image);
    delete s;
}

mrsim_status mrsim_simulate_ex(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                               mrsim_precision prec, void *stream, double *signal_out, int64_t n_adc,
                               const mrsim_options *opt) {
    Range nvtx_range("mrsim_simulate");
    if (!ctx) return MRSIM_EINVAL;
    if (!ph || !seq) return fail(ctx, MRSIM_EINVAL, "NULL phantom or sequence");
    if (ph->ctx != ctx || seq->ctx != ctx) return fail(ctx, MRSIM_EINVAL, "handle belongs to another context");
    if (!normalize_precision(prec)) return fail(ctx, MRSIM_EINVAL, "unknown precision");
    if (n_adc != seq->prog->host.n_adc)
        return fail(ctx, MRSIM_EINVAL, "n_adc = " + std::to_string(n_adc) + " but the sequence has " +
                                           std::to_string(seq->prog->host.n_adc) + " samples");
    if (n_adc > 0 && !signal_out) return fail(ctx, MRSIM_EINVAL, "NULL signal_out");
    const int mode = launch_mode(prec);
    const bool fp64 = mode != MODE_F32;  // float64 program and layouts (float64, double-float)
    mrsim_options o{};
    if (opt) o = *opt;
    if ((o.flags & MRSIM_TUNE) && !o.spins_per_thread && !o.threads_per_block &&
        !ctx->tuned.count(tune_key(prec, ph, seq))) {
        mrsim_options t{};
        mrsim_status ts = mrsim_autotune(ctx, ph, seq, prec, stream, &t);
        if (ts != MRSIM_OK) return ts;
    }
    Launch L = choose_launch(ctx, fp64, ph->n);
    auto tu = ctx->tuned.find(tune_key(prec, ph, seq));
    if (tu != ctx->tuned.end()) L = Launch{tu->second.k, tu->second.threads};
    if (o.spins_per_thread) L.k = o.spins_per_thread;
    if (o.threads_per_block) L.threads = o.threads_per_block;
    const bool k_ok = fp64 ? (L.k == 1 || L.k == 2) : (L.k == 1 || L.k == 2 || L.k == 4 || L.k == 8);
    if (!k_ok || L.threads < 32 || L.threads % 32 || L.threads > (fp64 || L.k == 8 ? 256 : 512))
        return fail(ctx, MRSIM_EINVAL, "unsupported spins_per_thread / threads_per_block");
    const Program &P = fp64 ? seq->p64 : seq->p32;
    if (fwd_smem_bytes(fp64, P, L.k, L.threads) > (size_t)ctx->max_smem_optin)
        return fail(ctx, MRSIM_EUNSUPPORTED, "shared memory of this launch shape exceeds the device limit");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t sig_bytes = (size_t)2 * (size_t)n_adc * sizeof(double);
    const bool host_sig = n_adc > 0 && !is_device_ptr(signal_out);
    double *dsig = signal_out;
    mrsim_status rs;
    if (host_sig) {
        if ((rs = grow(ctx, &ctx->d_sig, &ctx->sig_cap, 2 * (size_t)n_adc)) != MRSIM_OK) return rs;
        dsig = ctx->d_sig;
        if (o.flags & MRSIM_ACCUMULATE)
            CK(cudaMemcpyAsync(dsig, signal_out, sig_bytes, cudaMemcpyHostToDevice, st), "copy signal in");
    }
    if (n_adc > 0 && !(o.flags & MRSIM_ACCUMULATE)) CK(cudaMemsetAsync(dsig, 0, sig_bytes, st), "clear signal");
    // state in / out (host buffers go through one scratch area: [in | out])
    const size_t st_n = (size_t)3 * (size_t)ph->n;
    const bool host_in = o.state_in && !is_device_ptr(o.state_in);
    const bool host_out = o.state_out && !is_device_ptr(o.state_out);
    const double *din = o.state_in;
    double *dout = o.state_out;
    if (host_in || host_out) {
        if ((rs = grow(ctx, &ctx->d_state, &ctx->state_cap, 2 * std::max<size_t>(st_n, 1))) != MRSIM_OK) return rs;
        if (host_in) {
            CK(cudaMemcpyAsync(ctx->d_state, o.state_in, st_n * sizeof(double), cudaMemcpyHostToDevice, st), "copy state in");
            din = ctx->d_state;
        }
        if (host_out) dout = ctx->d_state + st_n;
    }
    // snapshots (host buffers go through their own scratch)
    const size_t snap_n = (size_t)seq->prog->host.n_snap * 3 * (size_t)ph->n;
    double *dsnap = o.snapshots;
    const bool host_snap = o.snapshots && snap_n > 0 && !is_device_ptr(o.snapshots);
    if (host_snap) {
        if ((rs = grow(ctx, &ctx->d_snap, &ctx->snap_cap, snap_n)) != MRSIM_OK) return rs;
        dsnap = ctx->d_snap;
    }
    FwdArgs a{};
    a.prog = P;
    a.params = ph->params;
    a.n_spins = ph->n;
    a.n_pad = ph->n_pad;
    a.state_in = din;
    a.state_out = dout;
    a.snap = snap_n > 0 ? dsnap : nullptr;
    a.signal = dsig;
    a.status = ctx->d_status;
    void *maps = nullptr;
    if ((rs = prepare_maps(ctx, seq, mode, a, stream, &maps)) != MRSIM_OK) return rs;
    int rc = mode == MODE_F64 ? launch_fwd_f64(a, L.k, L.threads, stream)
             : mode == MODE_DF ? launch_fwd_df(a, L.k, L.threads, stream)
                               : launch_fwd_f32(a, L.k, L.threads, stream);
    if (maps) cudaFreeAsync(maps, st);
    if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "launch forward kernel");
    if (host_out) CK(cudaMemcpyAsync(o.state_out, dout, st_n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy state out");
    if (host_snap) CK(cudaMemcpyAsync(o.snapshots, dsnap, snap_n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy snapshots");
    if (host_sig) CK(cudaMemcpyAsync(signal_out, dsig, sig_bytes, cudaMemcpyDeviceToHost, st), "copy signal out");
    if (host_sig || host_out || host_snap) return mrsim_stream_status(ctx, stream);
    return MRSIM_OK;
}

mrsim_status mrsim_simulate_coils(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq,
                                  mrsim_precision prec, void *stream, int32_t n_coils, const double *sens,
                                  double *signal_out, int64_t n_adc) {
    Range nvtx_range("mrsim_simulate_coils");
    if (!ctx) return MRSIM_EINVAL;
    if (!ph || !seq) return fail(ctx, MRSIM_EINVAL, "NULL phantom or sequence");
    if (ph->ctx != ctx || seq->ctx != ctx) return fail(ctx, MRSIM_EINVAL, "handle belongs to another context");
    if (!normalize_precision(prec, true)) return fail(ctx, MRSIM_EINVAL, "unknown precision");
    if (n_coils < 1 || n_coils > MAX_COILS)
        return fail(ctx, MRSIM_EINVAL, "n_coils must be 1.." + std::to_string(MAX_COILS));
    if (n_adc != seq->prog->host.n_adc)
        return fail(ctx, MRSIM_EINVAL, "n_adc = " + std::to_string(n_adc) + " but the sequence has " +
                                           std::to_string(seq->prog->host.n_adc) + " samples");
    if (ph->n > 0 && !sens) return fail(ctx, MRSIM_EINVAL, "NULL sensitivities");
    if (n_adc > 0 && !signal_out) return fail(ctx, MRSIM_EINVAL, "NULL signal buffer");
    const bool fp64 = prec == MRSIM_FP64;
    const int threads = 128, k = fp64 ? 1 : coil_spins_per_thread_f32(n_coils);
    const Program &P = fp64 ? seq->p64 : seq->p32;
    if (fwd_smem_bytes(fp64, P, k, threads) > (size_t)ctx->max_smem_optin)
        return fail(ctx, MRSIM_EUNSUPPORTED, "shared memory of this program exceeds the device limit");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    mrsim_status rs;
    // sensitivities into the kernel's layout (validated on the device)
    const int64_t n = ph->n;
    const double *dsrc = sens;
    if (n > 0 && !is_device_ptr(sens)) {
        if ((rs = grow(ctx, &ctx->d_stage, &ctx->stage_cap, (size_t)2 * n_coils * (size_t)n)) != MRSIM_OK) return rs;
        CK(cudaMemcpyAsync(ctx->d_stage, sens, sizeof(double) * 2 * (size_t)n_coils * (size_t)n, cudaMemcpyHostToDevice, st),
           "copy sensitivities");
        dsrc = ctx->d_stage;
    }
    const size_t sens_doubles = (size_t)n_coils * (size_t)ph->n_pad * (fp64 ? 2 : 1);
    if ((rs = grow(ctx, &ctx->d_sens, &ctx->sens_cap, std::max<size_t>(sens_doubles, 1))) != MRSIM_OK) return rs;
    if (n > 0) {
        const int big = 0x7fffffff;
        int bad = big;
        CK(cudaMemcpyAsync(ctx->d_bad, &big, sizeof(int), cudaMemcpyHostToDevice, st), "reset check");
        const int rc = pack_sens(n_coils, n, ph->n_pad, dsrc, ctx->d_sens, !fp64, ctx->d_bad, st);
        if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "pack sensitivities");
        CK(cudaMemcpyAsync(&bad, ctx->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read check");
        CK(cudaStreamSynchronize(st), "stream synchronize");
        if (bad != big) return fail(ctx, MRSIM_EINVAL, "sensitivity " + std::to_string(bad) + " is not finite");
    }
    const size_t sig_doubles = (size_t)n_coils * 2 * (size_t)n_adc;
    const bool host_sig = n_adc > 0 && !is_device_ptr(signal_out);
    double *dsig = signal_out;
    if (host_sig) {
        if ((rs = grow(ctx, &ctx->d_sig, &ctx->sig_cap, sig_doubles)) != MRSIM_OK) return rs;
        dsig = ctx->d_sig;
    }
    if (n_adc > 0) CK(cudaMemsetAsync(dsig, 0, sig_doubles * sizeof(double), st), "clear signal");
    FwdArgs a{};
    a.prog = P;
    a.params = ph->params;
    a.n_spins = ph->n;
    a.n_pad = ph->n_pad;
    a.signal = dsig;
    a.status = ctx->d_status;
    a.sens = ctx->d_sens;
    a.n_coils = n_coils;
    void *maps = nullptr;
    if ((rs = prepare_maps(ctx, seq, fp64 ? MODE_F64 : MODE_F32, a, stream, &maps)) != MRSIM_OK) return rs;
    const int rc = fp64 ? launch_fwd_coils_f64(a, threads, stream) : launch_fwd_coils_f32(a, threads, stream);
    if (maps) cudaFreeAsync(maps, st);
    if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "launch forward kernel (coils)");
    if (host_sig) {
        CK(cudaMemcpyAsync(signal_out, dsig, sig_doubles * sizeof(double), cudaMemcpyDeviceToHost, st), "copy signal out");
        return mrsim_stream_status(ctx, stream);
    }
    return MRSIM_OK;
}

mrsim_status mrsim_kt_simulate(mrsim_ctx *ctx, int64_t n_sets, const double *t1, const double *t2,
                               const double *b1, const double *df, int64_t n_steps, const mrsim_kt_step *steps,
                               int32_t max_order, mrsim_precision prec, void *stream, double *signal_out,
                               int64_t n_samples) {
    Range nvtx_range("mrsim_kt_simulate");
    if (!ctx) return MRSIM_EINVAL;
    if (!normalize_precision(prec, true)) return fail(ctx, MRSIM_EINVAL, "unknown precision");
    if (n_sets < 0 || n_steps < 0) return fail(ctx, MRSIM_EINVAL, "negative count");
    if (max_order < 0 || max_order > KT_MAX_ORDER)
        return fail(ctx, MRSIM_EINVAL, "max_order must be 0.." + std::to_string(KT_MAX_ORDER));
    if (n_sets > 0 && (!t1 || !t2)) return fail(ctx, MRSIM_EINVAL, "NULL T1/T2 array");
    if (n_steps > 0 && (!steps || is_device_ptr(steps))) return fail(ctx, MRSIM_EINVAL, "steps must be in host memory");
    // steps: validate and precompute the pulse's phase terms (float64, host)
    std::vector<KtStepDev> hs((size_t)n_steps);
    int64_t cnt = 0;
    for (int64_t k = 0; k < n_steps; ++k) {
        const mrsim_kt_step &q = steps[k];
        if (!std::isfinite(q.alpha) || !std::isfinite(q.phi) || !std::isfinite(q.tau) || !std::isfinite(q.adc_phase) ||
            q.tau < 0.0 || (q.sample != 0 && q.sample != 1) || q.shift < -KT_MAX_SHIFT || q.shift > KT_MAX_SHIFT)
            return fail(ctx, MRSIM_EINVAL, "step " + std::to_string(k) + ": non-finite field, tau < 0, sample not 0/1 or |shift| > " +
                                               std::to_string(KT_MAX_SHIFT));
        KtStepDev &d = hs[(size_t)k];
        d.alpha = q.alpha;
        d.cphi = std::cos(q.phi);
        d.sphi = std::sin(q.phi);
        d.c2phi = std::cos(2.0 * q.phi);
        d.s2phi = std::sin(2.0 * q.phi);
        d.tau = q.tau;
        d.cadc = std::cos(q.adc_phase);
        d.sadc = std::sin(q.adc_phase);
        d.shift = q.shift;
        d.sample = q.sample;
        cnt += q.sample;
    }
    if (cnt != n_samples)
        return fail(ctx, MRSIM_EINVAL, "n_samples = " + std::to_string(n_samples) + " but the steps take " +
                                           std::to_string(cnt) + " samples");
    if (n_sets > 0 && n_samples > 0 && !signal_out) return fail(ctx, MRSIM_EINVAL, "NULL signal buffer");
    if (n_sets == 0) return MRSIM_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    mrsim_status rs;
    // scratch: [steps | t1 | t2 | b1 | df] (parameters staged only when they are host arrays)
    const size_t step_doubles = (size_t)n_steps * sizeof(KtStepDev) / sizeof(double);
    const size_t need = step_doubles + 4 * (size_t)n_sets;
    if ((rs = grow(ctx, &ctx->d_kt, &ctx->kt_cap, std::max<size_t>(need, 1))) != MRSIM_OK) return rs;
    if (n_steps > 0) {
        if (prec == MRSIM_FP64) {
            CK(cudaMemcpyAsync(ctx->d_kt, hs.data(), hs.size() * sizeof(KtStepDev), cudaMemcpyHostToDevice, st),
               "copy steps");
        } else {
            std::vector<KtStepF> hf(hs.size());
            for (size_t k = 0; k < hs.size(); ++k) {
                const KtStepDev &d = hs[k];
                hf[k] = KtStepF{(float)d.alpha, (float)d.cphi, (float)d.sphi, (float)d.c2phi, (float)d.s2phi,
                                (float)d.tau, (float)d.cadc, (float)d.sadc, d.shift, d.sample};
            }
            CK(cudaMemcpyAsync(ctx->d_kt, hf.data(), hf.size() * sizeof(KtStepF), cudaMemcpyHostToDevice, st),
               "copy steps");
            CK(cudaStreamSynchronize(st), "stream synchronize");  // hf is a local buffer
        }
    }
    const double *src[4] = {t1, t2, b1, df};
    const double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4; ++i) {
        if (!src[i]) continue;
        if (is_device_ptr(src[i])) {
            dev[i] = src[i];
        } else {
            double *d = ctx->d_kt + step_doubles + (size_t)i * (size_t)n_sets;
            CK(cudaMemcpyAsync(d, src[i], sizeof(double) * (size_t)n_sets, cudaMemcpyHostToDevice, st), "copy parameters");
            dev[i] = d;
        }
    }
    {
        const int big = 0x7fffffff;
        int bad = big;
        CK(cudaMemcpyAsync(ctx->d_bad, &big, sizeof(int), cudaMemcpyHostToDevice, st), "reset check");
        const int rc = check_kt_params(n_sets, dev[0], dev[1], dev[2], dev[3], ctx->d_bad, st);
        if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "check parameters");
        CK(cudaMemcpyAsync(&bad, ctx->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st), "read check");
        CK(cudaStreamSynchronize(st), "stream synchronize");
        if (bad != big) return fail(ctx, MRSIM_EINVAL, "ensemble " + std::to_string(bad) + ": T1/T2 <= 0 or NaN, or non-finite B1/df");
    }
    const size_t sig_doubles = (size_t)n_sets * 2 * (size_t)n_samples;
    const bool host_sig = sig_doubles > 0 && !is_device_ptr(signal_out);
    double *dsig = signal_out;
    if (host_sig) {
        if ((rs = grow(ctx, &ctx->d_sig, &ctx->sig_cap, sig_doubles)) != MRSIM_OK) return rs;
        dsig = ctx->d_sig;
    }
    KtArgs a{};
    a.steps = ctx->d_kt;
    a.n_steps = n_steps;
    a.n_sets = n_sets;
    a.n_samples = n_samples;
    a.t1 = dev[0];
    a.t2 = dev[1];
    a.b1 = dev[2];
    a.df = dev[3];
    a.max_order = max_order;
    a.signal = dsig;
    const int rc = launch_kt(a, prec == MRSIM_FP64, stream);
    if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "launch K-t kernel");
    if (host_sig) {
        CK(cudaMemcpyAsync(signal_out, dsig, sig_doubles * sizeof(double), cudaMemcpyDeviceToHost, st), "copy signal out");
        return mrsim_stream_status(ctx, stream);
    }
    return MRSIM_OK;
}

mrsim_status mrsim_max_config_k(int64_t n_events, const mrsim_event *events, double gamma_hz_per_t,
                                double kmax_rad_per_m[3]) {
    if (!kmax_rad_per_m || n_events < 0 || (n_events > 0 && !events)) return MRSIM_EINVAL;
    if (!(gamma_hz_per_t > 0.0) || !std::isfinite(gamma_hz_per_t)) return MRSIM_EINVAL;
    const double two_pi_gamma = 2.0 * M_PI * gamma_hz_per_t;
    double total[3] = {0, 0, 0}, seg[3] = {0, 0, 0}, best[3] = {0, 0, 0};
    bool started = false;
    for (int64_t i = 0; i < n_events; ++i) {
        const mrsim_event &e = events[i];
        const double g[3] = {e.gx, e.gy, e.gz};
        if (!std::isfinite(e.dt) || e.dt < 0.0 || !std::isfinite(e.rf_flip) || !std::isfinite(g[0]) ||
            !std::isfinite(g[1]) || !std::isfinite(g[2]))
            return MRSIM_EINVAL;
        if (e.rf_flip != 0.0) {  // the pulse at the event's start closes the current segment
            if (started)
                for (int a = 0; a < 3; ++a) {
                    total[a] += std::fabs(seg[a]);
                    seg[a] = 0.0;
                }
            started = true;
        }
        if (!started) continue;
        for (int a = 0; a < 3; ++a) {
            seg[a] += two_pi_gamma * g[a] * e.dt;  // |k| is linear within the event: check its end
            best[a] = std::max(best[a], total[a] + std::fabs(seg[a]));
        }
    }
    for (int a = 0; a < 3; ++a) kmax_rad_per_m[a] = best[a];
    return MRSIM_OK;
}

mrsim_status mrsim_autotune(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq, mrsim_precision prec,
                            void *stream, mrsim_options *best) {
    Range nvtx_range("mrsim_autotune");
    if (!ctx) return MRSIM_EINVAL;
    if (!ph || !seq || !best) return fail(ctx, MRSIM_EINVAL, "NULL argument");
    if (ph->ctx != ctx || seq->ctx != ctx) return fail(ctx, MRSIM_EINVAL, "handle belongs to another context");
    if (!normalize_precision(prec)) return fail(ctx, MRSIM_EINVAL, "unknown precision");
    const int mode = launch_mode(prec);
    const bool fp64 = mode != MODE_F32;
    std::memset(best, 0, sizeof *best);
    Launch def = choose_launch(ctx, fp64, ph->n);
    if (ph->n == 0) {
        best->spins_per_thread = def.k;
        best->threads_per_block = def.threads;
        return MRSIM_OK;
    }
    const auto known = ctx->tuned.find(tune_key(prec, ph, seq));  // tuned before, or in the cache file
    if (known != ctx->tuned.end()) {
        best->spins_per_thread = known->second.k;
        best->threads_per_block = known->second.threads;
        return MRSIM_OK;
    }
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // time a prefix of the program that is long enough to contain the sequence's structure
    Program P = fp64 ? seq->p64 : seq->p32;
    const double ev_per_op = (double)std::max<int64_t>(seq->n_events, 1) / (double)std::max(P.n_ops, 1);
    const double target = 3e9;  // spin-steps per trial
    int64_t nt = (int64_t)std::ceil(target / ((double)ph->n * ev_per_op));
    nt = std::max<int64_t>(nt, std::min<int64_t>(P.n_ops, 256));
    P.n_ops = (int32_t)std::min<int64_t>(nt, P.n_ops);
    mrsim_status rs = grow(ctx, &ctx->d_sig, &ctx->sig_cap, 2 * (size_t)std::max<int64_t>(P.n_adc, 1));
    if (rs != MRSIM_OK) return rs;
    static const int f32k[] = {1, 2, 4, 8}, f64k[] = {1, 2};
    static const int thr[] = {32, 64, 96, 128, 160, 192, 224, 256, 320, 384, 448, 512};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ee = cudaEventCreate(&e0);
    if (ee == cudaSuccess) ee = cudaEventCreate(&e1);
    if (ee != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ctx, ee, "event");
    }
    // the train maps, once for every trial: the shapes are timed running the trains as the
    // simulation will
    void *tmaps = nullptr;
    {
        FwdArgs ma{};
        ma.prog = P;
        ma.params = ph->params;
        ma.n_spins = ph->n;
        ma.n_pad = ph->n_pad;
        if ((rs = prepare_maps(ctx, seq, mode, ma, stream, &tmaps)) != MRSIM_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rs;
        }
    }
    // time one launch of the prefix in shape (k, t); < 0 if the shape cannot run
    const int32_t short_ops = P.n_ops;
    const int32_t long_ops = (int32_t)std::min<int64_t>((int64_t)short_ops * 3, (fp64 ? seq->p64 : seq->p32).n_ops);
    auto trial = [&](int k, int t) -> float {
        FwdArgs a{};
        a.prog = P;
        a.params = ph->params;
        a.n_spins = ph->n;
        a.n_pad = ph->n_pad;
        a.signal = ctx->d_sig;
        a.status = ctx->d_status;
        a.maps = tmaps;
        cudaEventRecord(e0, st);
        const int rc = mode == MODE_F64 ? launch_fwd_f64(a, k, t, stream)
                       : mode == MODE_DF ? launch_fwd_df(a, k, t, stream)
                                         : launch_fwd_f32(a, k, t, stream);
        cudaEventRecord(e1, st);
        if (rc != 0 || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            return -1.0f;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // pass 1: every shape that fits, once after a warm-up launch; pass 2: the three fastest on a
    // three times longer prefix, twice each, so that timing noise does not pick the shape
    std::vector<TunedShape> cand;
    for (int k : (fp64 ? std::vector<int>(f64k, f64k + 2) : std::vector<int>(f32k, f32k + 4))) {
        for (int t : thr) {
            if (t > (fp64 || k == 8 ? 256 : 512)) continue;
            const size_t smem = fwd_smem_bytes(fp64, P, k, t);
            if (smem > (size_t)ctx->max_smem_optin || fwd_blocks_per_sm(mode, k, t, smem) == 0) continue;
            if (trial(k, t) < 0.0f) continue;
            const float ms = trial(k, t);
            if (ms >= 0.0f) cand.push_back(TunedShape{k, t, ms});
        }
    }
    std::sort(cand.begin(), cand.end(), [](const TunedShape &x, const TunedShape &y) { return x.ms < y.ms; });
    if (cand.size() > 3) cand.resize(3);
    P.n_ops = long_ops;
    for (TunedShape &c : cand) {
        c.ms = 1e30f;
        for (int r = 0; r < 2; ++r) {
            const float ms = trial(c.k, c.threads);
            if (ms >= 0.0f) c.ms = std::min(c.ms, ms);
        }
    }
    TunedShape win;
    win.ms = 1e30f;
    for (const TunedShape &c : cand)
        if (c.ms < win.ms) win = c;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (tmaps) cudaFreeAsync(tmaps, st);
    mrsim_status ss = mrsim_stream_status(ctx, stream);
    if (ss != MRSIM_OK) return ss;
    if (win.k == 0) return fail(ctx, MRSIM_EUNSUPPORTED, "no launch shape fits this program on the device");
    ctx->tuned[tune_key(prec, ph, seq)] = win;
    save_tune_entry(ctx, tune_key(prec, ph, seq), win);
    best->spins_per_thread = win.k;
    best->threads_per_block = win.threads;
    return MRSIM_OK;
}

mrsim_status mrsim_simulate(mrsim_ctx *ctx, const mrsim_phantom *ph, const mrsim_sequence *seq, mrsim_precision prec,
                            void *stream, double *signal_out, int64_t n_adc) {
    return mrsim_simulate_ex(ctx, ph, seq, prec, stream, signal_out, n_adc, nullptr);
}

mrsim_status mrsim_debug_compile(int64_t n_events, const mrsim_event *events, double gamma, mrsim_program_dump *d) {
    return mrsim_debug_compile_snapshots(n_events, events, gamma, 0, nullptr, d);
}

mrsim_status mrsim_debug_compile_snapshots(int64_t n_events, const mrsim_event *events, double gamma, int64_t n_snap,
                                           const int64_t *snap_after, mrsim_program_dump *d) {
    if (!d) return MRSIM_EINVAL;
    Compiled c;
    std::string err;
    int rc = compile_sequence(events, n_events, gamma, c, err, n_snap, snap_after);
    if (rc != MRSIM_OK) return (mrsim_status)rc;
    const int64_t n_train = (int64_t)c.train.size() / 2;
    if ((d->ops && (int64_t)c.ops64.size() > d->n_ops) || (d->pcls && c.n_pcls > d->n_pcls) ||
        (d->e1 && c.n_e1 > d->n_e1) || (d->e2 && c.n_e2 > d->n_e2) || (d->train && n_train > d->n_train) ||
        (d->demod && c.n_adc > d->n_adc))
        return MRSIM_EINVAL;
    if (d->ops) std::memcpy(d->ops, c.ops64.data(), c.ops64.size() * sizeof(OpF64));
    if (d->pcls) std::memcpy(d->pcls, c.pcls.data(), c.pcls.size() * sizeof(double));
    if (d->e1) std::memcpy(d->e1, c.e1.data(), c.e1.size() * sizeof(double));
    if (d->e2) std::memcpy(d->e2, c.e2.data(), c.e2.size() * sizeof(double));
    if (d->train) std::memcpy(d->train, c.train.data(), c.train.size() * sizeof(double));
    if (d->demod) std::memcpy(d->demod, c.demod.data(), c.demod.size() * sizeof(double));
    d->n_ops = (int64_t)c.ops64.size();
    d->n_pcls = c.n_pcls;
    d->n_e1 = c.n_e1;
    d->n_e2 = c.n_e2;
    d->n_train = (int32_t)n_train;
    d->n_adc = c.n_adc;
    return MRSIM_OK;
}

namespace {

// Work items for tiles of S spins, longest sequences first (longest-processing-time order), and
// the launch geometry of the persistent kernel.
mrsim_status batch_layout(mrsim_batch *b, int k, int threads) {
    mrsim_ctx *ctx = b->ctx;
    const int mode = launch_mode(b->prec);
    const bool fp64 = mode != MODE_F32;
    const int64_t S = (int64_t)k * threads;
    std::vector<int> order(b->descs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->seq[x]->n_events > b->seq[y]->n_events; });
    std::vector<BatchItem> items;
    size_t smem = 0;
    for (int d : order) {
        const int64_t tiles = (b->descs[d].n_spins + S - 1) / S;
        if (tiles > INT32_MAX) return fail(ctx, MRSIM_EINVAL, "too many tiles");
        for (int64_t t = 0; t < tiles; ++t) items.push_back(BatchItem{d, (int32_t)t});
        smem = std::max(smem, fwd_smem_bytes(fp64, b->descs[d].prog, k, threads));
    }
    if (smem > (size_t)ctx->max_smem_optin) return fail(ctx, MRSIM_EUNSUPPORTED, "launch shape exceeds shared memory");
    const int per_sm = batch_blocks_per_sm(mode, k, threads, smem);
    if (per_sm <= 0) return fail(ctx, MRSIM_EUNSUPPORTED, "launch shape cannot be resident");
    if (items.size() > (size_t)INT32_MAX) return fail(ctx, MRSIM_EINVAL, "too many work items");
    cudaFree(b->d_items);
    b->d_items = nullptr;
    if (!items.empty()) {
        CK(ctx_malloc(ctx, &b->d_items, items.size() * sizeof(BatchItem)), "cudaMalloc batch items");
        CK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice), "upload items");
    }
    b->items.swap(items);
    b->k = k;
    b->threads = threads;
    b->smem = smem;
    b->grid = (int)std::min<int64_t>((int64_t)per_sm * ctx->num_sms, std::max<size_t>(b->items.size(), 1));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return MRSIM_OK;
}

// zero outputs, reset the queue, run the persistent kernel (all asynchronous on `st`)
mrsim_status batch_enqueue(mrsim_batch *b, const FwdArgs *d_descs, cudaStream_t st) {
    mrsim_ctx *ctx = b->ctx;
    if (b->items.empty()) return MRSIM_OK;
    int rc = zero_signals(d_descs, (int)b->descs.size(), st);
    if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "zero batch signals");
    CK(cudaMemsetAsync(b->d_head, 0, sizeof(int), st), "reset work queue");
    for (size_t i = 0; i < b->descs.size(); ++i) {  // train maps of the phantoms that have some
        const FwdArgs &d = b->descs[i];
        if (!d.maps) continue;
        rc = launch_train_maps(launch_mode(b->prec), d, b->seq[i]->d_train64, const_cast<void *>(d.maps), st);
        if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "batch train maps");
    }
    BatchArgs a{};
    a.descs = d_descs;
    a.items = b->d_items;
    a.n_items = (int32_t)b->items.size();
    a.head = b->d_head;
    rc = launch_batch(launch_mode(b->prec), a, b->k, b->threads, b->smem, b->grid, st);
    if (rc != 0) return cuda_fail(ctx, (cudaError_t)rc, "launch batch kernel");
    return MRSIM_OK;
}

}  // namespace

mrsim_status mrsim_batch_create(mrsim_ctx *ctx, int32_t n, const mrsim_phantom *const *phantoms,
                                const mrsim_sequence *const *seqs, mrsim_precision prec, double *const *signals_out,
                                mrsim_batch **out) {
    if (!ctx || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (n < 0 || (n > 0 && (!phantoms || !seqs || !signals_out)))
        return fail(ctx, MRSIM_EINVAL, "invalid batch arrays");
    if (!normalize_precision(prec)) return fail(ctx, MRSIM_EINVAL, "unknown precision");
    cudaSetDevice(ctx->device);
    mrsim_batch *b = new (std::nothrow) mrsim_batch();
    if (!b) return fail(ctx, MRSIM_ENOMEM, "host allocation failed");
    b->ctx = ctx;
    b->prec = prec;
    int64_t max_n = 0;
    for (int i = 0; i < n; ++i) {
        const mrsim_phantom *p = phantoms[i];
        const mrsim_sequence *q = seqs[i];
        if (!p || !q || p->ctx != ctx || q->ctx != ctx) {
            delete b;
            return fail(ctx, MRSIM_EINVAL, "batch entry " + std::to_string(i) + ": NULL handle or another context");
        }
        if (q->prog->host.n_adc > 0 && !is_device_ptr(signals_out[i])) {
            delete b;
            return fail(ctx, MRSIM_EINVAL, "batch entry " + std::to_string(i) + ": signal buffer must be device memory");
        }
        FwdArgs a{};
        a.prog = prec != MRSIM_FP32 ? q->p64 : q->p32;  // float64 program for float64 and double-float
        a.params = p->params;
        a.n_spins = p->n;
        a.n_pad = p->n_pad;
        a.signal = signals_out[i];
        a.status = ctx->d_status;
        b->ph.push_back(p);
        b->seq.push_back(q);
        b->descs.push_back(a);
        b->spin_steps += p->n * q->n_events;
        max_n = std::max(max_n, p->n);
    }
    auto bail = [&](mrsim_status st) {
        mrsim_batch_destroy(b);
        return st;
    };
    // every phantom's train maps in one buffer, rebuilt by each launch (a phantom's device memory
    // may change between launches)
    const int bmode = launch_mode(prec);
    if (ctx->train_maps) {
        size_t total = 0;
        std::vector<size_t> off(b->descs.size(), 0);
        for (size_t i = 0; i < b->descs.size(); ++i) {
            const FwdArgs &a = b->descs[i];
            if (a.prog.n_tmap <= 0 || a.n_spins <= 0) continue;
            off[i] = total;
            total += (train_map_bytes(bmode, a.prog, a.n_pad) + 255) / 256 * 256;
        }
        if (total > 0) {
            cudaError_t e = ctx_malloc(ctx, &b->d_maps, total);
            if (e != cudaSuccess) {
                mrsim_batch_destroy(b);
                return cuda_fail(ctx, e, "batch train maps");
            }
            for (size_t i = 0; i < b->descs.size(); ++i)
                if (b->descs[i].prog.n_tmap > 0 && b->descs[i].n_spins > 0) b->descs[i].maps = b->d_maps + off[i];
        }
    }
    if (n > 0) {
        cudaError_t e = ctx_malloc(ctx, &b->d_descs, b->descs.size() * sizeof(FwdArgs));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_descs, b->descs.data(), b->descs.size() * sizeof(FwdArgs), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = ctx_malloc(ctx, &b->d_head, sizeof(int));
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "batch descriptors"));
    }
    // default shape: the single-phantom heuristic for the largest phantom, shrunk until it fits
    Launch L = choose_launch(ctx, prec != MRSIM_FP32, max_n);
    mrsim_status st = batch_layout(b, L.k, L.threads);
    for (int t : {64, 32}) {
        if (st != MRSIM_EUNSUPPORTED) break;
        st = batch_layout(b, 1, t);
    }
    if (st != MRSIM_OK) return bail(st);
    *out = b;
    return MRSIM_OK;
}

int64_t mrsim_batch_num_items(const mrsim_batch *b) { return b ? (int64_t)b->items.size() : -1; }

mrsim_status mrsim_batch_autotune(mrsim_batch *b, void *stream, mrsim_options *best) {
    if (!b) return MRSIM_EINVAL;
    mrsim_ctx *ctx = b->ctx;
    if (!best) return fail(ctx, MRSIM_EINVAL, "NULL best");
    std::memset(best, 0, sizeof *best);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = b->prec != MRSIM_FP32;
    if (b->descs.empty()) return MRSIM_OK;
    // Time prefixes of every program, the same fraction of each so that the mix of programs is
    // that of the whole batch: pass 1 every shape on about 2e10 spin-steps in all, pass 2 the
    // three fastest on about 3e11 (a short prefix over-weights the per-spin set-up and the first
    // TRs).  Warm-up launches run an 8-operation prefix so that each kernel is loaded first.
    const size_t nd = b->descs.size();
    std::vector<FwdArgs> sets[3] = {b->descs, b->descs, b->descs};  // pass 1, pass 2, warm-up
    const double fracs[2] = {std::min(1.0, 2e10 / (double)std::max<int64_t>(b->spin_steps, 1)),
                             std::min(1.0, 3e11 / (double)std::max<int64_t>(b->spin_steps, 1))};
    for (size_t i = 0; i < nd; ++i) {
        for (int q = 0; q < 2; ++q) {
            FwdArgs &a = sets[q][i];
            const int64_t nt = std::max<int64_t>((int64_t)std::ceil(a.prog.n_ops * fracs[q]), 8);
            a.prog.n_ops = (int32_t)std::min<int64_t>(nt, a.prog.n_ops);
        }
        sets[2][i].prog.n_ops = std::min<int32_t>(sets[2][i].prog.n_ops, 8);
    }
    size_t max_adc = 0;
    for (auto &a : b->descs) max_adc = std::max<size_t>(max_adc, (size_t)a.prog.n_adc);
    mrsim_status rs = grow(ctx, &ctx->d_sig, &ctx->sig_cap, 2 * std::max<size_t>(max_adc, 1));
    if (rs != MRSIM_OK) return rs;
    for (auto &v : sets)
        for (auto &a : v) a.signal = ctx->d_sig;  // the tuning runs all add into one scratch buffer
    FwdArgs *d_sets = nullptr;
    CK(ctx_malloc(ctx, &d_sets, 3 * nd * sizeof(FwdArgs)), "cudaMalloc tuning descriptors");
    cudaError_t ue = cudaSuccess;
    for (int q = 0; q < 3 && ue == cudaSuccess; ++q)
        ue = cudaMemcpy(d_sets + q * nd, sets[q].data(), nd * sizeof(FwdArgs), cudaMemcpyHostToDevice);
    if (ue != cudaSuccess) {
        cudaFree(d_sets);
        return cuda_fail(ctx, ue, "upload tuning descriptors");
    }
    const FwdArgs *d_pass[2] = {d_sets, d_sets + nd}, *d_warm = d_sets + 2 * nd;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ee = cudaEventCreate(&e0);
    if (ee == cudaSuccess) ee = cudaEventCreate(&e1);
    if (ee != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaFree(d_sets);
        return cuda_fail(ctx, ee, "event");
    }
    // one warm-up launch and one timed launch of shape (k, t); < 0 if the shape cannot run
    auto trial = [&](int k, int t, const FwdArgs *d_descs) -> float {
        std::string keep = ctx->err;
        if (batch_layout(b, k, t) != MRSIM_OK) {
            ctx->err = keep;
            return -1.0f;
        }
        if (batch_enqueue(b, d_warm, st) != MRSIM_OK) {
            cudaGetLastError();
            return -1.0f;
        }
        cudaEventRecord(e0, st);
        mrsim_status q = batch_enqueue(b, d_descs, st);
        cudaEventRecord(e1, st);
        if (q != MRSIM_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            return -1.0f;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    static const int f32k[] = {1, 2, 4, 8}, f64k[] = {1, 2};
    static const int thr[] = {32, 64, 96, 128, 160, 192, 224, 256, 320, 384, 448, 512};
    std::vector<TunedShape> cand;
    for (int k : (fp64 ? std::vector<int>(f64k, f64k + 2) : std::vector<int>(f32k, f32k + 4)))
        for (int t : thr) {
            if (t > (fp64 || k == 8 ? 256 : 512)) continue;
            const float ms = trial(k, t, d_pass[0]);
            if (ms >= 0.0f) cand.push_back(TunedShape{k, t, ms});
        }
    std::sort(cand.begin(), cand.end(), [](const TunedShape &x, const TunedShape &y) { return x.ms < y.ms; });
    if (cand.size() > 3) cand.resize(3);
    int bk = 0, bt = 0;
    float bms = 1e30f;
    for (const TunedShape &c : cand) {
        const float ms = trial(c.k, c.threads, d_pass[1]);
        if (ms >= 0.0f && ms < bms) {
            bms = ms;
            bk = c.k;
            bt = c.threads;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_sets);
    mrsim_status ss = mrsim_stream_status(ctx, stream);
    if (ss != MRSIM_OK) return ss;
    if (!bk) return fail(ctx, MRSIM_EUNSUPPORTED, "no launch shape fits this batch");
    mrsim_status ls = batch_layout(b, bk, bt);
    if (ls != MRSIM_OK) return ls;
    best->spins_per_thread = bk;
    best->threads_per_block = bt;
    return MRSIM_OK;
}

mrsim_status mrsim_batch_set_shape(mrsim_batch *b, int32_t spins_per_thread, int32_t threads_per_block) {
    if (!b) return MRSIM_EINVAL;
    const bool fp64 = b->prec != MRSIM_FP32;
    const int k = spins_per_thread, t = threads_per_block;
    const bool ok = fp64 ? (k == 1 || k == 2) : (k == 1 || k == 2 || k == 4 || k == 8);
    if (!ok || t < 32 || t % 32 || t > (fp64 || k == 8 ? 256 : 512))
        return fail(b->ctx, MRSIM_EINVAL, "unsupported spins_per_thread / threads_per_block");
    cudaSetDevice(b->ctx->device);
    return batch_layout(b, k, t);
}

mrsim_status mrsim_batch_launch(mrsim_batch *b, void *stream) {
    Range nvtx_range("mrsim_batch_launch");
    if (!b) return MRSIM_EINVAL;
    cudaSetDevice(b->ctx->device);
    return batch_enqueue(b, b->d_descs, (cudaStream_t)stream);
}

mrsim_status mrsim_batch_launch_graph(mrsim_batch *b, void *stream) {
    Range nvtx_range("mrsim_batch_launch_graph");
    if (!b) return MRSIM_EINVAL;
    mrsim_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    if (!b->graph) {
        if (!b->capture) CK(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "create capture stream");
        CK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
        mrsim_status st = batch_enqueue(b, b->d_descs, b->capture);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->capture, &g);
        if (st != MRSIM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return cuda_fail(ctx, e, "instantiate graph");
        }
    }
    CK(cudaGraphLaunch(b->graph, (cudaStream_t)stream), "graph launch");
    return MRSIM_OK;
}

void mrsim_batch_destroy(mrsim_batch *b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->d_descs);
    cudaFree(b->d_items);
    cudaFree(b->d_head);
    cudaFree(b->d_maps);
    delete b;
}

mrsim_status mrsim_simulate_batch(mrsim_ctx *ctx, int32_t n, const mrsim_phantom *const *phantoms,
                                  const mrsim_sequence *const *seqs, mrsim_precision prec, void *stream,
                                  double *const *signals_out) {
    mrsim_batch *b = nullptr;
    mrsim_status st = mrsim_batch_create(ctx, n, phantoms, seqs, prec, signals_out, &b);
    if (st != MRSIM_OK) return st;
    st = mrsim_batch_launch(b, stream);
    if (st == MRSIM_OK) st = mrsim_stream_status(ctx, stream);
    mrsim_batch_destroy(b);
    return st;
}

}  // extern "C"
