// internal.h -- device program format shared by the host sequence compiler and the kernels.
//
// A sequence of elementary sequences (§4.1) is compiled once, in float64, into a
// stream of operations that every spin of a thread block executes in lock-step
// (every thread sees the same operation, so branches on the operation never
// diverge: the "codelet" idea of §6.3, one specialised code path per operation
// kind).  Spin-independent work is done here once per sequence, as the paper's
// master process does (§6.3):
//   * gradient moments k = γ/2π · G · Δt in cycles/m;
//   * runs of events without RF and ADC merged into one precession
//     (analytic solutions span long intervals in one step, §3.3);
//   * T1 recovery applied lazily, once per RF pulse, over the time since the
//     previous pulse (Mz only matters at the next pulse);
//   * the transverse magnetisation is carried in a frame rotated about z by
//     the phase ψ of the most recent RF pulse, u + jv = (Mx + jMy)·exp(-jψ).
//     In that frame every hard pulse (Eq. 3.19) turns about the frame's x
//     axis: u' = u, v' = cos α·v + sin α·Mz, Mz' = cos α·Mz − sin α·v.
//     A pulse with another phase first turns the frame (one complex product by
//     a constant); precession commutes with the frame; the frame angle at each
//     sample is folded into the sample's demodulation factor;
//   * recurring precession intervals (same moment and Δt) become "classes"
//     whose per-spin phasor E2·exp(-j2π(k·x + Δf·Δt)) each thread block
//     evaluates once per spin in float64 and then reuses, e.g. for every
//     sample of a constant-gradient readout.  The host tracks which class the
//     kernel holds in registers and marks the operations that must reload it.
#pragma once
#include <cstddef>
#include <cstdint>

#include "../../include/mrsim.h"

namespace mrsim {

enum OpKind : uint8_t {
    OP_END = 0,      // lazy T1 over f[10]; f[0], f[1] = cos ψ, sin ψ of the final frame
    OP_RF = 1,       // general pulse: [frame turn f[2],f[3]] [lazy T1] rotation f[0]=cos α, f[1]=sin α
                     // [fused class precession] [single sample]
    OP_RF_FAST = 2,  // sub-pulse of a train: lazy T1 with the cached class, rotation, cached precession
    OP_PREC = 3,     // precession + T2 over one interval: cached class or inline; [single sample]
    OP_RUN = 4,      // [inline precession] then n consecutive samples, each after one precession by the cached class
    OP_RF_TRAIN = 5, // n fast sub-pulses whose (cos α, sin α) are train-table entries adc0 .. adc0+n-1
    OP_SNAP = 6,     // snapshot adc0 of every spin's state: lazy T1 over f[10] (the T1 clock restarts),
                     // then (Mx + jMy, Mz) with f[0], f[1] = cos ψ, sin ψ of the current frame
};

enum OpFlags : uint16_t {
    F_ADC = 1,       // one sample (index adc0) after the operation
    F_PCLS = 2,      // precession by the cached phasor class
    F_PLOAD = 4,     // load phasor class pcls into the register cache first
    F_INLINE = 8,    // PREC, RUN: phase from the op's own moment and Δt (a run applies it before its samples)
    F_E1CLS = 16,    // RF/END: lazy T1 factor from the cached T1 class
    F_E1LOAD = 32,   // load T1 class ecls into the register cache first
    F_E1INL = 64,    // RF/END: lazy T1 factor computed from f[10]
    F_E2CLS = 128,   // inline PREC: T2 factor from class ecls
    F_ANCHOR = 256,  // RUN: state after the run = state before it (and its inline precession) * phasor class acls
    F_FRAME = 512,   // RF: turn the frame by exp(-jδ), f[2] = cos δ, f[3] = sin δ
    F_KX = 1024,     // inline PREC: which phase terms are non-zero
    F_KY = 2048,
    F_KZ = 4096,
    F_DT = 8192,
    F_RFTAB = 16384,  // RF, RF_FAST: (cos α, sin α) from sub-pulse table entry `tab` (a parametric pulse)
    F_TMAP = 32768,   // RF_TRAIN: a recurring train; a launch given train maps applies map `tab` instead
};

// float32 program: 64 bytes.  Inline PREC payload: kx, ky, kz, Δt as (hi, lo) float pairs
// (f[0..7]) and Δt in f[8].
struct alignas(16) OpF32 {
    uint8_t kind;
    uint8_t rsv0;
    uint16_t flags;
    int32_t n;
    int32_t adc0;
    int16_t pcls, ecls;
    int16_t acls, tab;  // tab: sub-pulse table entry of a parametric pulse (F_RFTAB)
    float f[11];
};
static_assert(sizeof(OpF32) == 64, "OpF32 must be 64 bytes");

// float64 program: 128 bytes.  Inline PREC payload: kx, ky, kz, Δt in f[0..3].
struct alignas(16) OpF64 {
    uint8_t kind;
    uint8_t rsv0;
    uint16_t flags;
    int32_t n;
    int32_t adc0;
    int16_t pcls, ecls;
    int16_t acls, tab;  // as in OpF32
    int32_t rsv2;
    double f[13];
};
static_assert(sizeof(OpF64) == 128, "OpF64 must be 128 bytes");

// Limits of the per-block class tables (shared memory grows with them).
constexpr int MAX_PCLS = 8;
constexpr int MAX_E1CLS = 4;
constexpr int MAX_E2CLS = 4;
// Samples held per block before they are added to global memory: float32 keeps one block-wide
// window (warps add into it with shared-memory atomics), float64 one row per warp.
constexpr int SAMPLE_WINDOW_F32 = 1024;
constexpr int SAMPLE_WINDOW_F64 = 256;
// Longest sample run of one operation (must fit either window).
constexpr int RUN_MAX = 256;
// Entries (cos α, sin α) of the de-duplicated sub-pulse table held in shared memory.
constexpr int TRAIN_TABLE_MAX = 2048;
// Train maps: a sub-pulse train that recurs at least TRAIN_MAP_MIN times with the same precession
// class, T1 class and table entries is, for each spin, one affine map of its state (the composition
// of its sub-pulses, Eq. 3.23), computed once per launch; at most TRAIN_MAP_MAX kinds per program.
constexpr int TRAIN_MAP_MIN = 4;
constexpr int TRAIN_MAP_MAX = 16;
constexpr int TRAIN_MAP_ROWS = 12;  // A (3 x 3, row-major) and c (3): (u, v, Mz) <- A (u, v, Mz) + c

// Ops staged in shared memory per bulk copy (two buffers).
constexpr int CHUNK_F32 = 64;
constexpr int CHUNK_F64 = 32;

// Per-spin parameter block on the device: 7 float64 SoA rows of n_pad values:
// x, y, z [m], Δf = Δω/2π [Hz], M0, R1 = 1/T1, R2 = 1/T2 [1/s] (0 for T = ∞).
constexpr int NPARAM = 7;
enum ParamRow { P_X = 0, P_Y, P_Z, P_DF, P_RHO, P_R1, P_R2 };

struct Program {
    const void *ops;
    int32_t n_ops;
    int32_t n_pcls, n_e1, n_e2;
    const double *pcls;  // 4 per class: kx, ky, kz [cycles/m], Δt [s]
    const double *e1;    // τ [s] per class
    const double *e2;    // Δt [s] per class
    const double *demod; // 2 per sample: exp(-j(adc_phase - ψ)) with ψ the frame at the sample
    const float *demod32;  // the same factors rounded to float32 (float32 path)
    const void *train;     // sub-pulse table: n_train (cos α, sin α) pairs, float2 or double2
    int32_t n_train;
    int64_t n_adc;
    float kmax[4];  // float32 program: max |k_hi| of the inline precessions per term (kx, ky, kz, Δt)
    const int32_t *tmap;  // 4 per train-map kind: phasor class, T1 class, first table entry, sub-pulses
    int32_t n_tmap;
};

struct FwdArgs {
    Program prog;
    const double *params;  // NPARAM x n_pad
    int64_t n_spins, n_pad;
    const double *state_in;  // NULL or 3 per spin (device), laboratory frame
    double *state_out;       // NULL or 3 per spin (device), laboratory frame
    double *signal;          // 2 * n_adc (device), accumulated with atomics; with coils n_coils x 2 * n_adc
    int *status;             // device status word (0 = ok)
    const void *sens;        // receive coils: n_coils x n_pad complex (float2 or double2), coil-major
    int32_t n_coils;         // 0 = no coil weighting
    double *snap;            // NULL or n_snap x n_spins x 3 (device), written by OP_SNAP (laboratory frame)
    const void *maps;        // NULL (trains run sub-pulse by sub-pulse) or the train maps of this phantom and
                             // program: n_tmap x TRAIN_MAP_ROWS rows of n_pad values in the launch's type
};

// One work item of the persistent batch kernel: tile `tile` of the phantom of descriptor `desc`.
struct BatchItem {
    int32_t desc;
    int32_t tile;
};

struct BatchArgs {
    const FwdArgs *descs;    // one forward description per phantom (device)
    const BatchItem *items;  // work items, longest first (device)
    int32_t n_items;
    int *head;               // work-queue counter, zero before the launch (device)
};

// Arithmetic of a launch: float32, float64, or double-float (float32 pairs carrying their
// rounding error: the compensated precision).  Double-float uses the float64 program and
// layouts (fp64 = mode != MODE_F32 wherever a layout or program is chosen).
enum LaunchMode : int { MODE_F32 = 0, MODE_F64 = 1, MODE_DF = 2 };
inline int launch_mode(mrsim_precision p) {
    return p == MRSIM_FP64 ? MODE_F64 : p == MRSIM_FP32_KAHAN ? MODE_DF : MODE_F32;
}

// Kernel launchers (fwd_f32.cu / fwd_f64.cu / fwd_df.cu).  Return a cudaError_t value.
int launch_batch(int mode, const BatchArgs &b, int spins_per_thread, int threads, size_t smem, int grid,
                 void *stream);
int batch_blocks_per_sm(int mode, int spins_per_thread, int threads, size_t smem);
int launch_fwd_f32(const FwdArgs &a, int spins_per_thread, int threads, void *stream);
int launch_fwd_f64(const FwdArgs &a, int spins_per_thread, int threads, void *stream);
int launch_fwd_df(const FwdArgs &a, int spins_per_thread, int threads, void *stream);
// one block whose bounded mbarrier wait runs out after limit_ns and records MRSIM_ETIMEOUT in *status
int launch_wait_probe(int *status, uint64_t limit_ns, void *stream);
size_t fwd_smem_bytes(bool fp64, const Program &p, int spins_per_thread, int threads);
// Train maps of a.prog for the spins of a.params (n_pad per row) into `maps`: float32, float64 or
// double-float values by mode, built in double-float (float64 for mode MODE_F64) from the float64
// sub-pulse table train64 (2 per entry: cos α, sin α).
size_t train_map_bytes(int mode, const Program &p, int64_t n_pad);
int launch_train_maps(int mode, const FwdArgs &a, const double *train64, void *maps, void *stream);
// K-t formalism (kt_kernel.cu): one step per elementary sequence, with the pulse's phase terms
// precomputed on the host.
struct KtStepDev {
    double alpha;              // flip [rad] before B1 scaling; 0 = no pulse
    double cphi, sphi;         // cos φ, sin φ
    double c2phi, s2phi;       // cos 2φ, sin 2φ
    double tau;                // interval [s]
    double cadc, sadc;         // cos, sin of the receiver phase
    int32_t shift, sample;     // order shift q of the interval's gradient; 1 = record a_0
};
static_assert(sizeof(KtStepDev) == 72, "KtStepDev layout");
struct KtStepF {  // the same in float32, for the float32 kernel
    float alpha, cphi, sphi, c2phi, s2phi, tau, cadc, sadc;
    int32_t shift, sample;
};
static_assert(sizeof(KtStepF) == 40, "KtStepF layout");
constexpr int KT_MAX_ORDER = 255;  // 8 slots of 32 lanes
constexpr int KT_MAX_SHIFT = 64;
struct KtArgs {
    const void *steps;  // KtStepDev (float64) or KtStepF (float32) records
    int64_t n_steps, n_sets, n_samples;
    const double *t1, *t2, *b1, *df;  // per ensemble; b1, df may be NULL (1, 0)
    int32_t max_order;
    double *signal;                   // n_sets x 2 * n_samples
};
int launch_kt(const KtArgs &a, bool fp64, void *stream);
// lowest index of an ensemble with T1/T2 <= 0 or NaN, or non-finite B1/Δf, into *bad
int check_kt_params(int64_t n, const double *t1, const double *t2, const double *b1, const double *df, int *bad,
                    void *stream);

// Forward launch with receive coils (a.sens, a.n_coils in 1..MAX_COILS): float32 with 2 spins per
// thread, float64 with 1; coil rows per sample are a.n_coils rounded up to 1, 2, 4 or 8.
constexpr int MAX_COILS = MRSIM_MAX_COILS;
int launch_fwd_coils_f32(const FwdArgs &a, int threads, void *stream);
// spins per thread of the float32 coil kernel for n_coils receive coils
int coil_spins_per_thread_f32(int n_coils);
int launch_fwd_coils_f64(const FwdArgs &a, int threads, void *stream);
// Registers per thread of a kernel instance (0 if the shape does not exist).
int fwd_regs(int mode, int spins_per_thread);
// Resident blocks per SM of a launch shape with `smem` dynamic shared memory (0 = cannot launch).
int fwd_blocks_per_sm(int mode, int spins_per_thread, int threads, size_t smem);
int zero_signals(const FwdArgs *descs, int n, void *stream);
// Validate receive sensitivities (complex float64, [n_coils][n], interleaved) and write them to
// dst as [n_coils][n_pad] float2 (f32) or double2, zero-padded; bad = lowest index of a
// non-finite value.
int pack_sens(int32_t n_coils, int64_t n, int64_t n_pad, const double *src, void *dst, bool f32, int *bad,
              void *stream);
int pack_params(int64_t n, int64_t n_pad, const double *x, const double *y, const double *z,
                const double *rho, const double *t1, const double *t2, const double *dw,
                double *params, int *bad, void *stream);

}  // namespace mrsim
