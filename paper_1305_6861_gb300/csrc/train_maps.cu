// train_maps.cu -- set-up of the train maps: for every spin, the composition of a recurring shaped
// pulse's sub-pulses (Eq. 3.23) as one affine map of its state, which the forward kernel applies in
// place of the train (OP_RF_TRAIN with F_TMAP).
#include <cuda_runtime.h>

#include "../../include/mrsim.h"
#include "dfloat.cuh"
#include "internal.h"
#include "packed.cuh"

namespace mrsim {
namespace dev {

// Train maps (set-up): thread (s, t) composes the sub-pulses of map kind t for spin s exactly as
// train_run steps them (lazy T1 with the kind's T1 class, the turn by the table entry, precession
// by the kind's phasor class) on the three unit states, which become the columns of A, and on the
// zero state, which becomes c (it carries the T1 recovery towards M0), in C arithmetic
// (double-float or float64); the classes come from the spin's parameters in float64 as the
// forward kernel's set-up forms them, the turns from the float64 table.  Stored rounded to R.
template <typename C, typename R>
__global__ void __launch_bounds__(256) train_map_kernel(const FwdArgs a, const double *train64, R *maps) {
    __shared__ C tab[2 * RUN_MAX];  // the kind's (cos α, sin α), converted to C once per block
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    const Program &P = a.prog;
    const int pc = P.tmap[4 * t], ec = P.tmap[4 * t + 1], off = P.tmap[4 * t + 2], n = P.tmap[4 * t + 3];
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) tab[i] = C(train64[2 * off + i]);
    __syncthreads();
    if (s >= a.n_pad) return;
    const bool valid = s < a.n_spins;
    const int64_t np = a.n_pad;
    const double x = valid ? a.params[P_X * np + s] : 0.0;
    const double y = valid ? a.params[P_Y * np + s] : 0.0;
    const double z = valid ? a.params[P_Z * np + s] : 0.0;
    const double df = valid ? a.params[P_DF * np + s] : 0.0;
    const double m0 = valid ? a.params[P_RHO * np + s] : 0.0;
    const double r1 = valid ? a.params[P_R1 * np + s] : 0.0;
    const double r2 = valid ? a.params[P_R2 * np + s] : 0.0;
    const double dt = P.pcls[4 * pc + 3];
    double th = P.pcls[4 * pc] * x + P.pcls[4 * pc + 1] * y + P.pcls[4 * pc + 2] * z + df * dt;
    th -= rint(th);
    double sn, cs;
    sincospi(2.0 * th, &sn, &cs);
    const double e2 = exp(-dt * r2);
    const double eps = -expm1(-P.e1[ec] * r1);
    const C wr = C(e2 * cs), wi = C(-e2 * sn), nwi = C(e2 * sn), ep = C(eps), nep = C(-eps), rho = C(m0);
    C U[4] = {C(1.0), C(0.0), C(0.0), C(0.0)}, V[4] = {C(0.0), C(1.0), C(0.0), C(0.0)};
    C Z[4] = {C(0.0), C(0.0), C(1.0), C(0.0)};
    for (int i = 0; i < n; ++i) {
        const C ca = tab[2 * i], sa = tab[2 * i + 1], nsa = -tab[2 * i + 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const C zt = k < 3 ? vfma(nep, Z[k], Z[k]) : vfma(ep, rho - Z[k], Z[k]);  // lazy T1
            const C v1 = vdot2(V[k], ca, zt, sa);                                       // turn
            Z[k] = vdot2(V[k], nsa, zt, ca);
            const C u1 = vdot2(v1, nwi, U[k], wr);  // precession
            V[k] = vdot2(v1, wr, U[k], wi);
            U[k] = u1;
        }
    }
    R *m = maps + (int64_t)t * TRAIN_MAP_ROWS * np + s;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m[(0 + k) * np] = R(double(U[k]));
        m[(3 + k) * np] = R(double(V[k]));
        m[(6 + k) * np] = R(double(Z[k]));
    }
    m[9 * np] = R(double(U[3]));
    m[10 * np] = R(double(V[3]));
    m[11 * np] = R(double(Z[3]));
}

}  // namespace dev

size_t train_map_bytes(int mode, const Program &p, int64_t n_pad) {
    return (size_t)p.n_tmap * TRAIN_MAP_ROWS * (size_t)n_pad * (mode == MODE_F32 ? sizeof(float) : sizeof(double));
}

int launch_train_maps(int mode, const FwdArgs &a, const double *train64, void *maps, void *stream) {
    if (a.prog.n_tmap <= 0 || a.n_pad <= 0) return 0;
    const dim3 grid((unsigned)((a.n_pad + 255) / 256), (unsigned)a.prog.n_tmap);
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == MODE_F64)
        dev::train_map_kernel<double, double><<<grid, 256, 0, st>>>(a, train64, static_cast<double *>(maps));
    else if (mode == MODE_DF)
        dev::train_map_kernel<dev::dfl, dev::dfl><<<grid, 256, 0, st>>>(a, train64, static_cast<dev::dfl *>(maps));
    else
        dev::train_map_kernel<dev::dfl, float><<<grid, 256, 0, st>>>(a, train64, static_cast<float *>(maps));
    return (int)cudaGetLastError();
}

}  // namespace mrsim
