// compiled.h -- host-side result of the sequence compiler (compile.cpp).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mrsim.h"
#include "internal.h"

namespace mrsim {

struct Compiled {
    std::vector<OpF32> ops32;
    std::vector<OpF64> ops64;
    std::vector<double> pcls;   // 4 per phasor class: kx, ky, kz [cycles/m], Δt [s]
    std::vector<double> e1;     // τ per T1 class
    std::vector<double> e2;     // Δt per T2 class
    std::vector<double> demod;  // 2 per sample
    std::vector<double> train;  // 2 per sub-pulse table entry: cos α, sin α
    int n_pcls = 0, n_e1 = 0, n_e2 = 0;
    int64_t n_adc = 0;
    int64_t n_snap = 0;  // snapshots (OP_SNAP operations) in the program
    std::vector<int32_t> tmap;  // 4 per train-map kind: phasor class, T1 class, first table entry, sub-pulses
};

// Returns an mrsim_status; on failure `err` says why.
// snap_after: NULL or n_snap strictly increasing event indices after which every spin's state is
// recorded (§7.2: magnetisation data at chosen times).
// rf_param: NULL, or per event a learnable-flip index in [0, n_params) or -1.  Events with an index
// become parametric pulses: their (cos α, sin α) are read at run time from sub-pulse table entry
// index (the table's first n_params entries, which the caller fills before each launch).  Only the
// float64 kernel reads such tables; the float32 program of a parametric compile is not runnable.
int compile_sequence(const mrsim_event *ev, int64_t n, double gamma_hz, Compiled &out, std::string &err,
                     int64_t n_snap = 0, const int64_t *snap_after = nullptr, const int32_t *rf_param = nullptr,
                     int32_t n_params = 0);

}  // namespace mrsim
