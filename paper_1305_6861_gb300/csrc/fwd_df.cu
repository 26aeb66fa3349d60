// fwd_df.cu -- double-float instantiations of the forward and batch kernels: the compensated
// precision (MRSIM_FP32_KAHAN), float32 pairs (hi, lo) on the FP32 pipe with the float64 program
// and layouts (K = 1 or 2 spins per thread, as float64).
#include "fwd_kernel.cuh"

namespace mrsim {

int launch_fwd_df(const FwdArgs &a, int k, int threads, void *stream) {
    switch (k) {
    case 1: return dev::launch_one<dev::dfl, 1, 256>(a, threads, stream);
    case 2: return dev::launch_one<dev::dfl, 2, 256>(a, threads, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

int launch_batch_df(const BatchArgs &b, int k, int threads, size_t smem, int grid, void *stream) {
    switch (k) {
    case 1: return dev::launch_batch_one<dev::dfl, 1, 256>(b, threads, smem, grid, stream);
    case 2: return dev::launch_batch_one<dev::dfl, 2, 256>(b, threads, smem, grid, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

int batch_blocks_per_sm_df(int k, int threads, size_t smem) {
    switch (k) {
    case 1: return dev::batch_blocks_per_sm<dev::dfl, 1, 256>(threads, smem);
    case 2: return dev::batch_blocks_per_sm<dev::dfl, 2, 256>(threads, smem);
    default: return 0;
    }
}

int fwd_blocks_per_sm_df(int k, int threads, size_t smem) {
    switch (k) {
    case 1: return dev::blocks_per_sm<dev::dfl, 1, 256>(threads, smem);
    case 2: return dev::blocks_per_sm<dev::dfl, 2, 256>(threads, smem);
    default: return 0;
    }
}

int fwd_regs_df(int k) {
    switch (k) {
    case 1: return dev::regs_of<dev::dfl, 1, 256>();
    case 2: return dev::regs_of<dev::dfl, 2, 256>();
    default: return 0;
    }
}

}  // namespace mrsim
