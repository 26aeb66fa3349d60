// fwd_f32.cu -- float32 instantiations of the forward kernel (K = spins per thread).
#include "fwd_kernel.cuh"

namespace mrsim {

int launch_fwd_f32(const FwdArgs &a, int k, int threads, void *stream) {
    switch (k) {
    case 1: return dev::launch_one<float, 1, 512>(a, threads, stream);
    case 2: return dev::launch_one<float, 2, 512>(a, threads, stream);
    case 4: return dev::launch_one<float, 4, 512>(a, threads, stream);
    case 8: return dev::launch_one<float, 8, 256>(a, threads, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

int fwd_blocks_per_sm_f32(int k, int threads, size_t smem) {
    switch (k) {
    case 1: return dev::blocks_per_sm<float, 1, 512>(threads, smem);
    case 2: return dev::blocks_per_sm<float, 2, 512>(threads, smem);
    case 4: return dev::blocks_per_sm<float, 4, 512>(threads, smem);
    case 8: return dev::blocks_per_sm<float, 8, 256>(threads, smem);
    default: return 0;
    }
}

int launch_batch_f32(const BatchArgs &b, int k, int threads, size_t smem, int grid, void *stream) {
    switch (k) {
    case 1: return dev::launch_batch_one<float, 1, 512>(b, threads, smem, grid, stream);
    case 2: return dev::launch_batch_one<float, 2, 512>(b, threads, smem, grid, stream);
    case 4: return dev::launch_batch_one<float, 4, 512>(b, threads, smem, grid, stream);
    case 8: return dev::launch_batch_one<float, 8, 256>(b, threads, smem, grid, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

int batch_blocks_per_sm_f32(int k, int threads, size_t smem) {
    switch (k) {
    case 1: return dev::batch_blocks_per_sm<float, 1, 512>(threads, smem);
    case 2: return dev::batch_blocks_per_sm<float, 2, 512>(threads, smem);
    case 4: return dev::batch_blocks_per_sm<float, 4, 512>(threads, smem);
    case 8: return dev::batch_blocks_per_sm<float, 8, 256>(threads, smem);
    default: return 0;
    }
}

int fwd_regs_f32(int k) {
    switch (k) {
    case 1: return dev::regs_of<float, 1, 512>();
    case 2: return dev::regs_of<float, 2, 512>();
    case 4: return dev::regs_of<float, 4, 512>();
    case 8: return dev::regs_of<float, 8, 256>();
    default: return 0;
    }
}

int coil_spins_per_thread_f32(int n_coils) { return n_coils > 2 ? 4 : 2; }

int launch_fwd_coils_f32(const FwdArgs &a, int threads, void *stream) {
    if (a.n_coils <= 1) return dev::launch_one<float, 2, 512, 1>(a, threads, stream);
    if (a.n_coils <= 2) return dev::launch_one<float, 2, 512, 2>(a, threads, stream);
    if (a.n_coils <= 4) return dev::launch_one<float, 4, 256, 4>(a, threads, stream);
    if (a.n_coils <= MAX_COILS) return dev::launch_one<float, 4, 256, 8>(a, threads, stream);
    return (int)cudaErrorInvalidValue;
}

}  // namespace mrsim
