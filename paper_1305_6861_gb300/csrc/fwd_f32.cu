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

}  // namespace mrsim
