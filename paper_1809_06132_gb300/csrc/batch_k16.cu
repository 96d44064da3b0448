// Batched sweep kernels with 16-row tiles (one and two planes per pass).
#include "batch_dev.cuh"

namespace ps {

const void* batch_kernel_th16(int kp) {
    return kp == 1 ? reinterpret_cast<const void*>(&batch_kernel<16, 1>)
                   : reinterpret_cast<const void*>(&batch_kernel<16, 2>);
}

}  // namespace ps

namespace ps {
PS_DEFINE_CHECK_READER(check_bits_batch16)
}  // namespace ps
