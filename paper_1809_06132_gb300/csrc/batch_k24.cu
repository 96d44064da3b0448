// Batched sweep kernels with 24-row tiles (one and two planes per pass).
#include "batch_dev.cuh"

namespace ps {

const void* batch_kernel_th24(int kp) {
    return kp == 1 ? reinterpret_cast<const void*>(&batch_kernel<24, 1>)
                   : reinterpret_cast<const void*>(&batch_kernel<24, 2>);
}

}  // namespace ps

namespace ps {
PS_DEFINE_CHECK_READER(check_bits_batch24)
}  // namespace ps
