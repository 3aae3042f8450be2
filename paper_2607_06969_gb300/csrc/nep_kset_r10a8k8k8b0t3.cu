// Kernel instance: n_rad=10 n_ang=8 k_rad=8 k_ang=8 has_4body=0 n_types=3.
#include "nep_train.cuh"

namespace nep {
NEP_DEFINE_KERNEL_SET(kset_r10a8k8k8b0t3, 10, 8, 8, 8, 0, 3)
}  // namespace nep
