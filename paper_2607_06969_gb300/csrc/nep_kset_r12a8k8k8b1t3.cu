// Kernel instance: n_rad=12 n_ang=8 k_rad=8 k_ang=8 has_4body=1 n_types=3.
#include "nep_train.cuh"

namespace nep {
NEP_DEFINE_KERNEL_SET(kset_r12a8k8k8b1t3, 12, 8, 8, 8, 1, 3)
}  // namespace nep
