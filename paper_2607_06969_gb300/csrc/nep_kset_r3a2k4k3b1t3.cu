// Kernel instance: n_rad=3 n_ang=2 k_rad=4 k_ang=3 has_4body=1 n_types=3.
#include "nep_train.cuh"

namespace nep {
NEP_DEFINE_KERNEL_SET(kset_r3a2k4k3b1t3, 3, 2, 4, 3, 1, 3)
}  // namespace nep
