// Table of the compiled hyper-parameter instances.
#include "nep_internal.h"

namespace nep {

extern const KernelSet kset_r8a6k8k8b1t3;    // 216-atom / 900k / training / replica workloads
extern const KernelSet kset_r12a8k8k8b1t3;   // 3.7M-atom workload (larger NEP)
extern const KernelSet kset_r10a8k8k8b0t3;   // the paper's Table 2 model (2+3-body)
extern const KernelSet kset_r3a2k4k3b1t3;    // small model for exhaustive gradient tests

const KernelSet* find_kernel_set(int n_rad, int n_ang, int k_rad, int k_ang, int has_4body,
                                 int n_types) {
    static const KernelSet* all[] = {&kset_r8a6k8k8b1t3, &kset_r12a8k8k8b1t3, &kset_r10a8k8k8b0t3,
                                     &kset_r3a2k4k3b1t3};
    for (const KernelSet* k : all)
        if (k->n_rad == n_rad && k->n_ang == n_ang && k->k_rad == k_rad && k->k_ang == k_ang &&
            k->has_4body == has_4body && k->n_types == n_types)
            return k;
    return nullptr;
}

}  // namespace nep
