// Mixed-precision leaf products on the bf16 tensor cores (tcgen05).
// Not built yet: mixed_available() reports 0 and SPAMM_MIXED returns
// SPAMM_ENOTSUP.
#include "common.cuh"

namespace spamm {

int mixed_available() { return 0; }

int gemm_mixed(spamm_ctx*, const spamm_mat*, const spamm_mat*, const Plan&, const Epilogue&,
               spamm_mat*, double*, double*, double*) {
    set_error("mixed-precision leaf products are not available in this build");
    return SPAMM_ENOTSUP;
}

}  // namespace spamm
