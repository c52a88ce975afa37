// lbm_step_f64.cu -- the FP64 instantiations of the fused step kernels (one-step and
// multi-step) for every tile configuration the autotuner may pick; compiled
// as a translation unit of its own so that the two precisions build in parallel.
#include "lbm_step_kernels.cuh"

namespace lbm {
namespace {
const Entry kF64[] = {
    LBM_CFG(double, 32, 8, 256, 1),  LBM_CFG(double, 64, 8, 256, 1), LBM_CFG(double, 32, 16, 256, 1),
    LBM_CFG(double, 64, 4, 256, 1),  LBM_CFG(double, 32, 8, 256, 2),  LBM_CFG(double, 64, 16, 256, 1),
    LBM_CFG(double, 32, 32, 256, 1),
};
}  // namespace

const Entry* step_table_f64(int* n) {
    *n = int(sizeof(kF64) / sizeof(kF64[0]));
    return kF64;
}

}  // namespace lbm
