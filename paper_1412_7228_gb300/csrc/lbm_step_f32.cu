// lbm_step_f32.cu -- the FP32 instantiations of the fused step kernels (one-step and
// multi-step) for every tile configuration the autotuner may pick; compiled
// as a translation unit of its own so that the two precisions build in parallel.
#include "lbm_step_kernels.cuh"

namespace lbm {
namespace {
const Entry kF32[] = {
    LBM_CFG(float, 128, 16, 512, 1), LBM_CFG(float, 64, 16, 256, 1), LBM_CFG(float, 128, 8, 256, 1),
    LBM_CFG(float, 64, 32, 512, 1),  LBM_CFG(float, 32, 32, 256, 1), LBM_CFG(float, 64, 16, 256, 2),
    LBM_CFG(float, 64, 8, 256, 2),   LBM_CFG(float, 32, 16, 256, 2),  LBM_CFG(float, 64, 16, 512, 2),
};
}  // namespace

const Entry* step_table_f32(int* n) {
    *n = int(sizeof(kF32) / sizeof(kF32[0]));
    return kF32;
}

}  // namespace lbm
