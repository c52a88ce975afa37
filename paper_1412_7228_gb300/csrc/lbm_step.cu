// lbm_step.cu -- the tile-configuration tables of the fused step kernels
// (lbm_step_kernels.cuh, instantiated per precision in lbm_step_f32.cu and
// lbm_step_f64.cu) behind the host interface of lbm_internal.cuh.
#include "lbm_step_kernels.cuh"

namespace lbm {

const Entry* step_table_f32(int* n);
const Entry* step_table_f64(int* n);

namespace {
const Entry* table(int prec, int* n) { return prec == LBM_FP32 ? step_table_f32(n) : step_table_f64(n); }
}  // namespace

int step_config_count(int prec) {
    int n;
    table(prec, &n);
    return n;
}

TileCfg step_config(int prec, int k) {
    int n;
    const Entry* e = table(prec, &n);
    return e[k].tc();
}

size_t step_smem_bytes(int prec, int k) {
    int n;
    const Entry* e = table(prec, &n);
    return e[k].smem();
}

cudaError_t step_prepare(int prec, int k) {
    int n;
    const Entry* e = table(prec, &n);
    return e[k].prepare();
}

cudaError_t step_launch(int prec, int k, const Inst* d_insts, const void* args, bool one, int ntiles, int parity,
                        unsigned long long timeout_ns, cudaStream_t st) {
    int n;
    const Entry* e = table(prec, &n);
    return e[k].launch(d_insts, args, one, ntiles, parity, timeout_ns, st);
}

bool run_supported(int prec, int k) {
    int n;
    const Entry* e = table(prec, &n);
    return k >= 0 && k < n && e[k].nbuf == 1;
}

cudaError_t run_launch(int prec, int k, const Inst* d_insts, const void* args, bool one, int ntiles, int nsteps,
                       unsigned long long timeout_ns, cudaStream_t st) {
    int n;
    const Entry* e = table(prec, &n);
    return e[k].run(d_insts, args, one, ntiles, nsteps, timeout_ns, st);
}

}  // namespace lbm
