// lbm_init.h -- the initial equilibrium of a time level written in row
// bands (lbm_aux.cu), for an initial field that reaches the device band by
// band: each band's kernel can start while the next band is still being
// copied from the host.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// f_a = f_eq,a(rho, u) (u = 0 where ux and uy are NULL) of the nodes of rows
// [y0, y1) into time level `parity` of one instance, at their streamed
// positions (periodic); rho, ux and uy are device arrays of the whole
// nx x ny field, FP32 when f32 is set, else FP64.  The ghost cells are left
// to aux_fill_ghosts once every row is written.  cudaErrorInvalidValue for
// an empty or out-of-range band.
cudaError_t aux_init_rows(const Inst& host, const Inst* d_inst, const void* rho, const void* ux, const void* uy,
                          bool f32, int parity, int y0, int y1, cudaStream_t st);

}  // namespace lbm
