// lbm_static.cu -- lbm_field_pressure_jump_static: the Laplace-law sums of
// lbm_batch_measure over a density field the caller already holds in device
// memory, with no device allocation of any kind.
//
// Who needs it: code that cannot call cudaMalloc -- for example a caller whose
// device memory is entirely owned by another allocator (a framework's caching
// allocator or a fixed arena reserved at start-up, where a fresh cudaMalloc
// fails or breaks the memory budget), or a latency-critical loop that must not
// pay for an allocation call that can synchronise the whole device.  Those
// callers pass the input field and a host output array and nothing else.
//
// Scratch: the per-block partial sums live in g_scratch, a file-scope
// __device__ array.  Every GPU that loads this library holds it (about 128 KiB)
// until the process exits.  Host code cannot use the symbol itself as a device
// address, so the first call on each device looks its address up with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture begins.  Every call copies its eight
// totals to host memory and synchronises its stream before it returns.  All
// calls share the array and it keeps the previous call's contents: each
// block writes every slot it later reads, so nothing has to be cleared, but
// two calls whose kernels overlap on the GPU (different streams or host
// threads) race on it.
//
// The field must be device memory of the current device: the call checks
// this (cudaPointerGetAttributes) and rejects anything else with
// LBM_EINVAL, as it rejects an equation of state that lbm_set_params would
// reject, before any GPU work.
#include <cmath>
#include <cstring>
#include <mutex>

#include "lbm_eos_host.h"
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticPerThread = 32;
constexpr int kStaticNodesPerBlock = kStaticThreads * kStaticPerThread;   // 8192
constexpr int kStaticMaxBlocks = LBM_STATIC_MAX_NODES / kStaticNodesPerBlock;
constexpr int kSlots = 8;
static_assert(LBM_STATIC_MAX_NODES % kStaticNodesPerBlock == 0, "maximum must be a whole number of blocks");

// partial sums of up to kStaticMaxBlocks blocks, then the 8 totals
static __device__ __align__(256) double g_scratch[kStaticMaxBlocks * kSlots + kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

// {sum rho, sum p_in, sum rho_in, n_in, sum p_out, sum rho_out, n_out, 0}
__global__ void __launch_bounds__(kStaticThreads)
    k_field_sums(const double* __restrict__ rho, int nx, int ny, Phys<double> P, double cxc, double cyc, double r_in,
                 double r_out, double* __restrict__ partials) {
    __shared__ double red[kStaticThreads / 32][kSlots];
    const long long N = static_cast<long long>(nx) * ny;
    const long long base = static_cast<long long>(blockIdx.x) * kStaticNodesPerBlock;
    double v[kSlots] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < kStaticPerThread; ++k) {
        const long long i = base + k * kStaticThreads + threadIdx.x;
        if (i >= N) break;
        const int x = static_cast<int>(i % nx), y = static_cast<int>(i / nx);
        const double r = rho[i];
        double dx = x - cxc, dy = y - cyc;
        dx -= nx * rint(dx / nx);
        dy -= ny * rint(dy / ny);
        const double d = sqrt(dx * dx + dy * dy);
        v[0] += r;
        if (d <= r_in) {
            v[1] += p_eos(P, r);
            v[2] += r;
            v[3] += 1.0;
        }
        if (d >= r_out) {
            v[4] += p_eos(P, r);
            v[5] += r;
            v[6] += 1.0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        double x = v[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][s] = x;
    }
    __syncthreads();
    if (threadIdx.x < kSlots) {
        double x = red[0][threadIdx.x];
        for (int w = 1; w < kStaticThreads / 32; ++w) x += red[w][threadIdx.x];
        partials[blockIdx.x * kSlots + threadIdx.x] = x;
    }
}

__global__ void k_field_sums_finish(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    const int s = threadIdx.x;
    if (s >= kSlots) return;
    double x = partials[s];
    for (int b = 1; b < nblocks; ++b) x += partials[b * kSlots + s];
    out[s] = x;
}

// Address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

// d_rho is device (or managed) memory whose device is the current one.
bool on_current_device(const void* p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // the query's own error, not a pending one of the caller
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_field_pressure_jump_static(const double* d_rho, int nx, int ny, const lbm_eos* eos, double cx,
                                              double cy, double r_in, double r_out, double* out, void* stream) {
    using namespace lbm;
    if (!d_rho || !out || nx < 1 || ny < 1 || !(r_in >= 0) || !(r_out >= 0)) return LBM_EINVAL;
    if (!std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(r_in) || !std::isfinite(r_out)) return LBM_EINVAL;
    if (!eos_valid_at(eos)) return LBM_EINVAL;   // the laws and temperatures lbm_set_params accepts
    const long long N = static_cast<long long>(nx) * ny;
    if (N > LBM_STATIC_MAX_NODES) return LBM_EINVAL;   // the static scratch holds partials for at most this many nodes
    if (!on_current_device(d_rho)) return LBM_EINVAL;
    double* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return LBM_ECUDA;

    Phys<double> P;
    std::memset(&P, 0, sizeof P);
    fill_eos(P, *eos);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int blocks = static_cast<int>((N + kStaticNodesPerBlock - 1) / kStaticNodesPerBlock);
    double* partials = scratch;
    double* totals = scratch + kStaticMaxBlocks * kSlots;
    // cudaLaunchKernel returns this launch's own error (never an earlier one)
    void* a1[] = {&d_rho, &nx, &ny, &P, &cx, &cy, &r_in, &r_out, &partials};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_field_sums), dim3(blocks), dim3(kStaticThreads), a1, 0, st) !=
        cudaSuccess)
        return LBM_ECUDA;
    void* a2[] = {&partials, &blocks, &totals};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_field_sums_finish), dim3(1), dim3(32), a2, 0, st) !=
        cudaSuccess)
        return LBM_ECUDA;
    double s[kSlots];
    if (cudaMemcpyAsync(s, totals, sizeof s, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ECUDA;

    const double p_in = s[3] > 0 ? s[1] / s[3] : NAN, rho_in = s[3] > 0 ? s[2] / s[3] : NAN;
    const double p_out = s[6] > 0 ? s[4] / s[6] : NAN, rho_out = s[6] > 0 ? s[5] / s[6] : NAN;
    const double ex = s[0] - rho_out * static_cast<double>(N);
    const double R_eq = std::sqrt((ex > 0 ? ex : 0.0) / (M_PI * (rho_in - rho_out)));
    const double vals[LBM_MEASURE_N] = {p_in, p_out, rho_in, rho_out, R_eq, s[0], s[3], s[6]};
    std::memcpy(out, vals, sizeof vals);
    return LBM_OK;
}
