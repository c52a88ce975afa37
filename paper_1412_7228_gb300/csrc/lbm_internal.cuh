// lbm_internal.cuh -- device data layout, per-instance descriptors and the
// PTX helpers (mbarrier, TMA) shared by the sm_103a kernels of liblbm.
//
// HBM layout of one instance in precision T (float: deviations from
// t_a rho_ref; double: same, rho_ref may be 0):
//   pop[k][a][Y][X],  k in {0,1} the two time levels, a = 0..8,
//   Y = y + GY (GY = 2 ghost rows above and below),
//   X = x + GX (GX = 32 bytes / sizeof(T) ghost columns on the left, so an
//   interior row starts on a 32-byte sector), row pitch a multiple of 32 B.
// The array holds post-collision populations at their source node ("pull"
// storage): the pre-collision f_a(x, t) is pop[a][x - e_a].  Ghost cells
// hold periodic images, written by the step kernel for border nodes, so a
// tile's halo is one rectangular TMA box with no wrap logic.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int GY = 2;          // ghost rows per side
constexpr int kMaxSched = 5;   // CTA schedules known to lbm_set_schedule (3: multi-step persistent, 4: cluster)

template <typename T> struct Prec;
template <> struct Prec<float> { static constexpr int GX = 8; static constexpr int HX = 4; };
template <> struct Prec<double> { static constexpr int GX = 4; static constexpr int HX = 2; };

// Lattice velocity components e_a.
__host__ __device__ constexpr int cx(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}

// Status bits of an instance (sticky until cleared or re-initialised).
constexpr int ST_UNSTABLE = 1;
constexpr int ST_TIMEOUT = 2;

// Physics parameters in the kernel's precision.
template <typename T> struct Phys {
    int eos;            // LBM_EOS_*
    unsigned flags;     // LBM_FLAG_*
    T K, a, b, b4, RT, aalpha;   // EOS; b4 = b/4 (CS), aalpha = a alpha(T) (PR)
    T A, kappa, G, two_over_G;   // Eq. 9, Eq. 23, Eq. 10
    T s[9];             // Lambda
    T hs[9];            // 1 - s/2, the forcing weight of Eq. 5
    T ns[9], nhs[9];    // -s, -hs
    T h2s7;             // 2 hs[7] (exact)
    T h6s1, nh6s2;      // 6 hs[1], -6 hs[2]: the forcing weights of S[1] = 6 v.F, S[2] = -6 v.F
    T c1, c2;           // C[1] = c1 tr Q, C[2] = c2 tr Q (Eq. 26)
    T rho_ref;          // deviation reference
    int interact;       // 0 when G == 0: no psi, F = Q = 0
    // density-dependent shear viscosity: nu(rho) linear between (rho_g, nu_g)
    // and (rho_l, nu_l), clamped; s_7 = s_8 = 1 / (3 nu + 1/2)
    int var_visc;
    T nu_g, dnu, visc_rho_g, visc_inv_drho;
};

// One lattice, as the kernels see it in global memory.  Its TMA tensor maps
// are not here: they travel in the kernel argument blocks below.
struct alignas(128) Inst {
    void* pop[2];
    int* status;
    int nx, ny, pitch, nyp;  // pitch, nyp in elements
    long long plane;         // pitch * nyp
    Phys<float> pf;
    Phys<double> pd;
    int prec;                // LBM_FP32 / LBM_FP64
    int pad_[3];
};

// Everything a single-lattice step needs, passed by value as a
// __grid_constant__ kernel argument: the tensor maps and constants then live
// in the parameter bank, and tile coordinates come from blockIdx.
template <typename T> struct StepArgs {   // CUtensorMap members give it their alignment
    CUtensorMap tmap[2];
    Phys<T> P;
    void* pop[2];
    int* status;
    long long plane;
    int nx, ny, pitch, tiles_x;
};

// What a batched launch needs, passed by value as a __grid_constant__
// kernel argument as well: for up to kBatchLaunchMax instances their tensor
// maps (in parameter space a map needs neither a load of its own nor a
// tensormap proxy fence, which a map in global memory needs before every
// first use in a CTA) and tile counts; in FP32 also their array addresses,
// sizes and constants, so that the FP32 step reads nothing but populations
// from global memory (FP64, bound by its FP64 pipe, reads those from the
// instance descriptors: 64 FP64 constant sets would not fit the 32 KB
// argument space).  Slot k's tiles are first[k] .. first[k+1]-1, row-major
// over tiles_x[k] columns; with a tile table (the interleaved schedule)
// entry t gives (slot, x0, y0) instead.  A batch with more instances is
// stepped by several launches.
constexpr int kBatchLaunchMax = 64;
struct SlotLattice {                     // the fields of Inst the step uses
    void* pop[2];
    int* status;
    long long plane;
    int nx, ny, pitch, pad_;
};
template <typename T> struct BatchPhys {};
template <> struct BatchPhys<float> {
    Phys<float> P[kBatchLaunchMax];
};
template <typename T> struct BatchArgs {
    CUtensorMap tmap[kBatchLaunchMax];   // maps of the source time level of slot k
    const int4* tiles;                   // tile table, or nullptr: tiles in slot order
    int first[kBatchLaunchMax + 1];      // first tile of slot k; first[n] = tiles of the launch
    int tiles_x[kBatchLaunchMax];        // tile columns of slot k
    unsigned div_m[kBatchLaunchMax];     // division by tiles_x[k]: see tile_row()
    int div_s[kBatchLaunchMax];
    int inst[kBatchLaunchMax];           // slot k -> index into the Inst array
    int n;                               // slots in use, 1..kBatchLaunchMax
    SlotLattice lat[kBatchLaunchMax];    // read by FP32 launches
    BatchPhys<T> phys;                   // FP32 only
};

// What a multi-step persistent launch needs (schedule 3): for up to
// kRunMax instances the tensor maps of both time levels, tile counts, array
// addresses and sizes, FP32 constants, and the launch's work counter and the
// per-tile step counters in global memory.  Work item w is step w / ntiles
// of tile w % ntiles (tiles in slot order, row-major within an instance); a
// CTA takes items in that order and starts step s of a tile once every tile
// within two nodes of it (periodic within the instance: its 3 x 3 tile
// neighbourhood, and the tile beyond a last tile row or column one node
// wide) has finished step s - 1.
constexpr int kRunMax = 32;
template <typename T> struct RunPhys {};
template <> struct RunPhys<float> {
    Phys<float> P[kRunMax];
};
template <typename T> struct RunArgs {
    CUtensorMap tmap[2][kRunMax];        // [time level][slot]
    int first[kRunMax + 1];              // first tile of slot k; first[n] = ntiles
    int tiles_x[kRunMax];                // tile columns of slot k
    int inst[kRunMax];                   // slot k -> index into the Inst array
    int n;                               // slots in use, 1..kRunMax
    int ntiles;                          // tiles of all slots
    int nsteps;                          // steps this launch performs
    int parity0;                         // time level the first step reads
    int* done;                           // per tile: steps it has completed in this launch
    unsigned long long* counter;         // next work item
    int* abort_flag;                     // set when a bounded wait gave up: every CTA stops
    SlotLattice lat[kRunMax];            // read by FP32 launches
    RunPhys<T> phys;                     // FP32 only
};

// kernel parameters are limited to 32,764 bytes
static_assert(sizeof(BatchArgs<float>) <= 32764 && sizeof(BatchArgs<double>) <= 32764, "argument block too large");
static_assert(sizeof(RunArgs<float>) <= 32764 && sizeof(RunArgs<double>) <= 32764, "argument block too large");

// floor(r / d) for 0 <= r < 2^31 and d >= 1 as one 64-bit multiply and a
// shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d), m = ceil(2^(31+l) / d) and
// s = 31 + l, m d - 2^s lies in [0, d - 1] and d <= 2^l, so
// r m / 2^s = r / d + e with 0 <= e < 1/d, which cannot reach the next
// integer; m < 2^32.  The host computes (m, s) per instance and checks the
// result for every tile it launches.
__host__ __device__ __forceinline__ int tile_row(int r, unsigned m, int s) {
    return static_cast<int>((static_cast<unsigned long long>(r) * m) >> s);
}
inline void tile_row_magic(int d, unsigned* m, int* s) {
    int l = 0;
    while ((1ll << l) < d) ++l;
    *s = 31 + l;
    *m = static_cast<unsigned>(((1ull << (31 + l)) + static_cast<unsigned long long>(d) - 1) /
                               static_cast<unsigned long long>(d));
}

template <typename T> __device__ __forceinline__ const Phys<T>& phys(const Inst* I);
template <> __device__ __forceinline__ const Phys<float>& phys<float>(const Inst* I) { return I->pf; }
template <> __device__ __forceinline__ const Phys<double>& phys<double>(const Inst* I) { return I->pd; }

// Pressure law (Eq. 21 / Eq. 29 / Carnahan-Starling); K scales the whole law.
template <typename T> __device__ __forceinline__ T p_eos(const Phys<T>& P, T rho) {
    if (P.eos == LBM_EOS_CS) {
        T n = P.b4 * rho;
        T q = T(1) - n;
        T num = T(1) + n * (T(1) + n * (T(1) - n));
        return P.K * (rho * P.RT * num / (q * q * q) - P.a * rho * rho);
    } else if (P.eos == LBM_EOS_VDW) {
        return P.K * (rho * P.RT / (T(1) - P.b * rho) - P.a * rho * rho);
    } else {
        T br = P.b * rho;
        return P.K * (rho * P.RT / (T(1) - br) - P.aalpha * rho * rho / (T(1) + T(2) * br - br * br));
    }
}

// Radicand of Eq. 10 with c = 1: psi^2 = 2 (p_EOS - rho/3) / G.
template <typename T> __device__ __forceinline__ T psi_radicand(const Phys<T>& P, T rho) {
    return P.two_over_G * (p_eos(P, rho) - rho * T(1.0 / 3.0));
}

// Division, reciprocal and square root of the fused step.  FP32 uses the
// hardware approximations (a couple of ulp, far inside the FP32 error budget
// of the stored populations).  FP64 refines the hardware estimates
// (rcp.approx / rsqrt.approx, accurate to about 2^-22) with two steps of a
// quadratically converging iteration, which leaves only the rounding of the
// last step: 1/d by Newton-Raphson (e = 1 - d r, r <- r + r e), sqrt(x) by
// Goldschmidt's coupled iteration (g -> sqrt(x), h -> 1/(2 sqrt(x)):
// r = 1/2 - g h, g <- g + g r, h <- h + h r).  Both stay within 1 ulp of the
// IEEE-rounded 1/d and sqrt(x), a * rcp(d) within 1 ulp of a/d
// (lbm_fp64_math_check measures this on the device); they take fewer FP64
// operations than the IEEE sequences, and the FP64 step is bound by its FP64
// pipe.  sqrt keeps sqrt(+-0) = +-0 and NaN for x < 0.
template <typename T> struct Fast;
template <> struct Fast<float> {
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
    static __device__ __forceinline__ float sqrt(float a) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
};
template <> struct Fast<double> {
    static __device__ __forceinline__ double rcp(double d) {
        double r;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
        double e = fma(-d, r, 1.0);
        r = fma(r, e, r);
        e = fma(-d, r, 1.0);
        return fma(r, e, r);
    }
    static __device__ __forceinline__ double div(double a, double b) { return a * rcp(b); }
    static __device__ __forceinline__ double sqrt(double x) {
        double y;
        asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
        double g = x * y, h = 0.5 * y;
        double r = fma(-g, h, 0.5);
        g = fma(g, r, g);
        h = fma(h, r, h);
        r = fma(-g, h, 0.5);
        g = fma(g, r, g);
        return (__double_as_longlong(x) << 1) == 0 ? x : g;   // +-0: rsqrt is infinite there
    }
};

// ---- PTX helpers --------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete, giving up after
// timeout_ns of wall time.  Returns true when the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

// Global-memory flags shared between the CTAs of one persistent launch.
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Orders this thread's earlier generic-proxy accesses (the acquire above)
// before its later async-proxy ones (a TMA load of data other CTAs stored).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// 3-D tiled TMA load of a box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace lbm

// ---- host-side interfaces between the translation units -----------------
namespace lbm {

struct TileCfg { int bx, by, threads, stages; };

// Fused step (lbm_step.cu).
int step_config_count(int prec);
TileCfg step_config(int prec, int k);
size_t step_smem_bytes(int prec, int k);
cudaError_t step_prepare(int prec, int k);   // sets the dynamic smem attribute
// args: a StepArgs<T> for a context of one lattice (one = true; tile
// coordinates from blockIdx), else a BatchArgs<T> of up to kBatchLaunchMax
// instances, T the context's precision.  ntiles: tiles this launch steps.
cudaError_t step_launch(int prec, int k, const Inst* d_insts, const void* args, bool one, int ntiles, int parity,
                        unsigned long long timeout_ns, cudaStream_t st);
// Multi-step persistent launch of tile configuration k (one box per CTA
// only; false otherwise): args a RunArgs<T>, one = a single instance.  The
// caller has zeroed the step counters, the work counter and the abort flag.
bool run_supported(int prec, int k);
cudaError_t run_launch(int prec, int k, const Inst* d_insts, const void* args, bool one, int ntiles, int nsteps,
                       unsigned long long timeout_ns, cudaStream_t st);

// One lattice held in the shared memory of a thread-block cluster for n
// steps (lbm_cluster.cu; schedule 4): whether this device can run it for an
// nx x ny lattice of precision prec, and the launch (host: the descriptor;
// the caller refills the ghost cells of the time level written last).
bool cluster_supported(int prec, int nx, int ny);
cudaError_t cluster_run(const Inst& host, int parity, int nsteps, cudaStream_t st);

// Auxiliary kernels (lbm_aux.cu); `host` is the host copy of the descriptor.
// Fields of nx*ny doubles, or floats with f32 (each widened to FP64 exactly).
cudaError_t aux_init(const Inst& host, const Inst* d_inst, const void* rho, const void* ux, const void* uy, bool f32,
                     int parity, cudaStream_t st);
cudaError_t aux_fill_ghosts(const Inst& host, const Inst* d_inst, int parity, cudaStream_t st);
// bad |= 1: a density not finite, positive and below rho_max; |= 2: a velocity not finite
cudaError_t aux_check_init(const void* rho, const void* ux, const void* uy, bool f32, long long N, double rho_max,
                           int* bad, cudaStream_t st);
cudaError_t aux_gather_plane(const Inst& host, const Inst* d_inst, int parity, int a, double* out,
                             cudaStream_t st);
// field: 0 rho, 1 ux, 2 uy, 3 psi; rows [y0, y1), written at their place in
// out (row-major, nx per row)
cudaError_t aux_field(const Inst& host, const Inst* d_inst, int parity, int field, int y0, int y1, void* out,
                      bool f32out, cudaStream_t st);   // f32out: floats, each the FP64 value rounded to nearest
// out: 4 device words (see lbm_fp64_math_check); default stream.
cudaError_t aux_math_check(long long n, double lo, double hi, unsigned long long* out);
// FP64 FMA throughput of the current device (see lbm_fp64_fma_rate).
cudaError_t aux_fp64_fma_rate(int iters, cudaStream_t st, double* flops_per_s, double* seconds);
constexpr int kReduceBlocks = 304;   // 2 CTAs per SM of a 152-SM GB300: partial sums of FP64 reductions
constexpr int kReduceSlots = 8;
cudaError_t aux_measure(const Inst& host, const Inst* d_inst, int parity, double cx, double cy,
                        double r_in, double r_out, double* partials, double* result,
                        cudaStream_t st);
cudaError_t aux_stats(const Inst& host, const Inst* d_inst, int parity, double* partials,
                      double* result, cudaStream_t st);

}  // namespace lbm
