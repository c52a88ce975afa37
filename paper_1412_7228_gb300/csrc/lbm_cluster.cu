// lbm_cluster.cu -- the fused step of a small lattice held in the shared
// memory of one thread-block cluster for all the steps of an lbm_step call
// (schedule 4).
//
// The lattice is cut into strips of BY rows, one per CTA of a cluster of up
// to 16 CTAs (one CTA per SM).  Each CTA keeps two boxes of its strip (all
// nine planes, the strip plus two halo rows above and below and the halo
// columns of the one-step kernel's TMA box) in shared memory: the step's
// input and output time levels.  Per step a CTA
//   1. computes rho and psi (Eq. 10) of its strip and 1-node ring from the
//      input box (the same psi_ring as the one-step kernels);
//   2. collides and streams every owned node into the output box (the same
//      collide_rows, with the output addressed into shared memory);
//   3. writes the periodic images of the output's edge columns (x) into its
//      halo columns, and stores its first two output rows into the bottom
//      halo rows of the CTA above it and its last two into the top halo rows
//      of the CTA below it (periodic in y through the cluster ranks), in
//      their shared memory (distributed shared memory of the cluster);
//   4. waits at a cluster barrier, after which every output box is complete.
// The per-node arithmetic is that of the one-step kernels on the same box
// contents, so every schedule gives the same bits.  Nothing goes to global
// memory between steps: the populations are read once at the start and
// written once at the end (their ghost cells are then refilled by the
// caller).  No wait in this kernel spins in software: the cluster barrier
// is the hardware's, every CTA of the cluster runs the same number of steps
// and none leaves early, and a CTA's shared memory is only written by the
// others between two barriers that it takes part in.
#include "lbm_step_kernels.cuh"

namespace lbm {
namespace {

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster: this CTA's shared-memory writes
// (local and remote) before the barrier are visible to all after it.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::
            : "memory");
}
// The address in the shared memory of cluster CTA `rank` of the same
// offset as the local shared-memory address `addr`.
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

template <typename T> struct ClusterArgs {
    Phys<T> P;
    const T* src;      // time level read by the first step
    T* dst;            // time level written by the last step
    long long plane;   // elements per plane of the global arrays
    int pitch;         // elements per row of the global arrays
    int nx, ny, nsteps;
    int* status;
};

template <typename T, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT, 1) k_cluster(const __grid_constant__ ClusterArgs<T> a) {
    using Gm = Geom<T, BX, BY, NT, 1>;
    constexpr int WB = Gm::WB, PB = Gm::PB, HX = Gm::HX;
    constexpr int GXg = Prec<T>::GX;   // ghost columns of the global arrays
    extern __shared__ __align__(1024) unsigned char smem[];
    T* const box0 = reinterpret_cast<T*>(smem);
    T* const box1 = reinterpret_cast<T*>(smem + Gm::buf_stride);
    T* const sp = reinterpret_cast<T*>(smem + 2 * Gm::buf_stride);
    const int tid = threadIdx.x, tx = tid % BX, ty = tid / BX;
    const unsigned rank = cluster_rank(), C = cluster_size();
    const int nx = a.nx, ny = a.ny;
    const int y0 = static_cast<int>(rank) * BY;
    const int h = min(BY, ny - y0);                       // rows of this strip (the host makes it >= 2)
    const int h_last = ny - static_cast<int>(C - 1) * BY;
    const unsigned up = (rank + C - 1) % C, down = (rank + 1) % C;
    const int h_up = up == C - 1 ? h_last : BY;           // rows of the strip above
    const Phys<T>& P = a.P;
    const int interact = P.interact;
    const bool fast = interact && !P.var_visc && nx == BX && h == BY;
    const EosRegs<T> E(P);
    const T rho_ref = P.rho_ref;
    const int wcols = nx + 4;                             // columns -2 .. nx + 1 carry data

    // the input box of the first step: rows y0 - 2 .. y0 + h + 1 and columns
    // -2 .. nx + 1 of the global array (its ghost cells are current)
    for (int e = tid; e < 9 * (h + 4) * wcols; e += NT) {
        const int c = e % wcols, r = (e / wcols) % (h + 4), q = e / (wcols * (h + 4));
        box0[q * PB + r * WB + (HX - 2 + c)] =
            a.src[q * a.plane + static_cast<long long>(y0 - GY + r + GY) * a.pitch + (GXg - 2 + c)];
    }
    cluster_barrier();   // also: every CTA of the cluster has started before any remote store

    bool bad = false;
#pragma unroll 1
    for (int s = 0; s < a.nsteps; ++s) {
        const T* bi = (s & 1) ? box1 : box0;
        T* bo = (s & 1) ? box0 : box1;
        if (interact) ring_dispatch<Gm>(fast, P.eos, bi, sp, E, rho_ref, tid, tx, ty);
        __syncthreads();
        // the output of node (x, y) of the strip goes to box row GY + y,
        // column HX + x: collide_rows addresses (y + GY) * pitch + x + GX
        const Regs<T> R(P);
        T* const o = bo - (Gm::GX - HX);
        if (fast)
            bad |= collide_rows<Gm, true, false>(bi, sp, P, R, o, PB, WB, 0, 0, nx, h, false, interact, tx, ty);
        else
            bad |= collide_rows<Gm, false, false>(bi, sp, P, R, o, PB, WB, 0, 0, nx, h, false, interact, tx, ty);
        __syncthreads();
        // from the collision's outputs only, so neither waits for the other:
        // periodic images in x (columns -2, -1 <- nx - 2, nx - 1; nx, nx + 1
        // <- 0, 1), one thread per (column, row); and the edge rows (their x
        // images read at the source) to the neighbours' halo rows, thread
        // row k < 4: rows GY, GY + 1 to rows GY + h_up, GY + h_up + 1 of the
        // CTA above, rows GY + h - 2, GY + h - 1 to rows 0, 1 of the CTA below
        if (tx < 4 && ty < h) {
            const int to = tx < 2 ? tx - 2 : nx + tx - 2;
            const int from = tx < 2 ? nx + tx - 2 : tx - 2;
            T* row = bo + (GY + ty) * WB + HX;
#pragma unroll
            for (int q = 0; q < 9; ++q) row[q * PB + to] = row[q * PB + from];
        }
        if (ty < 4) {
            const int from = ty < 2 ? GY + ty : GY + h - 4 + ty;
            const int to = ty < 2 ? GY + h_up + ty : ty - 2;
            const uint32_t rbase = cluster_map(smem_u32(bo), ty < 2 ? up : down);
            for (int c = tx; c < wcols; c += BX) {
                const int x = c - 2, xs = x < 0 ? x + nx : (x >= nx ? x - nx : x);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    st_cluster(rbase + static_cast<uint32_t>((q * PB + to * WB + HX + x) * sizeof(T)),
                               bo[q * PB + from * WB + HX + xs]);
            }
        }
        cluster_barrier();
    }

    // the last output box's strip to the global array (ghost cells: the caller)
    const T* fin = (a.nsteps & 1) ? box1 : box0;
    for (int e = tid; e < 9 * h * nx; e += NT) {
        const int x = e % nx, r = (e / nx) % h, q = e / (nx * h);
        a.dst[q * a.plane + static_cast<long long>(y0 + r + GY) * a.pitch + (GXg + x)] =
            fin[q * PB + (GY + r) * WB + HX + x];
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(a.status, ST_UNSTABLE);
}

// A cluster configuration: strips of BY rows of at most BX nodes, NT threads.
template <typename T, int BX, int BY, int NT> struct ClusterCfg {
    using Gm = Geom<T, BX, BY, NT, 1>;
    static constexpr size_t smem = 2 * Gm::buf_stride + Gm::psi_stride;
    static_assert(smem <= 232448, "two boxes and the psi tile must fit in a CTA's shared memory");
    static constexpr int max_ctas = 16;
    static bool fits(int nx, int ny) {
        const int C = (ny + BY - 1) / BY;
        return nx >= 2 && nx <= BX && C <= max_ctas && ny - (C - 1) * BY >= 2;
    }
    // the launch of one cluster of C CTAs (attributes set on the kernel first)
    static cudaError_t config(unsigned C, cudaStream_t st, cudaLaunchConfig_t& cfg, cudaLaunchAttribute& attr) {
        const auto fn = &k_cluster<T, BX, BY, NT>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = C;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        return e;
    }
    // whether the device can hold a cluster of this lattice's CTAs at all
    static bool launchable(int ny) {
        const unsigned C = static_cast<unsigned>((ny + BY - 1) / BY);
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr;
        int n = 0;
        if (config(C, nullptr, cfg, attr) != cudaSuccess) return false;
        return cudaOccupancyMaxActiveClusters(&n, &k_cluster<T, BX, BY, NT>, &cfg) == cudaSuccess && n > 0;
    }
    static cudaError_t run(const ClusterArgs<T>& args, cudaStream_t st) {
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr;
        cudaError_t e = config(static_cast<unsigned>((args.ny + BY - 1) / BY), st, cfg, attr);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, &k_cluster<T, BX, BY, NT>, args);
    }
};

// One node per thread.  FP32: strips of 16 rows up to 64 nodes wide, or of
// 8 rows up to 128 wide; FP64, bound by its FP64 pipe, on as many SMs as a
// cluster has: strips of 4 rows up to 64 high, else of 8 rows, up to 64
// nodes wide.
using CF32a = ClusterCfg<float, 64, 16, 1024>;
using CF32b = ClusterCfg<float, 128, 8, 1024>;
using CF64a = ClusterCfg<double, 64, 4, 256>;
using CF64b = ClusterCfg<double, 64, 8, 512>;

template <typename T>
ClusterArgs<T> cluster_args(const Inst& h, const Phys<T>& P, int parity, int nsteps) {
    ClusterArgs<T> a;
    a.P = P;
    a.src = static_cast<const T*>(h.pop[parity]);
    a.dst = static_cast<T*>(h.pop[parity ^ (nsteps & 1)]);
    a.plane = h.plane;
    a.pitch = h.pitch;
    a.nx = h.nx;
    a.ny = h.ny;
    a.nsteps = nsteps;
    a.status = h.status;
    return a;
}

}  // namespace

bool cluster_supported(int prec, int nx, int ny) {
    if (prec == LBM_FP32) {
        if (CF32a::fits(nx, ny)) return CF32a::launchable(ny);
        return CF32b::fits(nx, ny) && CF32b::launchable(ny);
    }
    if (CF64a::fits(nx, ny)) return CF64a::launchable(ny);
    return CF64b::fits(nx, ny) && CF64b::launchable(ny);
}

cudaError_t cluster_run(const Inst& h, int parity, int nsteps, cudaStream_t st) {
    if (nsteps <= 0) return cudaSuccess;
    if (h.prec == LBM_FP32) {
        const ClusterArgs<float> a = cluster_args<float>(h, h.pf, parity, nsteps);
        if (CF32a::fits(h.nx, h.ny)) return CF32a::run(a, st);
        if (CF32b::fits(h.nx, h.ny)) return CF32b::run(a, st);
        return cudaErrorInvalidValue;
    }
    const ClusterArgs<double> a = cluster_args<double>(h, h.pd, parity, nsteps);
    if (CF64a::fits(h.nx, h.ny)) return CF64a::run(a, st);
    if (CF64b::fits(h.nx, h.ny)) return CF64b::run(a, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
