// lbm_aux.cu -- kernels around the fused step: initial equilibrium, ghost
// images, read-back of populations and macroscopic fields, and the FP64
// reductions behind Laplace's law (Eq. 22) and the run statistics.
// None of these is on the per-step path.
#include "lbm_internal.cuh"
#include "lbm_init.h"

namespace lbm {
namespace {

constexpr int kThreads = 256;

// Lattice weights t_a of the D2Q9 equilibrium (4/9, 1/9, 1/36).
__device__ __forceinline__ double tw(int a) { return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

template <typename T> __device__ __forceinline__ T* popk(const Inst* I, int parity) {
    return static_cast<T*>(I->pop[parity]);
}

// Element (a, x, y) of a time level; x in [-GX, pitch-GX), y in [-2, ny+2).
template <typename T> __device__ __forceinline__ long long at(const Inst* I, int a, int x, int y) {
    return a * I->plane + static_cast<long long>(y + GY) * I->pitch + (x + Prec<T>::GX);
}

// Node loops over a lattice: rows y by blockIdx.y, columns x by the
// threads of blockIdx.x (grid from grid_2d), so that no thread divides by
// the lattice width.
#define LBM_FOR_NODES(nx, ny)                                      \
    for (int y = blockIdx.y; y < (ny); y += gridDim.y)             \
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < (nx); x += gridDim.x * blockDim.x)

// ---- initial state: f_a(z) = f_eq,a(rho(z), u(z)); pull storage keeps it at z - e_a
// REST: no velocity field given (u = 0), where the equilibrium's velocity
// terms are exact zeros and the deviation is t_a (rho - rho_ref): FP64
// keeps the FP64 products; FP32 rounds rho - rho_ref (formed in FP64, so
// that no digit of a small difference is lost) to FP32 once and multiplies
// by the weights in FP32 (within 1.5 ulp of the correctly rounded value, and
// two FP64 operations per node instead of seven: GB300's FP64 pipe would
// otherwise bound the initialisation).  Rows [y0, y1) of the field; rho,
// ux and uy index the whole field.
template <typename T, bool REST, typename R>
__global__ void k_init(const Inst* __restrict__ I, const R* __restrict__ rho, const R* __restrict__ ux,
                       const R* __restrict__ uy, int parity, int y0, int y1) {
    const int nx = I->nx, ny = I->ny;
    T* p = popk<T>(I, parity);
    const double rr = static_cast<double>(phys<T>(I).rho_ref);
    for (int y = y0 + static_cast<int>(blockIdx.y); y < y1; y += gridDim.y)
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
            const long long i = static_cast<long long>(y) * nx + x;
            const double r = rho[i], u = !REST && ux ? double(ux[i]) : 0.0, v = !REST && uy ? double(uy[i]) : 0.0;
            const double u2 = u * u + v * v;
            // at rest: the three weights' products
            const double d = r - rr;
            T rest[3];
            if constexpr (sizeof(T) == 4) {
                const float df = static_cast<float>(d);
                rest[0] = __fmul_rn(4.0f / 9.0f, df);
                rest[1] = __fmul_rn(1.0f / 9.0f, df);
                rest[2] = __fmul_rn(1.0f / 36.0f, df);
            } else {
                rest[0] = tw(0) * d;
                rest[1] = tw(1) * d;
                rest[2] = tw(5) * d;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const double eu = cx(a) * u + cy(a) * v;
                // textbook second-order equilibrium, minus t_a rho_ref
                const double dev = REST ? 0.0 : tw(a) * ((r - rr) + r * (3.0 * eu + 4.5 * eu * eu - 1.5 * u2));
                int xs = x - cx(a), ys = y - cy(a);
                xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
                p[at<T>(I, a, xs, ys)] = REST ? rest[a == 0 ? 0 : (a < 5 ? 1 : 2)] : static_cast<T>(dev);
            }
        }
}

// The checks of an initial field, on the device: bit 1 of *bad when a
// density is not finite, not positive or not below rho_max, bit 2 when a
// velocity is not finite (the caller has zeroed *bad).
// Bit patterns of the field's type as signed integers, and the exponent field.
__device__ __forceinline__ long long bits_of(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ long long bits_of(float v) { return __float_as_int(v); }
template <typename R> __host__ __device__ constexpr long long exp_mask() {
    return sizeof(R) == 8 ? 0x7ff0000000000000ll : 0x7f800000ll;
}
template <typename R>
__global__ void k_check_init(const R* __restrict__ rho, const R* __restrict__ ux, const R* __restrict__ uy,
                             long long N, double rho_max, int* bad) {
    // on the bit patterns, as integers (no FP64 work): for rho_max > 0,
    // 0 < r < rho_max with r finite is 0 < bits(r) < bits(top), top = rho_max
    // in FP64, or for FP32 fields the smallest float not below rho_max
    // (positive values order as their patterns; negatives and -0 have the
    // sign bit, NaN and inf patterns lie above every finite value); finite is
    // an exponent field below all ones
    const long long top = sizeof(R) == 8 ? bits_of(rho_max) : bits_of(__double2float_ru(rho_max));
    constexpr long long kExp = exp_mask<R>();
    auto finite = [](R v) { return (bits_of(v) & kExp) != kExp; };
    int b = 0;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = bits_of(rho[i]);
        if (!(r > 0 && r < top)) b |= 1;
        if ((ux && !finite(ux[i])) || (uy && !finite(uy[i]))) b |= 2;
    }
    b = __reduce_or_sync(0xffffffffu, b);
    if (b && (threadIdx.x & 31) == 0) atomicOr(bad, b);
}

// Ghost cells x in [-2,0) U [nx,nx+2), y in [-2,0) U [ny,ny+2) of every
// plane, and only those: per plane the rows y = -2, -1, ny, ny + 1 over
// x in [-2, nx + 2) (4 (nx + 4) cells), then the columns x = -2, -1, nx,
// nx + 1 over y in [0, ny) (4 ny cells).  Each copies its periodic image
// inside the lattice.
template <typename T> __global__ void k_ghosts(const Inst* __restrict__ I, int parity) {
    const int nx = I->nx, ny = I->ny;
    const int W = nx + 4, per = 4 * W + 4 * ny;
    const long long M = 9ll * per;
    T* p = popk<T>(I, parity);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < M;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int a = static_cast<int>(i / per);
        const int r = static_cast<int>(i - static_cast<long long>(a) * per);
        int x, y;
        if (r < 4 * W) {
            const int row = r / W;
            x = r - row * W - 2;
            y = row < 2 ? row - 2 : ny + row - 2;
        } else {
            const int q = r - 4 * W, col = q / ny;
            y = q - col * ny;
            x = col < 2 ? col - 2 : nx + col - 2;
        }
        const int xs = ((x % nx) + nx) % nx, ys = ((y % ny) + ny) % ny;
        p[at<T>(I, a, x, y)] = p[at<T>(I, a, xs, ys)];
    }
}

// f_a(z, t) = pop_a(z - e_a) + t_a rho_ref, for one plane a.
template <typename T>
__global__ void k_gather(const Inst* __restrict__ I, int parity, int a, double* __restrict__ out) {
    const int nx = I->nx, ny = I->ny;
    const T* p = popk<T>(I, parity);
    const double off = tw(a) * static_cast<double>(phys<T>(I).rho_ref);
    const int ex = cx(a), ey = cy(a);
    LBM_FOR_NODES(nx, ny) {
        out[static_cast<long long>(y) * nx + x] = static_cast<double>(p[at<T>(I, a, x - ex, y - ey)]) + off;
    }
}

// rho and momentum sum f e of node (x, y), x in [-1, nx], y in [-1, ny].
template <typename T>
__device__ __forceinline__ double node_rho(const Inst* I, const T* p, int x, int y, double* jx, double* jy) {
    double r = 0.0, mx = 0.0, my = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const double v = static_cast<double>(p[at<T>(I, a, x - cx(a), y - cy(a))]);
        r += v;
        mx += cx(a) * v;
        my += cy(a) * v;
    }
    if (jx) *jx = mx;
    if (jy) *jy = my;
    return r + static_cast<double>(phys<T>(I).rho_ref);
}

// rho of an FP32 node from its nine deviations: their sum as an unevaluated
// pair hi + lo (Knuth's TwoSum gives the exact error of each addition; the
// errors are summed in FP32), then hi + lo + rho_ref in FP64.  Within about
// 2^-45 of the FP64 sum relative to the deviations' sum, and three FP64
// operations per node instead of eighteen: GB300's FP64 pipe would
// otherwise bound the density read-back.
__device__ __forceinline__ double node_rho_f32(const Inst* I, const float* p, int x, int y) {
    float hi = 0.0f, lo = 0.0f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const float v = p[at<float>(I, a, x - cx(a), y - cy(a))];
        const float sum = __fadd_rn(hi, v);
        const float bv = __fsub_rn(sum, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bv)), __fsub_rn(v, bv));
        hi = sum;
        lo = __fadd_rn(lo, err);
    }
    return (static_cast<double>(hi) + static_cast<double>(lo)) + static_cast<double>(I->pf.rho_ref);
}

__device__ __forceinline__ double psi_of(const Phys<double>& P, double rho) {
    return sqrt(psi_radicand(P, rho));
}

// rho, velocity (Eq. 9 force, rho u = sum f e + F/2) and psi of node (x, y).
template <typename T>
__device__ void node_fields(const Inst* I, const T* p, int x, int y, double* rho, double* ux, double* uy,
                            double* psi) {
    const Phys<double>& P = I->pd;
    const int nx = I->nx, ny = I->ny;
    double jx, jy;
    const double r = node_rho<T>(I, p, x, y, &jx, &jy);
    double Fx = 0.0, Fy = 0.0, ps = 0.0;
    if (P.interact) {
        ps = psi_of(P, r);
        double gx1 = 0, gy1 = 0, gx2 = 0, gy2 = 0;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            int xn = x + cx(a), yn = y + cy(a);
            xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
            yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
            const double pn = psi_of(P, node_rho<T>(I, p, xn, yn, nullptr, nullptr));
            const double w = (a < 5) ? 1.0 / 3.0 : 1.0 / 12.0;
            gx1 += w * pn * cx(a);
            gy1 += w * pn * cy(a);
            gx2 += w * pn * pn * cx(a);
            gy2 += w * pn * pn * cy(a);
        }
        Fx = -P.G * (0.5 * P.A * gx2 + (1.0 - P.A) * ps * gx1);
        Fy = -P.G * (0.5 * P.A * gy2 + (1.0 - P.A) * ps * gy1);
    }
    *rho = r;
    *ux = (jx + 0.5 * Fx) / r;
    *uy = (jy + 0.5 * Fy) / r;
    *psi = ps;
}

// One macroscopic field per launch (0 rho, 1 u_x, 2 u_y, 3 psi), each its
// own kernel: the density read-back keeps the registers of a plain gather.
// Rows [y0, y1) of the field, at their place in out (row-major nx x ny).
template <typename T, int FIELD, typename O>
__global__ void k_field(const Inst* __restrict__ I, int parity, int y0, int y1, O* __restrict__ out) {
    const int nx = I->nx;
    const T* p = popk<T>(I, parity);
    for (int y = y0 + static_cast<int>(blockIdx.y); y < y1; y += gridDim.y)
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
            const long long i = static_cast<long long>(y) * nx + x;
            double v;
            if constexpr (FIELD == 0 && sizeof(T) == 4) {
                v = node_rho_f32(I, p, x, y);
            } else if constexpr (FIELD == 0) {
                v = node_rho<T>(I, p, x, y, nullptr, nullptr);
            } else if constexpr (FIELD == 3) {
                v = I->pd.interact ? psi_of(I->pd, node_rho<T>(I, p, x, y, nullptr, nullptr)) : 0.0;
            } else {
                double r, u, w, s;
                node_fields<T>(I, p, x, y, &r, &u, &w, &s);
                v = FIELD == 1 ? u : w;
            }
            out[i] = static_cast<O>(v);
        }
}

// ---- FP64 block reductions ----------------------------------------------
// Each block writes kReduceSlots partial sums (slot `max_slot` is a max);
// k_finish adds the partials in a fixed order, so results are deterministic.
__device__ __forceinline__ void block_reduce_store(double (&v)[kReduceSlots], int max_slot, double* partials) {
    __shared__ double red[kThreads / 32][kReduceSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kReduceSlots; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = (k == max_slot) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kReduceSlots) {
        const int k = threadIdx.x;
        double x = red[0][k];
        for (int w = 1; w < kThreads / 32; ++w) x = (k == max_slot) ? fmax(x, red[w][k]) : x + red[w][k];
        partials[blockIdx.x * kReduceSlots + k] = x;
    }
}

__global__ void k_finish(const double* __restrict__ partials, int nblocks, int max_slot, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= kReduceSlots) return;
    double x = partials[k];
    for (int b = 1; b < nblocks; ++b) {
        const double y = partials[b * kReduceSlots + k];
        x = (k == max_slot) ? fmax(x, y) : x + y;
    }
    out[k] = x;
}

// Sums for Laplace's law: {sum rho, sum p_in, sum rho_in, n_in, sum p_out,
// sum rho_out, n_out, 0}; p = p_EOS(rho) (equal to rho/3 + G psi^2/2, Eq. 10).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_measure(const Inst* __restrict__ I, int parity, double cxc, double cyc,
                                                       double r_in, double r_out, double* __restrict__ partials) {
    const int nx = I->nx, ny = I->ny;
    const long long N = static_cast<long long>(nx) * ny;
    const T* p = popk<T>(I, parity);
    double v[kReduceSlots] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % nx), y = static_cast<int>(i / nx);
        const double r = node_rho<T>(I, p, x, y, nullptr, nullptr);
        double dx = x - cxc, dy = y - cyc;
        dx -= nx * rint(dx / nx);
        dy -= ny * rint(dy / ny);
        const double d = sqrt(dx * dx + dy * dy);
        v[0] += r;
        if (d <= r_in) {
            v[1] += p_eos(I->pd, r);
            v[2] += r;
            v[3] += 1.0;
        }
        if (d >= r_out) {
            v[4] += p_eos(I->pd, r);
            v[5] += r;
            v[6] += 1.0;
        }
    }
    block_reduce_store(v, -1, partials);
}

// {mass, sum rho u_x, sum rho u_y, sum rho |u|^2 / 2, max |u|, 0, 0, 0}
template <typename T>
__global__ void __launch_bounds__(kThreads) k_stats(const Inst* __restrict__ I, int parity, double* __restrict__ partials) {
    const int nx = I->nx, ny = I->ny;
    const long long N = static_cast<long long>(nx) * ny;
    const T* p = popk<T>(I, parity);
    double v[kReduceSlots] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % nx), y = static_cast<int>(i / nx);
        double r, u, w, s;
        node_fields<T>(I, p, x, y, &r, &u, &w, &s);
        v[0] += r;
        v[1] += r * u;
        v[2] += r * w;
        v[3] += 0.5 * r * (u * u + w * w);
        v[4] = fmax(v[4], sqrt(u * u + w * w));
    }
    block_reduce_store(v, 4, partials);
}

int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 8 * kReduceBlocks) b = 8 * kReduceBlocks;
    return static_cast<int>(b);
}

// Grid of the node loops (LBM_FOR_NODES): up to 8 blocks across a row, the
// rest down the rows, 8 * kReduceBlocks blocks at most.
dim3 grid_2d(int nx, int ny) {
    int gx = (nx + kThreads - 1) / kThreads;
    if (gx > 8) gx = 8;
    if (gx < 1) gx = 1;
    int gy = 8 * kReduceBlocks / gx;
    if (gy > ny) gy = ny;
    if (gy < 1) gy = 1;
    return dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
}

// ---- the FP64 step's division, reciprocal and square root against IEEE --
// Distance in units in the last place; values of opposite sign or NaN count
// as infinitely far.
__device__ __forceinline__ unsigned long long ulp_distance(double a, double b) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    if (x == y) return 0;
    if (!(a == a) || !(b == b) || ((x ^ y) < 0)) return ~0ull;
    return static_cast<unsigned long long>(x > y ? x - y : y - x);
}

// out[0..2]: largest distance of Fast<double>::rcp(d), div(a, d), sqrt(d)
// from 1/d, a/d, sqrt(d) (IEEE-rounded: this file keeps nvcc's default
// -prec-div and -prec-sqrt) over n values of d spread evenly over [lo, hi],
// a in [0.37, 0.87); out[3] = 1 if sqrt keeps +0, -0 and gives NaN for -1.
__global__ void k_math_check(long long n, double lo, double hi, unsigned long long* out) {
    unsigned long long m0 = 0, m1 = 0, m2 = 0;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const double d = lo + (hi - lo) * (static_cast<double>(i) / static_cast<double>(n));
        const double a = 0.37 + 0.5 * static_cast<double>((i * 2654435761ll) & 0xffff) / 65536.0;
        m0 = max(m0, ulp_distance(Fast<double>::rcp(d), 1.0 / d));
        m1 = max(m1, ulp_distance(Fast<double>::div(a, d), a / d));
        m2 = max(m2, ulp_distance(Fast<double>::sqrt(d), sqrt(d)));
    }
    atomicMax(&out[0], m0);
    atomicMax(&out[1], m1);
    atomicMax(&out[2], m2);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double pz = Fast<double>::sqrt(0.0), nz = Fast<double>::sqrt(-0.0), neg = Fast<double>::sqrt(-1.0);
        out[3] = (__double_as_longlong(pz) == 0 && __double_as_longlong(nz) == __double_as_longlong(-0.0) &&
                  !(neg == neg))
                     ? 1ull
                     : 0ull;
    }
}

// FP64 fused multiply-add throughput: every thread runs kFmaChains
// independent chains x <- x m + c (m < 1, so x stays finite) for `iters`
// iterations.  The chains' sum is compared with a value it cannot take, so
// the compiler keeps every FMA; nothing is stored.
constexpr int kFmaChains = 8;
constexpr int kFmaThreads = 256;
__device__ double g_fma_sink;
__global__ void __launch_bounds__(kFmaThreads) k_fp64_fma(int iters, double m, double c) {
    double x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = fma(x[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += x[k];
    if (s == -1.0) g_fma_sink = s;
}

}  // namespace

cudaError_t aux_fp64_fma_rate(int iters, cudaStream_t st, double* flops_per_s, double* seconds) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (2048 / kFmaThreads);   // every SM full
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best = 0.0f;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {   // the first launch warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            k_fp64_fma<<<blocks, kFmaThreads, 0, st>>>(iters, 0.999, 1e-3);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * blocks * kFmaThreads * static_cast<double>(kFmaChains) * iters;
    *seconds = best * 1e-3;
    *flops_per_s = flops / (*seconds);
    return cudaSuccess;
}

template <typename R>
cudaError_t init_rows_t(const Inst& h, const Inst* d, const R* rho, const R* ux, const R* uy, int parity, int y0,
                        int y1, cudaStream_t st) {
    const dim3 g = grid_2d(h.nx, y1 - y0);
    const bool rest = !ux && !uy;
    if (h.prec == LBM_FP32 && rest) k_init<float, true, R><<<g, kThreads, 0, st>>>(d, rho, ux, uy, parity, y0, y1);
    else if (h.prec == LBM_FP32) k_init<float, false, R><<<g, kThreads, 0, st>>>(d, rho, ux, uy, parity, y0, y1);
    else if (rest) k_init<double, true, R><<<g, kThreads, 0, st>>>(d, rho, ux, uy, parity, y0, y1);
    else k_init<double, false, R><<<g, kThreads, 0, st>>>(d, rho, ux, uy, parity, y0, y1);
    return cudaGetLastError();
}

cudaError_t aux_init(const Inst& h, const Inst* d, const void* rho, const void* ux, const void* uy, bool f32,
                     int parity, cudaStream_t st) {
    const cudaError_t e = aux_init_rows(h, d, rho, ux, uy, f32, parity, 0, h.ny, st);
    return e != cudaSuccess ? e : aux_fill_ghosts(h, d, parity, st);
}

cudaError_t aux_init_rows(const Inst& h, const Inst* d, const void* rho, const void* ux, const void* uy, bool f32,
                          int parity, int y0, int y1, cudaStream_t st) {
    if (y0 < 0 || y1 > h.ny || y0 >= y1) return cudaErrorInvalidValue;
    if (f32)
        return init_rows_t(h, d, static_cast<const float*>(rho), static_cast<const float*>(ux),
                           static_cast<const float*>(uy), parity, y0, y1, st);
    return init_rows_t(h, d, static_cast<const double*>(rho), static_cast<const double*>(ux),
                       static_cast<const double*>(uy), parity, y0, y1, st);
}

cudaError_t aux_check_init(const void* rho, const void* ux, const void* uy, bool f32, long long N, double rho_max,
                           int* bad, cudaStream_t st) {
    if (f32)
        k_check_init<float><<<grid_for(N), kThreads, 0, st>>>(static_cast<const float*>(rho),
                                                               static_cast<const float*>(ux),
                                                               static_cast<const float*>(uy), N, rho_max, bad);
    else
        k_check_init<double><<<grid_for(N), kThreads, 0, st>>>(static_cast<const double*>(rho),
                                                                static_cast<const double*>(ux),
                                                                static_cast<const double*>(uy), N, rho_max, bad);
    return cudaGetLastError();
}

cudaError_t aux_fill_ghosts(const Inst& h, const Inst* d, int parity, cudaStream_t st) {
    const long long M = 9ll * (4 * (h.nx + 4) + 4 * h.ny);
    if (h.prec == LBM_FP32)
        k_ghosts<float><<<grid_for(M), kThreads, 0, st>>>(d, parity);
    else
        k_ghosts<double><<<grid_for(M), kThreads, 0, st>>>(d, parity);
    return cudaGetLastError();
}

cudaError_t aux_gather_plane(const Inst& h, const Inst* d, int parity, int a, double* out, cudaStream_t st) {
    if (h.prec == LBM_FP32)
        k_gather<float><<<grid_2d(h.nx, h.ny), kThreads, 0, st>>>(d, parity, a, out);
    else
        k_gather<double><<<grid_2d(h.nx, h.ny), kThreads, 0, st>>>(d, parity, a, out);
    return cudaGetLastError();
}

template <typename O>
cudaError_t field_t(const Inst& h, const Inst* d, int parity, int field, int y0, int y1, O* out, cudaStream_t st) {
    const dim3 g = grid_2d(h.nx, y1 - y0);
    auto go = [&](auto k) { k<<<g, kThreads, 0, st>>>(d, parity, y0, y1, out); };
    const bool f32 = h.prec == LBM_FP32;
    switch (field) {
    case 0: f32 ? go(k_field<float, 0, O>) : go(k_field<double, 0, O>); break;
    case 1: f32 ? go(k_field<float, 1, O>) : go(k_field<double, 1, O>); break;
    case 2: f32 ? go(k_field<float, 2, O>) : go(k_field<double, 2, O>); break;
    default: f32 ? go(k_field<float, 3, O>) : go(k_field<double, 3, O>); break;
    }
    return cudaGetLastError();
}

cudaError_t aux_field(const Inst& h, const Inst* d, int parity, int field, int y0, int y1, void* out, bool f32out,
                      cudaStream_t st) {
    if (f32out) return field_t(h, d, parity, field, y0, y1, static_cast<float*>(out), st);
    return field_t(h, d, parity, field, y0, y1, static_cast<double*>(out), st);
}

cudaError_t aux_measure(const Inst& h, const Inst* d, int parity, double cxc, double cyc, double r_in,
                        double r_out, double* partials, double* result, cudaStream_t st) {
    if (h.prec == LBM_FP32)
        k_measure<float><<<kReduceBlocks, kThreads, 0, st>>>(d, parity, cxc, cyc, r_in, r_out, partials);
    else
        k_measure<double><<<kReduceBlocks, kThreads, 0, st>>>(d, parity, cxc, cyc, r_in, r_out, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish<<<1, 32, 0, st>>>(partials, kReduceBlocks, -1, result);
    return cudaGetLastError();
}

cudaError_t aux_stats(const Inst& h, const Inst* d, int parity, double* partials, double* result, cudaStream_t st) {
    if (h.prec == LBM_FP32)
        k_stats<float><<<kReduceBlocks, kThreads, 0, st>>>(d, parity, partials);
    else
        k_stats<double><<<kReduceBlocks, kThreads, 0, st>>>(d, parity, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish<<<1, 32, 0, st>>>(partials, kReduceBlocks, 4, result);
    return cudaGetLastError();
}

cudaError_t aux_math_check(long long n, double lo, double hi, unsigned long long* out) {
    k_math_check<<<1024, kThreads>>>(n, lo, hi, out);
    return cudaGetLastError();
}

}  // namespace lbm
