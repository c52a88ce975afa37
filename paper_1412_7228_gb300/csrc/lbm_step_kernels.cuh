// lbm_step_kernels.cuh -- the fused per-timestep kernel of the pseudo-potential MRT
// lattice Boltzmann method (Hu, Li & Uddin, arXiv:1412.7228, Sections 2 and
// 3.2) for sm_103a.
//
// One CTA owns a BX x BY tile of one instance.  Per step it
//   1. loads the tile's populations plus a halo (x -HX..BX+HX, y -2..BY+2)
//      of all nine planes with ONE 3-D TMA box into shared memory (the
//      halo rows/columns are periodic images kept in ghost cells, so no
//      wrap logic is needed);
//   2. computes rho and psi (Eq. 10) for the tile and its 1-node ring in
//      shared memory;
//   3. for every owned node: gathers f_a(x) = pop_a(x - e_a) ("pull"),
//      evaluates the hybrid force (Eq. 9) and the modifying tensor Q
//      (Eq. 23, scaled by G/2), transforms to moments, applies the relaxation
//      with the forcing (I - Lambda/2) S (Eqs. 5-6) and the source C
//      (Eqs. 25-26), transforms back, and stores the nine post-collision
//      values at the node (plus their periodic ghost images at borders).
// Each population is read from and written to HBM once per step; the halo
// re-reads of neighbouring tiles are served from L2.  No tensor cores: the
// 9x9 transforms have integer entries and are unrolled into adds.
#pragma once

#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

template <typename T, int BX_, int BY_, int NT_, int NBUF_> struct Geom {
    static constexpr int BX = BX_, BY = BY_, NT = NT_;
    static constexpr int NBUF = NBUF_;          // 1: one tile per CTA; 2: persistent, double-buffered
    static constexpr int HX = Prec<T>::HX;      // halo columns in the box (16 bytes)
    static constexpr int GX = Prec<T>::GX;      // ghost columns in HBM (32 bytes)
    static constexpr int WB = BX + 2 * HX;      // box width
    static constexpr int HB = BY + 2 * GY;      // box height
    static constexpr int PB = WB * HB;          // box elements per plane
    static constexpr int WP = BX + 2;           // psi tile (tile + 1 ring)
    static constexpr int HP = BY + 2;
    static constexpr int TY = NT / BX;          // thread rows
    static constexpr int ROWS = BY / TY;        // nodes per thread
    static constexpr size_t box_bytes = size_t(9) * PB * sizeof(T);
    static constexpr size_t buf_stride = (box_bytes + 127) / 128 * 128;      // box buffers
    static constexpr size_t psi_off = NBUF * buf_stride;
    static constexpr size_t psi_stride = (size_t(WP) * HP * sizeof(T) + 127) / 128 * 128;   // psi tiles
    static constexpr size_t smem = psi_off + NBUF * psi_stride;
    static_assert(NT % BX == 0 && BY % TY == 0, "thread layout must tile the block");
    static_assert(WB <= 256 && HB <= 256, "TMA box dimensions are limited to 256");
    static_assert((WB * sizeof(T)) % 16 == 0, "TMA box rows must be a multiple of 16 bytes");
    static_assert(BX >= 2, "the ring's extra columns are taken by threads tx = 0, 1");
};

// sum_a f_a grouped so that the result is invariant under the lattice's
// mirror symmetries (x -> -x swaps 1<->3, 5<->6, 7<->8; y -> -y swaps 2<->4,
// 5<->8, 6<->7): with commutative rounding a mirror-symmetric state stays
// bitwise mirror-symmetric, so rounding cannot push a symmetric drop off its
// centre (translation is a neutral mode of a static droplet).
template <typename T> __device__ __forceinline__ T rho_dev(const T (&f)[9]) {
    const T Sa = (f[1] + f[3]) + (f[2] + f[4]);
    const T Sd = (f[5] + f[7]) + (f[6] + f[8]);
    return f[0] + Sa + Sd;
}

// Rounding is fixed by the source, not by the compiler: the translation
// units that instantiate these kernels are built with -fmad=false and every
// fused multiply-add is an explicit fma().  The
// results are then the same bits for every tile shape, pipeline variant and
// launch path the autotuner may pick.
//
// Product rounded on its own: never fused into an FMA with a neighbouring
// add.  Used where a mirror swaps two product terms (p1^2 - p3^2, ...):
// fma(a, a, -b*b) is not antisymmetric in a and b, a difference of two
// rounded products is.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// The parameters one node needs, copied into registers once per tile (the
// descriptor lives in global memory, and the compiler may not keep values
// read through it across the node loop's stores).
// FP32 keeps them as values; FP64, bound by its FP64 pipe rather than by
// issue slots, keeps references and spends its registers on occupancy.
template <typename T, typename V> struct RegsOf {
    V ns1, ns2, ns4, ns6, ns7, ns8, h6s1, nh6s2, nhs4, nhs6, h2s7, hs8, c1, c2, rho_ref;   // ns = -s, nhs = -hs
    int var_visc;
    V nu_g, dnu, visc_rho_g, visc_inv_drho;
    __device__ __forceinline__ explicit RegsOf(const Phys<T>& P)
        : ns1(P.ns[1]), ns2(P.ns[2]), ns4(P.ns[4]), ns6(P.ns[6]), ns7(P.ns[7]), ns8(P.ns[8]), h6s1(P.h6s1),
          nh6s2(P.nh6s2), nhs4(P.nhs[4]), nhs6(P.nhs[6]), h2s7(P.h2s7), hs8(P.hs[8]), c1(P.c1), c2(P.c2),
          rho_ref(P.rho_ref), var_visc(P.var_visc), nu_g(P.nu_g), dnu(P.dnu), visc_rho_g(P.visc_rho_g),
          visc_inv_drho(P.visc_inv_drho) {}
};
template <typename T> struct RegsSel { using type = RegsOf<T, const T&>; };
template <> struct RegsSel<float> { using type = RegsOf<float, float>; };
template <typename T> using Regs = typename RegsSel<T>::type;

// Moment-space collision of one node in deviation form (Eqs. 2-6, 25, 26).
// Every expression maps onto itself (or its negative) under the mirrors
// above, which keeps symmetric states symmetric to the last bit.
// f: pre-collision f_a - t_a rho_ref; out: post-collision, same form.
// P: the relaxation constants (register copies for FP32, references into the
// descriptor for FP64).
// VISC = false: the tile's lattice has fixed shear rates (no per-node
// viscosity law), decided once per tile by the caller.
template <typename T, bool VISC, typename RP>
__device__ __forceinline__ void collide(const RP& P, const T (&f)[9], T Fx, T Fy, T Qxx, T Qyy, T Qxy,
                                        T (&out)[9]) {
    const T Sa = (f[1] + f[3]) + (f[2] + f[4]);
    const T Sd = (f[5] + f[7]) + (f[6] + f[8]);
    const T rt = f[0] + Sa + Sd;                       // rho - rho_ref, as rho_dev()
    const T rho = T(P.rho_ref) + rt;
    const T inv = Fast<T>::rcp(rho);
    const T d13 = f[1] - f[3], d24 = f[2] - f[4];
    const T Dxd = (f[5] - f[7]) + (f[8] - f[6]);
    const T Dyd = (f[5] - f[7]) + (f[6] - f[8]);
    const T jx = d13 + Dxd, jy = d24 + Dyd;
    const T rux = fma(T(0.5), Fx, jx), ruy = fma(T(0.5), Fy, jy);   // rho v = j + F/2
    const T ux = rux * inv, uy = ruy * inv;
    const T ru2 = mul_rn(rux, ux) + mul_rn(ruy, uy);   // rho |v|^2
    const T vF = mul_rn(ux, Fx) + mul_rn(uy, Fy);
    const T trQ = Qxx + Qyy;

    // a product with a power of two is exact, so fma(2^k, x, y) rounds like
    // the separate multiply and add it replaces: same bits, one instruction
    const T m1 = fma(T(-4), f[0], fma(T(2), Sd, -Sa));
    const T m2 = fma(T(4), f[0], fma(T(-2), Sa, Sd));
    const T m4 = fma(T(-2), d13, Dxd);
    const T m6 = fma(T(-2), d24, Dyd);
    const T m7 = (f[1] + f[3]) - (f[2] + f[4]);
    const T m8 = (f[5] + f[7]) - (f[6] + f[8]);

    // m - m_eq for e and eps (Eq. 4): m1 + 2 rt - 3 rho|v|^2, m2 - rt + 3 rho|v|^2
    const T n1 = fma(T(-3), ru2, fma(T(2), rt, m1));
    const T n2 = fma(T(3), ru2, m2 - rt);
    // S[1] = 6 v.F, S[2] = -6 v.F (Eq. 6): the 6 is folded into h6s1 = 6 hs1, nh6s2 = -6 hs2
    const T ms1 = fma(T(P.c1), trQ, fma(T(P.h6s1), vF, fma(T(P.ns1), n1, m1)));
    const T ms2 = fma(T(P.c2), trQ, fma(T(P.nh6s2), vF, fma(T(P.ns2), n2, m2)));
    const T ms3 = jx + Fx;                             // = m3 - s_j (m3 - rho v_x) + (1 - s_j/2) F_x
    const T ms4 = fma(T(P.nhs4), Fx, fma(T(P.ns4), m4 + rux, m4));
    const T ms5 = jy + Fy;
    const T ms6 = fma(T(P.nhs6), Fy, fma(T(P.ns6), m6 + ruy, m6));
    // shear rates: fixed, or from the density-dependent viscosity (Section 4.2)
    T ns7 = T(P.ns7), ns8 = T(P.ns8), h2s7 = T(P.h2s7), hs8 = T(P.hs8);   // h2s7 = 2 hs7
    if (VISC && P.var_visc) {
        const T w = fmin(fmax((rho - T(P.visc_rho_g)) * T(P.visc_inv_drho), T(0)), T(1));
        const T sn = Fast<T>::rcp(fma(T(3), fma(w, T(P.dnu), T(P.nu_g)), T(0.5)));
        ns7 = ns8 = -sn;
        hs8 = fma(T(-0.5), sn, T(1));
        h2s7 = T(2) - sn;                                 // = 2 hs8 exactly
    }
    const T ms7 = fma(ns7, Qxx - Qyy,
                      fma(h2s7, mul_rn(ux, Fx) - mul_rn(uy, Fy),
                          fma(ns7, m7 - (mul_rn(rux, ux) - mul_rn(ruy, uy)), m7)));
    const T ms8 = fma(ns8, Qxy, fma(hs8, mul_rn(ux, Fy) + mul_rn(uy, Fx), fma(ns8, m8 - mul_rn(rux, uy), m8)));

    // f* = M^-1 m* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
    // The rows of a1..a8 sum to zero over the nine outputs, so the mass of the
    // node is 9 a0: a0 is rt/9 correctly rounded (one residual FMA), not
    // rt * fl(1/9), whose constant is 7e-9 too large in FP32 and would add that
    // bias to the mass at every step of a steady state.
    const T c9 = T(1.0 / 9.0);
    const T q9 = rt * c9;
    const T a0 = fma(fma(q9, T(-9), rt), c9, q9);
    const T a1 = mul_rn(ms1, T(1.0 / 36.0)), a2 = mul_rn(ms2, T(1.0 / 36.0));
    const T a3 = mul_rn(ms3, T(1.0 / 6.0)), a4 = mul_rn(ms4, T(1.0 / 12.0));
    const T a5 = mul_rn(ms5, T(1.0 / 6.0)), a6 = mul_rn(ms6, T(1.0 / 12.0));
    // a7 = ms7 / 4 and a8 = ms8 / 4 are exact: folded into the last add
    const T bax = fma(T(-2), a2, a0 - a1);
    const T bdg = fma(T(2), a1, a0) + a2;
    const T X = fma(T(-2), a4, a3), Y = fma(T(-2), a6, a5);
    const T DX = a3 + a4, DY = a5 + a6;
    out[0] = fma(T(4), a2, fma(T(-4), a1, a0));
    out[1] = fma(T(0.25), ms7, bax + X);
    out[2] = fma(T(-0.25), ms7, bax + Y);
    out[3] = fma(T(0.25), ms7, bax - X);
    out[4] = fma(T(-0.25), ms7, bax - Y);
    out[5] = fma(T(0.25), ms8, bdg + DX + DY);
    out[6] = fma(T(-0.25), ms8, bdg - DX + DY);
    out[7] = fma(T(0.25), ms8, bdg - DX - DY);
    out[8] = fma(T(-0.25), ms8, bdg + DX - DY);
}

// Equation-of-state constants in registers.
template <typename T, typename V> struct EosOf {
    int eos;
    V K, a, b, b4, RT, aalpha, two_over_G;
    __device__ __forceinline__ explicit EosOf(const Phys<T>& P)
        : eos(P.eos), K(P.K), a(P.a), b(P.b), b4(P.b4), RT(P.RT), aalpha(P.aalpha), two_over_G(P.two_over_G) {}
};
template <typename T> struct EosSel { using type = EosOf<T, const T&>; };
template <> struct EosSel<float> { using type = EosOf<float, float>; };
template <typename T> using EosRegs = typename EosSel<T>::type;

// Eq. 10 radicand with the pressure laws of lbm_internal.cuh, using Fast<T>.
// EOSK = LBM_EOS_* fixes the law at compile time; 0 reads it from the constants.
template <int EOSK, typename T> __device__ __forceinline__ T radicand_step(const EosRegs<T>& P, T rho) {
    const int eos = EOSK ? EOSK : P.eos;
    T p;
    if (eos == LBM_EOS_CS) {
        const T n = P.b4 * rho, q = T(1) - n;
        const T num = fma(n, fma(n, T(1) - n, T(1)), T(1));
        p = P.K * fma(-P.a * rho, rho, Fast<T>::div(rho * P.RT * num, q * q * q));
    } else if (eos == LBM_EOS_VDW) {
        p = P.K * fma(-P.a * rho, rho, Fast<T>::div(rho * P.RT, fma(-P.b, rho, T(1))));
    } else {
        const T br = P.b * rho;
        p = P.K * (Fast<T>::div(rho * P.RT, T(1) - br) - Fast<T>::div(P.aalpha * rho * rho, fma(br, T(2) - br, T(1))));
    }
    return P.two_over_G * fma(rho, T(-1.0 / 3.0), p);
}

// psi of Eq. 10 in FP64 with the law's division(s) and the square root
// folded into one reciprocal square root.  Each law's radicand
// (2/G)(p_EOS - rho/3) is written as W / D with D > 0 inside the law's range:
//   Carnahan-Starling  D = q^3, q = 1 - b rho/4,  W = rho [kR num - (kA rho + k3) q^3]
//                      (num = 1 + n + n^2 - n^3, n = b rho/4);
//   van der Waals      D = d, d = 1 - b rho,       W = rho [kR - (kA rho + k3) d];
//   Peng-Robinson      D = d e, e = 1 + 2 b rho - (b rho)^2,
//                      W = rho [kR e - (kAa rho + k3 e) d];
// with kR = (2/G) K R T, kA = (2/G) K a, kAa = (2/G) K a alpha(T),
// k3 = (2/G)/3.  Then psi = W / sqrt(W D); 1/(2 sqrt(x)) comes from the
// hardware estimate refined by two Goldschmidt steps, as in
// Fast<double>::sqrt.  A negative radicand gives NaN (as the square root
// does), psi(W = 0) = 0.
__device__ __forceinline__ double psi_fold_fp64(double W, double D) {
    const double x = W * D;
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double g0 = x * y, h0 = 0.5 * y;
    const double r0 = fma(-g0, h0, 0.5);
    const double g1 = fma(g0, r0, g0), h1 = fma(h0, r0, h0);
    const double r1 = fma(-g1, h1, 0.5);
    const double h2 = fma(h1, r1, h1);
    return W == 0.0 ? 0.0 : (W + W) * h2;
}

template <int EOSK>
__device__ __forceinline__ double psi_fp64(const EosRegs<double>& E, double kR, double kA, double kAa, double k3,
                                           double rho) {
    const int eos = EOSK ? EOSK : E.eos;
    if (eos == LBM_EOS_CS) {
        const double n = E.b4 * rho, q = 1.0 - n;
        const double num = fma(n, fma(n, 1.0 - n, 1.0), 1.0);
        const double q3 = q * q * q;
        return psi_fold_fp64(rho * fma(-fma(kA, rho, k3), q3, kR * num), q3);
    }
    const double br = E.b * rho, d = 1.0 - br;
    if (eos == LBM_EOS_VDW) return psi_fold_fp64(rho * fma(-fma(kA, rho, k3), d, kR), d);
    const double e = fma(br, 2.0 - br, 1.0);
    return psi_fold_fp64(rho * fma(-fma(kAa, rho, k3 * e), d, kR * e), d * e);
}

// Hybrid force (Eq. 9) and modifying tensor (Eq. 23, x G/2) of one node
// from psi at the node (p0) and its eight neighbours (p_a at x + e_a).
// The lattice sums are formed with the integer weights 12 w_a (4 on the
// axes, 1 on the diagonals) and the common factor 1/12 is folded into the
// constants: negGw = -G/12, kGw = kappa G/24; hA = A/2, omA = 1 - A.
// q_a = p_a^2, rounded on their own (the caller slides them down a column
// with the psi values, so each square is formed once).
template <typename T>
__device__ __forceinline__ void force_q(T negGw, T hA, T omA, T kGw, T p0, T p1, T p2, T p3, T p4, T p5, T p6,
                                        T p7, T p8, T q0, T q1, T q2, T q3, T q4, T q5, T q6, T q7, T q8, T& Fx,
                                        T& Fy, T& Qxx, T& Qyy, T& Qxy) {
    // Eq. 9: F = -G [ (A/2) sum w psi_n^2 e + (1-A) psi sum w psi_n e ]
    const T a57 = p5 - p7, a86 = p8 - p6, b57 = q5 - q7, b86 = q8 - q6;
    const T gx1 = fma(T(4), p1 - p3, a57 + a86), gy1 = fma(T(4), p2 - p4, a57 - a86);
    const T gx2 = fma(T(4), q1 - q3, b57 + b86), gy2 = fma(T(4), q2 - q4, b57 - b86);
    const T c = omA * p0;
    Fx = negGw * fma(c, gx1, hA * gx2);
    Fy = negGw * fma(c, gy1, hA * gy2);
    // Eq. 23 (x G/2): sums of w (psi_n - psi) e e and w (psi_n^2 - psi^2) e e;
    // sum w e_x^2 = sum w e_y^2 = 1 (12 with the integer weights) and
    // sum w e_x e_y = 0 over the ring
    const T s57 = p5 + p7, s68 = p6 + p8, t57 = q5 + q7, t68 = q6 + q8;
    const T d1 = s57 + s68, d2 = t57 + t68;
    const T sxx1 = fma(T(-12), p0, fma(T(4), p1 + p3, d1)), syy1 = fma(T(-12), p0, fma(T(4), p2 + p4, d1));
    const T sxx2 = fma(T(-12), q0, fma(T(4), q1 + q3, d2)), syy2 = fma(T(-12), q0, fma(T(4), q2 + q4, d2));
    const T sxy1 = s57 - s68, sxy2 = t57 - t68;
    Qxx = kGw * fma(c, sxx1, hA * sxx2);
    Qyy = kGw * fma(c, syy1, hA * syy2);
    Qxy = kGw * fma(c, sxy1, hA * sxy2);
}

// The constants of the lattice a tile belongs to: in the argument block
// (parameter space), or for a batched FP64 launch in the instance's
// descriptor in global memory.
template <typename T>
__device__ __forceinline__ const Phys<T>& phys_of(const StepArgs<T>& a, const Inst*, int) {
    return a.P;
}
__device__ __forceinline__ const Phys<float>& phys_of(const BatchArgs<float>& a, const Inst*, int slot) {
    return a.phys.P[slot];
}
__device__ __forceinline__ const Phys<double>& phys_of(const BatchArgs<double>&, const Inst* I, int) {
    return phys<double>(I);
}

// rho and psi (Eq. 10) of the tile and its 1-node ring, into sp.  A density
// outside the EOS's psi domain gives a negative radicand and a NaN psi
// (square root), which reaches every output of the owned node (F and Q are
// linear in psi, 0 x NaN is NaN): the collision's NaN check records it.
// Ring nodes beyond the lattice's ghost images feed no owned node.
template <typename Gm, int EOSK, typename T>
__device__ __forceinline__ void psi_ring(const T* sf, T* sp, const EosRegs<T>& E, T rho_ref, int tid, int tx,
                                         int ty) {
    constexpr int BX = Gm::BX;
    // FP64: psi_fp64 on every path (the law fixed at compile time or read at
    // run time), so that every tile computes the same bits
    const T kR = E.two_over_G * E.K * E.RT, kA = E.two_over_G * E.K * E.a, kAa = E.two_over_G * E.K * E.aalpha;
    const T k3 = E.two_over_G * T(1.0 / 3.0);
    auto ring = [&](int i, int j) {
        const T* q = sf + (j + 1) * Gm::WB + (i + Gm::HX - 1);
        T g[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = q[a * Gm::PB - cy(a) * Gm::WB - cx(a)];
        const T rho = rho_ref + rho_dev(g);
        T psi;
        if constexpr (sizeof(T) == 8) {
            psi = psi_fp64<EOSK>(E, kR, kA, kAa, k3, rho);
        } else {
            psi = Fast<T>::sqrt(radicand_step<EOSK>(E, rho));
        }
        sp[j * Gm::WP + i] = psi;
    };
    // rows ty, ty + TY, ... (unrolled where a thread owns several rows; the
    // one-row shapes run under a tighter register bound); the two right-hand
    // ring columns go to the threads the last row pass leaves idle when there
    // are enough, so that no warp evaluates more ring nodes than the busiest
    // row pass gives it
    constexpr int K = (Gm::HP + Gm::TY - 1) / Gm::TY;
    constexpr bool kMerge = Gm::ROWS > 1 && (K * Gm::TY - Gm::HP) * BX >= 2 * Gm::HP;
    if constexpr (Gm::ROWS > 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = ty + k * Gm::TY;
            if (j < Gm::HP) {
                ring(tx, j);
            } else if (kMerge && k == K - 1) {
                const int e = (j - Gm::HP) * BX + tx;
                if (e < 2 * Gm::HP) ring(BX + (e & 1), e >> 1);
            }
        }
    } else {
        for (int j = ty; j < Gm::HP; j += Gm::TY) ring(tx, j);
    }
    if (!kMerge)
        for (int e = tid; e < 2 * Gm::HP; e += Gm::NT) ring(BX + (e & 1), e >> 1);
}

// Force, modifying tensor, collision and store of the thread's ROWS nodes
// (consecutive rows of column tx).  Returns true when a node's results are
// NaN.  FAST: every node of the tile lies inside the lattice (no bounds
// checks), G != 0 and the shear rates are fixed; GHOST: the tile is within
// two rows or columns of the lattice's edge, so its nodes there also write
// their periodic images.  Both are decided once per tile.
template <typename Gm, bool FAST, bool GHOST, typename T, typename RP>
__device__ __forceinline__ bool collide_rows(const T* sf, const T* sp, const Phys<T>& P, const RP& R, T* __restrict__ dst,
                                             long long plane, int pitch, int x0, int y0, int nx, int ny, bool border,
                                             bool interact_rt, int tx, int ty) {
    const bool interact = FAST || interact_rt;
    // periodic images in the ghost cells read by the neighbouring tiles
    auto ghost = [&](T* o, int x, int y, const T (&v)[9]) {
        const bool xl = x < 2, xr = x >= nx - 2, yl = y < 2, yr = y >= ny - 2;
        if (!(xl || xr || yl || yr)) return;
        const int oxs[3] = {0, xl ? nx : 0, xr ? -nx : 0};
        const int oys[3] = {0, yl ? ny : 0, yr ? -ny : 0};
        const bool hx[3] = {true, xl, xr};
        const bool hy[3] = {true, yl, yr};
        for (int iy = 0; iy < 3; ++iy)
            for (int ix = 0; ix < 3; ++ix) {
                if (!(hx[ix] && hy[iy]) || (ix == 0 && iy == 0)) continue;
                T* g = o + static_cast<long long>(oys[iy]) * pitch + oxs[ix];
#pragma unroll
                for (int a = 0; a < 9; ++a) g[a * plane] = v[a];
            }
    };

    // each thread owns ROWS consecutive rows of one column; the 3x3 psi
    // neighbourhood slides down with it (three new loads per node)
    const T G = P.G, A = P.A;
    const T negGw = -G * T(1.0 / 12.0), hA = T(0.5) * A, omA = T(1) - A;
    const T kGw = P.kappa * G * T(1.0 / 24.0);
    const int ly0 = ty * Gm::ROWS;
    const T* s0 = sp + (ly0 + 1) * Gm::WP + (tx + 1);   // psi of node (tx, ly0)
    // FP64 slides the squares of the window too (six FP64 products fewer
    // per node); FP32 forms them per node, which keeps it to fewer
    // registers and measured faster
    constexpr bool kSlideSquares = sizeof(T) == 8;
    T wm0 = T(0), wm1 = T(0), wm2 = T(0), w00 = T(0), w01 = T(0), w02 = T(0);
    T qm0 = T(0), qm1 = T(0), qm2 = T(0), q00 = T(0), q01 = T(0), q02 = T(0);   // their squares
    if (interact) {
        wm0 = s0[-Gm::WP - 1];
        wm1 = s0[-Gm::WP];
        wm2 = s0[-Gm::WP + 1];
        w00 = s0[-1];
        w01 = s0[0];
        w02 = s0[1];
        if (kSlideSquares) {
            qm0 = mul_rn(wm0, wm0);
            qm1 = mul_rn(wm1, wm1);
            qm2 = mul_rn(wm2, wm2);
            q00 = mul_rn(w00, w00);
            q01 = mul_rn(w01, w01);
            q02 = mul_rn(w02, w02);
        }
    }

    bool bad = false;
    T* o = dst + static_cast<long long>(y0 + ly0 + GY) * pitch + (x0 + tx + Gm::GX);
#pragma unroll
    for (int r = 0; r < Gm::ROWS; ++r, o += pitch) {
        const int ly = ly0 + r;
        const int x = x0 + tx, y = y0 + ly;
        T wp0 = T(0), wp1 = T(0), wp2 = T(0), qp0 = T(0), qp1 = T(0), qp2 = T(0);
        if (interact) {
            const T* sr = s0 + (r + 1) * Gm::WP;
            wp0 = sr[-1];
            wp1 = sr[0];
            wp2 = sr[1];
            if (kSlideSquares) {
                qp0 = mul_rn(wp0, wp0);
                qp1 = mul_rn(wp1, wp1);
                qp2 = mul_rn(wp2, wp2);
            }
        }
        if (FAST || (x < nx && y < ny)) {
            const T* q = sf + (ly + GY) * Gm::WB + (tx + Gm::HX);
            T f[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) f[a] = q[a * Gm::PB - cy(a) * Gm::WB - cx(a)];

            T Fx = T(0), Fy = T(0), Qxx = T(0), Qyy = T(0), Qxy = T(0);
            if (interact) {
                if (!kSlideSquares) {
                    qp0 = mul_rn(wp0, wp0);
                    qp1 = mul_rn(wp1, wp1);
                    qp2 = mul_rn(wp2, wp2);
                    qm0 = mul_rn(wm0, wm0);
                    qm1 = mul_rn(wm1, wm1);
                    qm2 = mul_rn(wm2, wm2);
                    q00 = mul_rn(w00, w00);
                    q01 = mul_rn(w01, w01);
                    q02 = mul_rn(w02, w02);
                }
                force_q<T>(negGw, hA, omA, kGw, w01, w02, wp1, w00, wm1, wp2, wp0, wm0, wm2, q01, q02, qp1, q00,
                           qm1, qp2, qp0, qm0, qm2, Fx, Fy, Qxx, Qyy, Qxy);
            }

            T out[9];
            collide<T, !FAST>(R, f, Fx, Fy, Qxx, Qyy, Qxy, out);
            if (!(out[0] == out[0])) bad = true;

#pragma unroll
            for (int a = 0; a < 9; ++a) o[a * plane] = out[a];
            if (GHOST && border) ghost(o, x, y, out);
        }
        wm0 = w00; wm1 = w01; wm2 = w02;
        w00 = wp0; w01 = wp1; w02 = wp2;
        qm0 = q00; qm1 = q01; qm2 = q02;
        q00 = qp0; q01 = qp1; q02 = qp2;
    }
    return bad;
}

// The tile's psi ring on the path chosen for it (see step_body).
template <typename Gm, typename T>
__device__ __forceinline__ void ring_dispatch(bool fast, int eos, const T* sf, T* sp, const EosRegs<T>& E, T rho_ref,
                                              int tid, int tx, int ty) {
    if (fast && eos == LBM_EOS_CS) psi_ring<Gm, LBM_EOS_CS>(sf, sp, E, rho_ref, tid, tx, ty);
    else if (fast && eos == LBM_EOS_VDW) psi_ring<Gm, LBM_EOS_VDW>(sf, sp, E, rho_ref, tid, tx, ty);
    else if (fast && eos == LBM_EOS_PR) psi_ring<Gm, LBM_EOS_PR>(sf, sp, E, rho_ref, tid, tx, ty);
    else psi_ring<Gm, 0>(sf, sp, E, rho_ref, tid, tx, ty);
}

// The tile's collision and store on the path chosen for it; true when a
// node's results are NaN.
template <typename Gm, typename T, typename RP>
__device__ __forceinline__ bool collide_dispatch(bool fast, bool border, const T* sf, const T* sp, const Phys<T>& P,
                                                 const RP& R, T* dst, long long plane, int pitch, int x0, int y0,
                                                 int nx, int ny, bool interact, int tx, int ty) {
    if (fast && !border)
        return collide_rows<Gm, true, false>(sf, sp, P, R, dst, plane, pitch, x0, y0, nx, ny, border, interact, tx,
                                             ty);
    if (fast)
        return collide_rows<Gm, true, true>(sf, sp, P, R, dst, plane, pitch, x0, y0, nx, ny, border, interact, tx,
                                            ty);
    return collide_rows<Gm, false, true>(sf, sp, P, R, dst, plane, pitch, x0, y0, nx, ny, border, interact, tx, ty);
}

// One kernel, two ways to find the work, both from a __grid_constant__
// argument block: ONE = a single lattice (StepArgs: constants and tensor
// maps; tile coordinates from the tile index); otherwise a BatchArgs over up
// to kBatchLaunchMax instances (tensor maps, tile counts, array addresses and
// sizes, FP32 constants; the tile's instance by a binary search of the tile
// counts' prefix sums, or from a tile table).
// NBUF = 2 makes the CTAs persistent with a two-stage TMA pipeline: while
// tile k is collided, the box of tile k+1 streams into the other
// shared-memory buffer.
// Each tile takes one of three code paths, chosen once per tile: the fast
// path (every node inside the lattice, G != 0, fixed shear rates; the EOS
// fixed at compile time) has no per-node checks, in two copies: with and
// without the periodic ghost images of tiles at the lattice's edge; the
// general path handles the rest.  All compute the same bits.
template <typename T, int BX, int BY, int NT, int NBUF, bool ONE, typename Args>
__device__ __forceinline__ void step_body(const Inst* __restrict__ insts, int ntiles, int parity,
                                          unsigned long long timeout_ns, const Args& a) {
    using Gm = Geom<T, BX, BY, NT, NBUF>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    int t = blockIdx.x;
    if (t >= ntiles) return;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // tile tt -> (slot, x0, y0); the slot indexes the argument block's instances
    auto tile_of = [&](int tt, int& slot, int& x0, int& y0) {
        if constexpr (ONE) {
            slot = 0;
            x0 = (tt % a.tiles_x) * BX;
            y0 = (tt / a.tiles_x) * BY;
        } else {
            if (a.tiles) {
                const int4 tl = a.tiles[tt];
                slot = tl.x;
                x0 = tl.y;
                y0 = tl.z;
            } else {
                int lo = 0, hi = a.n - 1;   // the last slot with first[slot] <= tt
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.first[mid] <= tt) lo = mid;
                    else hi = mid - 1;
                }
                const int r = tt - a.first[lo];
                const int q = tile_row(r, a.div_m[lo], a.div_s[lo]);   // r / tiles_x
                slot = lo;
                x0 = (r - q * a.tiles_x[lo]) * BX;
                y0 = q * BY;
            }
        }
    };
    auto issue = [&](int tt, int bb) {
        int slot, x0, y0;
        tile_of(tt, slot, x0, y0);
        const CUtensorMap* map;
        if constexpr (ONE) map = &a.tmap[parity];
        else map = &a.tmap[slot];
        mbar_arrive_expect_tx(&bar[bb], static_cast<uint32_t>(Gm::box_bytes));
        tma_load_3d(smem + bb * Gm::buf_stride, map, x0 + Gm::GX - Gm::HX, y0, 0, &bar[bb]);
    };
    if (tid == 0) issue(t, 0);

#pragma unroll 1
    for (int k = 0; t < ntiles; ++k, t += gridDim.x) {
        const int b = NBUF == 2 ? (k & 1) : 0;
        const uint32_t ph = NBUF == 2 ? ((k >> 1) & 1) : (k & 1);
        const T* sf = reinterpret_cast<const T*>(smem + b * Gm::buf_stride);
        T* sp = reinterpret_cast<T*>(smem + Gm::psi_off + b * Gm::psi_stride);
        int slot, x0, y0;
        tile_of(t, slot, x0, y0);
        const Inst* I = nullptr;
        if constexpr (!ONE && sizeof(T) == 8) I = insts + a.inst[slot];
        const Phys<T>& P = phys_of(a, I, slot);
        int nx, ny;
        int* status;
        if constexpr (ONE) {
            nx = a.nx;
            ny = a.ny;
            status = a.status;
        } else if constexpr (sizeof(T) == 4) {
            nx = a.lat[slot].nx;
            ny = a.lat[slot].ny;
            status = a.lat[slot].status;
        } else {
            nx = I->nx;
            ny = I->ny;
            status = I->status;
        }
        const int interact = P.interact;
        const EosRegs<T> E(P);
        const T rho_ref = P.rho_ref;
        const bool border = x0 < 2 || x0 + BX > nx - 2 || y0 < 2 || y0 + BY > ny - 2;
        // the fast path: every node of the tile inside the lattice, G != 0,
        // fixed shear rates
        const bool fast = interact && !P.var_visc && x0 + BX <= nx && y0 + BY <= ny;
        const int eos = P.eos;

        bool ok = mbar_wait_bounded(&bar[b], ph, timeout_ns);
        if (k == 0 && (P.flags & LBM_FLAG_TEST_FORCE_TIMEOUT)) {
            // the phase after the completed first load: nothing completes it
            ok = ok && mbar_wait_bounded(&bar[0], 1, 2000000ull);
        }

        // ---- rho and psi of the tile and its ring (Eq. 10) ---------------
        if (interact && ok) ring_dispatch<Gm>(fast, eos, sf, sp, E, rho_ref, tid, tx, ty);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(status, ST_TIMEOUT);
                mbar_wait_bounded(&bar[b], ph, timeout_ns);   // let a late copy land before exit
            }
            return;
        }
        // every thread is past its reads of the other buffer: prefetch the next tile into it
        if (NBUF == 2 && tid == 0 && t + static_cast<int>(gridDim.x) < ntiles) issue(t + gridDim.x, b ^ 1);

        // ---- collide and stream every owned node -------------------------
        T* dst;
        long long plane;
        int pitch;
        if constexpr (ONE) {
            dst = static_cast<T*>(a.pop[parity ^ 1]);
            plane = a.plane;
            pitch = a.pitch;
        } else if constexpr (sizeof(T) == 4) {
            dst = static_cast<T*>(a.lat[slot].pop[parity ^ 1]);
            plane = a.lat[slot].plane;
            pitch = a.lat[slot].pitch;
        } else {
            dst = static_cast<T*>(I->pop[parity ^ 1]);
            plane = I->plane;
            pitch = I->pitch;
        }
        const Regs<T> R(P);
        const bool bad = collide_dispatch<Gm>(fast, border, sf, sp, P, R, dst, plane, pitch, x0, y0, nx, ny, interact,
                                              tx, ty);
        if (bad) atomicOr(status, ST_UNSTABLE);
    }
}

// The constants of a tile's lattice in a multi-step launch: the argument
// block (FP32) or the instance descriptor (FP64), as for a batched step.
__device__ __forceinline__ const Phys<float>& phys_of(const RunArgs<float>& a, const Inst*, int slot) {
    return a.phys.P[slot];
}
__device__ __forceinline__ const Phys<double>& phys_of(const RunArgs<double>&, const Inst* I, int) {
    return phys<double>(I);
}

// A work item of a multi-step launch, w = s * ntiles + t: step s of tile t,
// which is tile (col, row) of the instance in slot `slot`.
struct RunItem {
    int s, t, slot, col, row;
};
template <bool ONE, typename T> __device__ __forceinline__ RunItem run_item(const RunArgs<T>& a, long long w) {
    RunItem it;
    it.s = static_cast<int>(w / a.ntiles);
    it.t = static_cast<int>(w - static_cast<long long>(it.s) * a.ntiles);
    it.slot = 0;
    if constexpr (!ONE) {
        int hi = a.n - 1;   // the last slot with first[slot] <= t
        while (it.slot < hi) {
            const int mid = (it.slot + hi + 1) >> 1;
            if (a.first[mid] <= it.t) it.slot = mid;
            else hi = mid - 1;
        }
    }
    const int ncol = a.tiles_x[it.slot];
    const int r = it.t - a.first[it.slot];
    it.row = r / ncol;
    it.col = r - it.row * ncol;
    return it;
}

// The step counter that lane `lane` (< 16) of the finding warp watches for
// item `it` (s > 0): step s - 1 of every tile whose nodes lie within two
// nodes of this tile's (periodically), i.e. the 3 x 3 tile neighbourhood
// and, across a last tile row or column only one node wide, the tile beyond
// it (the fourth candidate row / column; otherwise a repeat).  Each of them
// wrote part of what this tile reads, and read part of what it will
// overwrite.  Lane k watches candidate (k / 4, k % 4).
template <int BX, int BY, typename T>
__device__ __forceinline__ const int* run_dep_flag(const RunArgs<T>& a, const RunItem& it, int lane) {
    const int ncol = a.tiles_x[it.slot], nrow = (a.first[it.slot + 1] - a.first[it.slot]) / ncol;
    int dr = lane / 4 - 1, dc = lane % 4 - 1;
    const int ny = a.lat[it.slot].ny, nx = a.lat[it.slot].nx;
    if (dr == 2) {
        const bool thin = ny - (nrow - 1) * BY == 1 && nrow > 2;
        dr = thin && it.row == nrow - 2 ? 2 : (thin && it.row == 0 ? -2 : 0);
    }
    if (dc == 2) {
        const bool thin = nx - (ncol - 1) * BX == 1 && ncol > 2;
        dc = thin && it.col == ncol - 2 ? 2 : (thin && it.col == 0 ? -2 : 0);
    }
    const int cc = (it.col + dc + 2 * ncol) % ncol, rr = (it.row + dr + 2 * nrow) % nrow;
    return a.done + a.first[it.slot] + rr * ncol + cc;
}

// Warp-wide bounded wait until every lane's flag (lanes with mine == true
// watch nothing) has reached s.  Gives up after timeout_ns, or when another
// CTA raised the abort flag; returns false then.  The warp barrier at the
// end orders every lane's acquire before the caller's later accesses.
__device__ __forceinline__ bool run_dep_wait(const int* flag, bool mine, int s, const int* abort_flag,
                                             unsigned long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; !__all_sync(0xffffffffu, mine); ++it) {
        if (!mine) mine = ld_acquire_gpu(flag) >= s;
        if ((it & 63u) == 63u) {
            int give_up = 0;
            if (lane == 0) give_up = globaltimer_ns() - t0 > timeout_ns || ld_acquire_gpu(abort_flag) != 0;
            if (__shfl_sync(0xffffffffu, give_up, 0)) {
                ok = false;
                break;
            }
        }
    }
    __syncwarp();
    return ok;
}

// Multi-step persistent body: every CTA takes work items (step s, tile t)
// from a global counter in step order, waits until every tile within two
// nodes of it has finished step s - 1 (each of those wrote part of this
// tile's box, directly or as a periodic ghost image, and read part of what
// this tile will overwrite), loads its
// box, runs the same psi ring, collision and store as the one-step kernels
// (same bits), and publishes that tile t has finished step s.  The grid is
// launched cooperatively (every CTA resident), and items are handed out in
// step order, so every item a CTA waits for is held by a running CTA whose
// own waits are on earlier steps.  Every wait is bounded (timeout_ns): one
// that gives up records ST_TIMEOUT, raises the launch's abort flag, and
// every CTA stops at its next item.
template <typename T, int BX, int BY, int NT, bool ONE>
__device__ __forceinline__ void run_body(const Inst* __restrict__ insts, unsigned long long timeout_ns,
                                         const RunArgs<T>& a) {
    using Gm = Geom<T, BX, BY, NT, 1>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_work[6];   // ok, step, tile, slot, x0, y0 of the item, written by thread 0
    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = tid / BX;
    const T* sf = reinterpret_cast<const T*>(smem);
    T* sp = reinterpret_cast<T*>(smem + Gm::psi_off);

    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t phase = 0;
    bool first = true;
    const long long total = static_cast<long long>(a.nsteps) * a.ntiles;
    // warp 0 finds the work: lane 0 takes items from the counter (the next
    // one is taken while the current one is computed), lanes 0-15 check the
    // step counters of the tiles it depends on together, lane 0 issues the
    // TMA load
    const int lane = tid & 31;
    long long next = 0;
    if (tid == 0) next = static_cast<long long>(atomicAdd(a.counter, 1ull));
#pragma unroll 1
    for (;;) {
        if (tid < 32) {
            const long long w = __shfl_sync(0xffffffffu, next, 0);
            int ok = w < total;
            if (lane == 0 && ok) ok = ld_acquire_gpu(a.abort_flag) == 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            RunItem it{0, 0, 0, 0, 0};
            if (ok) {
                it = run_item<ONE>(a, w);
                if (it.s > 0) {
                    const int* flag = lane < 16 ? run_dep_flag<BX, BY>(a, it, lane) : nullptr;
                    ok = run_dep_wait(flag, lane >= 16 || ld_acquire_gpu(flag) >= it.s, it.s, a.abort_flag,
                                      timeout_ns);
                    if (!ok && lane == 0) {
                        atomicExch(a.abort_flag, 1);
                        atomicOr(a.lat[it.slot].status, ST_TIMEOUT);
                    }
                }
                if (ok && lane == 0) {
                    fence_proxy_async_global();   // the neighbours' stores, then this CTA's TMA read of them
                    mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(Gm::box_bytes));
                    tma_load_3d(smem, &a.tmap[(a.parity0 + it.s) & 1][it.slot], it.col * BX + Gm::GX - Gm::HX,
                                it.row * BY, 0, &bar);
                }
            }
            if (lane == 0) {
                if (ok) next = static_cast<long long>(atomicAdd(a.counter, 1ull));   // the item after this one
                s_work[0] = ok;
                s_work[1] = it.s;
                s_work[2] = it.t;
                s_work[3] = it.slot;
                s_work[4] = it.col * BX;
                s_work[5] = it.row * BY;
            }
        }
        __syncthreads();
        if (!s_work[0]) break;   // no copy in flight: nothing was issued
        const int s = s_work[1], t = s_work[2], slot = ONE ? 0 : s_work[3];
        const int x0 = s_work[4], y0 = s_work[5];
        const int parity = (a.parity0 + s) & 1;
        const Inst* I = nullptr;
        if constexpr (sizeof(T) == 8) I = insts + a.inst[slot];
        const Phys<T>& P = phys_of(a, I, slot);
        const int nx = a.lat[slot].nx, ny = a.lat[slot].ny;
        int* const status = a.lat[slot].status;
        T* const dst = static_cast<T*>(a.lat[slot].pop[parity ^ 1]);
        const long long plane = a.lat[slot].plane;
        const int pitch = a.lat[slot].pitch;
        const int interact = P.interact;
        const EosRegs<T> E(P);
        const T rho_ref = P.rho_ref;
        const bool border = x0 < 2 || x0 + BX > nx - 2 || y0 < 2 || y0 + BY > ny - 2;
        const bool fast = interact && !P.var_visc && x0 + BX <= nx && y0 + BY <= ny;

        bool ok = mbar_wait_bounded(&bar, phase, timeout_ns);
        phase ^= 1u;
        if (first && (P.flags & LBM_FLAG_TEST_FORCE_TIMEOUT)) {
            // the phase after the completed load: nothing completes it
            ok = ok && mbar_wait_bounded(&bar, phase, 2000000ull);
        }
        first = false;
        if (interact && ok) ring_dispatch<Gm>(fast, P.eos, sf, sp, E, rho_ref, tid, tx, ty);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(status, ST_TIMEOUT);
                atomicExch(a.abort_flag, 1);
                mbar_wait_bounded(&bar, phase ^ 1u, timeout_ns);   // let a late copy land before exit
            }
            return;
        }
        const Regs<T> R(P);
        const bool bad = collide_dispatch<Gm>(fast, border, sf, sp, P, R, dst, plane, pitch, x0, y0, nx, ny, interact,
                                              tx, ty);
        if (bad) atomicOr(status, ST_UNSTABLE);
        __syncthreads();   // every store of the tile, and every read of its box, is done
        // warp 1 publishes the tile's step while warp 0 already finds the next
        // item and issues its load; warp 0 never waits for warp 1 except through
        // the step counter, so an item that depends on this one simply waits a
        // little longer.  The release store is cumulative: the barrier above
        // orders every thread's stores of the tile before it, so a CTA that
        // acquires the counter sees them all
        if (tid == 32) st_release_gpu(a.done + t, s + 1);
    }
}

// The kernels.  FP32 launches ask for 1024 resident threads per SM (two
// CTAs of 512), which caps their registers at 64 (except the batched
// persistent variant, which would spill); FP64 leaves the register count to
// the compiler, except for one-tile-per-CTA tiles of one node row per thread
// (k_step_row), which ask for three resident CTAs: they fit in 85 registers
// without spilling, and the compiler's own choice for the batched variant
// (94-98) would leave two.
template <typename T, bool ONE> using ArgsOf = typename std::conditional<ONE, StepArgs<T>, BatchArgs<T>>::type;

template <typename T, int BX, int BY, int NT, int NBUF, bool ONE>
__global__ void __launch_bounds__(NT) k_step(const Inst* __restrict__ insts, int ntiles, int parity,
                                             unsigned long long timeout_ns,
                                             const __grid_constant__ ArgsOf<T, ONE> args) {
    step_body<T, BX, BY, NT, NBUF, ONE>(insts, ntiles, parity, timeout_ns, args);
}
template <typename T, int BX, int BY, int NT, int NBUF, bool ONE>
__global__ void __launch_bounds__(NT, 3) k_step_row(const Inst* __restrict__ insts, int ntiles, int parity,
                                                    unsigned long long timeout_ns,
                                                    const __grid_constant__ ArgsOf<T, ONE> args) {
    step_body<T, BX, BY, NT, NBUF, ONE>(insts, ntiles, parity, timeout_ns, args);
}
template <int BX, int BY, int NT, int NBUF, bool ONE>
__global__ void __launch_bounds__(NT, (ONE || NBUF == 1) ? 1024 / NT : 1) k_step_f32(const Inst* __restrict__ insts,
                                                            int ntiles, int parity, unsigned long long timeout_ns,
                                                            const __grid_constant__ ArgsOf<float, ONE> args) {
    step_body<float, BX, BY, NT, NBUF, ONE>(insts, ntiles, parity, timeout_ns, args);
}
template <typename T, int BX, int BY, int NT, bool ONE>
__global__ void __launch_bounds__(NT, 2) k_run(const Inst* __restrict__ insts, unsigned long long timeout_ns,
                                            const __grid_constant__ RunArgs<T> args) {
    run_body<T, BX, BY, NT, ONE>(insts, timeout_ns, args);
}
template <typename T, int BX, int BY, int NT, bool ONE>
__global__ void __launch_bounds__(NT, 3) k_run_row(const Inst* __restrict__ insts, unsigned long long timeout_ns,
                                                   const __grid_constant__ RunArgs<T> args) {
    run_body<T, BX, BY, NT, ONE>(insts, timeout_ns, args);
}
// CTAs of the multi-step FP32 kernel that fit on an SM: 1024 threads, and
// the SM's 228 KB of shared memory (1 KB of it reserved per CTA)
template <int BX, int BY, int NT> constexpr int run_ctas_f32() {
    constexpr int by_smem = static_cast<int>(233472 / (Geom<float, BX, BY, NT, 1>::smem + 2048));
    return by_smem < 1024 / NT ? (by_smem > 0 ? by_smem : 1) : 1024 / NT;
}
template <int BX, int BY, int NT, bool ONE>
__global__ void __launch_bounds__(NT, (run_ctas_f32<BX, BY, NT>())) k_run_f32(const Inst* __restrict__ insts,
                                                                          unsigned long long timeout_ns,
                                                                          const __grid_constant__ RunArgs<float> args) {
    run_body<float, BX, BY, NT, ONE>(insts, timeout_ns, args);
}
// the multi-step kernel of a (precision, ONE) launch, with the launch bounds of the one-step kernel
template <typename T, int BX, int BY, int NT, bool ONE,
          int KIND = std::is_same<T, float>::value ? 2 : (BX * BY == NT ? 1 : 0)>
struct RSel {
    static constexpr auto fn = &k_run<T, BX, BY, NT, ONE>;
};
template <typename T, int BX, int BY, int NT, bool ONE> struct RSel<T, BX, BY, NT, ONE, 1> {
    static constexpr auto fn = &k_run_row<T, BX, BY, NT, ONE>;
};
template <typename T, int BX, int BY, int NT, bool ONE> struct RSel<T, BX, BY, NT, ONE, 2> {
    static constexpr auto fn = &k_run_f32<BX, BY, NT, ONE>;
};

// the kernel a (precision, ONE) launch uses
template <typename T, int BX, int BY, int NT, int NBUF, bool ONE,
          int KIND = std::is_same<T, float>::value ? 2 : (BX * BY == NT && NBUF == 1 ? 1 : 0)>
struct KSel {
    static constexpr auto fn = &k_step<T, BX, BY, NT, NBUF, ONE>;
};
template <typename T, int BX, int BY, int NT, int NBUF, bool ONE> struct KSel<T, BX, BY, NT, NBUF, ONE, 1> {
    static constexpr auto fn = &k_step_row<T, BX, BY, NT, NBUF, ONE>;
};
template <typename T, int BX, int BY, int NT, int NBUF, bool ONE> struct KSel<T, BX, BY, NT, NBUF, ONE, 2> {
    static constexpr auto fn = &k_step_f32<BX, BY, NT, NBUF, ONE>;
};

// ---- tile configurations ------------------------------------------------
template <typename T, int BX, int BY, int NT, int NBUF> struct Cfg {
    using Gm = Geom<T, BX, BY, NT, NBUF>;
    static int grid_cap[2];   // resident CTAs on the device (persistent grid), per kernel variant
    static int run_cap[2];    // resident CTAs of the multi-step kernels (one box per CTA only)
    template <bool ONE> static cudaError_t prep_run() {
        if constexpr (NBUF != 1) {
            return cudaSuccess;
        } else {
            const auto fn = RSel<T, BX, BY, NT, ONE>::fn;
            cudaError_t e =
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(Gm::smem));
            if (e != cudaSuccess) return e;
            int dev = 0, sms = 0, occ = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT, Gm::smem)) != cudaSuccess) return e;
            run_cap[ONE ? 1 : 0] = occ * sms;
            return cudaSuccess;
        }
    }
    // every CTA of the grid resident (cooperative launch), no more CTAs than
    // work items, and no more than two per tile: beyond that the extra CTAs of
    // a small lattice would only wait for steps their neighbours have not
    // finished, and hold SM slots that other launches could use
    static cudaError_t run(const Inst* d, const void* args, bool one, int ntiles, int nsteps, unsigned long long to,
                           cudaStream_t st) {
        if constexpr (NBUF != 1) {
            return cudaErrorNotSupported;
        } else {
            const long long items = static_cast<long long>(ntiles) * nsteps;
            const int cap = run_cap[one ? 1 : 0];
            if (cap < 1) return cudaErrorNotSupported;
            long long grid = items < cap ? items : cap;
            if (grid > 2ll * ntiles) grid = 2ll * ntiles;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(static_cast<unsigned>(grid));
            cfg.blockDim = dim3(NT);
            cfg.dynamicSmemBytes = Gm::smem;
            cfg.stream = st;
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeCooperative;
            attr.val.cooperative = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            const RunArgs<T>& a = *static_cast<const RunArgs<T>*>(args);
            if (one) return cudaLaunchKernelEx(&cfg, RSel<T, BX, BY, NT, true>::fn, d, to, a);
            return cudaLaunchKernelEx(&cfg, RSel<T, BX, BY, NT, false>::fn, d, to, a);
        }
    }
    static TileCfg tc() { return TileCfg{BX, BY, NT, NBUF}; }
    static size_t smem() { return Gm::smem; }
    template <bool ONE> static cudaError_t prep_one() {
        cudaError_t e = cudaFuncSetAttribute(KSel<T, BX, BY, NT, NBUF, ONE>::fn,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(Gm::smem));
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, KSel<T, BX, BY, NT, NBUF, ONE>::fn, NT,
                                                                Gm::smem)) != cudaSuccess)
            return e;
        grid_cap[ONE ? 1 : 0] = (occ > 0 ? occ : 1) * sms;
        return cudaSuccess;
    }
    static cudaError_t prepare() {
        cudaError_t e = prep_one<false>();
        if (e == cudaSuccess) e = prep_one<true>();
        if (e == cudaSuccess) e = prep_run<false>();
        if (e == cudaSuccess) e = prep_run<true>();
        return e;
    }
    static cudaError_t launch(const Inst* d, const void* args, bool one, int n, int parity, unsigned long long to,
                              cudaStream_t st) {
        // one CTA per tile, or a persistent grid of resident CTAs striding over the tiles
        const int cap = grid_cap[one ? 1 : 0];
        const int grid = NBUF == 1 ? n : (n < cap ? n : cap);
        if (one)
            KSel<T, BX, BY, NT, NBUF, true>::fn<<<grid, NT, Gm::smem, st>>>(d, n, parity, to,
                                                                            *static_cast<const StepArgs<T>*>(args));
        else
            KSel<T, BX, BY, NT, NBUF, false>::fn<<<grid, NT, Gm::smem, st>>>(d, n, parity, to,
                                                                             *static_cast<const BatchArgs<T>*>(args));
        return cudaGetLastError();
    }
};
template <typename T, int BX, int BY, int NT, int NBUF> int Cfg<T, BX, BY, NT, NBUF>::grid_cap[2] = {1, 1};
template <typename T, int BX, int BY, int NT, int NBUF> int Cfg<T, BX, BY, NT, NBUF>::run_cap[2] = {0, 0};

}  // namespace

// A tile configuration: its shape, shared memory, set-up and launches.
struct Entry {
    TileCfg (*tc)();
    size_t (*smem)();
    cudaError_t (*prepare)();
    cudaError_t (*launch)(const Inst*, const void*, bool, int, int, unsigned long long, cudaStream_t);
    cudaError_t (*run)(const Inst*, const void*, bool, int, int, unsigned long long, cudaStream_t);
    int nbuf;
};

#define LBM_CFG(T, BX, BY, NT, NB)                                                                    \
    Entry {                                                                                          \
        &Cfg<T, BX, BY, NT, NB>::tc, &Cfg<T, BX, BY, NT, NB>::smem, &Cfg<T, BX, BY, NT, NB>::prepare, \
            &Cfg<T, BX, BY, NT, NB>::launch, &Cfg<T, BX, BY, NT, NB>::run, NB                         \
    }

}  // namespace lbm
