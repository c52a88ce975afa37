// lbm_step.cu -- the fused per-timestep kernel of the pseudo-potential MRT
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
#include "lbm_internal.cuh"

namespace lbm {
namespace {

template <typename T, int BX_, int BY_, int NT_> struct Geom {
    static constexpr int BX = BX_, BY = BY_, NT = NT_;
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
    static constexpr size_t psi_off = (box_bytes + 127) / 128 * 128;
    static constexpr size_t smem = psi_off + size_t(WP) * HP * sizeof(T);
    static_assert(NT % BX == 0 && BY % TY == 0, "thread layout must tile the block");
    static_assert(WB <= 256 && HB <= 256, "TMA box dimensions are limited to 256");
    static_assert((WB * sizeof(T)) % 16 == 0, "TMA box rows must be a multiple of 16 bytes");
};

// Moment-space collision of one node in deviation form (Eqs. 2-6, 25, 26).
// f: pre-collision f_a - t_a rho_ref; out: post-collision, same form.
template <typename T>
__device__ __forceinline__ void collide(const Phys<T>& P, const T (&f)[9], T Fx, T Fy, T Qxx, T Qyy,
                                        T Qxy, T (&out)[9]) {
    const T Sa = (f[1] + f[3]) + (f[2] + f[4]);
    const T Sd = (f[5] + f[7]) + (f[6] + f[8]);
    const T rt = f[0] + Sa + Sd;                       // rho - rho_ref
    const T rho = P.rho_ref + rt;
    const T inv = T(1) / rho;
    const T d13 = f[1] - f[3], d24 = f[2] - f[4];
    const T Dxd = (f[5] - f[7]) + (f[8] - f[6]);
    const T Dyd = (f[5] - f[7]) + (f[6] - f[8]);
    const T jx = d13 + Dxd, jy = d24 + Dyd;
    const T rux = jx + T(0.5) * Fx, ruy = jy + T(0.5) * Fy;   // rho v = j + F/2
    const T ux = rux * inv, uy = ruy * inv;
    const T ru2 = rux * ux + ruy * uy;                 // rho |v|^2
    const T vF = ux * Fx + uy * Fy;
    const T trQ = Qxx + Qyy;

    const T m1 = T(2) * Sd - Sa - T(4) * f[0];
    const T m2 = Sd - T(2) * Sa + T(4) * f[0];
    const T m4 = Dxd - T(2) * d13;
    const T m6 = Dyd - T(2) * d24;
    const T m7 = (f[1] + f[3]) - (f[2] + f[4]);
    const T m8 = (f[5] + f[7]) - (f[6] + f[8]);

    const T e1 = T(3) * ru2 - T(2) * rt;               // m_eq deviations (Eq. 4)
    const T e2 = rt - T(3) * ru2;
    const T ms1 = m1 - P.s[1] * (m1 - e1) + P.hs[1] * (T(6) * vF) + P.c1 * trQ;
    const T ms2 = m2 - P.s[2] * (m2 - e2) - P.hs[2] * (T(6) * vF) + P.c2 * trQ;
    const T ms3 = jx + Fx;                             // = m3 - s_j (m3 - rho v_x) + (1 - s_j/2) F_x
    const T ms4 = m4 - P.s[4] * (m4 + rux) - P.hs[4] * Fx;
    const T ms5 = jy + Fy;
    const T ms6 = m6 - P.s[6] * (m6 + ruy) - P.hs[6] * Fy;
    const T ms7 = m7 - P.s[7] * (m7 - (rux * ux - ruy * uy)) + P.hs[7] * (T(2) * (ux * Fx - uy * Fy)) -
                  P.s[7] * (Qxx - Qyy);
    const T ms8 = m8 - P.s[8] * (m8 - rux * uy) + P.hs[8] * (ux * Fy + uy * Fx) - P.s[8] * Qxy;

    // f* = M^-1 m* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const T a0 = rt * T(1.0 / 9.0), a1 = ms1 * T(1.0 / 36.0), a2 = ms2 * T(1.0 / 36.0);
    const T a3 = ms3 * T(1.0 / 6.0), a4 = ms4 * T(1.0 / 12.0);
    const T a5 = ms5 * T(1.0 / 6.0), a6 = ms6 * T(1.0 / 12.0);
    const T a7 = ms7 * T(0.25), a8 = ms8 * T(0.25);
    const T bax = a0 - a1 - T(2) * a2;
    const T bdg = a0 + T(2) * a1 + a2;
    const T X = a3 - T(2) * a4, Y = a5 - T(2) * a6;
    const T DX = a3 + a4, DY = a5 + a6;
    out[0] = a0 - T(4) * a1 + T(4) * a2;
    out[1] = bax + X + a7;
    out[2] = bax + Y - a7;
    out[3] = bax - X + a7;
    out[4] = bax - Y - a7;
    out[5] = bdg + DX + DY + a8;
    out[6] = bdg - DX + DY - a8;
    out[7] = bdg - DX - DY + a8;
    out[8] = bdg + DX - DY - a8;
}

template <typename T, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT) k_step(const Inst* __restrict__ insts, const int4* __restrict__ tiles,
                                             int parity, unsigned long long timeout_ns) {
    using Gm = Geom<T, BX, BY, NT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    T* sf = reinterpret_cast<T*>(smem);
    T* sp = reinterpret_cast<T*>(smem + Gm::psi_off);
    const int tid = threadIdx.x;

    const int4 tile = tiles[blockIdx.x];
    const Inst* I = insts + tile.x;
    const int x0 = tile.y, y0 = tile.z;
    const CUtensorMap* map = &I->tmap[parity];

    if (tid == 0) {
        acquire_tmap(map);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, static_cast<uint32_t>(Gm::box_bytes));
        tma_load_3d(sf, map, x0 + Gm::GX - Gm::HX, y0, 0, &bar);
    }

    const Phys<T>& P = phys<T>(I);
    const int nx = I->nx, ny = I->ny;
    const unsigned flags = P.flags;

    bool ok = mbar_wait_bounded(&bar, 0, timeout_ns);
    if (flags & LBM_FLAG_TEST_FORCE_TIMEOUT) {
        // parity 1 is the phase after the completed load: nothing completes it
        ok = ok && mbar_wait_bounded(&bar, 1, 2000000ull);
    }
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicOr(I->status, ST_TIMEOUT);
            mbar_wait_bounded(&bar, 0, timeout_ns);   // let a late copy land before exit
        }
        return;
    }

    // ---- rho and psi of the tile and its ring (Eq. 10) -------------------
    const int interact = P.interact;
    const T rho_ref = P.rho_ref;
    bool bad = false;
    if (interact) {
        for (int idx = tid; idx < Gm::WP * Gm::HP; idx += NT) {
            const int i = idx % Gm::WP, j = idx / Gm::WP;
            const T* q = sf + (j + 1) * Gm::WB + (i + Gm::HX - 1);
            T r = T(0);
#pragma unroll
            for (int a = 0; a < 9; ++a) r += q[a * Gm::PB - cy(a) * Gm::WB - cx(a)];
            const T rad = psi_radicand(P, rho_ref + r);
            sp[idx] = sqrt(rad);
            const int x = x0 - 1 + i, y = y0 - 1 + j;
            if (i >= 1 && i <= BX && j >= 1 && j <= BY && x < nx && y < ny && !(rad >= T(0))) bad = true;
        }
    }
    __syncthreads();

    // ---- collide and stream every owned node -----------------------------
    const int tx = tid % BX, ty = tid / BX;
    T* __restrict__ dst = static_cast<T*>(I->pop[parity ^ 1]);
    const long long plane = I->plane;
    const int pitch = I->pitch;
    const T G = P.G, A = P.A;
    const T hA = T(0.5) * A, omA = T(1) - A;
    const T kG2 = P.kappa * G * T(0.5);
    constexpr T w1 = T(1.0 / 3.0), w2 = T(1.0 / 12.0);

#pragma unroll 1
    for (int k = 0; k < Gm::ROWS; ++k) {
        const int ly = ty + k * Gm::TY;
        const int x = x0 + tx, y = y0 + ly;
        if (x >= nx || y >= ny) continue;
        const T* q = sf + (ly + GY) * Gm::WB + (tx + Gm::HX);
        T f[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a] = q[a * Gm::PB - cy(a) * Gm::WB - cx(a)];

        T Fx = T(0), Fy = T(0), Qxx = T(0), Qyy = T(0), Qxy = T(0);
        if (interact) {
            const T* s = sp + (ly + 1) * Gm::WP + (tx + 1);
            const T p0 = s[0];
            const T p1 = s[1], p2 = s[Gm::WP], p3 = s[-1], p4 = s[-Gm::WP];
            const T p5 = s[Gm::WP + 1], p6 = s[Gm::WP - 1], p7 = s[-Gm::WP - 1], p8 = s[-Gm::WP + 1];
            const T q1 = p1 * p1, q2 = p2 * p2, q3 = p3 * p3, q4 = p4 * p4;
            const T q5 = p5 * p5, q6 = p6 * p6, q7 = p7 * p7, q8 = p8 * p8;
            // Eq. 9: F = -G [ (A/2) sum w psi_n^2 e + (1-A) psi sum w psi_n e ]
            const T gx1 = w1 * (p1 - p3) + w2 * ((p5 - p7) + (p8 - p6));
            const T gy1 = w1 * (p2 - p4) + w2 * ((p5 - p7) + (p6 - p8));
            const T gx2 = w1 * (q1 - q3) + w2 * ((q5 - q7) + (q8 - q6));
            const T gy2 = w1 * (q2 - q4) + w2 * ((q5 - q7) + (q6 - q8));
            Fx = -G * (hA * gx2 + omA * p0 * gx1);
            Fy = -G * (hA * gy2 + omA * p0 * gy1);
            // Eq. 23 (x G/2): sums of w (psi_n - psi) e e and w (psi_n^2 - psi^2) e e;
            // sum w e_x^2 = sum w e_y^2 = 1 and sum w e_x e_y = 0 over the ring
            const T d1 = w2 * ((p5 + p7) + (p6 + p8));
            const T d2 = w2 * ((q5 + q7) + (q6 + q8));
            const T q0 = p0 * p0;
            const T sxx1 = w1 * (p1 + p3) + d1 - p0, syy1 = w1 * (p2 + p4) + d1 - p0;
            const T sxy1 = w2 * ((p5 + p7) - (p6 + p8));
            const T sxx2 = w1 * (q1 + q3) + d2 - q0, syy2 = w1 * (q2 + q4) + d2 - q0;
            const T sxy2 = w2 * ((q5 + q7) - (q6 + q8));
            const T c = omA * p0;
            Qxx = kG2 * (c * sxx1 + hA * sxx2);
            Qyy = kG2 * (c * syy1 + hA * syy2);
            Qxy = kG2 * (c * sxy1 + hA * sxy2);
        }

        T out[9];
        collide(P, f, Fx, Fy, Qxx, Qyy, Qxy, out);
        if (!(out[0] == out[0])) bad = true;

        T* o = dst + static_cast<long long>(y + GY) * pitch + (x + Gm::GX);
#pragma unroll
        for (int a = 0; a < 9; ++a) o[a * plane] = out[a];

        // periodic images in the ghost cells read by the neighbouring tiles
        const bool xl = x < 2, xr = x >= nx - 2, yl = y < 2, yr = y >= ny - 2;
        if (xl || xr || yl || yr) {
            const int oxs[3] = {0, xl ? nx : 0, xr ? -nx : 0};
            const int oys[3] = {0, yl ? ny : 0, yr ? -ny : 0};
            const bool hx[3] = {true, xl, xr};
            const bool hy[3] = {true, yl, yr};
            for (int iy = 0; iy < 3; ++iy)
                for (int ix = 0; ix < 3; ++ix) {
                    if (!(hx[ix] && hy[iy]) || (ix == 0 && iy == 0)) continue;
                    T* g = o + static_cast<long long>(oys[iy]) * pitch + oxs[ix];
#pragma unroll
                    for (int a = 0; a < 9; ++a) g[a * plane] = out[a];
                }
        }
    }
    if (bad) atomicOr(I->status, ST_UNSTABLE);
}

// ---- tile configurations ------------------------------------------------
template <typename T, int BX, int BY, int NT> struct Cfg {
    using Gm = Geom<T, BX, BY, NT>;
    static TileCfg tc() { return TileCfg{BX, BY, NT}; }
    static size_t smem() { return Gm::smem; }
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(k_step<T, BX, BY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(Gm::smem));
    }
    static cudaError_t launch(const Inst* d, const int4* t, int n, int parity, unsigned long long to,
                              cudaStream_t st) {
        k_step<T, BX, BY, NT><<<n, NT, Gm::smem, st>>>(d, t, parity, to);
        return cudaGetLastError();
    }
};

struct Entry {
    TileCfg (*tc)();
    size_t (*smem)();
    cudaError_t (*prepare)();
    cudaError_t (*launch)(const Inst*, const int4*, int, int, unsigned long long, cudaStream_t);
};

#define LBM_CFG(T, BX, BY, NT) \
    Entry { &Cfg<T, BX, BY, NT>::tc, &Cfg<T, BX, BY, NT>::smem, &Cfg<T, BX, BY, NT>::prepare, &Cfg<T, BX, BY, NT>::launch }

const Entry kF32[] = {
    LBM_CFG(float, 64, 16, 256), LBM_CFG(float, 32, 16, 256), LBM_CFG(float, 64, 8, 256),
    LBM_CFG(float, 128, 8, 256), LBM_CFG(float, 128, 16, 512), LBM_CFG(float, 32, 32, 256),
};
const Entry kF64[] = {
    LBM_CFG(double, 32, 8, 256), LBM_CFG(double, 64, 8, 256), LBM_CFG(double, 32, 16, 256),
    LBM_CFG(double, 64, 4, 256),
};

const Entry* table(int prec, int* n) {
    if (prec == LBM_FP32) { *n = int(sizeof(kF32) / sizeof(kF32[0])); return kF32; }
    *n = int(sizeof(kF64) / sizeof(kF64[0]));
    return kF64;
}

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

cudaError_t step_launch(int prec, int k, const Inst* d_insts, const int4* d_tiles, int ntiles, int parity,
                        unsigned long long timeout_ns, cudaStream_t st) {
    int n;
    const Entry* e = table(prec, &n);
    return e[k].launch(d_insts, d_tiles, ntiles, parity, timeout_ns, st);
}

}  // namespace lbm
