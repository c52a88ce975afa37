/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the per-timestep update of
 * Kupershtokh et al.'s hybrid pseudo-potential model in the D2Q9 MRT form,
 * with the kappa-scaled pressure-tensor modification of
 *   A. Hu, L. Li, R. Uddin, "Surface tension adjustment in a pseudo-potential
 *   lattice Boltzmann model", arXiv:1412.7228 (Sections 2 and 3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path, and it never calls
 * into it.
 *
 * Everything is FP64 with plain loops over the nine velocities, in the order
 * the paper states the method: density and pseudo-potential (Eq. 10), the
 * hybrid force (Eq. 9), the modifying tensor (Eq. 23), the moment-space
 * collision with forcing and source (Eqs. 2-6, 25, 26), back-transform and
 * streaming (Eq. 1).  It is compiled with -ffp-contract=off so that no fused
 * multiply-add changes the rounding between machines.
 *
 * Storage: f[a*ny*nx + y*nx + x] holds the pre-collision population f_a(x,t)
 * of node (x, y); x is the fastest index.
 *
 * Threads: the per-node loops carry OpenMP work-sharing pragmas.  Built
 * without -fopenmp (liboracle.so) they are ignored; built with it
 * (liboracle_omp.so) the nodes of a loop are shared among threads.  Every
 * node's arithmetic is the same either way and no loop accumulates across
 * nodes, so both builds give the same bits.
 *
 * Readings of the paper taken here (each is pinned by a CPU test):
 *  R1  The paper does not print M.  Its moment order (rho, e, eps, j_x, q_x,
 *      j_y, q_y, p_xx, p_xy) in Eq. 4 is that of Lallemand & Luo, whose rows
 *      are typed below with the velocity order e_0..e_8.  M^-1 is derived from
 *      M (its rows are orthogonal), not typed.
 *  R2  The velocity v in Eq. 4 and Eq. 6 is rho*v = sum_a f_a e_a + F/2.
 *  R3  Eq. 23 carries no G although its expansion Eq. 24 carries G/12, G/6;
 *      Q is therefore kappa*(G/2)*[...], which expands exactly to Eq. 24.
 *  R4  The eighth entry of C (Eq. 26) is -s_nu (Q_xx - Q_yy), the coefficient
 *      that gives the (1 - kappa) of Eq. 28.
 *  R5  The third entry of C is 0 (the paper's choice); Li et al.'s
 *      -1.5 s_eps (Q_xx + Q_yy) is available through li_eps.
 *  R6  The ninth entry of S (Eq. 6) is v_x F_y + v_y F_x.
 *  R7  c = 1 in Eq. 10, so psi = sqrt(2 (p_EOS - rho/3) / G).
 *  R8  K multiplies the whole equation of state (Eq. 21).
 *  R11 With G = 0 the interaction force and Q vanish and psi is not
 *      evaluated.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q9 9

/* orc_params must match oracle/__init__.py (ctypes mirror). */
typedef struct {
    int eos;          /* 1 Carnahan-Starling, 2 van der Waals (Eq. 21), 3 Peng-Robinson (Eq. 29) */
    double a, b, R, K, T, omega;   /* EOS constants; omega: PR acentric factor */
    double Tc;        /* PR only: critical temperature in alpha(T) */
    double A;         /* hybrid-force weight of Eq. 9 */
    double kappa;     /* surface-tension parameter of Eq. 23 */
    double G;         /* interaction strength; only its sign matters */
    double s[Q9];     /* diagonal of Lambda, Eq. 2, in moment order */
    int li_eps;       /* 1: third entry of C = -1.5 s_eps (Qxx+Qyy) (Li et al.) */
    int no_q;         /* 1: Q and C are not evaluated at all (unmodified model) */
    double fext_x, fext_y;  /* test-only constant body-force density */
    int walls_y;      /* test-only: half-way bounce-back walls at y=-1/2 and y=ny-1/2 */
    /* Density-dependent shear viscosity (Section 4.2): when var_visc is set,
     * nu(rho) is linear between (rho_g, nu_g) and (rho_l, nu_l), clamped to
     * that range, and s_7 = s_8 = 1/(3 nu + 1/2). */
    int var_visc;
    double nu_g, nu_l, visc_rho_g, visc_rho_l;
} orc_params;

/* D2Q9 velocities e_0..e_8: rest, four axis neighbours, four diagonals. */
static const int EX[Q9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Interaction weights w(|e|^2) of Eq. 7: w(1) = 1/3, w(2) = 1/12 (w(0) unused). */
static double w_int(int a) {
    int e2 = EX[a] * EX[a] + EY[a] * EY[a];
    if (e2 == 1) return 1.0 / 3.0;
    if (e2 == 2) return 1.0 / 12.0;
    return 0.0;
}

/* Lallemand-Luo rows, moment order of Eq. 4 (reading R1). */
static const double MROW[Q9][Q9] = {
    /* rho  */ { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    /* e    */ {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    /* eps  */ { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    /* j_x  */ { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    /* q_x  */ { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    /* j_y  */ { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    /* q_y  */ { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    /* p_xx */ { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    /* p_xy */ { 0,  0,  0,  0,  0,  1, -1,  1, -1},
};

/* M^-1 = M^T (M M^T)^-1; M M^T is diagonal because the rows are orthogonal. */
static void minv_build(double Minv[Q9][Q9]) {
    for (int k = 0; k < Q9; ++k) {
        double n2 = 0.0;
        for (int a = 0; a < Q9; ++a) n2 += MROW[k][a] * MROW[k][a];
        for (int a = 0; a < Q9; ++a) Minv[a][k] = MROW[k][a] / n2;
    }
}

void orc_matrices(double *M, double *Minv) {
    double Mi[Q9][Q9];
    minv_build(Mi);
    for (int i = 0; i < Q9; ++i)
        for (int j = 0; j < Q9; ++j) {
            M[i * Q9 + j] = MROW[i][j];
            Minv[i * Q9 + j] = Mi[i][j];
        }
}

void orc_velocities(int *ex, int *ey, double *w) {
    for (int a = 0; a < Q9; ++a) { ex[a] = EX[a]; ey[a] = EY[a]; w[a] = w_int(a); }
}

/* Equations of state.  Carnahan-Starling in its usual attractive form,
 * van der Waals Eq. 21, Peng-Robinson Eq. 29; K scales the whole law (R8). */
double orc_pressure(const orc_params *p, double rho) {
    double RT = p->R * p->T;
    if (p->eos == 1) {
        double eta = p->b * rho / 4.0;
        double num = 1.0 + eta + eta * eta - eta * eta * eta;
        double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
        return p->K * (rho * RT * num / den - p->a * rho * rho);
    }
    if (p->eos == 2) {
        return p->K * (rho * RT / (1.0 - p->b * rho) - p->a * rho * rho);
    }
    if (p->eos == 3) {
        double m = 0.37464 + 1.54226 * p->omega - 0.26992 * p->omega * p->omega;
        double sq = 1.0 + m * (1.0 - sqrt(p->T / p->Tc));
        double alpha = sq * sq;
        double bb = p->b * rho;
        return p->K * (rho * RT / (1.0 - bb) -
                       p->a * alpha * rho * rho / (1.0 + 2.0 * bb - bb * bb));
    }
    return NAN;
}

void orc_pressure_array(const orc_params *p, const double *rho, double *out, long n) {
    for (long i = 0; i < n; ++i) out[i] = orc_pressure(p, rho[i]);
}

/* Eq. 10 with c = 1 (R7): p_EOS = rho/3 + G psi^2 / 2.  Returns 0 when the
 * radicand is negative or not a number. */
static int psi_of_rho(const orc_params *p, double rho, double *psi) {
    double r = 2.0 * (orc_pressure(p, rho) - rho / 3.0) / p->G;
    if (!(r >= 0.0)) { *psi = NAN; return 0; }
    *psi = sqrt(r);
    return 1;
}

/* Eq. 4: equilibrium moments. */
void orc_meq(double rho, double vx, double vy, double *meq) {
    double v2 = vx * vx + vy * vy;
    meq[0] = rho;
    meq[1] = rho * (-2.0 + 3.0 * v2);
    meq[2] = rho * (1.0 - 3.0 * v2);
    meq[3] = rho * vx;
    meq[4] = -rho * vx;
    meq[5] = rho * vy;
    meq[6] = -rho * vy;
    meq[7] = rho * (vx * vx - vy * vy);
    meq[8] = rho * vx * vy;
}

/* Eq. 6 with the ninth entry read as v_x F_y + v_y F_x (R6). */
void orc_source_s(double vx, double vy, double Fx, double Fy, double *S) {
    double vF = vx * Fx + vy * Fy;
    S[0] = 0.0;
    S[1] = 6.0 * vF;
    S[2] = -6.0 * vF;
    S[3] = Fx;
    S[4] = -Fx;
    S[5] = Fy;
    S[6] = -Fy;
    S[7] = 2.0 * (vx * Fx - vy * Fy);
    S[8] = vx * Fy + vy * Fx;
}

/* Eq. 26 (readings R4, R5): the source that modifies the pressure tensor. */
void orc_source_c(const orc_params *p, double Qxx, double Qyy, double Qxy, double *C) {
    for (int k = 0; k < Q9; ++k) C[k] = 0.0;
    C[1] = 1.5 * p->s[1] * (Qxx + Qyy);
    if (p->li_eps) C[2] = -1.5 * p->s[2] * (Qxx + Qyy);
    C[7] = -p->s[7] * (Qxx - Qyy);
    C[8] = -p->s[8] * Qxy;
}

/* Eq. 9 (hybrid force, with U = G psi^2 / 2) and Eq. 23 (modifying tensor,
 * scaled by G/2 per R3) from a given psi field, periodic in x and y. */
void orc_force_q(const orc_params *p, int nx, int ny, const double *psi,
                 double *Fx, double *Fy, double *Qxx, double *Qyy, double *Qxy) {
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long i = (long)y * nx + x;
            double ps = psi[i];
            double fx = 0.0, fy = 0.0;
            double qxx = 0.0, qyy = 0.0, qxy = 0.0;
            for (int a = 1; a < Q9; ++a) {
                int xn = (x + EX[a] + nx) % nx;
                int yn = (y + EY[a] + ny) % ny;
                double pn = psi[(long)yn * nx + xn];
                double U = p->G * pn * pn / 2.0;
                double w = w_int(a);
                /* -A sum w U(x+e) e - (1-A) G psi(x) sum w psi(x+e) e */
                fx += -p->A * w * U * EX[a] - (1.0 - p->A) * p->G * ps * w * pn * EX[a];
                fy += -p->A * w * U * EY[a] - (1.0 - p->A) * p->G * ps * w * pn * EY[a];
                /* (1-A) psi(x) w (psi(x+e) - psi(x)) e e + (A/2) w (psi^2(x+e) - psi^2(x)) e e */
                double t = (1.0 - p->A) * ps * w * (pn - ps) + 0.5 * p->A * w * (pn * pn - ps * ps);
                qxx += t * EX[a] * EX[a];
                qyy += t * EY[a] * EY[a];
                qxy += t * EX[a] * EY[a];
            }
            Fx[i] = fx;
            Fy[i] = fy;
            double g2 = p->kappa * p->G / 2.0;
            Qxx[i] = g2 * qxx;
            Qyy[i] = g2 * qyy;
            Qxy[i] = g2 * qxy;
        }
}

/* Eq. 25 at one node: m* = m - Lambda (m - m_eq) + (I - Lambda/2) S + C,
 * then f* = M^-1 m*.  Velocity by R2. */
/* Relaxation rate of the shear moments (p_xx, p_xy) at density rho. */
static double shear_rate(const orc_params *p, double rho) {
    if (!p->var_visc) return p->s[7];
    double w = (rho - p->visc_rho_g) / (p->visc_rho_l - p->visc_rho_g);
    if (w < 0.0) w = 0.0;
    if (w > 1.0) w = 1.0;
    double nu = p->nu_g + w * (p->nu_l - p->nu_g);
    return 1.0 / (3.0 * nu + 0.5);
}

static void collide(const orc_params *p, double Minv[Q9][Q9], const double *f, double Fx,
                    double Fy, double Qxx, double Qyy, double Qxy, double *fout) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q9; ++a) {
        rho += f[a];
        jx += f[a] * EX[a];
        jy += f[a] * EY[a];
    }
    double vx = (jx + Fx / 2.0) / rho;
    double vy = (jy + Fy / 2.0) / rho;
    double m[Q9], meq[Q9], S[Q9], C[Q9], ms[Q9];
    for (int k = 0; k < Q9; ++k) {
        m[k] = 0.0;
        for (int a = 0; a < Q9; ++a) m[k] += MROW[k][a] * f[a];
    }
    orc_meq(rho, vx, vy, meq);
    orc_source_s(vx, vy, Fx, Fy, S);
    /* the rates of this node: the shear pair may depend on density */
    orc_params pl = *p;
    pl.s[7] = pl.s[8] = shear_rate(p, rho);
    if (p->no_q) {
        for (int k = 0; k < Q9; ++k) C[k] = 0.0;
    } else {
        orc_source_c(&pl, Qxx, Qyy, Qxy, C);
    }
    for (int k = 0; k < Q9; ++k) {
        ms[k] = m[k] - pl.s[k] * (m[k] - meq[k]) + (1.0 - pl.s[k] / 2.0) * S[k];
        if (!p->no_q) ms[k] = ms[k] + C[k];
    }
    for (int a = 0; a < Q9; ++a) {
        fout[a] = 0.0;
        for (int k = 0; k < Q9; ++k) fout[a] += Minv[a][k] * ms[k];
    }
}

void orc_collide_node(const orc_params *p, const double *f, double Fx, double Fy,
                      double Qxx, double Qyy, double Qxy, double *fout) {
    double Minv[Q9][Q9];
    minv_build(Minv);
    collide(p, Minv, f, Fx, Fy, Qxx, Qyy, Qxy, fout);
}

/* f = M^-1 m_eq(rho, u): the initial state used by every experiment. */
void orc_init_equilibrium(int nx, int ny, const double *rho, const double *ux,
                          const double *uy, double *f) {
    double Minv[Q9][Q9];
    minv_build(Minv);
    long N = (long)nx * ny;
    for (long i = 0; i < N; ++i) {
        double meq[Q9];
        orc_meq(rho[i], ux ? ux[i] : 0.0, uy ? uy[i] : 0.0, meq);
        for (int a = 0; a < Q9; ++a) {
            double v = 0.0;
            for (int k = 0; k < Q9; ++k) v += Minv[a][k] * meq[k];
            f[a * N + i] = v;
        }
    }
}

/* Density and psi of every node (Eq. 10).  Returns 0 on a bad radicand. */
static int rho_psi(const orc_params *p, int nx, int ny, const double *f, double *rho, double *psi) {
    long N = (long)nx * ny;
    int ok = 1;
#pragma omp parallel for reduction(&:ok)
    for (long i = 0; i < N; ++i) {
        double r = 0.0;
        for (int a = 0; a < Q9; ++a) r += f[a * N + i];
        rho[i] = r;
        if (p->G == 0.0) {
            psi[i] = 0.0;
        } else if (!psi_of_rho(p, r, &psi[i])) {
            ok = 0;
        }
        if (!(r == r)) ok = 0;
    }
    return ok;
}

/* Interaction force and Q of every node; with G = 0 both vanish (R11). */
static void forces(const orc_params *p, int nx, int ny, const double *psi, double *Fx,
                   double *Fy, double *Qxx, double *Qyy, double *Qxy) {
    long N = (long)nx * ny;
    if (p->G == 0.0) {
        for (long i = 0; i < N; ++i) Fx[i] = Fy[i] = Qxx[i] = Qyy[i] = Qxy[i] = 0.0;
    } else {
        orc_force_q(p, nx, ny, psi, Fx, Fy, Qxx, Qyy, Qxy);
    }
    for (long i = 0; i < N; ++i) {
        Fx[i] += p->fext_x;
        Fy[i] += p->fext_y;
    }
}

/* Macroscopic fields of the current state: rho, v (R2), psi, F. */
int orc_macro(const orc_params *p, int nx, int ny, const double *f, double *rho,
              double *ux, double *uy, double *psi, double *Fx, double *Fy) {
    long N = (long)nx * ny;
    double *Qs = (double *)malloc(sizeof(double) * 3 * N);
    if (!Qs) return -2;
    int ok = rho_psi(p, nx, ny, f, rho, psi);
    forces(p, nx, ny, psi, Fx, Fy, Qs, Qs + N, Qs + 2 * N);
    for (long i = 0; i < N; ++i) {
        double jx = 0.0, jy = 0.0;
        for (int a = 0; a < Q9; ++a) {
            jx += f[a * N + i] * EX[a];
            jy += f[a * N + i] * EY[a];
        }
        ux[i] = (jx + Fx[i] / 2.0) / rho[i];
        uy[i] = (jy + Fy[i] / 2.0) / rho[i];
    }
    free(Qs);
    return ok ? 0 : 1;
}

/* Index of the opposite velocity (for the test-only bounce-back walls). */
static int opposite(int a) {
    for (int b = 0; b < Q9; ++b)
        if (EX[b] == -EX[a] && EY[b] == -EY[a]) return b;
    return -1;
}

/* nsteps full time steps of Eq. 1 / Eq. 25 on f (in place).  Returns 0 on
 * success, 1 if a density left the EOS's psi domain or became NaN (the step
 * that found it is not applied), -1 on bad arguments, -2 on allocation. */
int orc_step(const orc_params *p, int nx, int ny, double *f, int nsteps) {
    if (nx < 1 || ny < 1 || nsteps < 0) return -1;
    if (p->walls_y && p->G != 0.0) return -1;
    long N = (long)nx * ny;
    double *work = (double *)malloc(sizeof(double) * (size_t)N * (9 + 7));
    if (!work) return -2;
    double *fpost = work;
    double *rho = work + 9 * N, *psi = rho + N, *Fx = psi + N, *Fy = Fx + N;
    double *Qxx = Fy + N, *Qyy = Qxx + N, *Qxy = Qyy + N;
    double Minv[Q9][Q9];
    minv_build(Minv);
    int rc = 0;
    for (int t = 0; t < nsteps; ++t) {
        if (!rho_psi(p, nx, ny, f, rho, psi)) { rc = 1; break; }
        forces(p, nx, ny, psi, Fx, Fy, Qxx, Qyy, Qxy);
#pragma omp parallel for
        for (long i = 0; i < N; ++i) {
            double fn[Q9], fo[Q9];
            for (int a = 0; a < Q9; ++a) fn[a] = f[a * N + i];
            collide(p, Minv, fn, Fx[i], Fy[i], Qxx[i], Qyy[i], Qxy[i], fo);
            for (int a = 0; a < Q9; ++a) fpost[a * N + i] = fo[a];
        }
        /* streaming: f_a(x + e_a, t+1) = f*_a(x, t), periodic in x and y
         * (or half-way bounce-back at the two y walls in the test-only mode);
         * every target is written by exactly one source */
#pragma omp parallel for
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int a = 0; a < Q9; ++a) {
                    double v = fpost[a * N + (long)y * nx + x];
                    int yt = y + EY[a];
                    int xt = (x + EX[a] + nx) % nx;
                    if (p->walls_y && (yt < 0 || yt >= ny)) {
                        f[opposite(a) * N + (long)y * nx + x] = v;
                    } else {
                        yt = (yt + ny) % ny;
                        f[a * N + (long)yt * nx + xt] = v;
                    }
                }
    }
    free(work);
    return rc;
}

/* Threads of the OpenMP build (n > 0 sets them); 1 without OpenMP. */
int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
