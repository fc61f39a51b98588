/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle of the axisymmetric MRT lattice
 * Boltzmann model for thermal flow in porous media (Liu, He & Li, arXiv 1409.5929).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the yardstick the CUDA path is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may build, load or call it.  It shares no code, header, table or
 * helper with the CUDA library; neither side includes or links the other.
 *
 * It follows the paper's per-node sequence literally, in double precision and on
 * the r-weighted populations of Eq. 17 (f carries a factor r; nothing is rescaled):
 *   pull streaming (Eq. 22, Eq. 33)
 *   -> wall nodes: non-equilibrium extrapolation (Sec. 4, ref. [47])
 *   -> T (Eq. 38), G (Eq. 7), rho (Eq. 26), v (Eq. 29), l (Eq. 30), u (Eq. 28)
 *   -> F (Eq. 6), F~ and a_r (Eq. 25), S (Eq. 24)
 *   -> m = M f (Eq. 16, 18), m_eq (Eq. 19-20), m+ (Eq. 21), f+ = M^-1 m+ (Eq. 22)
 *   -> g+ (Eq. 33, 35-37).
 * Readings where the paper is silent (node placement, boundary details, start
 * state, Nusselt stencil, residual) are stated beside the code that takes them.
 *
 * Storage convention: the state between steps is the post-collision population
 * set f+, g+ at every node, population-major, z fastest:
 *   f[i*nr*nz + kr*nz + kz], i = 0..8;  g[i*nr*nz + kr*nz + kz], i = 0..4.
 * The macroscopic fields "of a state" are those a pull of that state yields.
 *
 * Parity status: every function here is pinned by the CPU tests (algebraic
 * identities of Eq. 18-24 and App. A, conservation, BGK limit, analytic
 * conduction and Brinkman solutions, Table 2), except the porous-annulus run at
 * epsilon = 0.6, Da = 1e-2, which no printed number pins beyond those invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- geometry -- */
enum { ORC_ANNULUS = 0, ORC_ANNULUS_PERIODIC_Z = 1, ORC_PIPE_PERIODIC_Z = 2, ORC_PIPE_INFLOW = 3 };
enum { ORC_FLUID = 0, ORC_WALL_IN = 1, ORC_WALL_OUT = 2, ORC_BOTTOM = 3, ORC_TOP = 4, ORC_AXIS = 5, ORC_INLET = 6,
       ORC_OUTLET = 7 };

typedef struct orc_params {
    int32_t nr, nz, geometry;
    int32_t collision;                   /* 0: MRT (Eq. 21, rates of Sec. 4); 1: BGK, every rate 1/tau (Sec. 3.1) */
    double radius_ratio;                 /* R* = r_o / r_i (annulus) */
    double Ra, Da, Pr, J, lambda;        /* Eq. 9 */
    double Ma;                           /* Mach number of Eq. 39 */
    double tau_nu;                       /* > 0: given; otherwise Eq. 39 */
    double F_eps;                        /* < 0: Ergun per node (Eq. 8); 0: no Forchheimer; > 0: constant */
    double eps_mean;                     /* mean porosity used to fix d_p from Da */
    double T_hot, T_cold;
    double body_accel_z;                 /* external acceleration a of Eq. 7, z component */
    double init_noise;                   /* amplitude of the uniform start-temperature noise */
    uint64_t seed;
    double u_in;                         /* inlet velocity U_in (pipe with inlet and outlet, Sec. 4.1) */
    double heater_len;                   /* > 0: isoflux discrete heater on the inner wall (Sec. 4.4), l / H */
    double heater_center;                /* its centre h / H */
} orc_params;

typedef struct orc_consts {
    double L, H, r0;                     /* r(kr) = r0 + kr */
    double tau, tauT, nu_e, nu, gbeta, T0, Ma;
    double Kbar;                         /* Da * L^2 */
    double s[9];                         /* diagonal of Lambda, Eq. 23 */
    int32_t cartesian;                   /* test hook: drop every axisymmetric term */
    int32_t pad0;
} orc_consts;

/* D2Q9 velocities of Eq. 14, c = 1, components (r, z). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EZ[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Eq. 32 weights. */
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* Image of each direction under r -> -r (specular axis reflection). */
static const int MIRROR9[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};
static const int MIRROR5[5] = {0, 3, 2, 1, 4};

static const double CS2 = 1.0 / 3.0;     /* c_s^2, D2Q9 */
static const double CS2T = 1.0 / 5.0;    /* c_sT^2, D2Q5, Sec. 3.2 */
static const double W0T = 3.0 / 5.0;     /* rest weight of Eq. 36 */

/* Eq. 18. */
static const double MMAT[9][9] = {
    { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  1, -1,  1, -1}};

static double MINV[9][9];
static int minv_ready = 0;

/* M^-1 = M^T diag(1 / (M M^T)_kk): the rows of Eq. 18 are mutually orthogonal. */
static void build_minv(void)
{
    if (minv_ready) return;
    for (int k = 0; k < 9; ++k) {
        double nk = 0;
        for (int i = 0; i < 9; ++i) nk += MMAT[k][i] * MMAT[k][i];
        for (int i = 0; i < 9; ++i) MINV[i][k] = MMAT[k][i] / nk;
    }
    minv_ready = 1;
}

void orc_matrices(double *M, double *Minv)
{
    build_minv();
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            M[a * 9 + b] = MMAT[a][b];
            Minv[a * 9 + b] = MINV[a][b];
        }
}

/* ------------------------------------------------------ parameters (Eq. 39) -- */
/*
 * L and r0.  Walls sit on nodes (non-equilibrium extrapolation needs them there):
 * annulus: L = nr - 1, H = nz - 1, r_i = L / (R* - 1), r(kr) = r_i + kr.
 * pipe: the axis lies half a cell below row 0, r(kr) = kr + 1/2, the wall node is
 * row nr - 1, and L is the pipe radius r(nr - 1) (Sec. 4.1 takes L = D / 2).
 */
int orc_derive(const orc_params *p, orc_consts *c)
{
    memset(c, 0, sizeof(*c));
    if (p->nr < 3 || p->nz < 3) return 1;
    if (p->geometry == ORC_PIPE_PERIODIC_Z || p->geometry == ORC_PIPE_INFLOW) {
        c->r0 = 0.5;
        c->L = (p->nr - 1) + 0.5;
    } else {
        if (!(p->radius_ratio > 1.0)) return 1;
        c->L = p->nr - 1;
        c->r0 = c->L / (p->radius_ratio - 1.0);
    }
    c->H = p->nz - 1;
    const double cs = sqrt(CS2);
    const double dT = p->T_hot - p->T_cold;
    if (p->tau_nu > 0) {
        c->tau = p->tau_nu;
        c->Ma = (p->Ra > 0) ? (c->tau - 0.5) * cs * sqrt(p->Ra) / (p->J * c->L * sqrt(p->Pr)) : 0.0;
    } else {
        if (!(p->Ra > 0)) return 1;
        c->Ma = p->Ma;
        c->tau = 0.5 + p->Ma * p->J * c->L * sqrt(p->Pr) / (cs * sqrt(p->Ra));   /* Eq. 39 */
    }
    if (!(c->tau > 0.5)) return 1;
    c->tauT = CS2 * p->lambda * (c->tau - 0.5) / (CS2T * p->J * p->Pr);         /* Eq. 39 */
    c->nu_e = CS2 * (c->tau - 0.5);                                               /* Eq. 31 */
    c->nu = c->nu_e / p->J;                                                       /* Eq. 9: J = nu_e / nu */
    /* U = Ma c_s (Ma = U / c_s) and U = sqrt(g beta dT L), Sec. 4. */
    if (p->Ra > 0) {
        if (dT == 0) return 1;
        const double U = c->Ma * cs;
        c->gbeta = U * U / (dT * c->L);
    } else {
        c->gbeta = 0.0;
    }
    /* Sec. 4.2; with the discrete heater T0 = T_o (Sec. 4.4) */
    c->T0 = p->heater_len > 0 ? p->T_cold : 0.5 * (p->T_hot + p->T_cold);
    c->Kbar = p->Da * c->L * c->L;                                                /* Eq. 9: Da = K / L^2 */
    /* Eq. 23 with the rates of Sec. 4; the BGK limit of Sec. 3.1 relaxes every moment
     * at 1/tau */
    const double s_nu = 1.0 / c->tau;
    const double s[9] = {1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, s_nu, s_nu};
    memcpy(c->s, s, sizeof(s));
    if (p->collision == 1)
        for (int k = 0; k < 9; ++k) c->s[k] = s_nu;
    return 0;
}

/*
 * Eq. 8 per node.  The particle diameter is fixed once from Da and the mean
 * porosity (K(eps_mean) = Da L^2); each node then takes K and F_phi from its own
 * porosity.  eps_mean = 1 means no solid matrix: K = Da L^2 everywhere.  A node
 * with phi = 1 inside a porous medium has infinite K (no drag).  Da <= 0 turns the
 * drag off.  Returns nu / K and F_phi / sqrt(K).
 */
void orc_porous(const orc_params *p, const orc_consts *c, double phi, double *lin, double *nl)
{
    double invK;
    if (!(p->Da > 0)) {
        invK = 0.0;
    } else if (p->eps_mean >= 1.0) {
        invK = 1.0 / c->Kbar;
    } else {
        const double em = p->eps_mean;
        const double dp2 = 150.0 * (1 - em) * (1 - em) * c->Kbar / (em * em * em);
        invK = (phi >= 1.0) ? 0.0 : 150.0 * (1 - phi) * (1 - phi) / (phi * phi * phi * dp2);
    }
    double Fphi;
    if (p->F_eps < 0) Fphi = 1.75 / sqrt(150.0 * phi * phi * phi);
    else Fphi = p->F_eps;
    *lin = c->nu * invK;
    *nl = Fphi * sqrt(invK);
}

/* ------------------------------------------- equilibria and source (Sec. 3.1) -- */
/* Eq. 32. */
void orc_feq(double r, double rho, double ur, double uz, double phi, double *feq)
{
    const double u2 = ur * ur + uz * uz;
    for (int i = 0; i < 9; ++i) {
        const double eu = EX[i] * ur + EZ[i] * uz;
        feq[i] = W9[i] * r * rho * (1 + eu / CS2 + eu * eu / (2 * phi * CS2 * CS2) - u2 / (2 * phi * CS2));
    }
}

/* Eq. 19-20. */
void orc_meq(double r, double rho, double ur, double uz, double phi, double *meq)
{
    const double u2 = ur * ur + uz * uz;
    meq[0] = r * rho;
    meq[1] = r * (-2 * rho + 3 * rho * u2 / phi);
    meq[2] = r * (rho - 3 * rho * u2 / phi);
    meq[3] = r * rho * ur;
    meq[4] = r * (-rho * ur);
    meq[5] = r * rho * uz;
    meq[6] = r * (-rho * uz);
    meq[7] = r * rho * (ur * ur - uz * uz) / phi;
    meq[8] = r * rho * ur * uz / phi;
}

/* Eq. 24. */
void orc_source(double r, double rho, double ur, double uz, double phi, double Ftr, double Ftz, double *S)
{
    const double uF = ur * Ftr + uz * Ftz;
    S[0] = 0;
    S[1] = r * rho * 6 * uF / phi;
    S[2] = r * rho * (-6 * uF / phi);
    S[3] = r * rho * Ftr;
    S[4] = r * rho * (-Ftr);
    S[5] = r * rho * Ftz;
    S[6] = r * rho * (-Ftz);
    S[7] = r * rho * 2 * (ur * Ftr - uz * Ftz) / phi;
    S[8] = r * rho * (ur * Ftz + uz * Ftr) / phi;
}

/* Eq. 35-36: D2Q5 equilibrium. */
static void geq5(double T, double ur, double uz, double *geq)
{
    const double wt[5] = {W0T, (1 - W0T) / 4, (1 - W0T) / 4, (1 - W0T) / 4, (1 - W0T) / 4};
    for (int i = 0; i < 5; ++i) geq[i] = wt[i] * T * (1 + (EX[i] * ur + EZ[i] * uz) / CS2T);
}

/* --------------------------------------------- macroscopic recovery (Sec. 3) -- */
/*
 * T (Eq. 38), rho (Eq. 26), G (Eq. 7), v (Eq. 29), l_j0 and l_1 (Eq. 30), u (Eq. 28).
 * Eq. 28 is used literally per component, with |v| = sqrt(v_r^2 + v_z^2); it is
 * exact only where l_r0 = l_z0.  The external acceleration a of Eq. 7 has only a
 * z component here (it is not the a_r of Eq. 25).
 */
void orc_macros(const orc_params *p, const orc_consts *c, double r, double phi, const double *f,
                const double *g, double *rho_o, double *ur_o, double *uz_o, double *T_o)
{
    double T = 0;
    for (int i = 0; i < 5; ++i) T += g[i];
    double sf = 0, jr = 0, jz = 0;
    for (int i = 0; i < 9; ++i) {
        sf += f[i];
        jr += EX[i] * f[i];
        jz += EZ[i] * f[i];
    }
    const double rho = sf / r;
    const double Gr = 0.0;
    const double Gz = c->gbeta * (T - c->T0) + p->body_accel_z;
    const double axi = c->cartesian ? 0.0 : 1.0;
    const double vr = (jr + 0.5 * r * phi * rho * Gr + axi * 0.5 * rho * CS2) / rho;
    const double vz = (jz + 0.5 * r * phi * rho * Gz) / rho;
    double lin, nl;
    orc_porous(p, c, phi, &lin, &nl);
    const double lr0 = 0.5 * ((r * r + axi * CS2 * (c->tau - 0.5)) / r + r * phi * 0.5 * lin);
    const double lz0 = 0.5 * (r + r * phi * 0.5 * lin);
    const double l1 = r * phi * 0.5 * nl;
    const double vmag = sqrt(vr * vr + vz * vz);
    *ur_o = vr / (lr0 + sqrt(lr0 * lr0 + l1 * vmag));
    *uz_o = vz / (lz0 + sqrt(lz0 * lz0 + l1 * vmag));
    *rho_o = rho;
    *T_o = T;
}

/* ------------------------------------------------------ collision (Eq. 21) -- */
/*
 * One node: forces (Eq. 6, 25), source (Eq. 24), MRT relaxation in moment space
 * (Eq. 21) and back-transform (Eq. 22), then the D2Q5 update (Eq. 33, 35, 37) with
 * the direction-dependent rate omega_g,i = (1 + e_ir tau_T / r) / (tau_T + 1/2).
 * rho, u and T are inputs so that wall nodes can impose u = 0 and T = T_b.
 */
void orc_collide(const orc_params *p, const orc_consts *c, double r, double phi, const double *f,
                 const double *g, double rho, double ur, double uz, double T, double *fo, double *go)
{
    build_minv();
    const double axi = c->cartesian ? 0.0 : 1.0;
    double lin, nl;
    orc_porous(p, c, phi, &lin, &nl);
    const double umag = sqrt(ur * ur + uz * uz);
    const double Gr = 0.0;
    const double Gz = c->gbeta * (T - c->T0) + p->body_accel_z;
    const double Fr = -phi * lin * ur - phi * nl * umag * ur + phi * Gr;             /* Eq. 6 */
    const double Fz = -phi * lin * uz - phi * nl * umag * uz + phi * Gz;
    const double ar = axi * CS2 * (1 - 2 * (c->tau - 0.5) * ur / r) / r;            /* after Eq. 25 */
    const double Ftr = Fr + ar, Ftz = Fz;                                            /* Eq. 25 */
    double S[9], meq[9], m[9], mp[9];
    orc_source(r, rho, ur, uz, phi, Ftr, Ftz, S);
    orc_meq(r, rho, ur, uz, phi, meq);
    for (int k = 0; k < 9; ++k) {                                                    /* Eq. 16 */
        m[k] = 0;
        for (int i = 0; i < 9; ++i) m[k] += MMAT[k][i] * f[i];
    }
    for (int k = 0; k < 9; ++k)                                                      /* Eq. 21 */
        mp[k] = m[k] - c->s[k] * (m[k] - meq[k]) + (1 - c->s[k] / 2) * S[k];
    for (int i = 0; i < 9; ++i) {                                                    /* Eq. 22 */
        fo[i] = 0;
        for (int k = 0; k < 9; ++k) fo[i] += MINV[i][k] * mp[k];
    }
    double geq[5];
    geq5(T, ur, uz, geq);
    for (int i = 0; i < 5; ++i) {                                                    /* Eq. 33, 37 */
        const double wg = (1 + axi * EX[i] * c->tauT / r) / (c->tauT + 0.5);
        const double psi = -axi * (ur / r) * geq[i];
        go[i] = g[i] - wg * (g[i] - geq[i]) + psi;
    }
}

/* -------------------------------------------------------- grid and classes -- */
static int periodic_z(const orc_params *p)
{
    return p->geometry == ORC_ANNULUS_PERIODIC_Z || p->geometry == ORC_PIPE_PERIODIC_Z;
}
static int is_pipe(const orc_params *p) { return p->geometry == ORC_PIPE_PERIODIC_Z || p->geometry == ORC_PIPE_INFLOW; }

/* Node classes (Fig. 1 and Fig. 3): walls on the outermost nodes; corners belong
 * to the side walls, so the Dirichlet temperature wins there.  Pipe with inlet and
 * outlet (Fig. 1): the wall is 0 < z < H, so the inlet row z = 0 and the outlet row
 * z = H own their corners. */
static int node_class(const orc_params *p, int kr, int kz)
{
    if (p->geometry == ORC_PIPE_INFLOW) {
        if (kz == 0) return ORC_INLET;
        if (kz == p->nz - 1) return ORC_OUTLET;
    }
    if (kr == p->nr - 1) return ORC_WALL_OUT;
    if (kr == 0) return is_pipe(p) ? ORC_AXIS : ORC_WALL_IN;
    if (!periodic_z(p)) {
        if (kz == 0) return ORC_BOTTOM;
        if (kz == p->nz - 1) return ORC_TOP;
    }
    return ORC_FLUID;
}

static int is_wall(int cls) { return (cls >= ORC_WALL_IN && cls <= ORC_TOP) || cls == ORC_INLET || cls == ORC_OUTLET; }

int orc_node_class(const orc_params *p, uint8_t *out)
{
    for (int kr = 0; kr < p->nr; ++kr)
        for (int kz = 0; kz < p->nz; ++kz) out[(size_t)kr * p->nz + kz] = (uint8_t)node_class(p, kr, kz);
    return 0;
}

/* Pull streaming (Eq. 22 and Eq. 33): f_i(x) = f_i+(x - e_i).  Periodic z wraps.
 * Below the axis (pipe) the ghost row kr = -1 is the mirror image of row 0 with
 * e_r reversed. */
static void pull(const orc_params *p, const double *fp, const double *gp, int kr, int kz,
                 double *f, double *g)
{
    const size_t N = (size_t)p->nr * p->nz;
    for (int i = 0; i < 9; ++i) {
        int sr = kr - EX[i], sz = kz - EZ[i], ii = i;
        if (periodic_z(p)) sz = (sz + p->nz) % p->nz;
        if (sr < 0) { sr = -sr - 1; ii = MIRROR9[i]; }
        f[i] = fp[ii * N + (size_t)sr * p->nz + sz];
    }
    for (int i = 0; i < 5; ++i) {
        int sr = kr - EX[i], sz = kz - EZ[i], ii = i;
        if (periodic_z(p)) sz = (sz + p->nz) % p->nz;
        if (sr < 0) { sr = -sr - 1; ii = MIRROR5[i]; }
        g[i] = gp[ii * N + (size_t)sr * p->nz + sz];
    }
}

/* The interior node a wall node extrapolates from: one step inward along the wall
 * normal; a corner uses the diagonal interior node. */
static void fluid_neighbour(const orc_params *p, int cls, int kr, int kz, int *fr, int *fz)
{
    *fr = kr;
    *fz = kz;
    if (cls == ORC_WALL_IN) *fr = 1;
    if (cls == ORC_WALL_OUT) *fr = p->nr - 2;
    if (cls == ORC_BOTTOM || cls == ORC_INLET) *fz = 1;
    if (cls == ORC_TOP || cls == ORC_OUTLET) *fz = p->nz - 2;
    if ((cls == ORC_INLET || cls == ORC_OUTLET) && kr == p->nr - 1) *fr = p->nr - 2;
    if ((cls == ORC_WALL_IN || cls == ORC_WALL_OUT) && !periodic_z(p)) {
        if (kz == 0) *fz = 1;
        if (kz == p->nz - 1) *fz = p->nz - 2;
    }
}

/*
 * Discrete heater (Sec. 4.4, Fig. 7): inner-wall node kz is heated when
 * |kz - h H| <= l H / 2 (H = nz - 1); the rest of the inner wall is insulated.
 */
static int in_heater(const orc_params *p, int kz)
{
    const double H = p->nz - 1;
    return fabs(kz - p->heater_center * H) <= 0.5 * p->heater_len * H;
}

/*
 * Non-equilibrium extrapolation (Sec. 4, ref. [47]) at a boundary node x_b:
 *   f(x_b) = f_eq(r_b, rho_b, u_b) + [f(x_f) - f_eq(r_f, rho_f, u_f)]
 *   g(x_b) = g_eq(T_b, u_b) + [g(x_f) - g_eq(T_f, u_f)]
 * with f(x_f), g(x_f) the post-streaming populations of the interior neighbour and
 * rho_f, u_f, T_f recovered from them.  Walls are no-slip (u_b = 0, rho_b = rho_f);
 * T_b is T_hot on the inner wall, T_cold on the outer wall and T_f on the adiabatic
 * top and bottom.  Pipe with inlet and outlet (Sec. 4.1): inlet u_b = (0, U_in),
 * rho_b = rho_f, T_b = T_hot (T_in); outlet zero gradient u_b = u_f, T_b = T_f, with
 * the density held at rho_0 = 1 there (the paper is silent on the outlet pressure).
 * The pipe wall is the outer wall, T_cold (T_w).  The non-equilibrium part is
 * copied unscaled, as in [47].
 */
static void rebuild(const orc_params *p, const orc_consts *c, const double *phi, const double *fp,
                    const double *gp, int cls, int kr, int kz, double *f, double *g, double *Tb, double *urb,
                    double *uzb)
{
    int fr, fz;
    fluid_neighbour(p, cls, kr, kz, &fr, &fz);
    double ff[9], gf[5];
    pull(p, fp, gp, fr, fz, ff, gf);
    const double rf = c->r0 + fr, rb = c->r0 + kr;
    const double phif = phi[(size_t)fr * p->nz + fz];
    const double phib = phi[(size_t)kr * p->nz + kz];
    double rho_f, ur_f, uz_f, T_f;
    orc_macros(p, c, rf, phif, ff, gf, &rho_f, &ur_f, &uz_f, &T_f);
    double rho_b = rho_f;
    *urb = 0;
    *uzb = 0;
    if (cls == ORC_INLET) {
        *uzb = p->u_in;
    } else if (cls == ORC_OUTLET) {
        *urb = ur_f;
        *uzb = uz_f;
        rho_b = 1.0;
    }
    double feq_b[9], feq_f[9], geq_b[5], geq_f[5];
    orc_feq(rb, rho_b, *urb, *uzb, phib, feq_b);
    orc_feq(rf, rho_f, ur_f, uz_f, phif, feq_f);
    for (int i = 0; i < 9; ++i) f[i] = feq_b[i] + (ff[i] - feq_f[i]);
    *Tb = (cls == ORC_WALL_IN || cls == ORC_INLET) ? p->T_hot : (cls == ORC_WALL_OUT) ? p->T_cold : T_f;
    if (cls == ORC_WALL_IN && p->heater_len > 0) {
        /* Sec. 4.4: q' = -k dT/dr on the heater (q' L / k = T_hot - T_cold), dT/dr = 0 on the
         * insulated rest.  The wall temperature solves the one-sided second-order
         * difference (-3 T_b + 4 T_1 - T_2) / 2 = -q'/k with T_1, T_2 the temperatures of
         * the next two nodes inward; the corners (diagonal neighbour) take T_f. */
        if (fz == kz) {
            double f2[9], g2[5];
            pull(p, fp, gp, 2, kz, f2, g2);
            double T2 = 0;
            for (int i = 0; i < 5; ++i) T2 += g2[i];
            const double G = in_heater(p, kz) ? (p->T_hot - p->T_cold) / c->L : 0.0;
            *Tb = (4 * T_f - T2 + 2 * G) / 3;
        } else {
            *Tb = T_f;
        }
    }
    geq5(*Tb, *urb, *uzb, geq_b);
    geq5(T_f, ur_f, uz_f, geq_f);
    for (int i = 0; i < 5; ++i) g[i] = geq_b[i] + (gf[i] - geq_f[i]);
}

/* Post-streaming populations and macroscopic fields of one node of a state. */
static void node_state(const orc_params *p, const orc_consts *c, const double *phi, const double *fp,
                       const double *gp, int kr, int kz, double *f, double *g, double *rho, double *ur,
                       double *uz, double *T)
{
    const int cls = node_class(p, kr, kz);
    const double r = c->r0 + kr;
    if (is_wall(cls)) {
        double Tb, urb, uzb;
        rebuild(p, c, phi, fp, gp, cls, kr, kz, f, g, &Tb, &urb, &uzb);
        double sf = 0;
        for (int i = 0; i < 9; ++i) sf += f[i];
        *rho = sf / r;                                                               /* Eq. 26 */
        *ur = urb;
        *uz = uzb;
        *T = Tb;
    } else {
        pull(p, fp, gp, kr, kz, f, g);
        orc_macros(p, c, r, phi[(size_t)kr * p->nz + kz], f, g, rho, ur, uz, T);
    }
}

/* ------------------------------------------------------------- time step -- */
static void step_once(const orc_params *p, const orc_consts *c, const double *phi, const double *fp,
                      const double *gp, double *fn, double *gn, int threads)
{
    const size_t N = (size_t)p->nr * p->nz;
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
    for (int kr = 0; kr < p->nr; ++kr) {
        for (int kz = 0; kz < p->nz; ++kz) {
            double f[9], g[5], fo[9], go[5], rho, ur, uz, T;
            node_state(p, c, phi, fp, gp, kr, kz, f, g, &rho, &ur, &uz, &T);
            const size_t n = (size_t)kr * p->nz + kz;
            orc_collide(p, c, c->r0 + kr, phi[n], f, g, rho, ur, uz, T, fo, go);
            for (int i = 0; i < 9; ++i) fn[i * N + n] = fo[i];
            for (int i = 0; i < 5; ++i) gn[i * N + n] = go[i];
        }
    }
}

/* Advance nsteps; f and g hold the state on entry and on return. */
int orc_run(const orc_params *p, const double *phi, double *f, double *g, int64_t nsteps, int threads)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    build_minv();
    const size_t N = (size_t)p->nr * p->nz;
    double *f2 = (double *)malloc(9 * N * sizeof(double));
    double *g2 = (double *)malloc(5 * N * sizeof(double));
    if (!f2 || !g2) { free(f2); free(g2); return 2; }
    for (int64_t s = 0; s < nsteps; ++s) {
        step_once(p, &c, phi, f, g, f2, g2, threads > 0 ? threads : 1);
        memcpy(f, f2, 9 * N * sizeof(double));
        memcpy(g, g2, 5 * N * sizeof(double));
    }
    free(f2);
    free(g2);
    return 0;
}

/* Fields of a state: rho, u_r, u_z, T at every node (walls: u = 0, T = T_b). */
int orc_moments(const orc_params *p, const double *phi, const double *f, const double *g, double *rho,
                double *ur, double *uz, double *T)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    build_minv();
    for (int kr = 0; kr < p->nr; ++kr)
        for (int kz = 0; kz < p->nz; ++kz) {
            double ff[9], gg[5];
            const size_t n = (size_t)kr * p->nz + kz;
            node_state(p, &c, phi, f, g, kr, kz, ff, gg, &rho[n], &ur[n], &uz[n], &T[n]);
        }
    return 0;
}

/* ----------------------------------------------------------- start state -- */
/* SplitMix64 (Steele, Lea & Flood 2014): output number n (0-based) of the stream
 * seeded with `seed` is mix(seed + (n + 1) * golden_gamma). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/*
 * Start state (the paper is silent).  Fields: rho = rho0 = 1 and either u = 0 with
 * T = T0 + noise * U(-1, 1) on non-wall nodes (cold start; draw number kr*nz + kz
 * of SplitMix64(seed), 53-bit uniform), or caller-given (u_r, u_z, T) (warm start).
 * Wall nodes take u = 0 and their wall temperature; top, bottom and the pipe outlet
 * take the start temperature of their interior neighbour; the pipe inlet takes
 * u = (0, U_in) and T_hot.  Pre-collision populations:
 *   f = M^-1 (m_eq - S / 2),   g = g_eq(T, u),
 * so that Eq. 29 returns the given u exactly when u = 0.  The stored state is those
 * populations after one collision at their own node (walls with u = 0, T = T_b).
 */
int orc_init(const orc_params *p, const double *phi, const double *ur_in, const double *uz_in,
             const double *T_in, double *f, double *g)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    build_minv();
    const size_t N = (size_t)p->nr * p->nz;
    double *Tst = (double *)malloc(N * sizeof(double));
    if (!Tst) return 2;
    for (int kr = 0; kr < p->nr; ++kr)
        for (int kz = 0; kz < p->nz; ++kz) {
            const size_t n = (size_t)kr * p->nz + kz;
            if (T_in) {
                Tst[n] = T_in[n];
            } else {
                const double u01 = (double)(orc_splitmix64(p->seed, n) >> 11) * (1.0 / 9007199254740992.0);
                Tst[n] = c.T0 + p->init_noise * (2 * u01 - 1);
            }
        }
    for (int kr = 0; kr < p->nr; ++kr)
        for (int kz = 0; kz < p->nz; ++kz) {
            const size_t n = (size_t)kr * p->nz + kz;
            const int cls = node_class(p, kr, kz);
            const double r = c.r0 + kr;
            double ur = 0, uz = 0, T = Tst[n];
            if (cls == ORC_WALL_IN && p->heater_len > 0) {
                int fr, fz;
                fluid_neighbour(p, cls, kr, kz, &fr, &fz);
                T = Tst[(size_t)fr * p->nz + fz];
            } else if (cls == ORC_WALL_IN) T = p->T_hot;
            else if (cls == ORC_WALL_OUT) T = p->T_cold;
            else if (cls == ORC_INLET) {
                T = p->T_hot;
                uz = p->u_in;
            } else if (cls == ORC_BOTTOM || cls == ORC_TOP || cls == ORC_OUTLET) {
                int fr, fz;
                fluid_neighbour(p, cls, kr, kz, &fr, &fz);
                T = Tst[(size_t)fr * p->nz + fz];
            } else if (ur_in && uz_in) {
                ur = ur_in[n];
                uz = uz_in[n];
            }
            /* forces at the start fields: Eq. 6, 7, 25 */
            double lin, nl;
            orc_porous(p, &c, phi[n], &lin, &nl);
            const double umag = sqrt(ur * ur + uz * uz);
            const double Gz = c.gbeta * (T - c.T0) + p->body_accel_z;
            const double Ftr = -phi[n] * lin * ur - phi[n] * nl * umag * ur
                               + CS2 * (1 - 2 * (c.tau - 0.5) * ur / r) / r;
            const double Ftz = -phi[n] * lin * uz - phi[n] * nl * umag * uz + phi[n] * Gz;
            double meq[9], S[9], fpre[9], gpre[5], fo[9], go[5];
            orc_meq(r, 1.0, ur, uz, phi[n], meq);
            orc_source(r, 1.0, ur, uz, phi[n], Ftr, Ftz, S);
            for (int i = 0; i < 9; ++i) {
                fpre[i] = 0;
                for (int k = 0; k < 9; ++k) fpre[i] += MINV[i][k] * (meq[k] - 0.5 * S[k]);
            }
            geq5(T, ur, uz, gpre);
            double rho, urr, uzz, TT;
            if (is_wall(cls)) {
                double sf = 0;
                for (int i = 0; i < 9; ++i) sf += fpre[i];
                rho = sf / r;
                urr = ur;
                uzz = uz;
                TT = T;
            } else {
                orc_macros(p, &c, r, phi[n], fpre, gpre, &rho, &urr, &uzz, &TT);
            }
            orc_collide(p, &c, r, phi[n], fpre, gpre, rho, urr, uzz, TT, fo, go);
            for (int i = 0; i < 9; ++i) f[i * N + n] = fo[i];
            for (int i = 0; i < 5; ++i) g[i * N + n] = go[i];
        }
    free(Tst);
    return 0;
}

/* ------------------------------------------------------------ diagnostics -- */
/*
 * Eq. 42: Nu_{i,o} = -(r_{i,o} / (H dT)) * integral_0^H (dT/dr)_{i,o} dz, with the
 * one-sided second-order wall derivative (-3 T_0 + 4 T_1 - T_2) / 2 (mirrored at
 * the outer wall) and the trapezoid rule over the nz wall nodes, H = nz - 1.
 */
int orc_nusselt(const orc_params *p, const double *T, double *nu_i, double *nu_o)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    const int nr = p->nr, nz = p->nz;
    const double ri = c.r0, ro = c.r0 + (nr - 1);
    double Ii = 0, Io = 0;
    for (int kz = 0; kz < nz; ++kz) {
        const double di = (-3 * T[kz] + 4 * T[(size_t)nz + kz] - T[(size_t)2 * nz + kz]) / 2;
        const double dO = (3 * T[(size_t)(nr - 1) * nz + kz] - 4 * T[(size_t)(nr - 2) * nz + kz]
                           + T[(size_t)(nr - 3) * nz + kz]) / 2;
        const double wz = (kz == 0 || kz == nz - 1) ? 0.5 : 1.0;
        Ii += wz * di;
        Io += wz * dO;
    }
    const double dT = p->T_hot - p->T_cold;
    *nu_i = -ri * Ii / (c.H * dT);
    *nu_o = -ro * Io / (c.H * dT);
    return 0;
}

/*
 * Convergence residual between two consecutive states' fields (the paper defines
 * none): max(|u^n - u^(n-1)|_2 / |u^n|_2, |T^n - T^(n-1)|_2 / |T^n|_2) over the
 * non-wall nodes.  Also returns the mass sum over all nodes of r * rho (= sum_i f_i).
 */
/*
 * Pipe with inlet and outlet (Sec. 4.1): local wall Nusselt number of Eq. 40,
 * Nu(z) = D (dT/dr)_w / (T_w - T_b), D = 2 r_i, at every column kz.  T_b is the
 * mixing-cup bulk temperature int_0^{r_i} u_z r T dr / int_0^{r_i} u_z r dr: Eq. 41
 * as printed omits u_z, but with that area mean the no-porous pipe gives Nu = 5.3
 * instead of the printed 3.674 (Table 1) and the classical 3.657, which the
 * mixing-cup mean reproduces.  Nodes sit at r = k + 1/2 with the wall node at r_i;
 * the integrals use the trapezoid rule on the points r = 0 (integrand 0), 1/2,
 * 3/2, ..., r_i.  (dT/dr)_w is the one-sided second-order difference
 * (3 T_w - 4 T_{w-1} + T_{w-2}) / 2.  Writes nu[0..nz-1].
 */
int orc_pipe_nusselt(const orc_params *p, const double *uz, const double *T, double *nu)
{
    orc_consts c;
    if (orc_derive(p, &c) || p->geometry != ORC_PIPE_INFLOW) return 1;
    const int nr = p->nr, nz = p->nz;
    const double ri = c.r0 + (nr - 1);
    for (int kz = 0; kz < nz; ++kz) {
        double num = 0.25 * (c.r0 * uz[kz] * T[kz]), den = 0.25 * (c.r0 * uz[kz]);   /* [0, 1/2] */
        for (int k = 0; k + 1 < nr; ++k) {
            const size_t a = (size_t)k * nz + kz, b = (size_t)(k + 1) * nz + kz;
            const double ra = c.r0 + k, rb = c.r0 + k + 1;
            num += 0.5 * (ra * uz[a] * T[a] + rb * uz[b] * T[b]);
            den += 0.5 * (ra * uz[a] + rb * uz[b]);
        }
        const double Tb = num / den;
        const double Tw = T[(size_t)(nr - 1) * nz + kz];
        const double dTdr = (3 * Tw - 4 * T[(size_t)(nr - 2) * nz + kz] + T[(size_t)(nr - 3) * nz + kz]) / 2;
        nu[kz] = 2 * ri * dTdr / (Tw - Tb);
    }
    return 0;
}

/*
 * Discrete heater (Sec. 4.4): local Nusselt number of Eq. 44 at the heated inner-wall
 * nodes, Nu(z) = q' L / (k (T_h - T_o)) = (T_hot - T_cold) / (T_h(z) - T_cold), and
 * its mean over the heater (Eq. 43; the heated nodes weigh equally).  nu_z[kz] is
 * NaN off the heater.  T: the fields of a state (T_h = the inner wall node's T).
 */
int orc_heater_nusselt(const orc_params *p, const double *T, double *nu_mean, double *nu_z)
{
    orc_consts c;
    if (orc_derive(p, &c) || !(p->heater_len > 0)) return 1;
    const double dT = p->T_hot - p->T_cold;
    double sum = 0;
    int n = 0;
    for (int kz = 0; kz < p->nz; ++kz) {
        const int heated = in_heater(p, kz) && node_class(p, 0, kz) == ORC_WALL_IN &&
                           (periodic_z(p) || (kz > 0 && kz < p->nz - 1));
        const double nu = heated ? dT / (T[kz] - p->T_cold) : NAN;
        if (nu_z) nu_z[kz] = nu;
        if (heated) {
            sum += nu;
            ++n;
        }
    }
    *nu_mean = n ? sum / n : NAN;
    return 0;
}

/*
 * Stokes stream function of the axisymmetric flow, behind the |psi|max columns of
 * Table 3 (the paper names psi without defining it; this is the textbook form for
 * Eq. 1):  r u_z = d psi / dr and r u_r = - d psi / dz, i.e.
 *     psi(r, z) = integral from r_s to r of r' u_z(r', z) dr',
 * with r_s the inner wall (annulus: no slip there, psi = 0 on it) or the axis (pipes:
 * psi = 0 on the axis; the first panel runs from r = 0, where the integrand is 0, to
 * the first row at r = 1/2).  The integral is the trapezoid rule over the rows.
 * Writes psi[nr*nz] (may be NULL) and the largest |psi| into *psi_max (lattice units).
 */
int orc_stream_function(const orc_params *p, const double *uz, double *psi, double *psi_max)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    const int nr = p->nr, nz = p->nz;
    double big = 0;
    for (int kz = 0; kz < nz; ++kz) {
        double acc = 0;
        if (is_pipe(p)) acc = 0.5 * c.r0 * (0.0 + c.r0 * uz[kz]);       /* panel [0, r0] */
        for (int kr = 0; kr < nr; ++kr) {
            if (kr > 0) {
                const double r_lo = c.r0 + (kr - 1), r_hi = c.r0 + kr;
                acc += 0.5 * (r_lo * uz[(size_t)(kr - 1) * nz + kz] + r_hi * uz[(size_t)kr * nz + kz]);
            }
            if (psi) psi[(size_t)kr * nz + kz] = acc;
            if (fabs(acc) > big) big = fabs(acc);
        }
    }
    if (psi_max) *psi_max = big;
    return 0;
}

int orc_residual(const orc_params *p, const double *rho_n, const double *ur_n, const double *uz_n,
                 const double *T_n, const double *ur_p, const double *uz_p, const double *T_p,
                 double *res, double *mass)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    double du = 0, u2 = 0, dt = 0, t2 = 0, m = 0;
    for (int kr = 0; kr < p->nr; ++kr)
        for (int kz = 0; kz < p->nz; ++kz) {
            const size_t n = (size_t)kr * p->nz + kz;
            m += (c.r0 + kr) * rho_n[n];
            if (is_wall(node_class(p, kr, kz))) continue;
            const double a = ur_n[n] - ur_p[n], b = uz_n[n] - uz_p[n], d = T_n[n] - T_p[n];
            du += a * a + b * b;
            u2 += ur_n[n] * ur_n[n] + uz_n[n] * uz_n[n];
            dt += d * d;
            t2 += T_n[n] * T_n[n];
        }
    const double ru = u2 > 0 ? sqrt(du / u2) : (du > 0 ? INFINITY : 0.0);
    const double rt = t2 > 0 ? sqrt(dt / t2) : (dt > 0 ? INFINITY : 0.0);
    *res = ru > rt ? ru : rt;
    *mass = m;
    return 0;
}

/* ------------------------------------------------------------- test hooks -- */
/*
 * One collision at one node with optional overrides, for the algebraic tests:
 * s_override (9 rates or NULL), cartesian = 1 drops every axisymmetric term
 * (c_s^2 terms of Eq. 27-30, a_r of Eq. 25, the e_ir/r part of omega_g, psi).
 * wall = 0: rho, u, T recovered (Eq. 26-30, 38); wall = 1: rho from Eq. 26,
 * u = 0, T = T_wall.  macro_out = (rho, u_r, u_z, T) used.
 */
int orc_collide_node(const orc_params *p, const double *s_override, int cartesian, double r, double phi,
                     const double *f, const double *g, int wall, double T_wall, double *fo, double *go,
                     double *macro_out)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    if (s_override) memcpy(c.s, s_override, sizeof(c.s));
    c.cartesian = cartesian;
    double rho, ur, uz, T;
    if (wall) {
        double sf = 0;
        for (int i = 0; i < 9; ++i) sf += f[i];
        rho = sf / r;
        ur = 0;
        uz = 0;
        T = T_wall;
    } else {
        orc_macros(p, &c, r, phi, f, g, &rho, &ur, &uz, &T);
    }
    orc_collide(p, &c, r, phi, f, g, rho, ur, uz, T, fo, go);
    macro_out[0] = rho;
    macro_out[1] = ur;
    macro_out[2] = uz;
    macro_out[3] = T;
    return 0;
}

/* Full update of one node (kr, kz) of a state: post-streaming populations and
 * fields (node_state) and the collision, without touching any other node.  Only
 * rows kr - 2 .. kr + 2 of f, g and phi are read. */
int orc_node_update(const orc_params *p, const double *phi, const double *f, const double *g, int kr, int kz,
                    double *fo, double *go, double *macro_out)
{
    orc_consts c;
    if (orc_derive(p, &c)) return 1;
    build_minv();
    double ff[9], gg[5], rho, ur, uz, T;
    node_state(p, &c, phi, f, g, kr, kz, ff, gg, &rho, &ur, &uz, &T);
    orc_collide(p, &c, c.r0 + kr, phi[(size_t)kr * p->nz + kz], ff, gg, rho, ur, uz, T, fo, go);
    macro_out[0] = rho;
    macro_out[1] = ur;
    macro_out[2] = uz;
    macro_out[3] = T;
    return 0;
}

int orc_derive_export(const orc_params *p, double *out)
{
    orc_consts c;
    const int rc = orc_derive(p, &c);
    out[0] = c.L; out[1] = c.H; out[2] = c.r0; out[3] = c.tau; out[4] = c.tauT; out[5] = c.nu_e;
    out[6] = c.nu; out[7] = c.gbeta; out[8] = c.T0; out[9] = c.Ma; out[10] = c.Kbar;
    return rc;
}
