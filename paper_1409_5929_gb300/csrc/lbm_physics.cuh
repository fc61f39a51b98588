// lbm_physics.cuh -- per-node arithmetic of the axisymmetric MRT-LB step
// (Liu, He & Li, arXiv 1409.5929, Sec. 3.1-3.2 and Sec. 4), device side.
//
// Variables.  The populations of Eq. 17 carry a factor r.  Between steps they are
// stored as deviations from the exact post-collision rest state (rho = 1, u = 0):
//     ft_i = f+_i - (r w_i + c_i),   c_i = e_ir w_i / 2,
//     gh_i = g+_i - wT_i (T0 + R(x)),
// where r w_i + c_i = M^-1 (m_eq + S/2) at rest (S_3 = rho c_s^2 from a_r of Eq. 25)
// and R(x) is a per-node reference temperature offset held in FP16 (a separate plane,
// refreshed from the current temperature by the rebase kernel).  The reference keeps
// the stored gh at the size of the temperature change since the last refresh instead
// of |T - T0|, so FP32 rounding no longer freezes slow thermal modes before they settle.
// Streaming maps the flow rest state onto the pre-collision rest state r w_i - c_i
// (because r - e_ir + e_ir/2 = r - e_ir/2), so the pulled pre-collision deviation
//     fv_i(x) = f_i(x) - (r w_i - c_i) = ft_i(x - e_i)
// is a plain copy (Eq. 22), also through the specular image of the axis row; the
// pulled thermal deviation is gh_i(x - e_i) + wT_i (R(x - e_i) - R(x)).  The
// moments of the deviations are mv = M fv = m - r (1, -2, 1, 0, ...) + (0, 0, 0, c_s^2/2,
// -c_s^2/2, 0, ...).  Eq. 21 applied to mv, with the constant c_s^2 of S_3 (and -c_s^2
// of S_4) removed from the source, gives exactly M ft+: the rest constants cancel.  All
// handled values are small, so FP32 (and FP16/BF16 storage) keep their precision.
// M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

enum { ANNULUS = 0, ANNULUS_PERIODIC_Z = 1, PIPE_PERIODIC_Z = 2, PIPE_INFLOW = 3 };
enum { FLUID = 0, WALL_IN = 1, WALL_OUT = 2, BOTTOM = 3, TOP = 4, AXIS = 5, INLET = 6, OUTLET = 7 };

// Lattice constants, in the arithmetic type R of the kernel that uses them.
template <typename R>
struct Consts {
    int nr, nz, geometry;
    int porous_mode;   // 0: no drag; 1: K = Da L^2 everywhere; 2: K(phi) from Eq. 8
    int ergun;         // 1: F_phi from Eq. 8 per node; 0: constant F_eps
    int periodic;      // 1: periodic in z (ANNULUS_PERIODIC_Z, PIPE_PERIODIC_Z)
    int heater;        // 1: isoflux discrete heater on the inner wall (Sec. 4.4)
    int hz0, hz1;      // heated inner-wall columns hz0 .. hz1
    R r0;              // r(kr = 0)
    R cs2tau;          // c_s^2 (tau - 1/2)
    R two_taum;        // 2 (tau - 1/2)
    R s_e, s_eps, s_j, s_q, s_nu;   // Eq. 23 with the rates of Sec. 4
    R h_e, h_eps, h_j, h_q, h_nu;   // 1 - s / 2 of each (the source weights of Eq. 21)
    R cs2_2tm;                      // c_s^2 2 (tau - 1/2)
    R tauT, wg_den;    // tau_T and 1 / (tau_T + 1/2)
    R gbeta, T0, az;   // buoyancy, reference temperature, external acceleration (z)
    R lin_coef;        // nu / K = lin_coef (mode 1) or lin_coef (1 - phi)^2 / phi^3 (mode 2)
    R nl_coef;         // F_phi / sqrt(K), see porous()
    R T_hot, T_cold;
    R u_in;               // inlet velocity (PIPE_INFLOW)
    R hG;                 // heater gradient q' / k = (T_hot - T_cold) / L
    const __half* tref;   // per-node reference offset R(x) (FP16, one plane)
    const uint2* fref;    // per-node references of 16-bit storage (A, J_r, J_z, R in FP16, see fref_delta)
};

template <typename R> __host__ __device__ constexpr R cs2() { return R(1) / R(3); }

__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }

// Reciprocals.  rcp_fast: hardware approximation (a few ulp), used only where an
// error of that size perturbs a parameter-like quantity (geometry, porous
// coefficients, small corrections).  rcp_acc: one Newton step on top (error well
// below one ulp, unbiased rounding), used wherever the result scales the conserved
// momentum that the next step reads back (1/rho and the Eq. 28 denominators): a
// biased factor there would act as a spurious force every step.
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_acc(float x) {
    const float y = __fdividef(1.0f, x);
    return fmaf(y, fmaf(-x, y, 1.0f), y);
}
__device__ __forceinline__ double rcp_acc(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }

// Node class (Fig. 1, Fig. 3): walls on the outermost nodes, corners on the side walls.
__host__ __device__ __forceinline__ bool periodic_z(int geometry) {
    return geometry == ANNULUS_PERIODIC_Z || geometry == PIPE_PERIODIC_Z;
}
__host__ __device__ __forceinline__ int node_class(int geometry, int nr, int nz, int kr, int kz) {
    if (geometry == PIPE_INFLOW) {   // Fig. 1: the wall is 0 < z < H; inlet and outlet own the corners
        if (kz == 0) return INLET;
        if (kz == nz - 1) return OUTLET;
    }
    if (kr == nr - 1) return WALL_OUT;
    if (kr == 0) return (geometry == PIPE_PERIODIC_Z || geometry == PIPE_INFLOW) ? AXIS : WALL_IN;
    if (geometry == ANNULUS) {
        if (kz == 0) return BOTTOM;
        if (kz == nz - 1) return TOP;
    }
    return FLUID;
}
// Boundary nodes rebuilt by non-equilibrium extrapolation (walls, inlet, outlet).
__host__ __device__ __forceinline__ bool is_wall(int cls) { return (cls >= WALL_IN && cls <= TOP) || cls >= INLET; }

// Interior neighbour a wall node extrapolates from (wall normal; corners diagonal).
__device__ __forceinline__ void fluid_neighbour(int geometry, int nr, int nz, int cls, int kr, int kz,
                                                int& fr, int& fz) {
    fr = kr;
    fz = kz;
    if (cls == WALL_IN) fr = 1;
    else if (cls == WALL_OUT) fr = nr - 2;
    else if (cls == BOTTOM || cls == INLET) fz = 1;
    else if (cls == TOP || cls == OUTLET) fz = nz - 2;
    if ((cls == INLET || cls == OUTLET) && kr == nr - 1) fr = nr - 2;
    if ((cls == WALL_IN || cls == WALL_OUT) && geometry == ANNULUS) {
        if (kz == 0) fz = 1;
        if (kz == nz - 1) fz = nz - 2;
    }
}

// Eq. 8 per node, in closed form.  With d_p fixed from Da and the mean porosity,
// 1/K(phi) = c_k (1 - phi)^2 / phi^3 and the Ergun F_phi / sqrt(K) = 1.75 sqrt(c_k / 150)
// (1 - phi) / phi^3, so one reciprocal 1/phi^3 gives nu / K, F_phi / sqrt(K) and 1/phi.
// porous_mode 0: no drag; 1: K = Da L^2 everywhere (F_phi from phi, or constant);
// 2: K(phi) per node.  lin = nu / K, nl = F_phi / sqrt(K).
template <typename R>
__device__ __forceinline__ void porous(const Consts<R>& c, R phi, R& lin, R& nl, R& inv_phi) {
    const R ip3 = rcp_fast(phi * phi * phi);
    inv_phi = phi * phi * ip3;
    if (c.porous_mode == 2) {
        const R om = R(1) - phi;
        lin = c.lin_coef * om * om * ip3;
        nl = c.ergun ? c.nl_coef * om * ip3 : c.nl_coef * om * sqrt_fast(ip3);
    } else if (c.porous_mode == 1) {
        lin = c.lin_coef;
        nl = c.ergun ? c.nl_coef * sqrt_fast(ip3) : c.nl_coef;
    } else {
        lin = R(0);
        nl = R(0);
    }
}

// Macroscopic fields of a non-wall node from its pre-collision deviations fv, gh:
// T (Eq. 38), rho (Eq. 26), G (Eq. 7), v (Eq. 29), l_j0, l_1 (Eq. 30), u (Eq. 28,
// literally per component with |v| = sqrt(v_r^2 + v_z^2)); lin, nl from porous().
template <typename R>
__device__ __forceinline__ void recover(const Consts<R>& c, R r, R inv_r, R phi, R lin, R nl, const R* fh,
                                        const R* gh, R rref, R& m0, R& rho, R& ur, R& uz, R& dT) {
    dT = gh[0] + gh[1] + gh[2] + gh[3] + gh[4];   // T - T0 - R(x)
    m0 = ((fh[0] + fh[1]) + (fh[2] + fh[3])) + ((fh[4] + fh[5]) + (fh[6] + fh[7])) + fh[8];
    rho = R(1) + m0 * inv_r;
    const R jr = (fh[1] - fh[3]) + (fh[5] - fh[6]) + (fh[8] - fh[7]);
    const R jz = (fh[2] - fh[4]) + (fh[5] + fh[6]) - (fh[7] + fh[8]);
    const R Gz = c.gbeta * (dT + rref) + c.az;
    const R inv_rho = rcp_acc(rho);
    // sum_i e_ir f_i = jr - c_s^2 / 2, so v_r = (jr - c_s^2/2) / rho + c_s^2 / 2 (Eq. 29)
    const R vr = (jr + R(0.5) * cs2<R>() * m0 * inv_r) * inv_rho;
    const R vz = jz * inv_rho + R(0.5) * r * phi * Gz;
    const R hd = R(0.25) * r * phi * lin;
    const R lr0 = R(0.5) * (r + c.cs2tau * inv_r) + hd;
    const R lz0 = R(0.5) * r + hd;
    // Eq. 28: u_j = v_j / D_j, D_j = l_j0 + sqrt(l_j0^2 + x) = 2 l_j0 + x / D_j with
    // x = l_1 |v|; the small Forchheimer part x / D_j is evaluated with fast operations.
    R Dr = R(2) * lr0, Dz = R(2) * lz0;
    if (nl != R(0)) {
        const R x = R(0.5) * r * phi * nl * sqrt_fast(vr * vr + vz * vz);
        Dr += x * rcp_fast(lr0 + sqrt_fast(lr0 * lr0 + x));
        Dz += x * rcp_fast(lz0 + sqrt_fast(lz0 * lz0 + x));
    }
    ur = vr * rcp_acc(Dr);
    uz = vz * rcp_acc(Dz);
}

// f = M^-1 m with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
template <typename R>
__device__ __forceinline__ void minv(const R* m, R* f) {
    const R a0 = m[0] * R(1.0 / 9), a1 = m[1] * R(1.0 / 36), a2 = m[2] * R(1.0 / 36);
    const R a3 = m[3] * R(1.0 / 6), a4 = m[4] * R(1.0 / 12), a5 = m[5] * R(1.0 / 6), a6 = m[6] * R(1.0 / 12);
    const R a7 = m[7] * R(0.25), a8 = m[8] * R(0.25);
    const R b14 = a0 - a1 - R(2) * a2;
    const R b58 = a0 + R(2) * a1 + a2;
    const R x3 = a3 - R(2) * a4, x5 = a5 - R(2) * a6;
    const R y3 = a3 + a4, y5 = a5 + a6;
    f[0] = a0 - R(4) * a1 + R(4) * a2;
    f[1] = b14 + x3 + a7;
    f[2] = b14 + x5 - a7;
    f[3] = b14 - x3 + a7;
    f[4] = b14 - x5 - a7;
    f[5] = b58 + y3 + y5 + a8;
    f[6] = b58 - y3 + y5 - a8;
    f[7] = b58 - y3 - y5 + a8;
    f[8] = b58 + y3 - y5 - a8;
}

// Collision of one node (in place: pre-collision deviations in, stored
// post-collision deviations out): forces (Eq. 6, 25), source (Eq. 24),
// MRT relaxation (Eq. 21) and f+ = M^-1 m+ (Eq. 22); D2Q5 update (Eq. 33, 35-37)
// with omega_g,i = (1 + e_ir tau_T / r) / (tau_T + 1/2).  rho, u, T are given so
// that wall nodes can impose u = 0 and their temperature; m0 = sum_i fh_i.
template <typename R>
__device__ __forceinline__ void collide(const Consts<R>& c, R r, R inv_r, R phi, R lin, R nl, R inv_phi, R* fh,
                                        R* gh, R rref, R m0, R rho, R ur, R uz, R dT) {
    const R Tb = c.T0 + rref;   // the node's reference temperature
    const R T = Tb + dT;
    const R u2 = ur * ur + uz * uz;
    const R um = sqrt_fast(u2);
    const R Gz = c.gbeta * (dT + rref) + c.az;
    const R drag = lin + nl * um;
    const R Fr = -phi * drag * ur;
    const R Ftr = Fr + (cs2<R>() - c.cs2_2tm * ur * inv_r) * inv_r;   // Eq. 25
    const R Ftz = -phi * drag * uz + phi * Gz;
    const R rr = r * rho;
    // Eq. 24; S_3 = r rho F~_r = c_s^2 + S3, the constant c_s^2 cancelling against
    // the rest offsets of the stored deviations
    const R S1 = R(6) * rr * (ur * Ftr + uz * Ftz) * inv_phi;
    const R S3 = cs2<R>() * m0 * inv_r + rr * Fr - rho * c.cs2_2tm * ur * inv_r;
    const R S5 = rr * Ftz;
    const R S7 = R(2) * rr * (ur * Ftr - uz * Ftz) * inv_phi;
    const R S8 = rr * (ur * Ftz + uz * Ftr) * inv_phi;
    // m = M f on the deviations (Eq. 16, 18)
    const R s14 = (fh[1] + fh[2]) + (fh[3] + fh[4]);
    const R s58 = (fh[5] + fh[6]) + (fh[7] + fh[8]);
    const R m1 = R(-4) * fh[0] - s14 + R(2) * s58;
    const R m2 = R(4) * fh[0] - R(2) * s14 + s58;
    const R d13 = fh[1] - fh[3], d24 = fh[2] - fh[4];
    const R x58 = (fh[5] - fh[7]), x68 = (fh[6] - fh[8]);
    const R m3 = d13 + x58 - x68;
    const R m4 = R(-2) * d13 + x58 - x68;
    const R m5 = d24 + x58 + x68;
    const R m6 = R(-2) * d24 + x58 + x68;
    const R m7 = (fh[1] + fh[3]) - (fh[2] + fh[4]);
    const R m8 = (fh[5] + fh[7]) - (fh[6] + fh[8]);
    // m_eq - r (1, -2, 1, 0, ...) (Eq. 19-20)
    const R q = R(3) * rr * u2 * inv_phi;
    const R e1 = R(-2) * m0 + q, e2 = m0 - q;
    const R e3 = rr * ur, e5 = rr * uz;
    const R e7 = rr * (ur * ur - uz * uz) * inv_phi, e8 = rr * ur * uz * inv_phi;
    // Eq. 21 with Lambda = diag(1, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu), as the
    // change dm = m+ - m (dm_0 = 0).  Eq. 22 is applied to the change only,
    // f+ = f + M^-1 dm, so the inexact float reciprocals of M^-1 scale the small
    // collision increment and not the conserved moments themselves (a factor like
    // 6 fl(1/6) = 1 + 3e-8 on the momentum every step would act as a spurious force).
    const R dm[9] = {R(0),
                     -c.s_e * (m1 - e1) + c.h_e * S1,
                     -c.s_eps * (m2 - e2) - c.h_eps * S1,
                     -c.s_j * (m3 - e3) + c.h_j * S3,
                     -c.s_q * (m4 + e3) - c.h_q * S3,
                     -c.s_j * (m5 - e5) + c.h_j * S5,
                     -c.s_q * (m6 + e5) - c.h_q * S5,
                     -c.s_nu * (m7 - e7) + c.h_nu * S7,
                     -c.s_nu * (m8 - e8) + c.h_nu * S8};
    R df[9];
    minv(dm, df);
#pragma unroll
    for (int i = 0; i < 9; ++i) fh[i] += df[i];
    // D2Q5 (Eq. 33, 35-37)
    const R k = c.tauT * inv_r;
    const R wd = c.wg_den;
    const R cu = -ur * inv_r;
    const R Tr = R(0.5) * T * ur, Tz = R(0.5) * T * uz;
    // g_eq - wT (T0 + R) (Eq. 35-36); the rest component is dT minus the other four so that
    // sum_i g_eq,i = T holds to rounding (0.6f + 4 * 0.1f is not 1)
    const R t1 = R(0.1) * dT;
    const R g1e = t1 + Tr, g3e = t1 - Tr;
    const R g2e = t1 + Tz, g4e = t1 - Tz;
    const R g0e = dT - R(4) * t1;
    const R wT0 = R(0.6) * Tb, wT1 = R(0.1) * Tb;
    gh[0] = gh[0] - wd * (gh[0] - g0e) + cu * (g0e + wT0);
    gh[1] = gh[1] - (R(1) + k) * wd * (gh[1] - g1e) + cu * (g1e + wT1);
    gh[2] = gh[2] - wd * (gh[2] - g2e) + cu * (g2e + wT1);
    gh[3] = gh[3] - (R(1) - k) * wd * (gh[3] - g3e) + cu * (g3e + wT1);
    gh[4] = gh[4] - wd * (gh[4] - g4e) + cu * (g4e + wT1);
}

// D2Q9 direction tables (Eq. 14) and weights (Eq. 32).
__host__ __device__ constexpr int ex9(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__host__ __device__ constexpr int ez9(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
__host__ __device__ constexpr int mirror9(int i) { return i == 1 ? 3 : i == 3 ? 1 : i == 5 ? 6 : i == 6 ? 5 : i == 7 ? 8 : i == 8 ? 7 : i; }
template <typename R> __host__ __device__ constexpr R w9(int i) { return i == 0 ? R(4) / R(9) : i < 5 ? R(1) / R(9) : R(1) / R(36); }

// Boundary node rebuild by non-equilibrium extrapolation (Sec. 4, ref. [47]) from the
// interior neighbour's pre-collision deviations (fhf at radius rf; iphif = 1/phi_f):
//   f_b = f_eq(r_b, rho_b, u_b) + [f_f - f_eq(r_f, rho_f, u_f)]      (Eq. 32)
// In deviations: fh_b,i = r_b w_i [drho_b + rho_b (3 eu_b + 4.5 eu_b^2 / phi_b - 1.5 u_b^2
// / phi_b)] + fh_f,i - r_f w_i [drho_f + rho_f (3 eu + 4.5 eu^2 / phi_f - 1.5 u^2 / phi_f)],
// drho = rho - 1, drho_f = m0f / r_f.  Walls: u_b = 0, rho_b = rho_f.
template <typename R>
__device__ __forceinline__ void rebuild_flow(R rb, R rf, R iphib, R iphif, R drhob, R rhob, R urb, R uzb, R m0f,
                                             R rhof, R urf, R uzf, const R* fhf, R* fh) {
    const R drho = m0f * rcp_acc(rf);
    const R u2 = urf * urf + uzf * uzf;
    const R ub2 = urb * urb + uzb * uzb;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = R(ex9(i)) * urf + R(ez9(i)) * uzf;
        const R q = drho + rhof * (R(3) * eu + R(4.5) * eu * eu * iphif - R(1.5) * u2 * iphif);
        const R eb = R(ex9(i)) * urb + R(ez9(i)) * uzb;
        const R qb = drhob + rhob * (R(3) * eb + R(4.5) * eb * eb * iphib - R(1.5) * ub2 * iphib);
        fh[i] = rb * w9<R>(i) * qb + fhf[i] - rf * w9<R>(i) * q;
    }
}

// Thermal part of the boundary rebuild: g_b = g_eq(T_b, u_b) + [g_f - g_eq(T_f, u_f)]
// (Eq. 35); in deviations gh_b,i = (g_eq,i(T_b, u_b) - wT_i Tb0) + gh_f,i - (g_eq,i(T_f, u_f)
// - wT_i Tf0) with dTb = T_b - Tb0, Tb0 = T0 + R_b, Tf0 = T0 + R_f the neighbour's reference,
// dTf = T_f - Tf0.
template <typename R>
__device__ __forceinline__ void rebuild_thermal(R Tf0, R dTf, R Tb0, R dTb, R urb, R uzb, R urf, R uzf, const R* ghf,
                                                R* gh) {
    const R Tf = Tf0 + dTf, Tb = Tb0 + dTb;
    const R tr = R(0.5) * Tf * urf, tz = R(0.5) * Tf * uzf;
    const R br = R(0.5) * Tb * urb, bz = R(0.5) * Tb * uzb;
    const R d = dTb - dTf;
    const R t1 = R(0.1) * d;
    gh[0] = ghf[0] + (d - R(4) * t1);
    gh[1] = ghf[1] + (t1 - tr + br);
    gh[2] = ghf[2] + (t1 - tz + bz);
    gh[3] = ghf[3] + (t1 + tr - br);
    gh[4] = ghf[4] + (t1 + tz - bz);
}

// References of 16-bit storage.  A 16-bit population stored against the rest state
// rounds at 2^-11 (FP16) or 2^-8 (BF16) of its deviation r w_i (3 e_i.u + ...), whose
// rounding jitter keeps convective runs from settling.  It is therefore stored against a
// per-node reference equilibrium instead:
//     s_i(y) = f+_i(y) - (r w_i + e_ir w_i / 2) - D_i(Q(y)),   D_i(Q) = w_i (A + 3 e_i.J),
// the part of Eq. 32's r-weighted f_eq linear in the deviations, with A = r (rho - 1) and
// J = r rho u of the node held in FP16 and refreshed from the state by the rebase kernel.
// The stored s_i then carry the second-order part of f_eq, the non-equilibrium part and
// the change since the last refresh.  The fourth FP16 of the node's 8-byte reference word
// is its temperature reference R(x) (see the thermal deviations above), so one load gives
// both.  Encoding and decoding use the same D_i(Q(y)) of the node y that wrote the value,
// evaluated in this fixed sequence of round-to-nearest operations (fref_delta2 in
// lbm_pair.cuh repeats it lane by lane), so the reference cancels exactly and any Q is a
// valid (if less effective) one.
struct Qf {
    float A, Jr, Jz, R;
};

__device__ __forceinline__ Qf fref_unpack(uint2 u) {
    const __half2 a = *reinterpret_cast<const __half2*>(&u.x), b = *reinterpret_cast<const __half2*>(&u.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return {fa.x, fa.y, fb.x, fb.y};
}

__device__ __forceinline__ uint2 fref_pack(__half A, __half Jr, __half Jz, __half R) {
    const __half2 a = __halves2half2(A, Jr), b = __halves2half2(Jz, R);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&a);
    u.y = *reinterpret_cast<const uint32_t*>(&b);
    return u;
}

__device__ __forceinline__ float fref_delta(int i, const Qf& q) {
    float eJ;
    switch (i) {
        case 0: eJ = 0.f; break;
        case 1: eJ = q.Jr; break;
        case 2: eJ = q.Jz; break;
        case 3: eJ = -q.Jr; break;
        case 4: eJ = -q.Jz; break;
        case 5: eJ = __fadd_rn(q.Jr, q.Jz); break;
        case 6: eJ = __fsub_rn(q.Jz, q.Jr); break;
        case 7: eJ = -__fadd_rn(q.Jr, q.Jz); break;
        default: eJ = -__fsub_rn(q.Jz, q.Jr); break;
    }
    return __fmul_rn(w9<float>(i), __fmaf_rn(eJ, 3.0f, q.A));
}

}  // namespace lbm
