// lbm_pair.cuh -- the per-node arithmetic of lbm_physics.cuh for two nodes at once, on
// the packed FP32 instructions of sm_100+ (fma/add/mul/sub .f32x2: two independent
// round-to-nearest FP32 operations per instruction, each lane bitwise equal to the scalar
// operation).  The two lanes are two z-adjacent nodes of one row, so every per-row
// quantity (r, 1/r and the constants built from them) is shared and every per-node
// quantity is a pair.  The algebra is that of recover() and collide() (Eq. 6-8, 21-30,
// 33-38); only the evaluation order differs where a multiply-add is written as one fused
// instruction.
//
// Flow reference of 16-bit storage (the encoding of lbm_physics.cuh's scalar
// fref_delta): the stored value of population i at node y is
//     s_i(y) = f+_i(y) - (r w_i + e_ir w_i / 2) - D_i(Q(y)),   D_i(Q) = w_i (A + 3 e_i.J),
// with (A, J_r, J_z) = (sum of the deviations, their e-weighted sums) of the node in FP16,
// refreshed by the rebase kernel.  fref_delta2 evaluates D with the same sequence of
// rounded operations as the scalar version (fma(eJ, 3, A) then the weight), so a value
// encoded by one and decoded by the other is unchanged.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_physics.cuh"

namespace lbm {

struct V2 {
    float2 v;
};

__device__ __forceinline__ V2 v2(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ V2 v2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) {
    unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a.v);
    unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b.v), rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    V2 d;
    d.v = *reinterpret_cast<float2*>(&rd);
    return d;
}
__device__ __forceinline__ V2 operator-(V2 a) { return {make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ V2 operator+(V2 a, float b) { return a + v2(b); }
__device__ __forceinline__ V2 operator+(float a, V2 b) { return v2(a) + b; }
__device__ __forceinline__ V2 operator-(V2 a, float b) { return a - v2(b); }
__device__ __forceinline__ V2 operator-(float a, V2 b) { return v2(a) - b; }
__device__ __forceinline__ V2 operator*(V2 a, float b) { return a * v2(b); }
__device__ __forceinline__ V2 operator*(float a, V2 b) { return v2(a) * b; }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) { return a = a + b; }
// a * b + c, one rounding per lane
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ V2 fma2(V2 a, float b, V2 c) { return fma2(a, v2(b), c); }
__device__ __forceinline__ V2 fma2(float a, V2 b, V2 c) { return fma2(v2(a), b, c); }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, float c) { return fma2(a, b, v2(c)); }
__device__ __forceinline__ V2 fma2(V2 a, float b, float c) { return fma2(a, v2(b), v2(c)); }
__device__ __forceinline__ V2 fma2(float a, V2 b, float c) { return fma2(v2(a), b, v2(c)); }

// Lane-wise reciprocal and square root: the hardware approximations (rcp.approx and
// sqrt.approx, one instruction each; sqrt(0) = 0, so no guard is needed), where the scalar
// path of lbm_physics.cuh goes through __fdividef and x rsqrt(x) with their range checks.
// rcp_acc adds one Newton step, as the scalar rcp_acc does.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ V2 rcp_fast(V2 x) { return v2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }
__device__ __forceinline__ V2 rcp_acc(V2 x) {
    const V2 y = rcp_fast(x);
    return fma2(y, fma2(-x, y, 1.0f), y);
}
__device__ __forceinline__ V2 sqrt_fast(V2 x) { return v2(sqrt_approx(x.v.x), sqrt_approx(x.v.y)); }

// Row constants of the recovery and collision, shared by both lanes.
struct RowC {
    float r, inv_r;
    float hr;      // r / 2
    float qr;      // r / 4
    float c1;      // c_s^2 / (2 r)
    float L0r;     // (r + c_s^2 (tau - 1/2) / r) / 2
    float kT;      // tau_T / r
    float cs2r;    // c_s^2 / r
    float c2r;     // c_s^2 2 (tau - 1/2) / r
};

__device__ __forceinline__ RowC row_consts(const Consts<float>& c, int kr) {
    RowC q;
    q.r = c.r0 + float(kr);
    q.inv_r = rcp_acc(q.r);
    q.hr = 0.5f * q.r;
    q.qr = 0.25f * q.r;
    q.c1 = 0.5f * cs2<float>() * q.inv_r;
    q.L0r = 0.5f * (q.r + c.cs2tau * q.inv_r);
    q.kT = c.tauT * q.inv_r;
    q.cs2r = cs2<float>() * q.inv_r;
    q.c2r = c.cs2_2tm * q.inv_r;
    return q;
}

// Eq. 8 per node (porous() of lbm_physics.cuh, lane-wise).
__device__ __forceinline__ void porous2(const Consts<float>& c, V2 phi, V2& lin, V2& nl, V2& inv_phi) {
    const V2 ph2 = phi * phi;
    const V2 ip3 = rcp_fast(ph2 * phi);
    inv_phi = ph2 * ip3;
    if (c.porous_mode == 2) {
        const V2 om = 1.0f - phi;
        lin = c.lin_coef * (om * om) * ip3;
        nl = c.ergun ? c.nl_coef * om * ip3 : c.nl_coef * om * sqrt_fast(ip3);
    } else if (c.porous_mode == 1) {
        lin = v2(c.lin_coef);
        nl = c.ergun ? c.nl_coef * sqrt_fast(ip3) : v2(c.nl_coef);
    } else {
        lin = v2(0.f);
        nl = v2(0.f);
    }
}

// recover() of lbm_physics.cuh (Eq. 26-30, 38) for two nodes; dT is relative to each
// node's reference temperature T0 + R(x), rref = R(x).
__device__ __forceinline__ void recover2(const Consts<float>& c, const RowC& q, V2 phi, V2 lin, V2 nl, const V2* fh,
                                         const V2* gh, V2 rref, V2& m0, V2& rho, V2& ur, V2& uz, V2& dT) {
    dT = ((gh[0] + gh[1]) + (gh[2] + gh[3])) + gh[4];
    m0 = ((fh[0] + fh[1]) + (fh[2] + fh[3])) + ((fh[4] + fh[5]) + (fh[6] + fh[7])) + fh[8];
    rho = fma2(m0, q.inv_r, 1.0f);
    const V2 jr = ((fh[1] - fh[3]) + (fh[5] - fh[6])) + (fh[8] - fh[7]);
    const V2 jz = ((fh[2] - fh[4]) + (fh[5] + fh[6])) - (fh[7] + fh[8]);
    const V2 Gz = fma2(v2(c.gbeta), dT + rref, v2(c.az));
    const V2 inv_rho = rcp_acc(rho);
    const V2 vr = fma2(m0, q.c1, jr) * inv_rho;
    const V2 vz = fma2(jz, inv_rho, (q.hr * phi) * Gz);
    const V2 hd = (q.qr * phi) * lin;
    const V2 lr0 = q.L0r + hd;
    const V2 lz0 = q.hr + hd;
    // Eq. 28 as in recover(), without a branch: x = 0 (no Forchheimer drag) adds 0
    const V2 x = (q.hr * phi) * nl * sqrt_fast(fma2(vr, vr, vz * vz));
    const V2 Dr = fma2(x, rcp_fast(lr0 + sqrt_fast(fma2(lr0, lr0, x))), lr0 + lr0);
    const V2 Dz = fma2(x, rcp_fast(lz0 + sqrt_fast(fma2(lz0, lz0, x))), lz0 + lz0);
    ur = vr * rcp_acc(Dr);
    uz = vz * rcp_acc(Dz);
}

// f = M^-1 m (minv of lbm_physics.cuh) for two nodes.
__device__ __forceinline__ void minv2(const V2* m, V2* f) {
    const V2 a0 = m[0] * (1.0f / 9), a1 = m[1] * (1.0f / 36), a2 = m[2] * (1.0f / 36);
    const V2 a3 = m[3] * (1.0f / 6), a4 = m[4] * (1.0f / 12), a5 = m[5] * (1.0f / 6), a6 = m[6] * (1.0f / 12);
    const V2 a7 = m[7] * 0.25f, a8 = m[8] * 0.25f;
    const V2 b14 = fma2(a2, -2.0f, a0 - a1);
    const V2 b58 = fma2(a1, 2.0f, a0 + a2);
    const V2 x3 = fma2(a4, -2.0f, a3), x5 = fma2(a6, -2.0f, a5);
    const V2 y3 = a3 + a4, y5 = a5 + a6;
    f[0] = fma2(a2 - a1, 4.0f, a0);
    f[1] = (b14 + x3) + a7;
    f[2] = (b14 + x5) - a7;
    f[3] = (b14 - x3) + a7;
    f[4] = (b14 - x5) - a7;
    f[5] = ((b58 + y3) + y5) + a8;
    f[6] = ((b58 - y3) + y5) - a8;
    f[7] = ((b58 - y3) - y5) + a8;
    f[8] = ((b58 + y3) - y5) - a8;
}

// collide() of lbm_physics.cuh (Eq. 6, 21-25, 33-37) for two nodes, in place; rref = R(x).
__device__ __forceinline__ void collide2(const Consts<float>& c, const RowC& q, V2 phi, V2 lin, V2 nl, V2 inv_phi,
                                         V2* fh, V2* gh, V2 rref, V2 m0, V2 rho, V2 ur, V2 uz, V2 dT) {
    const V2 Tb = c.T0 + rref;   // the nodes' reference temperatures
    const V2 T = Tb + dT;
    const V2 u2 = fma2(ur, ur, uz * uz);
    const V2 um = sqrt_fast(u2);
    const V2 Gz = fma2(v2(c.gbeta), dT + rref, v2(c.az));
    const V2 drag = fma2(nl, um, lin);
    const V2 pd = phi * drag;
    const V2 Fr = -(pd * ur);
    const V2 Ftr = fma2(fma2(-q.c2r, ur, v2(cs2<float>())), q.inv_r, Fr);   // Eq. 25
    const V2 Ftz = fma2(phi, Gz, -(pd * uz));
    const V2 rr = q.r * rho;
    const V2 rri = rr * inv_phi;
    // Eq. 24 without the rest constant c_s^2 of S_3 (see collide())
    const V2 S1 = (6.0f * rri) * fma2(ur, Ftr, uz * Ftz);
    const V2 S3 = fma2(m0, q.cs2r, fma2(rr, Fr, -(rho * (q.c2r * ur))));
    const V2 S5 = rr * Ftz;
    const V2 S7 = (2.0f * rri) * fma2(ur, Ftr, -(uz * Ftz));
    const V2 S8 = rri * fma2(ur, Ftz, uz * Ftr);
    // m = M f on the deviations (Eq. 16, 18)
    const V2 s14 = (fh[1] + fh[2]) + (fh[3] + fh[4]);
    const V2 s58 = (fh[5] + fh[6]) + (fh[7] + fh[8]);
    const V2 m1 = fma2(fh[0], -4.0f, fma2(s58, 2.0f, -s14));
    const V2 m2 = fma2(fh[0], 4.0f, fma2(s14, -2.0f, s58));
    const V2 d13 = fh[1] - fh[3], d24 = fh[2] - fh[4];
    const V2 x58 = fh[5] - fh[7], x68 = fh[6] - fh[8];
    const V2 xm = x58 - x68, xp = x58 + x68;
    const V2 m3 = d13 + xm;
    const V2 m4 = fma2(d13, -2.0f, xm);
    const V2 m5 = d24 + xp;
    const V2 m6 = fma2(d24, -2.0f, xp);
    const V2 m7 = (fh[1] + fh[3]) - (fh[2] + fh[4]);
    const V2 m8 = (fh[5] + fh[7]) - (fh[6] + fh[8]);
    // m_eq - r (1, -2, 1, 0, ...) (Eq. 19-20)
    const V2 qq = (3.0f * rri) * u2;
    const V2 e1 = fma2(m0, -2.0f, qq), e2 = m0 - qq;
    const V2 e3 = rr * ur, e5 = rr * uz;
    const V2 e7 = rri * fma2(ur, ur, -(uz * uz)), e8 = rri * (ur * uz);
    // Eq. 21 as the change dm = m+ - m (dm_0 = 0); Eq. 22 on the change only
    V2 dm[9];
    dm[0] = v2(0.f);
    dm[1] = fma2(v2(c.h_e), S1, (-c.s_e) * (m1 - e1));
    dm[2] = fma2(v2(-c.h_eps), S1, (-c.s_eps) * (m2 - e2));
    dm[3] = fma2(v2(c.h_j), S3, (-c.s_j) * (m3 - e3));
    dm[4] = fma2(v2(-c.h_q), S3, (-c.s_q) * (m4 + e3));
    dm[5] = fma2(v2(c.h_j), S5, (-c.s_j) * (m5 - e5));
    dm[6] = fma2(v2(-c.h_q), S5, (-c.s_q) * (m6 + e5));
    dm[7] = fma2(v2(c.h_nu), S7, (-c.s_nu) * (m7 - e7));
    dm[8] = fma2(v2(c.h_nu), S8, (-c.s_nu) * (m8 - e8));
    V2 df[9];
    minv2(dm, df);
#pragma unroll
    for (int i = 0; i < 9; ++i) fh[i] += df[i];
    // D2Q5 (Eq. 33, 35-37), relative to T0 + R(x)
    const V2 wd = v2(c.wg_den);
    const V2 cu = -(ur * q.inv_r);
    const V2 hT = 0.5f * T;
    const V2 Tr = hT * ur, Tz = hT * uz;
    const V2 t1 = 0.1f * dT;
    const V2 g1e = t1 + Tr, g3e = t1 - Tr;
    const V2 g2e = t1 + Tz, g4e = t1 - Tz;
    const V2 g0e = fma2(t1, -4.0f, dT);
    const V2 wT0 = 0.6f * Tb, wT1 = 0.1f * Tb;
    const V2 wp = (1.0f + q.kT) * wd, wm = (1.0f - q.kT) * wd;
    gh[0] = fma2(cu, g0e + wT0, fma2(-wd, gh[0] - g0e, gh[0]));
    gh[1] = fma2(cu, g1e + wT1, fma2(-wp, gh[1] - g1e, gh[1]));
    gh[2] = fma2(cu, g2e + wT1, fma2(-wd, gh[2] - g2e, gh[2]));
    gh[3] = fma2(cu, g3e + wT1, fma2(-wm, gh[3] - g3e, gh[3]));
    gh[4] = fma2(cu, g4e + wT1, fma2(-wd, gh[4] - g4e, gh[4]));
}

// ------------------------------------------------------ flow reference, packed --
// Q of two nodes as floats: (A, J_r, J_z, R) per lane.
struct Q2 {
    V2 A, Jr, Jz, R;
};

// D_i(Q) for both lanes, in the rounded operations of fref_delta (lbm_physics.cuh).
__device__ __forceinline__ V2 fref_delta2(int i, const Q2& Q) {
    V2 eJ;
    switch (i) {
        case 0: eJ = v2(0.f); break;
        case 1: eJ = Q.Jr; break;
        case 2: eJ = Q.Jz; break;
        case 3: eJ = -Q.Jr; break;
        case 4: eJ = -Q.Jz; break;
        case 5: eJ = Q.Jr + Q.Jz; break;
        case 6: eJ = Q.Jz - Q.Jr; break;
        case 7: eJ = -(Q.Jr + Q.Jz); break;
        default: eJ = -(Q.Jz - Q.Jr); break;
    }
    return w9<float>(i) * fma2(eJ, 3.0f, Q.A);
}

}  // namespace lbm
