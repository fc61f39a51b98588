// lbm.cu -- kernels and host runtime behind the C ABI of include/lbm.h.
//
// Axisymmetric D2Q9 MRT flow + D2Q5 temperature lattice Boltzmann step for porous
// media (Liu, He & Li, arXiv 1409.5929, Sec. 3-4) on one GB300 (sm_103a).
//
// Data layout in HBM (per handle):
//   state A, state B: 14 planes (f_0..f_8, g_0..g_4), each nr*nz elements, z fastest,
//                     plane stride padded to 64 elements; f planes in the storage
//                     type (FP32, FP16 or BF16), g planes in FP32, holding the
//                     deviations of lbm_physics.cuh.  A step reads one buffer and
//                     writes the other.
//   phi:              nr*nz porosity values (FP32).
//   tref:             nr*nz temperature references R(x) (FP16).
//   fref:             nr*nz flow references Q(x), 4 x FP16 each (16-bit storage).
//   macro snapshots, reduction scratch, staging: only for diagnostics.
//
// A step is two launches on the handle's stream:
//   k_bulk  every non-wall node: pull (Eq. 22, 33), recovery (Eq. 26-30, 38),
//           collision (Eq. 21-24, 33-37), store.  Grid (nz / 128, nr).  With
//           16-bit storage k_bulk_pair: two z-adjacent nodes per thread on the
//           packed FP32 instructions (lbm_pair.cuh).
//   k_wall  every wall node: rebuild from the interior neighbour by
//           non-equilibrium extrapolation (Sec. 4, ref. [47]), collision with
//           u = 0 and the wall temperature, store.  One thread per wall node.
// Both read only the source buffer and write disjoint nodes of the destination.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_pair.cuh"
#include "lbm_physics.cuh"

using namespace lbm;

// ------------------------------------------------------------ storage types --
// Flow populations in the storage type; temperature populations always FP32 (in
// 16 bits the per-step change of g - wT T0, of order 0.05, falls below the format's
// resolution and the temperature field stagnates); porosity always FP32 (in FP16 its
// half-ulp, 2.4e-4 relative near 0.7, moves the Darcy drag of Eq. 8 by about 2e-3).
__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ void stv(float* p, float v) { *p = v; }
__device__ __forceinline__ void stv(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void stv(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <int STO> struct St;
template <> struct St<LBM_F32> { using TF = float; using TG = float; using P = float; };
template <> struct St<LBM_F16> { using TF = __half; using TG = float; using P = float; };
template <> struct St<LBM_BF16> { using TF = __nv_bfloat16; using TG = float; using P = float; };

// One state buffer: nine flow planes then five temperature planes.
template <int STO> struct Buf {
    typename St<STO>::TF* f;
    typename St<STO>::TG* g;
};

static size_t f_size(int sto) { return sto == LBM_F32 ? 4 : 2; }
static size_t g_size(int) { return 4; }
static size_t phi_size(int) { return 4; }
static size_t state_bytes(int sto, int64_t plane) { return (size_t)plane * (9 * f_size(sto) + 5 * g_size(sto)); }

constexpr int BULK_THREADS = 128;
#ifndef LBM_BULK_RPT
#define LBM_BULK_RPT 4
#endif
constexpr int BULK_RPT = LBM_BULK_RPT;  // rows per thread of the bulk kernel (32-bit indexing)
#ifndef LBM_BULK_RPT_MIN_BLOCKS
#define LBM_BULK_RPT_MIN_BLOCKS 16
#endif
// BULK_RPT rows per thread only where the grid keeps at least this many blocks per SM
constexpr int BULK_RPT_MIN_BLOCKS = LBM_BULK_RPT_MIN_BLOCKS;

// ------------------------------------------------------------- layouts --
// Where the post-collision population i of node y is kept between steps:
//   LAY_N  two state buffers (A/B): slot i at y of the buffer last written;
//   LAY_S  one buffer (in place), after an even number of steps: slot opp(i) at y;
//   LAY_L  one buffer, after an odd number of steps: slot i at y + e_i (z wraps when
//          periodic; populations leaving through the pipe axis are kept where the axis
//          row's pull reads them: f+_3(0, z) at (1, (0, z)), f+_6(0, z) at (5, (0, z + 1)),
//          f+_7(0, z) at (8, (0, z - 1)); other populations leaving the domain are dropped).
// A step of the in-place scheme reads S and writes L, or reads L and writes S: every
// location a node reads is one it writes and no other node touches it, so one buffer
// suffices.  The same layouts hold for the five temperature populations.
enum { LAY_N = 0, LAY_S = 1, LAY_L = 2 };
__host__ __device__ constexpr int opp9(int i) { return i == 0 ? 0 : i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5; }

// ------------------------------------------------------------- pull (Eq. 22) --
// Sources of the pulled populations at (kr, kz): the node src[i] whose post-collision
// population sp[i] streams into population i, i.e. (kr - e_ir) nz + (kz - e_iz), and in the
// pipe's axis row for the e_r = +1 populations the node's mirror image (population
// mirror(i) of row 0); and, for layout LAY, where that value is kept: node loc[i], slot
// lp[i].  Periodic z wraps.
template <int LAY, typename R, typename I>
__device__ __forceinline__ void pull_sources(const Consts<R>& c, int kr, int kz, I* src, int* sp, I* loc, int* lp) {
    const bool pz = c.periodic != 0;
    const int zm = (pz && kz == 0) ? c.nz - 1 : kz - 1;       // source column for e_z = +1
    const int zp = (pz && kz == c.nz - 1) ? 0 : kz + 1;       // source column for e_z = -1
    const I row = (I)kr * c.nz;
    const I rowm = row - c.nz, rowp = row + c.nz;
    const bool axis = (kr == 0);                              // reached only in the pipe
    src[0] = row + kz;        sp[0] = 0;
    src[1] = (axis ? row : rowm) + kz;  sp[1] = axis ? 3 : 1;
    src[2] = row + zm;        sp[2] = 2;
    src[3] = rowp + kz;       sp[3] = 3;
    src[4] = row + zp;        sp[4] = 4;
    src[5] = (axis ? row : rowm) + zm;  sp[5] = axis ? 6 : 5;
    src[6] = rowp + zm;       sp[6] = 6;
    src[7] = rowp + zp;       sp[7] = 7;
    src[8] = (axis ? row : rowm) + zp;  sp[8] = axis ? 7 : 8;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        loc[i] = LAY == LAY_L ? row + kz : src[i];
        lp[i] = LAY == LAY_N ? sp[i] : LAY == LAY_S ? opp9(sp[i]) : i;
    }
}

// Where node (kr, kz) keeps its post-collision population i in layout LAY (false: dropped).
template <int LAY, typename R, typename I>
__device__ __forceinline__ bool own_slot(const Consts<R>& c, int kr, int kz, int i, I& node, int& slot) {
    if (LAY != LAY_L) {
        node = (I)kr * c.nz + kz;
        slot = LAY == LAY_N ? i : opp9(i);
        return true;
    }
    int r = kr + ex9(i), z = kz + ez9(i);
    slot = i;
    if (r < 0) {   // leaving through row 0: kept only on the pipe axis, as its mirror image
        if (c.geometry != PIPE_PERIODIC_Z && c.geometry != PIPE_INFLOW) return false;
        r = 0;         // the mirror image keeps the z motion: (0, z + e_iz)
        slot = i == 3 ? 1 : i == 6 ? 5 : 8;
    }
    if (r >= c.nr) return false;
    if (z < 0 || z >= c.nz) {
        if (!c.periodic) return false;
        z = z < 0 ? z + c.nz : z - c.nz;
    }
    node = (I)r * c.nz + z;
    return true;
}

// Flow populations stored against a per-node reference (16-bit storage, see fref_delta).
template <int STO> __host__ __device__ constexpr bool has_fref() { return STO != LBM_F32; }

// Pre-collision deviations at (kr, kz) from the post-collision state A in layout LAY: a
// plain copy of ft_i(x - e_i) (see lbm_physics.cuh), plus, with 16-bit storage, the
// reference part D_pop(Q(source)) of the value the source node stored.  src receives the
// source nodes (for the temperature reference).
template <int STO, int LAY, typename R, typename I>
__device__ __forceinline__ void pull_raw(const Consts<R>& c, const Buf<STO>& A, I plane, int kr, int kz, R* fh,
                                         R* gh, I* src) {
    I loc[9];
    int sp[9], lp[9];
    pull_sources<LAY, R, I>(c, kr, kz, src, sp, loc, lp);
    const auto* __restrict__ F = A.f;
    const auto* __restrict__ G = A.g;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float v = ldv(F + lp[i] * plane + loc[i]);
        if constexpr (has_fref<STO>()) v += fref_delta(sp[i], fref_unpack(c.fref[src[i]]));
        fh[i] = R(v);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) gh[i] = R(ldv(G + lp[i] * plane + loc[i]));
}

// Re-reference pulled thermal deviations to the node's R(x): gh_i += wT_i (R(x - e_i) - R(x))
// with r0 = R(x) and rm, zm, rp, zp the offsets of the sources of g_1 .. g_4.
template <typename R>
__device__ __forceinline__ void reref(R* gh, R r0, R rm, R zm, R rp, R zp) {
    gh[1] += R(0.1) * (rm - r0);
    gh[2] += R(0.1) * (zm - r0);
    gh[3] += R(0.1) * (rp - r0);
    gh[4] += R(0.1) * (zp - r0);
}

// Every storage type keeps the temperature reference R(x): the FP32 temperature populations
// stored against T0 alone would carry deviations of size |T - T0|, on which FP32 arithmetic
// biases the thermal update and freezes slow modes short of their fixed point.
template <int STO> __host__ __device__ constexpr bool has_ref() { return true; }

// R(x) of node n: its own FP16 plane with FP32 storage, the fourth FP16 of the node's
// reference word with 16-bit storage.
template <int STO, typename R, typename I>
__device__ __forceinline__ float tref_at(const Consts<R>& c, I n) {
    if constexpr (has_fref<STO>()) {
        const uint32_t w = c.fref[n].y;
        return __high2float(*reinterpret_cast<const __half2*>(&w));
    } else {
        return __half2float(c.tref[n]);
    }
}

// Pull (Eq. 22) from layout LAY with the thermal deviations re-referenced to R(x), which
// *rref receives (on the pipe axis row g_1 comes from the node's own mirror image).
template <int STO, typename R, typename I = int64_t, int LAY = LAY_N>
__device__ __forceinline__ void pull(const Consts<R>& c, const Buf<STO>& A, I plane, int kr, int kz, R* fh, R* gh,
                                     R& rref) {
    I src[9];
    pull_raw<STO, LAY, R, I>(c, A, plane, kr, kz, fh, gh, src);
    rref = R(tref_at<STO>(c, (I)kr * c.nz + kz));
    reref(gh, rref, R(tref_at<STO>(c, src[1])), R(tref_at<STO>(c, src[2])), R(tref_at<STO>(c, src[3])),
          R(tref_at<STO>(c, src[4])));
}

// Store the post-collision deviations of node (kr, kz) = n in layout LAY (16-bit storage:
// against the node's own flow reference Q(n)).
template <int STO, typename R, typename I = int64_t, int LAY = LAY_N>
__device__ __forceinline__ void store(const Consts<float>& c, const Buf<STO>& B, I plane, int kr, int kz, I n,
                                      const R* fh, const R* gh) {
    Qf q;
    if constexpr (has_fref<STO>()) q = fref_unpack(c.fref[n]);
    if constexpr (LAY == LAY_N) {
        // two buffers: the nine flow planes, then the five temperature planes (measured 7 %
        // faster than interleaved)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float v = float(fh[i]);
            if constexpr (has_fref<STO>()) v -= fref_delta(i, q);
            stv(B.f + i * plane + n, v);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) stv(B.g + i * plane + n, float(gh[i]));
    } else {
        // in place: f_i and g_i of one direction together, at the location own_slot gives
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            I m;
            int slot;
            if (!own_slot<LAY, float, I>(c, kr, kz, i, m, slot)) continue;
            float v = float(fh[i]);
            if constexpr (has_fref<STO>()) v -= fref_delta(i, q);
            stv(B.f + slot * plane + m, v);
            if (i < 5) stv(B.g + slot * plane + m, float(gh[i]));
        }
    }
}

// Boundary node state: rebuild (Sec. 4, ref. [47]) from the interior neighbour, then
// rho from Eq. 26.  Walls: u_b = 0, rho_b = rho_f, T_b = T_hot (inner), T_cold (outer),
// T_f (adiabatic top and bottom).  Pipe inlet: u_b = (0, u_in), rho_b = rho_f, T_b = T_hot;
// outlet: u_b = u_f, T_b = T_f, rho_b = 1 (zero gradient of u and T, density held).
template <int STO, typename R, int LAY = LAY_N>
__device__ __forceinline__ void wall_state(const Consts<R>& c, const Buf<STO> A,
                                           const typename St<STO>::P* __restrict__ phi, int64_t plane, int cls,
                                           int kr, int kz, R* fh, R* gh, R& m0, R& rho, R& urb, R& uzb, R& dTb,
                                           R& refb) {
    int fr, fz;
    fluid_neighbour(c.geometry, c.nr, c.nz, cls, kr, kz, fr, fz);
    R fhf[9], ghf[5], reff;
    pull<STO, R, int64_t, LAY>(c, A, plane, fr, fz, fhf, ghf, reff);
    const R rf = c.r0 + R(fr), rb = c.r0 + R(kr);
    const R phif = R(ldv(phi + (int64_t)fr * c.nz + fz));
    R m0f, rhof, urf, uzf, dTf, lin, nl, ipf;
    porous(c, phif, lin, nl, ipf);
    recover(c, rf, rcp_acc(rf), phif, lin, nl, fhf, ghf, reff, m0f, rhof, urf, uzf, dTf);
    R drhob = m0f * rcp_acc(rf), rhob = rhof;
    urb = R(0);
    uzb = R(0);
    R ipb = R(1);
    if (cls == INLET) {
        uzb = c.u_in;
    } else if (cls == OUTLET) {
        urb = urf;
        uzb = uzf;
        drhob = R(0);
        rhob = R(1);
    }
    if (cls >= INLET) ipb = rcp_acc(R(ldv(phi + (int64_t)kr * c.nz + kz)));
    rebuild_flow(rb, rf, ipb, ipf, drhob, rhob, urb, uzb, m0f, rhof, urf, uzf, fhf, fh);
    // deviations relative to this boundary node's own reference R_b
    refb = R(tref_at<STO>(c, (int64_t)kr * c.nz + kz));
    dTb = (cls == WALL_IN || cls == INLET) ? (c.T_hot - c.T0) - refb
          : cls == WALL_OUT                 ? (c.T_cold - c.T0) - refb
                                            : (dTf + reff) - refb;
    if (cls == WALL_IN && c.heater) {
        // Sec. 4.4: q' = -k dT/dr on the heater, dT/dr = 0 on the rest of the inner wall;
        // (-3 T_b + 4 T_1 - T_2) / 2 = -q'/k with the next two nodes inward (T_1 = T_f);
        // corners (diagonal neighbour) take T_f
        if (fz == kz) {
            R f2[9], g2[5], ref2;
            pull<STO, R, int64_t, LAY>(c, A, plane, 2, kz, f2, g2, ref2);
            const R T1 = (c.T0 + reff) + dTf;
            const R T2 = (c.T0 + ref2) + (((g2[0] + g2[1]) + (g2[2] + g2[3])) + g2[4]);
            const R G = (kz >= c.hz0 && kz <= c.hz1) ? c.hG : R(0);
            dTb = (R(4) * T1 - T2 + R(2) * G) * R(1.0 / 3.0) - (c.T0 + refb);
        } else {
            dTb = (dTf + reff) - refb;
        }
    }
    rebuild_thermal(c.T0 + reff, dTf, c.T0 + refb, dTb, urb, uzb, urf, uzf, ghf, gh);
    m0 = ((fh[0] + fh[1]) + (fh[2] + fh[3])) + ((fh[4] + fh[5]) + (fh[6] + fh[7])) + fh[8];
    rho = R(1) + m0 * rcp_acc(rb);
}

// Boundary node t -> (kr, kz): inner wall (annulus), outer wall, then bottom and top
// without the corners (closed annulus).  Pipe with inlet: inlet row, outlet row, then
// the wall without the corners.
__device__ __forceinline__ void wall_node(int geometry, int nr, int nz, int t, int& kr, int& kz) {
    if (geometry == PIPE_INFLOW) {
        if (t < nr) { kr = t; kz = 0; return; }
        t -= nr;
        if (t < nr) { kr = t; kz = nz - 1; return; }
        t -= nr;
        kr = nr - 1;
        kz = 1 + t;
        return;
    }
    if (geometry != PIPE_PERIODIC_Z) {
        if (t < nz) { kr = 0; kz = t; return; }
        t -= nz;
    }
    if (t < nz) { kr = nr - 1; kz = t; return; }
    t -= nz;
    if (t < nr - 2) { kr = 1 + t; kz = 0; return; }
    t -= nr - 2;
    kr = 1 + t;
    kz = nz - 1;
}

static int wall_count(int geometry, int nr, int nz) {
    if (geometry == ANNULUS) return 2 * nz + 2 * (nr - 2);
    if (geometry == ANNULUS_PERIODIC_Z) return 2 * nz;
    if (geometry == PIPE_INFLOW) return 2 * nr + nz - 2;
    return nz;
}

// ------------------------------------------------------------------ kernels --
// Update `rows` consecutive non-wall nodes of column kz from row kr0 on (rows past the
// last row are skipped); shared by the single-problem and the batched bulk kernels.
// I: index type.
template <int STO, typename I, int LIN = LAY_N, int LOUT = LAY_N>
__device__ __forceinline__ void update_column(const Consts<float>& c, const Buf<STO>& A, const Buf<STO>& B,
                                              const typename St<STO>::P* __restrict__ phi, I plane, int kr0,
                                              int rows, int kz) {
    // node_class split into its column and row parts: the end columns are boundary
    // nodes unless z is periodic; row nr - 1 is a wall, row 0 too unless it is a pipe axis
    const bool zwall = !c.periodic && (kz == 0 || kz == c.nz - 1);
    const bool row0_wall = c.geometry == ANNULUS || c.geometry == ANNULUS_PERIODIC_Z;
#pragma unroll 1
    for (int j = 0; j < rows; ++j) {
        const int kr = kr0 + j;
        if (kr >= c.nr) break;
        if (zwall || kr == c.nr - 1 || (kr == 0 && row0_wall)) continue;
        float fh[9], gh[5], ref;
        pull<STO, float, I, LIN>(c, A, plane, kr, kz, fh, gh, ref);
        const I n = (I)kr * c.nz + kz;
        const float r = c.r0 + float(kr), inv_r = rcp_acc(r);
        const float ph = ldv(phi + n);
        float m0, rho, ur, uz, dT, lin, nl, iph;
        porous(c, ph, lin, nl, iph);
        recover(c, r, inv_r, ph, lin, nl, fh, gh, ref, m0, rho, ur, uz, dT);
        collide(c, r, inv_r, ph, lin, nl, iph, fh, gh, ref, m0, rho, ur, uz, dT);
        store<STO, float, I, LOUT>(c, B, plane, kr, kz, n, fh, gh);
    }
}

// ------------------------------------------- packed pair update (16-bit storage) --
// Two z-adjacent nodes (kz0, kz0 + 1) per thread, their arithmetic on the packed FP32
// instructions of lbm_pair.cuh.  Loads of the node's own columns are single vector loads
// when the row's first element index is even (VEC: nz even, kz0 even); the shifted
// columns of the e_z = +-1 populations are two scalar loads.  Flow populations carry the
// flow reference: the pull adds D_pop(Q(source)), the store subtracts D_i(Q(own)).
__device__ __forceinline__ V2 ld2(const __half* p, int a, int b, bool vec) {
    if (vec) return {__half22float2(__ldg(reinterpret_cast<const __half2*>(p + a)))};
    return v2(__half2float(__ldg(p + a)), __half2float(__ldg(p + b)));
}
__device__ __forceinline__ V2 ld2(const __nv_bfloat16* p, int a, int b, bool vec) {
    if (vec) return {__bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p + a)))};
    return v2(__bfloat162float(__ldg(p + a)), __bfloat162float(__ldg(p + b)));
}
__device__ __forceinline__ V2 ld2(const float* p, int a, int b, bool vec) {
    if (vec) return {__ldg(reinterpret_cast<const float2*>(p + a))};
    return v2(__ldg(p + a), __ldg(p + b));
}
__device__ __forceinline__ Q2 ldq2(const uint2* q, int a, int b, bool vec) {
    uint2 ua, ub;
    if (vec) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(q + a));
        ua = make_uint2(u.x, u.y);
        ub = make_uint2(u.z, u.w);
    } else {
        ua = __ldg(q + a);
        ub = __ldg(q + b);
    }
    const Qf x = fref_unpack(ua), y = fref_unpack(ub);
    return {v2(x.A, y.A), v2(x.Jr, y.Jr), v2(x.Jz, y.Jz), v2(x.R, y.R)};
}

__device__ __forceinline__ void st2(__half* p, int a, V2 v, bool s0, bool s1, bool vec) {
    const __half2 h = __floats2half2_rn(v.v.x, v.v.y);
    if (vec && s0 && s1) {
        *reinterpret_cast<__half2*>(p + a) = h;
    } else {
        if (s0) p[a] = __low2half(h);
        if (s1) p[a + 1] = __high2half(h);
    }
}
__device__ __forceinline__ void st2(__nv_bfloat16* p, int a, V2 v, bool s0, bool s1, bool vec) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.v.x, v.v.y);
    if (vec && s0 && s1) {
        *reinterpret_cast<__nv_bfloat162*>(p + a) = h;
    } else {
        if (s0) p[a] = __low2bfloat16(h);
        if (s1) p[a + 1] = __high2bfloat16(h);
    }
}
__device__ __forceinline__ void st2(float* p, int a, V2 v, bool s0, bool s1, bool vec) {
    if (vec && s0 && s1) {
        *reinterpret_cast<float2*>(p + a) = v.v;
    } else {
        if (s0) p[a] = v.v.x;
        if (s1) p[a + 1] = v.v.y;
    }
}

// The rest of one row of a column pair once its sources are loaded: the flow reference
// added back (D_pop of each source's word; g_1 .. g_4 re-expressed against the node's own
// temperature reference), the recovery and collision, and the store with the own word's
// D_i removed.  qw(rs, cs): the two reference words of the sources in row kr - 1 + rs and
// columns (kz0 - 1, kz0), (kz0, kz0 + 1) or (kz0 + 1, kz0 + 2) for cs = 0, 1, 2.
template <int STO, bool VEC, class QW>
__device__ __forceinline__ void pair_finish(const Consts<float>& c, const Buf<STO>& B, int plane, int kr, int row,
                                            int kz0, int p1, int p5, int p8, V2 (&fh)[9], V2 (&gh)[5], V2 ph,
                                            const QW& qw, bool st0, bool st1) {
    // the reference words of the sources: the flow part D_pop of the pulled values and,
    // in their fourth slot, the temperature references R that re-express g_1 .. g_4
    // against the node's own R(x)
    const Q2 q0o = qw(1, 1);
    const V2 rref = q0o.R;
    {
        const Q2 qmo = qw(0, 1), qml = qw(0, 0), qmr = qw(0, 2);
        fh[1] += fref_delta2(p1, qmo);
        fh[5] += fref_delta2(p5, qml);
        fh[8] += fref_delta2(p8, qmr);
        gh[1] += 0.1f * (qmo.R - rref);
        const Q2 q0l = qw(1, 0), q0r = qw(1, 2);
        fh[0] += fref_delta2(0, q0o);
        fh[2] += fref_delta2(2, q0l);
        fh[4] += fref_delta2(4, q0r);
        gh[2] += 0.1f * (q0l.R - rref);
        gh[4] += 0.1f * (q0r.R - rref);
        const Q2 qpo = qw(2, 1), qpl = qw(2, 0), qpr = qw(2, 2);
        fh[3] += fref_delta2(3, qpo);
        fh[6] += fref_delta2(6, qpl);
        fh[7] += fref_delta2(7, qpr);
        gh[3] += 0.1f * (qpo.R - rref);
    }
    const RowC q = row_consts(c, kr);
    V2 lin, nl, iph, m0, rho, ur, uz, dT;
    porous2(c, ph, lin, nl, iph);
    recover2(c, q, ph, lin, nl, fh, gh, rref, m0, rho, ur, uz, dT);
    collide2(c, q, ph, lin, nl, iph, fh, gh, rref, m0, rho, ur, uz, dT);
    auto* __restrict__ Fo = B.f;
    float* __restrict__ Go = B.g;
#pragma unroll
    for (int i = 0; i < 9; ++i) fh[i] = fh[i] - fref_delta2(i, q0o);
    if (VEC && st0 && st1) {   // both lanes stored, aligned: one vector store per population
#pragma unroll
        for (int i = 0; i < 9; ++i) st2(Fo + i * plane, row + kz0, fh[i], true, true, true);
#pragma unroll
        for (int i = 0; i < 5; ++i) st2(Go + i * plane, row + kz0, gh[i], true, true, true);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) st2(Fo + i * plane, row + kz0, fh[i], st0, st1, false);
#pragma unroll
        for (int i = 0; i < 5; ++i) st2(Go + i * plane, row + kz0, gh[i], st0, st1, false);
    }
}

// Update rows kr0 .. kr0 + rows - 1 (non-wall rows below nr) of the column pair starting
// at the even column kz0.  VEC: nz is even, so every row's first element index is even
// and the own-column pairs are aligned for vector loads and stores.
template <int STO, bool VEC>
__device__ __forceinline__ void update_pair(const Consts<float>& c, const Buf<STO>& A, const Buf<STO>& B,
                                            const float* __restrict__ phi, int plane, int kr0, int rows, int kz0) {
    static_assert(has_fref<STO>(), "the packed pair update serves 16-bit storage");
    const int nz = c.nz;
    const bool pz = c.periodic != 0;
    // a lane past the last column, or on the end column of a closed geometry (a boundary
    // node), computes on clamped indices and is not stored
    const bool in1 = kz0 + 1 < nz;
    const bool st0 = pz || (kz0 > 0 && kz0 < nz - 1);   // (kz0 = nz - 1 when nz is odd)
    const bool st1 = in1 && (pz || kz0 + 1 < nz - 1);
    if (!st0 && !st1) return;
    const int zc1 = in1 ? kz0 + 1 : kz0;
    const int zm0 = kz0 > 0 ? kz0 - 1 : (pz ? nz - 1 : 0);          // e_z = +1 source, lane 0
    const int zp0 = in1 ? kz0 + 1 : (pz ? 0 : nz - 1);              // e_z = -1 source, lane 0
    const int zp1 = kz0 + 2 < nz ? kz0 + 2 : (pz ? kz0 + 2 - nz : nz - 1);   // e_z = -1, lane 1
    const bool row0_wall = c.geometry == ANNULUS || c.geometry == ANNULUS_PERIODIC_Z;
    const auto* __restrict__ F = A.f;
    const float* __restrict__ G = A.g;
    const uint2* __restrict__ Qp = c.fref;
#pragma unroll 1
    for (int j = 0; j < rows; ++j) {
        const int kr = kr0 + j;
        if (kr >= c.nr) break;
        if (kr == c.nr - 1 || (kr == 0 && row0_wall)) continue;
        const bool axis = kr == 0;   // pipe axis row: e_r = +1 sources are the mirror image
        const int row = kr * nz, rowp = row + nz, rowm = axis ? row : row - nz;
        const int p1 = axis ? 3 : 1, p5 = axis ? 6 : 5, p8 = axis ? 7 : 8;
        // own (kz0, zc1), left (zm0, kz0) and right (zp0, zp1) columns of a row
        V2 fh[9], gh[5];
        fh[0] = ld2(F, row + kz0, row + zc1, VEC);
        fh[1] = ld2(F + p1 * plane, rowm + kz0, rowm + zc1, VEC);
        fh[2] = ld2(F + 2 * plane, row + zm0, row + kz0, false);
        fh[3] = ld2(F + 3 * plane, rowp + kz0, rowp + zc1, VEC);
        fh[4] = ld2(F + 4 * plane, row + zp0, row + zp1, false);
        fh[5] = ld2(F + p5 * plane, rowm + zm0, rowm + kz0, false);
        fh[6] = ld2(F + 6 * plane, rowp + zm0, rowp + kz0, false);
        fh[7] = ld2(F + 7 * plane, rowp + zp0, rowp + zp1, false);
        fh[8] = ld2(F + p8 * plane, rowm + zp0, rowm + zp1, false);
        gh[0] = ld2(G, row + kz0, row + zc1, VEC);
        gh[1] = ld2(G + p1 * plane, rowm + kz0, rowm + zc1, VEC);
        gh[2] = ld2(G + 2 * plane, row + zm0, row + kz0, false);
        gh[3] = ld2(G + 3 * plane, rowp + kz0, rowp + zc1, VEC);
        gh[4] = ld2(G + 4 * plane, row + zp0, row + zp1, false);
        const V2 ph = ld2(phi, row + kz0, row + zc1, VEC);
        const auto qw = [&](int rs, int cs) {   // words of row kr - 1 + rs, columns left / own / right
            const int r = rs == 0 ? rowm : (rs == 1 ? row : rowp);
            if (cs == 1) return ldq2(Qp, r + kz0, r + zc1, VEC);
            if (cs == 0) return ldq2(Qp, r + zm0, r + kz0, false);
            return ldq2(Qp, r + zp0, r + zp1, false);
        };
        pair_finish<STO, VEC>(c, B, plane, kr, row, kz0, p1, p5, p8, fh, gh, ph, qw, st0, st1);
    }
}

// Reference word of a node from its post-collision deviations d_i = f+_i - rest_i
// (A = sum d_i, J = sum e_i d_i) and its temperature reference R: each rounded to FP16
// after clamping to its range (a clamped or otherwise inexact reference only stores
// larger values).
__device__ __forceinline__ uint2 fref_make(float A, float Jr, float Jz, __half R) {
    auto h = [](float x) { return __float2half_rn(fminf(fmaxf(x, -60000.0f), 60000.0f)); };
    return fref_pack(h(A), h(Jr), h(Jz), R);
}

// One thread per column segment of RPT rows: the column's index arithmetic, the
// kernel-argument loads and the class checks are shared by RPT nodes.
// I: index type; 32-bit when the state buffer holds fewer than 2^31 elements.
// Resident blocks of 128 threads per SM the register allocation must allow (0: no
// constraint).  16-bit flow storage is issue-bound: ten blocks (48 registers) beat the
// compiler's nine (measured 0.5303 vs 0.5425 ms at 4096 x 8192); FP32 is bandwidth-bound
// and does best with the compiler's own allocation (56 registers, 0.6079 ms; 0.6119 with
// nine blocks required, 0.6376 with ten).
// In place with 16-bit storage (one node per thread, shifted reads or stores): eight blocks
// (64 registers) measured 0.693 ms at 4096 x 8192 against 0.716 with nine and 0.737 with
// ten (48 registers, 36 bytes spilled).
#ifndef LBM_INPLACE16_MIN_BLOCKS
#define LBM_INPLACE16_MIN_BLOCKS 8
#endif
template <int STO, int LIN = LAY_N>
constexpr int bulk_min_blocks() { return STO == LBM_F32 ? 0 : (LIN == LAY_N ? 10 : LBM_INPLACE16_MIN_BLOCKS); }

template <int STO, typename I, int RPT, int LIN = LAY_N, int LOUT = LAY_N>
__global__ void __launch_bounds__(BULK_THREADS, bulk_min_blocks<STO, LIN>()) k_bulk(const Consts<float> c, const Buf<STO> A, const Buf<STO> B,
                                                       const typename St<STO>::P* __restrict__ phi, I plane) {
    const int kz = blockIdx.x * BULK_THREADS + threadIdx.x;
    if (kz >= c.nz) return;
    update_column<STO, I, LIN, LOUT>(c, A, B, phi, plane, blockIdx.y * RPT, RPT, kz);
}

// 16-bit storage: one column pair per thread (2 BULK_THREADS columns per block).
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 6
#endif
template <int STO, bool VEC, int RPT>
__global__ void __launch_bounds__(BULK_THREADS, LBM_PAIR_MIN_BLOCKS) k_bulk_pair(const Consts<float> c, const Buf<STO> A, const Buf<STO> B,
                                                            const float* __restrict__ phi, int plane) {
    const int kz0 = 2 * (blockIdx.x * BULK_THREADS + threadIdx.x);
    if (kz0 >= c.nz) return;
    update_pair<STO, VEC>(c, A, B, phi, plane, blockIdx.y * RPT, RPT, kz0);
}

// 16-bit storage, staged (even nz): a block of NT threads covers the columns [z0, z0 + 2 NT)
// of RPT rows.  For each row it needs one run of columns [a, b) = [z0 - 1, z0 + 2 NT + 1)
// (clipped to the row) of the source row of every population plane, the porosity of its
// own columns and the reference words of three rows.  Thread 0 copies each run into shared
// memory with a 1-D bulk copy (cp.async.bulk) of the 16-byte-aligned window around it
// (the window may take a few elements of the neighbouring row, never of another plane:
// planes are multiples of 64 elements), completion counted in bytes on an mbarrier per
// buffer; the next row's copies are in flight while the current row computes from the
// other buffer.  Reference words live in a ring of four rows (row mod 4; the pipe axis
// row's mirror row -1 holds row 0's words), so each row after the first copies one new
// row of them.  At a closed z end the clipped runs serve every stored lane (a lane on an
// end column is not stored, as in update_pair; it reads one column past the run, inside
// the shared block, and computes on whatever it finds there);
// blocks at a periodic z end run update_pair.  Every wait is bounded: a wait that runs
// out sets *status to LBM_ERR_TIMEOUT, and the block then waits (with the drain bound)
// for the copies it has in flight and stops.
constexpr int STAGE_SPIN = 1 << 22;   // try_wait rounds of one bounded wait (a few seconds)
template <int NT>
struct __align__(16) PairStage {
    static constexpr int F = 2 * NT + 16, G = 2 * NT + 8, Q = 2 * NT + 4, P = 2 * NT + 4;   // window capacities
    uint4 pad;                   // column -1 of the first window (read by an unstored lane) lands here
    unsigned short f[2][9][F];   // 16-bit flow sources, two rows in flight
    float g[2][5][G];            // thermal sources
    float ph[2][P];              // porosity of the own columns
    uint2 q[4][Q];               // reference words, ring over row mod 4
    unsigned long long bar[2];   // one mbarrier per buffer
};

// The 16-byte-aligned window of elements (U per 16 bytes, ES bytes each) around columns
// [a, b) of row R of a plane with row stride nz: its first element, the window index of
// column a, and its length in bytes.
struct Win {
    int start, off;
    uint32_t bytes;
};
template <int U, int ES>
__device__ __forceinline__ Win win(int R, int nz, int a, int b) {
    const int e0 = R * nz + a, s = e0 & -U, e1 = (R * nz + b + U - 1) & -U;
    return {s, e0 - s, (uint32_t)((e1 - s) * ES)};
}

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sm_addr(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Bounded wait for the completion of phase `phase` of an mbarrier.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t phase, int spin) {
    for (int i = 0; i < spin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ V2 h16x2(uint32_t w, const __half*) {
    return {__half22float2(*reinterpret_cast<const __half2*>(&w))};
}
__device__ __forceinline__ V2 h16x2(uint32_t w, const __nv_bfloat16*) {
    return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w))};
}
__device__ __forceinline__ float h16(unsigned short u, const __half*) { return __half2float(__ushort_as_half(u)); }
__device__ __forceinline__ float h16(unsigned short u, const __nv_bfloat16*) {
    return __bfloat162float(__ushort_as_bfloat16(u));
}
__device__ __forceinline__ Q2 q2_of(uint2 ua, uint2 ub) {
    const Qf x = fref_unpack(ua), y = fref_unpack(ub);
    return {v2(x.A, y.A), v2(x.Jr, y.Jr), v2(x.Jz, y.Jz), v2(x.R, y.R)};
}

// One staged block: rows r0 .. r0 + RPT - 1 (at most), columns z0 .. z0 + 2 NT - 1 (see above).
// spin: try_wait rounds of the per-row waits (the final drain always uses STAGE_SPIN).
// ALN: nz is a multiple of 8 and the blocks at both z ends run update_pair, so every staged
// block starts its runs at column z0 - 1 = 7 mod 8 of a row that starts 16-byte aligned
// (the window index of each column is a constant offset from it) and stores both lanes of
// every thread.
template <int STO, int NT, bool ALN>
__device__ __forceinline__ void stage_block(const Consts<float>& c, const Buf<STO>& A, const Buf<STO>& B,
                                            const float* __restrict__ phi, int plane, int r0, int RPT, int z0,
                                            int spin, int* __restrict__ status, PairStage<NT>& sb) {
    using TF = typename St<STO>::TF;
    const int nz = c.nz, t = threadIdx.x, kz0 = z0 + 2 * t;
    if (nz & 1) {   // launched for even nz only: the pair reads below assume it
        if (t == 0) atomicExch(status, LBM_ERR_INVALID);
        return;
    }
    if ((ALN && (z0 == 0 || z0 + 2 * NT + 8 > nz)) || (c.periodic && (z0 == 0 || z0 + 2 * NT >= nz))) {   // global loads
        if (kz0 < nz) update_pair<STO, true>(c, A, B, phi, plane, r0, RPT, kz0);
        return;
    }
    const bool row0_wall = c.geometry == ANNULUS || c.geometry == ANNULUS_PERIODIC_Z;
    const auto computes = [&](int kr) { return kr < c.nr - 1 && (kr > 0 || !row0_wall); };
    const TF* __restrict__ F = A.f;
    const float* __restrict__ G = A.g;
    const uint2* __restrict__ Qp = c.fref;
    const int rows = min(RPT, c.nr - r0);
    const int a = ALN ? z0 - 1 : max(z0 - 1, 0);   // first column of the runs; they end at min(z0 + 2 NT + 1, nz)
    const uint32_t bar0 = sm_addr(&sb.bar[0]), bar1 = sm_addr(&sb.bar[1]);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // thread 0: copy the sources of row r0 + j into buffer j & 1, and the reference words
    // it needs first (rows kr - 1 .. kr + 1 for the first row, then row kr + 1)
    const auto issue = [&](int j) {
        const int kr = r0 + j, bf = j & 1;
        const uint32_t bar = bf ? bar1 : bar0;
        const int q_lo = j == 0 ? kr - 1 : kr + 1, q_hi = min(kr + 1, c.nr - 1);
        const bool axis = kr == 0 && !row0_wall;   // pipe axis: row -1 mirrors row 0
        const bool comp = computes(kr);
        const int Rm = axis ? kr : kr - 1, b = min(z0 + 2 * NT + 1, nz), pb = min(z0 + 2 * NT, nz);
        const Win wf[3] = {win<8, 2>(Rm, nz, a, b), win<8, 2>(kr, nz, a, b), win<8, 2>(kr + 1, nz, a, b)};
        const Win wg[3] = {win<4, 4>(Rm, nz, a, b), win<4, 4>(kr, nz, a, b), win<4, 4>(kr + 1, nz, a, b)};
        const Win wp = win<4, 4>(kr, nz, z0, pb);
        uint32_t bytes = 0;
        if (comp)   // three flow slots per row group; thermal slots 0, 2, 4 in row kr, 1 and 3 in the others
            bytes = 3 * (wf[0].bytes + wf[1].bytes + wf[2].bytes) + 3 * wg[1].bytes + wg[0].bytes + wg[2].bytes +
                    wp.bytes;
        for (int qr = q_lo; qr <= q_hi; ++qr)
            if (qr >= 0 || axis) bytes += win<2, 8>(max(qr, 0), nz, a, b).bytes;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // after the reads of the buffer's last use
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        if (comp) {
            const int p1 = axis ? 3 : 1, p5 = axis ? 6 : 5, p8 = axis ? 7 : 8;
            // flow slot i: plane and row group (0: row kr - 1 or its mirror, 1: kr, 2: kr + 1)
            const int fpl[9] = {0, p1, 2, 3, 4, p5, 6, 7, p8};
            const int frg[9] = {1, 0, 1, 2, 1, 0, 2, 2, 0};
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const Win& w = wf[frg[i]];
                bulk_copy(sb.f[bf][i], F + fpl[i] * plane + w.start, w.bytes, bar);
            }
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const Win& w = wg[frg[i]];
                bulk_copy(sb.g[bf][i], G + fpl[i] * plane + w.start, w.bytes, bar);
            }
            bulk_copy(sb.ph[bf], phi + wp.start, wp.bytes, bar);
        }
        for (int qr = q_lo; qr <= q_hi; ++qr)
            if (qr >= 0 || axis) {
                const Win w = win<2, 8>(max(qr, 0), nz, a, b);
                bulk_copy(sb.q[qr & 3], Qp + w.start, w.bytes, bar);
            }
    };
    if (t == 0) issue(0);
    const bool active = ALN || kz0 < nz;
    bool ok = true;
#pragma unroll 1
    for (int j = 0; j < rows; ++j) {
        if (t == 0 && j + 1 < rows) issue(j + 1);
        const int kr = r0 + j, bf = j & 1;
        ok = bar_wait(bf ? bar1 : bar0, (j >> 1) & 1, spin);
        if (active && computes(kr)) {
            const bool axis = kr == 0;
            const int p1 = axis ? 3 : 1, p5 = axis ? 6 : 5, p8 = axis ? 7 : 8;
            const int Rm = axis ? kr : kr - 1;
            // window index of the own column kz0 in row group rg (the left column is one
            // below, the right columns one and two above)
            const auto wo = [&](int R, int U) { return kz0 - a + (ALN ? U - 1 : ((R * nz + a) & (U - 1))); };
            const int of[3] = {wo(Rm, 8), wo(kr, 8), wo(kr + 1, 8)};
            const int og[3] = {wo(Rm, 4), wo(kr, 4), wo(kr + 1, 4)};
            const auto own = [&](int i, int rg) {
                return h16x2(*reinterpret_cast<const uint32_t*>(&sb.f[bf][i][of[rg]]), F);
            };
            const auto fat = [&](int i, int rg, int d) {   // columns kz0 + d, kz0 + d + 1
                return v2(h16(sb.f[bf][i][of[rg] + d], F), h16(sb.f[bf][i][of[rg] + d + 1], F));
            };
            const auto gown = [&](int i, int rg) { return V2{*reinterpret_cast<const float2*>(&sb.g[bf][i][og[rg]])}; };
            const auto gat = [&](int i, int rg, int d) {
                return v2(sb.g[bf][i][og[rg] + d], sb.g[bf][i][og[rg] + d + 1]);
            };
            V2 fh[9], gh[5];
            fh[0] = own(0, 1);
            fh[1] = own(1, 0);
            fh[2] = fat(2, 1, -1);
            fh[3] = own(3, 2);
            fh[4] = fat(4, 1, 1);
            fh[5] = fat(5, 0, -1);
            fh[6] = fat(6, 2, -1);
            fh[7] = fat(7, 2, 1);
            fh[8] = fat(8, 0, 1);
            gh[0] = gown(0, 1);
            gh[1] = gown(1, 0);
            gh[2] = gat(2, 1, -1);
            gh[3] = gown(3, 2);
            gh[4] = gat(4, 1, 1);
            const V2 ph{*reinterpret_cast<const float2*>(&sb.ph[bf][kz0 - z0 + (ALN ? 0 : (kr * nz + z0) & 3)])};
            const auto qw = [&](int rs, int cs) {
                const int qr = kr - 1 + rs;
                const uint2* q = sb.q[qr & 3];
                const int o = kz0 - a + (ALN ? 1 : ((max(qr, 0) * nz + a) & 1));
                const uint4 u = *reinterpret_cast<const uint4*>(q + o);   // the own pair's two words
                if (cs == 1) return q2_of(make_uint2(u.x, u.y), make_uint2(u.z, u.w));
                if (cs == 0) return q2_of(q[o - 1], make_uint2(u.x, u.y));
                return q2_of(make_uint2(u.z, u.w), q[o + 2]);
            };
            const bool st0 = ALN || kz0 > 0 || c.periodic, st1 = ALN || kz0 + 1 < nz - 1 || c.periodic;
            pair_finish<STO, true>(c, B, plane, kr, kr * nz, kz0, p1, p5, p8, fh, gh, ph, qw, st0, st1);
        }
        if (__syncthreads_or(!ok)) {   // a wait ran out: drain what is in flight and stop
            if (t == 0) {
                atomicExch(status, LBM_ERR_TIMEOUT);
                bar_wait(bf ? bar1 : bar0, (j >> 1) & 1, STAGE_SPIN);
                if (j + 1 < rows) bar_wait(bf ? bar0 : bar1, ((j + 1) >> 1) & 1, STAGE_SPIN);
            }
            return;
        }
    }
}

#ifndef LBM_STAGE_MIN_BLOCKS
#define LBM_STAGE_MIN_BLOCKS 6
#endif
template <int STO, int RPT, bool ALN>
__global__ void __launch_bounds__(BULK_THREADS, LBM_STAGE_MIN_BLOCKS) k_bulk_stage(const Consts<float> c, const Buf<STO> A, const Buf<STO> B,
                                                             const float* __restrict__ phi, int plane, int spin,
                                                             int* __restrict__ status) {
    __shared__ PairStage<BULK_THREADS> sb;
    stage_block<STO, BULK_THREADS, ALN>(c, A, B, phi, plane, blockIdx.y * RPT, RPT, blockIdx.x * 2 * BULK_THREADS, spin,
                                        status, sb);
}

// The staged kernel keeps sizeof(PairStage<BULK_THREADS>) (30.7 KB) of shared memory per
// block; at LBM_STAGE_MIN_BLOCKS blocks per SM that needs the largest shared-memory carveout.
template <int STO>
static cudaError_t stage_carveout() {
    cudaError_t e = cudaFuncSetAttribute(k_bulk_stage<STO, BULK_RPT, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bulk_stage<STO, BULK_RPT, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

// Wall nodes; LIN / LOUT: layouts read and written (in-place storage alternates S and L).
template <int STO, int LIN = LAY_N, int LOUT = LAY_N>
__global__ void k_wall(const Consts<float> c, const Buf<STO> A,
                       const Buf<STO> B, const typename St<STO>::P* __restrict__ phi,
                       int64_t plane, int count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int kr, kz;
    wall_node(c.geometry, c.nr, c.nz, t, kr, kz);
    const int cls = node_class(c.geometry, c.nr, c.nz, kr, kz);
    float fh[9], gh[5], m0, rho, urb, uzb, dTb, refb;
    wall_state<STO, float, LIN>(c, A, phi, plane, cls, kr, kz, fh, gh, m0, rho, urb, uzb, dTb, refb);
    const int64_t n = (int64_t)kr * c.nz + kz;
    const float r = c.r0 + float(kr), ph = ldv(phi + n);
    float lin, nl, iph;
    porous(c, ph, lin, nl, iph);
    collide(c, r, rcp_acc(r), ph, lin, nl, iph, fh, gh, refb, m0, rho, urb, uzb, dTb);
    store<STO, float, int64_t, LOUT>(c, B, plane, kr, kz, n, fh, gh);
}

// Fields of a state at every node (NULL outputs skipped).
template <int STO, int LAY = LAY_N>
__global__ void k_moments(const Consts<float> c, const Buf<STO> A,
                          const typename St<STO>::P* __restrict__ phi, int64_t plane, float* rho_o, float* ur_o,
                          float* uz_o, float* T_o) {
    const int kz = blockIdx.x * blockDim.x + threadIdx.x;
    const int kr = blockIdx.y;
    if (kz >= c.nz) return;
    const int cls = node_class(c.geometry, c.nr, c.nz, kr, kz);
    const int64_t n = (int64_t)kr * c.nz + kz;
    float fh[9], gh[5], m0, rho, ur = 0.f, uz = 0.f, dT, ref;
    if (is_wall(cls)) {
        wall_state<STO, float, LAY>(c, A, phi, plane, cls, kr, kz, fh, gh, m0, rho, ur, uz, dT, ref);
    } else {
        pull<STO, float, int64_t, LAY>(c, A, plane, kr, kz, fh, gh, ref);
        const float r = c.r0 + float(kr), ph = ldv(phi + n);
        float lin, nl, iph;
        porous(c, ph, lin, nl, iph);
        recover(c, r, rcp_acc(r), ph, lin, nl, fh, gh, ref, m0, rho, ur, uz, dT);
    }
    if (rho_o) rho_o[n] = rho;
    if (ur_o) ur_o[n] = ur;
    if (uz_o) uz_o[n] = uz;
    if (T_o) T_o[n] = (c.T0 + ref) + dT;
}

// Start state (FP64 arithmetic, one launch per initialisation): pre-collision
// f = M^-1(m_eq - S/2) at rho = 1 (Eq. 19-20, 24), g = g_eq(T, u) (Eq. 35), then one
// collision at the node.  Cold start: T = T0 + noise * U(-1, 1) from SplitMix64.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double start_T(const Consts<double>& c, const float* T_in, double noise, uint64_t seed,
                                          int64_t n) {
    if (T_in) return (double)T_in[n];
    const double u01 = (double)(splitmix64(seed, (uint64_t)n) >> 11) * (1.0 / 9007199254740992.0);
    return c.T0 + noise * (2 * u01 - 1);
}

template <int STO>
__global__ void k_init(const Consts<double> c, const Buf<STO> B,
                       const typename St<STO>::P* __restrict__ phi, int64_t plane, const float* ur_in,
                       const float* uz_in, const float* T_in, double noise, uint64_t seed, __half* __restrict__ tref,
                       uint2* __restrict__ fref, int inplace) {
    const int kz = blockIdx.x * blockDim.x + threadIdx.x;
    const int kr = blockIdx.y;
    if (kz >= c.nz) return;
    const int64_t n = (int64_t)kr * c.nz + kz;
    const int cls = node_class(c.geometry, c.nr, c.nz, kr, kz);
    const double r = c.r0 + kr, inv_r = 1.0 / r;
    double T = start_T(c, T_in, noise, seed, n), ur = 0, uz = 0;
    if (cls == WALL_IN && c.heater) {
        int fr, fz;
        fluid_neighbour(c.geometry, c.nr, c.nz, cls, kr, kz, fr, fz);
        T = start_T(c, T_in, noise, seed, (int64_t)fr * c.nz + fz);
    } else if (cls == WALL_IN) T = c.T_hot;
    else if (cls == WALL_OUT) T = c.T_cold;
    else if (cls == INLET) {
        T = c.T_hot;
        uz = c.u_in;
    } else if (cls == BOTTOM || cls == TOP || cls == OUTLET) {
        int fr, fz;
        fluid_neighbour(c.geometry, c.nr, c.nz, cls, kr, kz, fr, fz);
        T = start_T(c, T_in, noise, seed, (int64_t)fr * c.nz + fz);
    } else if (ur_in && uz_in) {
        ur = ur_in[n];
        uz = uz_in[n];
    }
    const double ph = (double)ldv(phi + n);
    double lin, nl, iphi;
    porous(c, ph, lin, nl, iphi);
    const double um = sqrt(ur * ur + uz * uz);
    const double Fr = -ph * (lin + nl * um) * ur;
    const double Ftr = Fr + cs2<double>() * (1 - c.two_taum * ur * inv_r) * inv_r;
    const double Ftz = -ph * (lin + nl * um) * uz + ph * (c.gbeta * (T - c.T0) + c.az);
    const double u2 = ur * ur + uz * uz;
    // deviation moments of f = M^-1 (m_eq - S/2) at rho = 1 (S_3 without its rest c_s^2)
    const double S1 = 6 * r * (ur * Ftr + uz * Ftz) * iphi, S5 = r * Ftz;
    const double S3 = r * Fr - cs2<double>() * c.two_taum * ur * inv_r;
    const double S7 = 2 * r * (ur * Ftr - uz * Ftz) * iphi, S8 = r * (ur * Ftz + uz * Ftr) * iphi;
    const double q = 3 * r * u2 * iphi;
    const double mpre[9] = {0.0,
                            q - 0.5 * S1,
                            -q + 0.5 * S1,
                            r * ur - 0.5 * S3,
                            -r * ur + 0.5 * S3,
                            r * uz - 0.5 * S5,
                            -r * uz + 0.5 * S5,
                            r * (ur * ur - uz * uz) * iphi - 0.5 * S7,
                            r * ur * uz * iphi - 0.5 * S8};
    double fh[9], gh[5];
    minv(mpre, fh);
    // reference offset R(x) = T - T0 in FP16; gh relative to T0 + R(x)
    const __half Rh = __float2half_rn(fminf(fmaxf((float)(T - c.T0), -60000.f), 60000.f));
    if constexpr (!has_fref<STO>()) tref[n] = Rh;
    const double ref = (double)__half2float(Rh);
    const double dTs = T - c.T0 - ref;
    gh[0] = 0.6 * dTs;
    gh[1] = 0.1 * dTs + 0.5 * T * ur;
    gh[2] = 0.1 * dTs + 0.5 * T * uz;
    gh[3] = 0.1 * dTs - 0.5 * T * ur;
    gh[4] = 0.1 * dTs - 0.5 * T * uz;
    double m0, rho, u_r = ur, u_z = uz, dT;   // boundary nodes keep their start velocity
    if (is_wall(cls)) {
        m0 = ((fh[0] + fh[1]) + (fh[2] + fh[3])) + ((fh[4] + fh[5]) + (fh[6] + fh[7])) + fh[8];
        rho = 1 + m0 * inv_r;
        dT = dTs;
    } else {
        recover(c, r, inv_r, ph, lin, nl, fh, gh, ref, m0, rho, u_r, u_z, dT);
    }
    collide(c, r, inv_r, ph, lin, nl, iphi, fh, gh, ref, m0, rho, u_r, u_z, dT);
    if constexpr (has_fref<STO>()) {
        // the start state's own flow reference: the moments of its deviations
        double A = 0, Jr = 0, Jz = 0;
        for (int i = 0; i < 9; ++i) {
            A += fh[i];
            Jr += ex9(i) * fh[i];
            Jz += ez9(i) * fh[i];
        }
        const uint2 qw = fref_make((float)A, (float)Jr, (float)Jz, Rh);
        fref[n] = qw;
        const Qf q = fref_unpack(qw);
        for (int i = 0; i < 9; ++i)
            stv(B.f + (inplace ? opp9(i) : i) * plane + n, (float)(fh[i] - (double)fref_delta(i, q)));
    } else {
        for (int i = 0; i < 9; ++i) stv(B.f + (inplace ? opp9(i) : i) * plane + n, (float)fh[i]);
    }
    // in-place storage starts in layout S: population i in slot opp(i) of its own node
    for (int i = 0; i < 5; ++i) stv(B.g + (inplace ? opp9(i) : i) * plane + n, (float)gh[i]);
}

template <int STO> __device__ __forceinline__ typename St<STO>::P mkp(float v);
template <> __device__ __forceinline__ float mkp<LBM_F32>(float v) { return v; }
template <> __device__ __forceinline__ float mkp<LBM_F16>(float v) { return v; }
template <> __device__ __forceinline__ float mkp<LBM_BF16>(float v) { return v; }

// Porosity upload: validate (0 < phi <= 1) and convert to the storage type.
__device__ __forceinline__ unsigned int bad_phi(float v) { return !(v > 0.f && v <= 1.f); }

// Porosity upload: count of values outside (0, 1] and conversion to the storage type.
// Grid-stride; 16-byte loads when src is 16-byte aligned (vec != 0), then the ragged tail
// one value at a time.
template <int STO>
__global__ void k_phi(const float* __restrict__ src, typename St<STO>::P* __restrict__ dst, int64_t n, int vec,
                      unsigned int* bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = vec ? n / 4 : 0;
    unsigned int cnt = 0;
    for (int64_t q = t; q < n4; q += stride) {
        const float4 v = reinterpret_cast<const float4*>(src)[q];
        cnt += bad_phi(v.x) + bad_phi(v.y) + bad_phi(v.z) + bad_phi(v.w);
        dst[4 * q] = mkp<STO>(v.x);
        dst[4 * q + 1] = mkp<STO>(v.y);
        dst[4 * q + 2] = mkp<STO>(v.z);
        dst[4 * q + 3] = mkp<STO>(v.w);
    }
    for (int64_t i = 4 * n4 + t; i < n; i += stride) {
        const float v = src[i];
        cnt += bad_phi(v);
        dst[i] = mkp<STO>(v);
    }
    if (cnt) atomicAdd(bad, cnt);
}

// Two result values written into mapped host memory by the kernel itself (no copy-engine
// transfer for 16 bytes).
__global__ void k_put2(const double* __restrict__ src, double* dst, int skip_first) {
    const int i = threadIdx.x;
    if (i < 2 && !(skip_first && i == 0)) dst[i] = src[i];
}

// Range check alone (FP32 storage: the checked staging buffer becomes the field); src is a
// staging buffer (cudaMalloc, 16-byte aligned).
__global__ void k_phi_check(const float* __restrict__ src, int64_t n, unsigned int* bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n / 4;
    unsigned int cnt = 0;
    for (int64_t q = t; q < n4; q += stride) {
        const float4 v = reinterpret_cast<const float4*>(src)[q];
        cnt += bad_phi(v.x) + bad_phi(v.y) + bad_phi(v.z) + bad_phi(v.w);
    }
    for (int64_t i = 4 * n4 + t; i < n; i += stride) cnt += bad_phi(src[i]);
    if (cnt) atomicAdd(bad, cnt);
}

// Blocks of 256 threads for the grid-stride porosity kernels over n values.
static unsigned int phi_blocks(int64_t n) {
    return (unsigned int)std::max<int64_t>(1, std::min<int64_t>((n / 4 + 255) / 256, 4096));
}

static int aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

template <int STO>
__global__ void k_phi_fill(typename St<STO>::P* __restrict__ dst, int64_t n, float v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = mkp<STO>(v);
}

__global__ void k_node_class(int geometry, int nr, int nz, uint8_t* out) {
    const int kz = blockIdx.x * blockDim.x + threadIdx.x;
    const int kr = blockIdx.y;
    if (kz < nz) out[(int64_t)kr * nz + kz] = (uint8_t)node_class(geometry, nr, nz, kr, kz);
}

// ----------------------------------------------------- FP64 reductions --
// Block sum of NV doubles per thread (warp shuffles, then shared memory).
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* out_if_thread0) {
    __shared__ double sh[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    if (lane == 0)
        for (int j = 0; j < NV; ++j) sh[warp][j] = v[j];
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double x = lane < nw ? sh[lane][j] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out_if_thread0[j] = x;
        }
    }
}

// Residual partials over nodes: |du|^2, |u|^2, dT^2, T^2 on non-wall nodes, mass
// r * rho on all nodes, and a count of non-finite values; one row of 6 per block.
constexpr int RES_NV = 6;
__global__ void k_resid_partial(int geometry, int nr, int nz, double r0, const float* __restrict__ cur,
                                const float* __restrict__ prev, int64_t fstride, double* __restrict__ partials) {
    double v[RES_NV] = {0, 0, 0, 0, 0, 0};
    const int64_t N = (int64_t)nr * nz;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int kr = (int)(n / nz), kz = (int)(n - (int64_t)kr * nz);
        const float rho = cur[n], ur = cur[fstride + n], uz = cur[2 * fstride + n], T = cur[3 * fstride + n];
        if (!isfinite(rho) || !isfinite(ur) || !isfinite(uz) || !isfinite(T)) v[5] += 1;
        v[4] += (r0 + kr) * (double)rho;
        if (is_wall(node_class(geometry, nr, nz, kr, kz))) continue;
        const double a = (double)ur - prev[fstride + n], b = (double)uz - prev[2 * fstride + n];
        const double d = (double)T - prev[3 * fstride + n];
        v[0] += a * a + b * b;
        v[1] += (double)ur * ur + (double)uz * uz;
        v[2] += d * d;
        v[3] += (double)T * T;
    }
    double out[RES_NV];
    block_sum<RES_NV>(v, out);
    if (threadIdx.x == 0)
        for (int j = 0; j < RES_NV; ++j) partials[blockIdx.x * RES_NV + j] = out[j];
}

__global__ void k_sum_rows(const double* __restrict__ partials, int rows, double* __restrict__ result) {
    double v[RES_NV] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < rows; b += blockDim.x)
        for (int j = 0; j < RES_NV; ++j) v[j] += partials[b * RES_NV + j];
    double out[RES_NV];
    block_sum<RES_NV>(v, out);
    if (threadIdx.x == 0)
        for (int j = 0; j < RES_NV; ++j) result[j] = out[j];
}

// Temperature of node (kr, kz) of a state: wall temperature, the interior
// neighbour's T on adiabatic walls, else sum of the pulled g (Eq. 38), in FP64.
template <int STO, int LAY = LAY_N>
__device__ double node_T(const Consts<float>& c, const Buf<STO> A, int64_t plane, int kr,
                         int kz) {
    const int cls = node_class(c.geometry, c.nr, c.nz, kr, kz);
    if (cls == WALL_IN || cls == INLET) return (double)c.T_hot;
    if (cls == WALL_OUT) return (double)c.T_cold;
    if (cls == BOTTOM || cls == TOP || cls == OUTLET) {
        int fr, fz;
        fluid_neighbour(c.geometry, c.nr, c.nz, cls, kr, kz, fr, fz);
        kr = fr;
        kz = fz;
    }
    float fh[9], gh[5], ref;
    pull<STO, float, int64_t, LAY>(c, A, plane, kr, kz, fh, gh, ref);
    return (double)c.T0 + (double)ref + (((double)gh[0] + gh[1]) + ((double)gh[2] + gh[3]) + gh[4]);
}

// Eq. 42 for both walls: one-sided second-order dT/dr, trapezoid in z.  One column per
// thread, a partial sum per block; k_nusselt_final adds the partials in block order.
template <int STO, int LAY = LAY_N>
__global__ void __launch_bounds__(128) k_nusselt(const Consts<float> c, const Buf<STO> A, int64_t plane,
                                                 double* __restrict__ partials) {
    double v[2] = {0, 0};
    for (int kz = blockIdx.x * blockDim.x + threadIdx.x; kz < c.nz; kz += gridDim.x * blockDim.x) {
        const double wz = (kz == 0 || kz == c.nz - 1) ? 0.5 : 1.0;
        const double t0 = node_T<STO, LAY>(c, A, plane, 0, kz), t1 = node_T<STO, LAY>(c, A, plane, 1, kz);
        const double t2 = node_T<STO, LAY>(c, A, plane, 2, kz);
        const double u0 = node_T<STO, LAY>(c, A, plane, c.nr - 1, kz);
        const double u1 = node_T<STO, LAY>(c, A, plane, c.nr - 2, kz);
        const double u2 = node_T<STO, LAY>(c, A, plane, c.nr - 3, kz);
        v[0] += wz * (-3 * t0 + 4 * t1 - t2) * 0.5;
        v[1] += wz * (3 * u0 - 4 * u1 + u2) * 0.5;
    }
    double out[2];
    block_sum<2>(v, out);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = out[0];
        partials[2 * blockIdx.x + 1] = out[1];
    }
}

__global__ void __launch_bounds__(256) k_nusselt_final(const double* __restrict__ partials, int blocks, double ri,
                                                       double ro, double H, double dTw, double* __restrict__ result) {
    double v[2] = {0, 0};
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
        v[0] += partials[2 * b];
        v[1] += partials[2 * b + 1];
    }
    double out[2];
    block_sum<2>(v, out);
    if (threadIdx.x == 0) {
        result[0] = -ri * out[0] / (H * dTw);
        result[1] = -ro * out[1] / (H * dTw);
    }
}

// Eq. 40 per column for the pipe with inlet and outlet: Nu(z) = D (dT/dr)_w / (T_w - T_b)
// with the mixing-cup T_b = int u_z r T dr / int u_z r dr (trapezoid on r = 0, r0, r0 + 1,
// ..., r_i; the integrand is 0 at r = 0) and the one-sided second-order wall derivative.
// uz, T: field planes (row stride nz).  One thread per column, FP64.
__global__ void k_pipe_nusselt(int nr, int nz, double r0, const float* __restrict__ uz, const float* __restrict__ T,
                               double* __restrict__ nu) {
    const int kz = blockIdx.x * blockDim.x + threadIdx.x;
    if (kz >= nz) return;
    double num = 0.25 * (r0 * (double)uz[kz] * (double)T[kz]), den = 0.25 * (r0 * (double)uz[kz]);
    for (int k = 0; k + 1 < nr; ++k) {
        const int64_t a = (int64_t)k * nz + kz, b = a + nz;
        const double ra = r0 + k, rb = r0 + k + 1;
        num += 0.5 * (ra * (double)uz[a] * (double)T[a] + rb * (double)uz[b] * (double)T[b]);
        den += 0.5 * (ra * (double)uz[a] + rb * (double)uz[b]);
    }
    const double Tw = T[(int64_t)(nr - 1) * nz + kz];
    const double dTdr = (3 * Tw - 4 * (double)T[(int64_t)(nr - 2) * nz + kz] + (double)T[(int64_t)(nr - 3) * nz + kz]) / 2;
    nu[kz] = 2 * (r0 + (nr - 1)) * dTdr / (Tw - num / den);
}

// Eq. 43-44 for the discrete heater: Nu(z) = dT / (T_h(z) - T_o) at the heated inner-wall
// columns hz0..hz1 (corners excluded unless z is periodic), NaN elsewhere, and the mean
// over the heated columns.  Th: the inner-wall row of the T field.  One block, FP64.
__global__ void __launch_bounds__(256) k_heater_nusselt(int nz, int hz0, int hz1, int periodic, double dT, double To,
                                                        const float* __restrict__ Th, double* __restrict__ nu_z,
                                                        double* __restrict__ result) {
    double v[2] = {0, 0};
    for (int kz = threadIdx.x; kz < nz; kz += blockDim.x) {
        const bool heated = kz >= hz0 && kz <= hz1 && (periodic || (kz > 0 && kz < nz - 1));
        const double nu = heated ? dT / ((double)Th[kz] - To) : NAN;
        nu_z[kz] = nu;
        if (heated) {
            v[0] += nu;
            v[1] += 1;
        }
    }
    double out[2];
    block_sum<2>(v, out);
    if (threadIdx.x == 0) result[0] = out[1] > 0 ? out[0] / out[1] : NAN;
}

// Stokes stream function of the axisymmetric flow (|psi|max of Table 3):
// psi(r, z) = int_{r_s}^{r} r' u_z dr' so that r u_z = d psi/dr and, by Eq. 1,
// r u_r = -d psi/dz; r_s is the inner wall (annulus) or the axis (pipes, whose first
// panel runs from r = 0 to the first row at r0).  One thread per column walks the rows
// (each row's read is coalesced across the block), accumulating in FP64; every block
// writes the largest |psi| of its columns to block_max[blockIdx.x].
__global__ void __launch_bounds__(128) k_stream_function(int nr, int nz, double r0, int from_axis,
                                                         const float* __restrict__ uz, float* __restrict__ psi,
                                                         double* __restrict__ block_max) {
    const int kz = blockIdx.x * blockDim.x + threadIdx.x;
    double big = 0;
    if (kz < nz) {
        double prev = r0 * (double)uz[kz];
        double s = from_axis ? 0.5 * r0 * prev : 0.0;
        psi[kz] = (float)s;
        big = fabs(s);
        for (int k = 1; k < nr; ++k) {
            const int64_t n = (int64_t)k * nz + kz;
            const double cur = (r0 + k) * (double)uz[n];
            s += 0.5 * (prev + cur);
            prev = cur;
            psi[n] = (float)s;
            big = fmax(big, fabs(s));
        }
    }
    for (int o = 16; o > 0; o >>= 1) big = fmax(big, __shfl_down_sync(0xffffffffu, big, o));
    __shared__ double sh[4];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = big;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w) big = fmax(big, sh[w]);
        block_max[blockIdx.x] = big;
    }
}

// FP64 export of rows [row0, row0 + nrows): raw post-collision populations
// f_i = ft_i + r w_i + e_ir w_i / 2, g_i = gh_i + wT_i (T0 + R(x)), from the state in layout
// LAY (NaN for a population that layout does not keep).
template <int STO, int LAY = LAY_N>
__global__ void k_export(const Consts<float> c, const Buf<STO> A, int64_t plane, int row0,
                         int nrows, double r0, double T0, double* __restrict__ out) {
    const int kz = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (kz >= c.nz || j >= nrows) return;
    const int kr = row0 + j;
    const int64_t n = (int64_t)kr * c.nz + kz, m = (int64_t)j * c.nz + kz, P = (int64_t)nrows * c.nz;
    const double r = r0 + kr;
    const double wt[5] = {0.6, 0.1, 0.1, 0.1, 0.1};
    const double Tb = T0 + (double)tref_at<STO>(c, n);
    for (int i = 0; i < 9; ++i) {
        int64_t at;
        int slot;
        if (!own_slot<LAY, float, int64_t>(c, kr, kz, i, at, slot)) {
            out[i * P + m] = NAN;
            if (i < 5) out[(9 + i) * P + m] = NAN;
            continue;
        }
        double ref = 0.0;
        if constexpr (has_fref<STO>()) ref = (double)fref_delta(i, fref_unpack(c.fref[n]));
        out[i * P + m] = (double)ldv(A.f + slot * plane + at) + ref + (r + 0.5 * ex9(i)) * w9<double>(i);
        if (i < 5) out[(9 + i) * P + m] = (double)ldv(A.g + slot * plane + at) + wt[i] * Tb;
    }
}

// Reference refresh: R(x) <- FP16(R(x) + sum_i gh_i(x)), gh re-expressed against the
// new reference (gh_0 += d - 4 d/10, gh_1..4 += d/10 with d = R_old - R_new).  The
// populations, and every field they give, are unchanged up to rounding.
// Node (kr, kz) = n, state in layout LAY: the locations of its own populations (own_slot);
// a population the layout does not keep counts as a zero deviation (any R is a valid one).
template <int STO, int LAY, typename I>
__device__ __forceinline__ void rebase_thermal_node(const Consts<float>& c, const Buf<STO>& A, I plane, int kr,
                                                    int kz, I n, __half* __restrict__ tref) {
    float g[5];
    I at[5];
    int slot[5];
    bool kept[5], all = true;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        kept[i] = own_slot<LAY, float, I>(c, kr, kz, i, at[i], slot[i]);
        all = all && kept[i];
        g[i] = kept[i] ? ldv(A.g + slot[i] * plane + at[i]) : 0.f;
    }
    // a boundary node whose outgoing populations the layout dropped keeps its reference
    // (the kept ones do not sum to its temperature)
    if (!all) return;
    const float r_old = __half2float(tref[n]);
    const float t = r_old + (((g[0] + g[1]) + (g[2] + g[3])) + g[4]);
    const __half h = __float2half_rn(fminf(fmaxf(t, -60000.f), 60000.f));
    const float d = r_old - __half2float(h), d1 = 0.1f * d;
    g[0] += d - 4.f * d1;
#pragma unroll
    for (int i = 1; i < 5; ++i) g[i] += d1;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        stv(A.g + slot[i] * plane + at[i], g[i]);
    tref[n] = h;
}

template <int STO, int LAY = LAY_N>
__global__ void k_rebase(const Consts<float> c, const Buf<STO> A, int64_t plane, int64_t N, __half* __restrict__ tref) {
    if constexpr (has_ref<STO>()) {
        for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
            rebase_thermal_node<STO, LAY, int64_t>(c, A, plane, (int)(n / c.nz), (int)(n % c.nz), n, tref);
    }
}

// Reference refresh (16-bit storage) of node n: decode its flow populations with the old
// reference word (as the pull does), take the new A, J from their deviation moments and the
// new R from the node's temperature (as rebase_thermal_node does), re-express the thermal
// deviations against the new R and re-encode the flow populations against the new A, J.
// The populations, and every field they give, are unchanged up to the storage rounding of
// the re-encoded (now small) values.
template <int STO, int LAY, typename I>
__device__ __forceinline__ void rebase_16_node(const Consts<float>& c, const Buf<STO>& S, I plane, int kr, int kz,
                                               I n, uint2* __restrict__ fref) {
    const Qf q0 = fref_unpack(fref[n]);
    float d[9], g[5];
    I at[9];
    int slot[9];
    bool kept[9], all = true;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        kept[i] = own_slot<LAY, float, I>(c, kr, kz, i, at[i], slot[i]);
        all = all && kept[i];
        d[i] = (kept[i] ? ldv(S.f + slot[i] * plane + at[i]) : 0.f) + fref_delta(i, q0);
        if (i < 5) g[i] = kept[i] ? ldv(S.g + slot[i] * plane + at[i]) : 0.f;
    }
    // a boundary node whose outgoing populations the layout dropped keeps its references:
    // the kept populations do not give its moments
    if (!all) return;
    const float a = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const float jr = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const float jz = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    const float t = q0.R + (((g[0] + g[1]) + (g[2] + g[3])) + g[4]);
    const __half h = __float2half_rn(fminf(fmaxf(t, -60000.f), 60000.f));
    const float dr = q0.R - __half2float(h), dr1 = 0.1f * dr;
    g[0] += dr - 4.f * dr1;
#pragma unroll
    for (int i = 1; i < 5; ++i) g[i] += dr1;
    const uint2 qw = fref_make(a, jr, jz, h);
    const Qf q1 = fref_unpack(qw);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        stv(S.f + slot[i] * plane + at[i], d[i] - fref_delta(i, q1));
        if (i < 5) stv(S.g + slot[i] * plane + at[i], g[i]);
    }
    fref[n] = qw;
}

template <int STO, int LAY = LAY_N>
__global__ void k_rebase_16(const Consts<float> c, const Buf<STO> S, int64_t plane, int64_t N,
                            uint2* __restrict__ fref) {
    if constexpr (has_fref<STO>()) {
        for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
            rebase_16_node<STO, LAY, int64_t>(c, S, plane, (int)(n / c.nz), (int)(n % c.nz), n, fref);
    }
}

// ------------------------------------------------------------ host runtime --
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            (void)cudaGetLastError();                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
        }                                                                                          \
    } while (0)

struct lbm_handle {
    lbm_params p;
    lbm_info info;
    Consts<float> cf;
    Consts<double> cd;
    int device = 0;
    int sms = 0;             // multiprocessors of the device
    cudaStream_t stream = nullptr;
    int64_t plane = 0;       // elements per plane (padded)
    int64_t N = 0;           // nr * nz
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;             // buffer holding the current state
    void* phi = nullptr;
    __half* tref = nullptr;  // per-node reference offset R(x) of the thermal deviations
    uint2* fref = nullptr;   // per-node flow reference Q(x) (16-bit storage)
    int64_t since_rebase = 0;  // steps since the last flow-reference refresh
    int aa = 0;              // 1: in-place storage (one state buffer, layouts S and L alternate)
    int aa_odd = 0;          // in-place: 0 = state in layout S, 1 = in layout L
    float* fstage = nullptr; // N floats: porosity / init field upload
    // lbm_set_porosity_async: its own copy stream, two staging buffers (the upload into one
    // overlaps the steps that read the other), events and an error count
    cudaStream_t copy_stream = nullptr;
    float* astage[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    int astage_i = 0;
    int phi_pending = -1;           // staging buffer uploaded but not yet converted into phi
    unsigned int* bad_async = nullptr;
    float* mac = nullptr;    // two snapshots of 4 planes: rho, ur, uz, T
    int64_t mstride = 0;
    double* partials = nullptr;
    int pblocks = 0;
    double* result = nullptr;   // 8 doubles
    unsigned int* bad = nullptr;
    uint8_t* cls = nullptr;
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // (bulk start, bulk end, wall start, wall end) per timed step
    int* wait_status = nullptr;    // 16-bit storage: LBM_ERR_TIMEOUT once a bounded wait of the staged kernel ran out
    int spin = STAGE_SPIN;         // try_wait rounds of its per-row waits
    int stage = 1;                 // 16-bit: the staged bulk kernel where it applies (lbm_set_staging)
};

static int derive(const lbm_params* p, lbm_info* o, Consts<double>* cd) {
    memset(o, 0, sizeof(*o));
    if (!p) return fail(LBM_ERR_INVALID, "params is NULL");
    if (p->nr < 3 || p->nz < 3) return fail(LBM_ERR_INVALID, "grid %d x %d: need nr, nz >= 3", p->nr, p->nz);
    if (p->nr > 65535) return fail(LBM_ERR_INVALID, "nr = %d exceeds 65535", p->nr);
    if (p->geometry < 0 || p->geometry > 3) return fail(LBM_ERR_INVALID, "unknown geometry %d", p->geometry);
    if (p->storage < 0 || p->storage > 2) return fail(LBM_ERR_INVALID, "unknown storage %d", p->storage);
    if (p->collision != LBM_MRT && p->collision != LBM_BGK)
        return fail(LBM_ERR_INVALID, "unknown collision %d", p->collision);
    if (p->inplace != 0 && p->inplace != 1) return fail(LBM_ERR_INVALID, "inplace must be 0 or 1");
    if (!(p->J > 0) || !(p->lambda > 0) || !(p->Pr > 0))
        return fail(LBM_ERR_INVALID, "J, lambda and Pr must be positive");
    if (!(p->eps_mean > 0 && p->eps_mean <= 1)) return fail(LBM_ERR_INVALID, "eps_mean %g outside (0, 1]", p->eps_mean);
    const double cs = std::sqrt(1.0 / 3.0);
    if (p->geometry == PIPE_PERIODIC_Z || p->geometry == PIPE_INFLOW) {
        o->r0 = 0.5;
        o->L = (p->nr - 1) + 0.5;
    } else {
        if (!(p->radius_ratio > 1)) return fail(LBM_ERR_INVALID, "radius_ratio %g must exceed 1", p->radius_ratio);
        o->L = p->nr - 1;
        o->r0 = o->L / (p->radius_ratio - 1);
    }
    o->H = p->nz - 1;
    const double dTw = p->T_hot - p->T_cold;
    if (p->tau_nu > 0) {
        o->tau_nu = p->tau_nu;
        o->Ma = p->Ra > 0 ? (o->tau_nu - 0.5) * cs * std::sqrt(p->Ra) / (p->J * o->L * std::sqrt(p->Pr)) : 0.0;
    } else {
        if (!(p->Ra > 0)) return fail(LBM_ERR_INVALID, "Ra must be positive when tau_nu is not given");
        o->Ma = p->Ma;
        o->tau_nu = 0.5 + p->Ma * p->J * o->L * std::sqrt(p->Pr) / (cs * std::sqrt(p->Ra));   // Eq. 39
    }
    if (!(o->tau_nu > 0.5)) return fail(LBM_ERR_INVALID, "tau_nu = %g must exceed 1/2", o->tau_nu);
    o->tau_T = (1.0 / 3.0) * p->lambda * (o->tau_nu - 0.5) / (0.2 * p->J * p->Pr);            // Eq. 39
    o->nu_e = (o->tau_nu - 0.5) / 3.0;                                                           // Eq. 31
    o->nu = o->nu_e / p->J;
    if (p->Ra > 0) {
        if (dTw == 0) return fail(LBM_ERR_INVALID, "T_hot == T_cold with Ra > 0");
        const double U = o->Ma * cs;                                                             // Ma = U / c_s
        o->gbeta = U * U / (dTw * o->L);                                                         // U^2 = g beta dT L
    }
    if (p->heater_len > 0) {
        if (p->geometry != LBM_ANNULUS && p->geometry != LBM_ANNULUS_PERIODIC_Z)
            return fail(LBM_ERR_INVALID, "the discrete heater needs an annulus geometry");
        if (p->nr < 4) return fail(LBM_ERR_INVALID, "the discrete heater needs nr >= 4");
        if (!(p->heater_len <= 1)) return fail(LBM_ERR_INVALID, "heater_len %g exceeds 1 (l / H)", p->heater_len);
        if (!(p->heater_center >= 0 && p->heater_center <= 1))
            return fail(LBM_ERR_INVALID, "heater_center %g outside [0, 1] (h / H)", p->heater_center);
    }
    if (p->geometry == LBM_PIPE_INFLOW && !(p->u_in >= 0 && p->u_in < 0.5))
        return fail(LBM_ERR_INVALID, "u_in = %g: the inlet velocity must lie in [0, 1/2)", p->u_in);
    o->T0 = p->heater_len > 0 ? p->T_cold : 0.5 * (p->T_hot + p->T_cold);   // Sec. 4.4: T0 = T_o
    o->Kbar = p->Da * o->L * o->L;
    const int64_t N = (int64_t)p->nr * p->nz;
    // populations read and written, porosity, and the references each node's pull reads:
    // R(x) (FP16) with FP32 storage, the reference word (A, J_r, J_z, R; 4 x FP16) with 16-bit
    // storage
    o->bytes_per_step = N * (int64_t)(2 * (9 * f_size(p->storage) + 5 * g_size(p->storage)) + phi_size(p->storage) +
                                      (p->storage == LBM_F32 ? sizeof(__half) : sizeof(uint2)));
    if (cd) {
        Consts<double>& c = *cd;
        memset(&c, 0, sizeof(c));
        c.nr = p->nr;
        c.nz = p->nz;
        c.geometry = p->geometry;
        c.periodic = periodic_z(p->geometry) ? 1 : 0;
        c.porous_mode = !(p->Da > 0) ? 0 : (p->eps_mean >= 1 ? 1 : 2);
        c.ergun = p->F_eps < 0;
        c.r0 = o->r0;
        c.cs2tau = (o->tau_nu - 0.5) / 3.0;
        c.two_taum = 2 * (o->tau_nu - 0.5);
        c.s_e = 1.1;
        c.s_eps = 1.1;
        c.s_j = 1.0;
        c.s_q = 1.2;
        c.s_nu = 1.0 / o->tau_nu;
        if (p->collision == LBM_BGK)   // Sec. 3.1: every moment relaxes at 1/tau
            c.s_e = c.s_eps = c.s_j = c.s_q = c.s_nu;
        c.h_e = 1 - 0.5 * c.s_e;
        c.h_eps = 1 - 0.5 * c.s_eps;
        c.h_j = 1 - 0.5 * c.s_j;
        c.h_q = 1 - 0.5 * c.s_q;
        c.h_nu = 1 - 0.5 * c.s_nu;
        c.cs2_2tm = c.two_taum / 3.0;
        c.tauT = o->tau_T;
        c.wg_den = 1.0 / (o->tau_T + 0.5);
        c.gbeta = o->gbeta;
        c.T0 = o->T0;
        c.az = p->body_accel_z;
        c.u_in = p->u_in;
        if (p->heater_len > 0) {
            const double H = p->nz - 1, h = p->heater_center * H, half = 0.5 * p->heater_len * H;
            c.heater = 1;
            c.hz0 = (int)std::max(0.0, std::ceil(h - half));
            c.hz1 = (int)std::min(H, std::floor(h + half));
            c.hG = (p->T_hot - p->T_cold) / o->L;
        }
        // Eq. 8 coefficients (see porous()): 1/K(phi) = c_k (1 - phi)^2 / phi^3 with
        // c_k = eps_mean^3 / ((1 - eps_mean)^2 Da L^2), i.e. K(eps_mean) = Da L^2.
        const double em = p->eps_mean;
        const double F = p->F_eps > 0 ? p->F_eps : 0.0;
        if (c.porous_mode == 2) {
            const double ck = em * em * em / ((1 - em) * (1 - em) * o->Kbar);
            c.lin_coef = o->nu * ck;
            c.nl_coef = c.ergun ? 1.75 * std::sqrt(ck / 150.0) : F * std::sqrt(ck);
        } else if (c.porous_mode == 1) {
            c.lin_coef = o->nu / o->Kbar;
            c.nl_coef = c.ergun ? 1.75 * std::sqrt(1.0 / (150.0 * o->Kbar)) : F / std::sqrt(o->Kbar);
        }
        c.T_hot = p->T_hot;
        c.T_cold = p->T_cold;
    }
    return LBM_OK;
}

static Consts<float> to_float(const Consts<double>& d) {
    Consts<float> f;
    f.nr = d.nr; f.nz = d.nz; f.geometry = d.geometry; f.porous_mode = d.porous_mode; f.ergun = d.ergun; f.periodic = d.periodic;
    f.heater = d.heater; f.hz0 = d.hz0; f.hz1 = d.hz1; f.hG = (float)d.hG;
    f.r0 = (float)d.r0; f.cs2tau = (float)d.cs2tau; f.two_taum = (float)d.two_taum;
    f.s_e = (float)d.s_e; f.s_eps = (float)d.s_eps; f.s_j = (float)d.s_j; f.s_q = (float)d.s_q; f.s_nu = (float)d.s_nu;
    f.h_e = (float)d.h_e; f.h_eps = (float)d.h_eps; f.h_j = (float)d.h_j; f.h_q = (float)d.h_q; f.h_nu = (float)d.h_nu;
    f.cs2_2tm = (float)d.cs2_2tm;
    f.tauT = (float)d.tauT; f.wg_den = (float)d.wg_den; f.gbeta = (float)d.gbeta; f.T0 = (float)d.T0;
    f.az = (float)d.az; f.lin_coef = (float)d.lin_coef; f.nl_coef = (float)d.nl_coef;
    f.T_hot = (float)d.T_hot; f.T_cold = (float)d.T_cold;
    f.u_in = (float)d.u_in;
    f.tref = d.tref;
    return f;
}

// Work that reads or writes the porosity field first waits for an asynchronous upload.
static dim3 grid2d(const lbm_handle* h, int threads) {
    return dim3((unsigned)((h->p.nz + threads - 1) / threads), (unsigned)h->p.nr);
}

// Dispatch a templated launch on the storage type.
#define DISPATCH_STO(sto, ...)                      \
    switch (sto) {                                  \
        case LBM_F32: { constexpr int S_ = LBM_F32; __VA_ARGS__; } break;  \
        case LBM_F16: { constexpr int S_ = LBM_F16; __VA_ARGS__; } break;  \
        default: { constexpr int S_ = LBM_BF16; __VA_ARGS__; } break;      \
    }

// Dispatch on the two 16-bit storage types.
#define DISPATCH_STO16(sto, ...)                                           \
    switch (sto) {                                                         \
        case LBM_F16: { constexpr int S_ = LBM_F16; __VA_ARGS__; } break;  \
        default: { constexpr int S_ = LBM_BF16; __VA_ARGS__; } break;      \
    }

// Layout of a state: A/B buffers, or in-place after an even (S) or odd (L) number of steps.
#define DISPATCH_LAY(lay, ...)                                             \
    switch (lay) {                                                         \
        case LAY_S: { constexpr int L_ = LAY_S; __VA_ARGS__; } break;      \
        case LAY_L: { constexpr int L_ = LAY_L; __VA_ARGS__; } break;      \
        default: { constexpr int L_ = LAY_N; __VA_ARGS__; } break;         \
    }

// rows per thread of the batched kernels: 1, 2 or 4 (the values the tuner tries)
#define DISPATCH_RPT(rpt, ...)                                             \
    switch (rpt) {                                                         \
        case 4: { constexpr int R_ = 4; __VA_ARGS__; } break;              \
        case 2: { constexpr int R_ = 2; __VA_ARGS__; } break;              \
        default: { constexpr int R_ = 1; __VA_ARGS__; } break;             \
    }

template <int STO> static Buf<STO> bufp(const lbm_handle* h, int which) {
    Buf<STO> b;
    char* base = (char*)h->buf[which];
    b.f = (typename St<STO>::TF*)base;
    b.g = (typename St<STO>::TG*)(base + 9 * h->plane * f_size(STO));
    return b;
}
template <int STO> using PP = typename St<STO>::P;

static int wait_phi(lbm_handle* h) {
    if (h->phi_pending >= 0) {
        // the newest upload becomes the field: on the compute stream, after everything
        // queued before (which read the old field) and after its copy
        const int i = h->phi_pending;
        h->phi_pending = -1;
        CK(cudaStreamWaitEvent(h->stream, h->copied[i], 0));
        const unsigned blocks = phi_blocks(h->N);
        // the field is FP32 for every storage type: check the staging buffer and swap it with
        // the field; the old field becomes staging buffer i once the work queued before has
        // read it
        k_phi_check<<<blocks, 256, 0, h->stream>>>(h->astage[i], h->N, h->bad_async);
        void* old = h->phi;
        h->phi = h->astage[i];
        h->astage[i] = (float*)old;
        CK(cudaGetLastError());
        CK(cudaEventRecord(h->consumed[i], h->stream));
    }
    return LBM_OK;
}

extern "C" {

void lbm_params_default(lbm_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nr = 48;
    p->nz = 96;
    p->geometry = LBM_ANNULUS;
    p->storage = LBM_F32;
    p->radius_ratio = 2.0;
    p->Ra = 1e3;
    p->Da = 1e-2;
    p->Pr = 1.0;
    p->J = 1.0;
    p->lambda = 1.0;
    p->Ma = 0.1;
    p->tau_nu = 0.0;
    p->F_eps = -1.0;
    p->eps_mean = 0.6;
    p->T_hot = 1.0;
    p->T_cold = 0.0;
    p->body_accel_z = 0.0;
    p->init_noise = 1e-3;
    p->seed = 1;
    p->heater_center = 0.5;
}

int lbm_derive(const lbm_params* p, lbm_info* out) {
    if (!out) return fail(LBM_ERR_INVALID, "out is NULL");
    return derive(p, out, nullptr);
}

int lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_OK;
    cudaSetDevice(h->device);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);   // an upload may still write phi
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* b : h->buf) cudaFree(b);
    cudaFree(h->tref);
    cudaFree(h->fref);
    cudaFree(h->phi);
    cudaFree(h->fstage);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (int i = 0; i < 2; ++i) {
        cudaFree(h->astage[i]);
        if (h->consumed[i]) cudaEventDestroy(h->consumed[i]);
        if (h->copied[i]) cudaEventDestroy(h->copied[i]);
    }
    cudaFree(h->bad_async);
    cudaFree(h->mac);
    cudaFree(h->partials);
    cudaFree(h->result);
    cudaFree(h->bad);
    cudaFree(h->cls);
    cudaFree(h->wait_status);
    for (auto e : h->ev) cudaEventDestroy(e);
    delete h;
    return LBM_OK;
}

static int launch_init(lbm_handle* h, const float* ur, const float* uz, const float* T) {
    if (int rc = wait_phi(h)) return rc;
    dim3 g = grid2d(h, 128);
    DISPATCH_STO(h->p.storage,
                 k_init<S_><<<g, 128, 0, h->stream>>>(h->cd, bufp<S_>(h, 0), (const PP<S_>*)h->phi, h->plane, ur, uz,
                                                      T, h->p.init_noise, h->p.seed, h->tref, h->fref, h->aa));
    CK(cudaGetLastError());
    h->cur = 0;
    h->aa_odd = 0;
    h->info.steps = 0;
    h->since_rebase = 0;
    return LBM_OK;
}

int lbm_create(const lbm_params* p, lbm_handle** out) {
    if (!out) return fail(LBM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    lbm_handle* h = new lbm_handle();
    int rc = derive(p, &h->info, &h->cd);
    if (rc) { delete h; return rc; }
    h->p = *p;
    h->cf = to_float(h->cd);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return fail(LBM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); }
    e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { delete h; return fail(LBM_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e)); }
    if (p->storage != LBM_F32) {
        e = p->storage == LBM_F16 ? stage_carveout<LBM_F16>() : stage_carveout<LBM_BF16>();
        if (e != cudaSuccess) { delete h; return fail(LBM_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)); }
    }
    h->N = (int64_t)p->nr * p->nz;
    h->plane = (h->N + 63) / 64 * 64;
    h->mstride = h->plane;
    h->pblocks = 1024;
#define ALLOC(ptr, bytes)                                                       \
    do {                                                                        \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                   \
        if (e_ != cudaSuccess) {                                                \
            (void)cudaGetLastError();                                           \
            lbm_destroy(h);                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, \
                        "cudaMalloc(%zu bytes): %s", (size_t)(bytes), cudaGetErrorString(e_)); \
        }                                                                       \
    } while (0)
    h->aa = p->inplace;
    ALLOC(h->buf[0], state_bytes(p->storage, h->plane));
    if (!h->aa) ALLOC(h->buf[1], state_bytes(p->storage, h->plane));
    if (p->storage == LBM_F32) {
        ALLOC(h->tref, h->plane * sizeof(__half));
        h->cd.tref = h->tref;
        h->cf.tref = h->tref;
    } else {
        ALLOC(h->fref, h->plane * sizeof(uint2));
        h->cd.fref = h->fref;
        h->cf.fref = h->fref;
        ALLOC(h->wait_status, sizeof(int));
        e = cudaMemset(h->wait_status, 0, sizeof(int));
        if (e != cudaSuccess) { lbm_destroy(h); return fail(LBM_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e)); }
    }
    ALLOC(h->phi, h->plane * phi_size(p->storage));
    ALLOC(h->partials, (size_t)h->pblocks * RES_NV * sizeof(double));
    ALLOC(h->result, 8 * sizeof(double));
    ALLOC(h->bad, sizeof(unsigned int));
#undef ALLOC
    // uniform porosity eps_mean, then the cold start
    const int thr = 256;
    const unsigned blocks = (unsigned)((h->N + thr - 1) / thr);
    DISPATCH_STO(p->storage, k_phi_fill<S_><<<blocks, thr, 0, h->stream>>>((PP<S_>*)h->phi, h->N, (float)p->eps_mean));
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        rc = launch_init(h, nullptr, nullptr, nullptr);
        if (rc) { lbm_destroy(h); return rc; }
        e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) {
        lbm_destroy(h);
        return fail(LBM_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e));
    }
    *out = h;
    return LBM_OK;
}

int lbm_set_stream(lbm_handle* h, void* stream) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    const cudaStream_t s = (cudaStream_t)stream;
    if (s == h->stream) return LBM_OK;
    CK(cudaSetDevice(h->device));
    // the new stream starts after everything already queued on the old one
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t err = cudaEventRecord(e, h->stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, e, 0);
    cudaEventDestroy(e);   // released once the recorded work has completed
    if (err != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_set_stream: %s", cudaGetErrorString(err));
    h->stream = s;
    return LBM_OK;
}

static int ensure_fstage(lbm_handle* h) {
    if (!h->fstage) CK(cudaMalloc((void**)&h->fstage, 3 * h->plane * sizeof(float)));
    return LBM_OK;
}

int lbm_set_porosity(lbm_handle* h, const float* phi, int on_device) {
    if (!h || !phi) return fail(LBM_ERR_INVALID, "NULL argument");
    CK(cudaSetDevice(h->device));
    if (int rc = wait_phi(h)) return rc;
    const float* src = phi;
    if (!on_device) {
        int rc = ensure_fstage(h);
        if (rc) return rc;
        CK(cudaMemcpyAsync(h->fstage, phi, h->N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        src = h->fstage;
    }
    CK(cudaMemsetAsync(h->bad, 0, sizeof(unsigned int), h->stream));
    DISPATCH_STO(h->p.storage, k_phi<S_><<<phi_blocks(h->N), 256, 0, h->stream>>>(src, (PP<S_>*)h->phi, h->N,
                                                                                   aligned16(src), h->bad));
    CK(cudaGetLastError());
    unsigned int bad = 0;
    CK(cudaMemcpyAsync(&bad, h->bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (bad) return fail(LBM_ERR_INVALID, "%u porosity values outside (0, 1]", bad);
    return LBM_OK;
}

int lbm_set_porosity_async(lbm_handle* h, const float* phi) {
    if (!h || !phi) return fail(LBM_ERR_INVALID, "NULL argument");
    CK(cudaSetDevice(h->device));
    if (!h->copy_stream) {
        CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            CK(cudaMalloc((void**)&h->astage[i], h->plane * sizeof(float)));   // may become the field
            CK(cudaEventCreateWithFlags(&h->consumed[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->copied[i], cudaEventDisableTiming));
        }
        CK(cudaMalloc((void**)&h->bad_async, sizeof(unsigned int)));
        CK(cudaMemsetAsync(h->bad_async, 0, sizeof(unsigned int), h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    const int i = h->astage_i;
    h->astage_i ^= 1;
    // on the copy stream: staging buffer i is free once its last conversion has run, then
    // copy; the conversion into phi waits for the next reader of the field (wait_phi), so
    // copies follow one another on the copy stream while the compute stream runs, and an
    // upload that no reader saw is superseded by the next one
    CK(cudaStreamWaitEvent(h->copy_stream, h->consumed[i], 0));
    CK(cudaMemcpyAsync(h->astage[i], phi, h->N * sizeof(float), cudaMemcpyHostToDevice, h->copy_stream));
    CK(cudaEventRecord(h->copied[i], h->copy_stream));
    h->phi_pending = i;
    return LBM_OK;
}

int lbm_porosity_errors(lbm_handle* h, uint32_t* count, int clear) {
    if (!h || !count) return fail(LBM_ERR_INVALID, "NULL argument");
    *count = 0;
    if (!h->bad_async) return LBM_OK;
    CK(cudaSetDevice(h->device));
    int rc = wait_phi(h);
    if (rc) return rc;
    unsigned int v = 0;
    CK(cudaMemcpyAsync(&v, h->bad_async, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    if (clear) CK(cudaMemsetAsync(h->bad_async, 0, sizeof(unsigned int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *count = v;
    return LBM_OK;
}

int lbm_init_fields(lbm_handle* h, const float* ur, const float* uz, const float* T, int on_device) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    if ((ur == nullptr) != (uz == nullptr)) return fail(LBM_ERR_INVALID, "give both u_r and u_z or neither");
    CK(cudaSetDevice(h->device));
    const float *dur = ur, *duz = uz, *dT = T;
    if (!on_device && (ur || T)) {
        int rc = ensure_fstage(h);
        if (rc) return rc;
        if (ur) {
            CK(cudaMemcpyAsync(h->fstage, ur, h->N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(h->fstage + h->plane, uz, h->N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
            dur = h->fstage;
            duz = h->fstage + h->plane;
        }
        if (T) {
            CK(cudaMemcpyAsync(h->fstage + 2 * h->plane, T, h->N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
            dT = h->fstage + 2 * h->plane;
        }
    }
    int rc = launch_init(h, dur, duz, dT);
    if (rc) return rc;
    if (!on_device) CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// With 16-bit storage the flow reference is refreshed every LBM_FREF_EVERY steps of
// lbm_step (and before every check interval of lbm_run): the stored values stay of the
// size of the change since the last refresh however long the run.
constexpr int64_t LBM_FREF_EVERY = 1024;
static int launch_rebase(lbm_handle* h);

static int cur_lay(const lbm_handle* h) { return !h->aa ? LAY_N : (h->aa_odd ? LAY_L : LAY_S); }

// One step with in-place storage: read the current layout, write the other one, in the
// same buffer.  The wall kernel runs first: it reads the pre-collision values of its
// interior neighbours, which the bulk kernel overwrites.  One node per thread (update_column)
// for every storage type.
static int launch_step_inplace(lbm_handle* h, int nw) {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};   // wall start / end, bulk start / end
    if (h->timing)
        for (auto& x : e) CK(cudaEventCreate(&x));
    const bool i32 = 14 * h->plane < ((int64_t)1 << 31);
    const int64_t zblocks = (h->p.nz + BULK_THREADS - 1) / BULK_THREADS;
    const int rpt = (i32 && zblocks * ((h->p.nr + BULK_RPT - 1) / BULK_RPT) >= (int64_t)BULK_RPT_MIN_BLOCKS * h->sms) ? BULK_RPT : 1;
    const dim3 gb((unsigned)zblocks, (unsigned)((h->p.nr + rpt - 1) / rpt));
    const bool odd = h->aa_odd != 0;   // reading L (odd) or S (even)
    if (h->timing) CK(cudaEventRecord(e[0], h->stream));
#define AA_LAUNCH(LIN_, LOUT_)                                                                                  \
    DISPATCH_STO(h->p.storage, {                                                                               \
        const auto S = bufp<S_>(h, 0);                                                                         \
        const auto* ph = (const PP<S_>*)h->phi;                                                                \
        k_wall<S_, LIN_, LOUT_><<<(nw + 127) / 128, 128, 0, h->stream>>>(h->cf, S, S, ph, h->plane, nw);       \
        if (h->timing) CK(cudaEventRecord(e[1], h->stream));                                                   \
        if (h->timing) CK(cudaEventRecord(e[2], h->stream));                                                   \
        if (rpt > 1)                                                                                           \
            k_bulk<S_, int, BULK_RPT, LIN_, LOUT_><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, S, S, ph,         \
                                                                                        (int)h->plane);         \
        else if (i32)                                                                                          \
            k_bulk<S_, int, 1, LIN_, LOUT_><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, S, S, ph, (int)h->plane); \
        else                                                                                                   \
            k_bulk<S_, int64_t, 1, LIN_, LOUT_><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, S, S, ph, h->plane);  \
    })
    if (odd) {
        AA_LAUNCH(LAY_L, LAY_S);
    } else {
        AA_LAUNCH(LAY_S, LAY_L);
    }
#undef AA_LAUNCH
    CK(cudaGetLastError());
    if (h->timing) {
        CK(cudaEventRecord(e[3], h->stream));
        // the (bulk start, bulk end, wall start, wall end) quadruple lbm_kernel_times reads
        h->ev.push_back(e[2]);
        h->ev.push_back(e[3]);
        h->ev.push_back(e[0]);
        h->ev.push_back(e[1]);
    }
    h->aa_odd ^= 1;
    h->info.steps += 1;
    h->since_rebase += 1;
    return LBM_OK;
}

static int launch_step(lbm_handle* h) {
    if (int rc = wait_phi(h)) return rc;
    if (h->fref && h->since_rebase >= LBM_FREF_EVERY)
        if (int rc = launch_rebase(h)) return rc;
    const int nw = wall_count(h->p.geometry, h->p.nr, h->p.nz);
    if (h->aa) return launch_step_inplace(h, nw);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e1b = nullptr, e2 = nullptr;
    if (h->timing) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventCreate(&e1b));
        CK(cudaEventCreate(&e2));
        CK(cudaEventRecord(e0, h->stream));
    }
    // BULK_RPT rows per thread where the grid keeps BULK_RPT_MIN_BLOCKS blocks per SM
    // (9 blocks of 128 threads are resident per SM), else one row per thread so that small
    // grids still fill the device
    const bool i32 = 14 * h->plane < ((int64_t)1 << 31);
    const bool pair = h->p.storage != LBM_F32 && i32;   // 16-bit storage: two columns per thread
    const int cols = pair ? 2 * BULK_THREADS : BULK_THREADS;
    const int64_t zblocks = (h->p.nz + cols - 1) / cols;
    const int rpt = (i32 && zblocks * ((h->p.nr + BULK_RPT - 1) / BULK_RPT) >= (int64_t)BULK_RPT_MIN_BLOCKS * h->sms) ? BULK_RPT : 1;
    const dim3 gb((unsigned)zblocks, (unsigned)((h->p.nr + rpt - 1) / rpt));
    if (pair) {
        const bool vec = (h->p.nz & 1) == 0;
        DISPATCH_STO16(h->p.storage, {
            auto A = bufp<S_>(h, h->cur);
            auto B = bufp<S_>(h, h->cur ^ 1);
            const float* ph = (const float*)h->phi;
            if (vec && rpt > 1 && h->stage && h->p.nz % 8 == 0) k_bulk_stage<S_, BULK_RPT, true><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, A, B, ph, (int)h->plane, h->spin, h->wait_status);
            else if (vec && rpt > 1 && h->stage) k_bulk_stage<S_, BULK_RPT, false><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, A, B, ph, (int)h->plane, h->spin, h->wait_status);
            else if (vec && rpt > 1) k_bulk_pair<S_, true, BULK_RPT><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, A, B, ph, (int)h->plane);
            else if (vec) k_bulk_pair<S_, true, 1><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, A, B, ph, (int)h->plane);
            else if (rpt > 1) k_bulk_pair<S_, false, BULK_RPT><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, A, B, ph, (int)h->plane);
            else k_bulk_pair<S_, false, 1><<<gb, BULK_THREADS, 0, h->stream>>>(h->cf, A, B, ph, (int)h->plane);
        });
    } else if (rpt > 1) {
        DISPATCH_STO(h->p.storage,
                     k_bulk<S_, int, BULK_RPT><<<gb, BULK_THREADS, 0, h->stream>>>(
                         h->cf, bufp<S_>(h, h->cur), bufp<S_>(h, h->cur ^ 1), (const PP<S_>*)h->phi, (int)h->plane));
    } else if (i32) {
        DISPATCH_STO(h->p.storage,
                     k_bulk<S_, int, 1><<<gb, BULK_THREADS, 0, h->stream>>>(
                         h->cf, bufp<S_>(h, h->cur), bufp<S_>(h, h->cur ^ 1), (const PP<S_>*)h->phi, (int)h->plane));
    } else {
        DISPATCH_STO(h->p.storage,
                     k_bulk<S_, int64_t, 1><<<gb, BULK_THREADS, 0, h->stream>>>(
                         h->cf, bufp<S_>(h, h->cur), bufp<S_>(h, h->cur ^ 1), (const PP<S_>*)h->phi, h->plane));
    }
    CK(cudaGetLastError());
    if (h->timing) {
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventRecord(e1b, h->stream));
    }
    // after the bulk kernel on the same stream (run beside it, the wall kernel took the
    // SMs the bulk kernel's memory pipeline needs: bulk 0.496 against 0.488 ms, FP16)
    DISPATCH_STO(h->p.storage,
                 k_wall<S_><<<(nw + 127) / 128, 128, 0, h->stream>>>(h->cf, bufp<S_>(h, h->cur), bufp<S_>(h, h->cur ^ 1),
                                                                     (const PP<S_>*)h->phi, h->plane, nw));
    CK(cudaGetLastError());
    if (h->timing) {
        CK(cudaEventRecord(e2, h->stream));
        // (bulk start, bulk end, wall start, wall end): the wall kernel starts where the bulk ends
        h->ev.push_back(e0);
        h->ev.push_back(e1);
        h->ev.push_back(e1b);
        h->ev.push_back(e2);
    }
    h->cur ^= 1;
    h->info.steps += 1;
    h->since_rebase += 1;
    return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    if (nsteps < 0) return fail(LBM_ERR_INVALID, "nsteps < 0");
    CK(cudaSetDevice(h->device));
    for (int64_t s = 0; s < nsteps; ++s) {
        int rc = launch_step(h);
        if (rc) return rc;
    }
    return LBM_OK;
}

static int launch_moments(lbm_handle* h, int which, float* rho, float* ur, float* uz, float* T) {
    if (int rc = wait_phi(h)) return rc;
    const dim3 g = grid2d(h, 128);
    DISPATCH_LAY(cur_lay(h), DISPATCH_STO(h->p.storage,
                 k_moments<S_, L_><<<g, 128, 0, h->stream>>>(h->cf, bufp<S_>(h, which), (const PP<S_>*)h->phi,
                                                             h->plane, rho, ur, uz, T)));
    CK(cudaGetLastError());
    return LBM_OK;
}

static int ensure_mac(lbm_handle* h) {
    if (!h->mac) CK(cudaMalloc((void**)&h->mac, 8 * h->mstride * sizeof(float)));
    return LBM_OK;
}

int lbm_moments(lbm_handle* h, float* rho, float* ur, float* uz, float* T, int on_device) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    CK(cudaSetDevice(h->device));
    if (on_device) return launch_moments(h, h->cur, rho, ur, uz, T);
    int rc = ensure_mac(h);
    if (rc) return rc;
    float* m = h->mac;
    rc = launch_moments(h, h->cur, m, m + h->mstride, m + 2 * h->mstride, m + 3 * h->mstride);
    if (rc) return rc;
    float* outs[4] = {rho, ur, uz, T};
    for (int j = 0; j < 4; ++j)
        if (outs[j])
            CK(cudaMemcpyAsync(outs[j], m + j * h->mstride, h->N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// Eq. 42 of the current state into h->result[0..1] (stream-ordered).
static int launch_nusselt(lbm_handle* h) {
    const double dTw = h->p.T_hot - h->p.T_cold;
    const double ri = h->info.r0, ro = h->info.r0 + (h->p.nr - 1);
    const int blocks = (int)std::min<int64_t>((h->p.nz + 127) / 128, h->pblocks);
    DISPATCH_LAY(cur_lay(h), DISPATCH_STO(h->p.storage, k_nusselt<S_, L_><<<blocks, 128, 0, h->stream>>>(
                                                            h->cf, bufp<S_>(h, h->cur), h->plane, h->partials)));
    k_nusselt_final<<<1, 256, 0, h->stream>>>(h->partials, blocks, ri, ro, h->info.H, dTw, h->result);
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_nusselt(lbm_handle* h, double* nu_inner, double* nu_outer) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    if (h->p.geometry == LBM_PIPE_INFLOW || h->p.heater_len > 0) {   // lbm_pipe_nusselt, lbm_heater_nusselt
        if (nu_inner) *nu_inner = NAN;
        if (nu_outer) *nu_outer = NAN;
        return LBM_OK;
    }
    CK(cudaSetDevice(h->device));
    if (int rc = launch_nusselt(h)) return rc;
    double r[2];
    CK(cudaMemcpyAsync(r, h->result, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (nu_inner) *nu_inner = h->p.geometry == LBM_PIPE_PERIODIC_Z ? NAN : r[0];
    if (nu_outer) *nu_outer = r[1];
    return LBM_OK;
}

int lbm_nusselt_async(lbm_handle* h, double* out) {
    if (!h || !out) return fail(LBM_ERR_INVALID, "NULL argument");
    if (h->p.geometry == LBM_PIPE_INFLOW || h->p.heater_len > 0) {   // lbm_pipe_nusselt, lbm_heater_nusselt
        out[0] = out[1] = NAN;
        return LBM_OK;
    }
    CK(cudaSetDevice(h->device));
    if (int rc = launch_nusselt(h)) return rc;
    // stream order keeps h->result intact until it has been read
    const int pipe = h->p.geometry == LBM_PIPE_PERIODIC_Z;
    if (pipe) out[0] = NAN;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
        k_put2<<<1, 32, 0, h->stream>>>(h->result, (double*)at.devicePointer, pipe);
        CK(cudaGetLastError());
    } else {
        (void)cudaGetLastError();   // pageable memory: an ordinary copy
        CK(cudaMemcpyAsync(out + pipe, h->result + pipe, (2 - pipe) * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
    }
    return LBM_OK;
}

int lbm_sync(lbm_handle* h) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    CK(cudaSetDevice(h->device));
    if (h->copy_stream) CK(cudaStreamSynchronize(h->copy_stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// FP64 residual sums between two field snapshots (4 planes each: rho, u_r, u_z, T):
// res = max(|du|_2 / |u|_2, |dT|_2 / |T|_2) over non-wall nodes, mass = sum r rho.
static int residual_between(lbm_handle* h, const float* cur, const float* prev, double* res, double* mass) {
    const int blocks = (int)std::min<int64_t>(h->pblocks, (h->N + 255) / 256);
    k_resid_partial<<<blocks, 256, 0, h->stream>>>(h->p.geometry, h->p.nr, h->p.nz, h->info.r0, cur, prev,
                                                   h->mstride, h->partials);
    CK(cudaGetLastError());
    k_sum_rows<<<1, 256, 0, h->stream>>>(h->partials, blocks, h->result);
    CK(cudaGetLastError());
    double s[RES_NV];
    CK(cudaMemcpyAsync(s, h->result, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (s[5] > 0) return fail(LBM_ERR_DIVERGED, "%.0f nodes hold NaN or Inf", s[5]);
    const double ru = s[1] > 0 ? std::sqrt(s[0] / s[1]) : (s[0] > 0 ? INFINITY : 0.0);
    const double rt = s[3] > 0 ? std::sqrt(s[2] / s[3]) : (s[2] > 0 ? INFINITY : 0.0);
    if (res) *res = ru > rt ? ru : rt;
    if (mass) *mass = s[4];
    return LBM_OK;
}

static int snapshot(lbm_handle* h, int which, float* m) {
    if (int rc = wait_phi(h)) return rc;
    return launch_moments(h, which, m, m + h->mstride, m + 2 * h->mstride, m + 3 * h->mstride);
}

int lbm_residual(lbm_handle* h, double* res, double* mass) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    if (h->aa)
        return fail(LBM_ERR_INVALID, "in-place storage keeps no previous state: use lbm_run, or two snapshots and "
                                     "lbm_field_residual_noalloc");
    if (h->info.steps < 1) return fail(LBM_ERR_INVALID, "residual needs at least one step since initialisation");
    CK(cudaSetDevice(h->device));
    int rc = ensure_mac(h);
    if (rc) return rc;
    float* cur = h->mac;
    float* prev = h->mac + 4 * h->mstride;
    if ((rc = snapshot(h, h->cur, cur)) || (rc = snapshot(h, h->cur ^ 1, prev))) return rc;
    return residual_between(h, cur, prev, res, mass);
}

// Steady-state iteration.  The criterion is the mean change per step over each check
// interval, |u^n - u^(n-k)|_2 / (k |u^n|_2) (likewise T): with FP32 or 16-bit state the
// change between two consecutive steps carries rounding jitter of order 1e-8 - 1e-7
// that does not decay, whereas the interval mean falls with the true drift.
int lbm_run(lbm_handle* h, int64_t max_steps, int64_t check_every, double tol, int64_t* steps_done, double* res) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    if (max_steps < 0 || check_every < 1) return fail(LBM_ERR_INVALID, "max_steps >= 0 and check_every >= 1 required");
    CK(cudaSetDevice(h->device));
    int rc = ensure_mac(h);
    if (rc) return rc;
    float* a = h->mac;
    float* b = h->mac + 4 * h->mstride;
    if ((rc = snapshot(h, h->cur, b))) return rc;
    int64_t done = 0;
    double r = INFINITY;
    while (done < max_steps) {
        const int64_t k = std::min(check_every, max_steps - done);
        if ((rc = lbm_rebase(h))) break;
        if ((rc = lbm_step(h, k))) break;
        done += k;
        if ((rc = lbm_wait_status(h, 0))) break;   // before the residual reads a state the timeout left invalid
        if ((rc = snapshot(h, h->cur, a))) break;
        double m;
        rc = residual_between(h, a, b, &r, &m);
        if (rc) break;
        r /= (double)k;
        std::swap(a, b);
        if (r <= tol) break;
    }
    if (steps_done) *steps_done = done;
    if (res) *res = r;
    return rc;
}

int lbm_pipe_nusselt(lbm_handle* h, double* nu, int32_t nz) {
    if (!h || !nu) return fail(LBM_ERR_INVALID, "NULL argument");
    if (h->p.geometry != LBM_PIPE_INFLOW) return fail(LBM_ERR_INVALID, "lbm_pipe_nusselt needs LBM_PIPE_INFLOW");
    if (nz != h->p.nz) return fail(LBM_ERR_INVALID, "nz = %d, the grid has %d", nz, h->p.nz);
    CK(cudaSetDevice(h->device));
    int rc = ensure_mac(h);
    if (rc) return rc;
    if ((rc = snapshot(h, h->cur, h->mac))) return rc;
    double* d = nullptr;
    CK(cudaMallocAsync((void**)&d, (size_t)nz * sizeof(double), h->stream));
    k_pipe_nusselt<<<(unsigned)((nz + 127) / 128), 128, 0, h->stream>>>(h->p.nr, nz, h->info.r0, h->mac + 2 * h->mstride,
                                                                       h->mac + 3 * h->mstride, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(nu, d, (size_t)nz * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "pipe Nusselt: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_heater_nusselt(lbm_handle* h, double* nu_mean, double* nu_z) {
    if (!h || !nu_mean) return fail(LBM_ERR_INVALID, "NULL argument");
    if (!(h->p.heater_len > 0)) return fail(LBM_ERR_INVALID, "lbm_heater_nusselt needs heater_len > 0");
    CK(cudaSetDevice(h->device));
    int rc = ensure_mac(h);
    if (rc) return rc;
    if ((rc = snapshot(h, h->cur, h->mac))) return rc;
    const int nz = h->p.nz;
    double* d = nullptr;
    CK(cudaMallocAsync((void**)&d, (size_t)(nz + 1) * sizeof(double), h->stream));
    k_heater_nusselt<<<1, 256, 0, h->stream>>>(nz, h->cf.hz0, h->cf.hz1, h->cf.periodic, h->p.T_hot - h->p.T_cold,
                                               h->p.T_cold, h->mac + 3 * h->mstride, d + 1, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(nu_mean, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && nu_z)
        e = cudaMemcpyAsync(nu_z, d + 1, (size_t)nz * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "heater Nusselt: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_stream_function(lbm_handle* h, float* psi, int on_device, double* psi_max) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    CK(cudaSetDevice(h->device));
    int rc = ensure_mac(h);
    if (rc) return rc;
    if ((rc = snapshot(h, h->cur, h->mac))) return rc;
    const int nz = h->p.nz;
    const unsigned blocks = (unsigned)((nz + 127) / 128);
    float* dst = (psi && on_device) ? psi : h->mac + 4 * h->mstride;
    const int from_axis = h->p.geometry == LBM_PIPE_PERIODIC_Z || h->p.geometry == LBM_PIPE_INFLOW;
    double* d = nullptr;
    CK(cudaMallocAsync((void**)&d, (size_t)blocks * sizeof(double), h->stream));
    std::vector<double> bm(blocks);
    k_stream_function<<<blocks, 128, 0, h->stream>>>(h->p.nr, nz, h->info.r0, from_axis, h->mac + 2 * h->mstride,
                                                     dst, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bm.data(), d, (size_t)blocks * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && psi && !on_device)
        e = cudaMemcpyAsync(psi, dst, (size_t)h->N * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "stream function: %s", cudaGetErrorString(e));
    double big = 0;
    for (double x : bm) big = std::max(big, x);
    if (psi_max) *psi_max = big;
    return LBM_OK;
}

// Refresh the references of the current state: the temperature reference R(x) with FP32
// storage, the reference word (A, J, R) with 16-bit storage.
static int launch_rebase(lbm_handle* h) {
    const unsigned blocks = (unsigned)std::min<int64_t>((h->N + 255) / 256, (int64_t)h->sms * 16);
    if (h->p.storage == LBM_F32) {
        DISPATCH_LAY(cur_lay(h), k_rebase<LBM_F32, L_><<<blocks, 256, 0, h->stream>>>(
                                     h->cf, bufp<LBM_F32>(h, h->cur), h->plane, h->N, h->tref));
    } else {
        DISPATCH_LAY(cur_lay(h), DISPATCH_STO16(h->p.storage, k_rebase_16<S_, L_><<<blocks, 256, 0, h->stream>>>(
                                                                  h->cf, bufp<S_>(h, h->cur), h->plane, h->N, h->fref)));
    }
    CK(cudaGetLastError());
    h->since_rebase = 0;
    return LBM_OK;
}

int lbm_rebase(lbm_handle* h) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    CK(cudaSetDevice(h->device));
    return launch_rebase(h);
}

int lbm_node_class(lbm_handle* h, uint8_t* out) {
    if (!h || !out) return fail(LBM_ERR_INVALID, "NULL argument");
    CK(cudaSetDevice(h->device));
    if (!h->cls) CK(cudaMalloc((void**)&h->cls, h->N));
    k_node_class<<<grid2d(h, 128), 128, 0, h->stream>>>(h->p.geometry, h->p.nr, h->p.nz, h->cls);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, h->cls, h->N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_export_populations(lbm_handle* h, int32_t row0, int32_t nrows, double* f, double* g) {
    if (!h || !f || !g) return fail(LBM_ERR_INVALID, "NULL argument");
    if (row0 < 0 || nrows < 1 || row0 + nrows > h->p.nr) return fail(LBM_ERR_INVALID, "row range outside the grid");
    CK(cudaSetDevice(h->device));
    const int64_t P = (int64_t)nrows * h->p.nz;
    double* d = nullptr;
    CK(cudaMallocAsync((void**)&d, 14 * P * sizeof(double), h->stream));
    dim3 grid((unsigned)((h->p.nz + 127) / 128), (unsigned)nrows);
    DISPATCH_LAY(cur_lay(h), DISPATCH_STO(h->p.storage, k_export<S_, L_><<<grid, 128, 0, h->stream>>>(
                                                            h->cf, bufp<S_>(h, h->cur), h->plane, row0, nrows,
                                                            h->info.r0, h->info.T0, d)));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, 9 * P * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, d + 9 * P, 5 * P * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "export: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_get_info(lbm_handle* h, lbm_info* out) {
    if (!h || !out) return fail(LBM_ERR_INVALID, "NULL argument");
    *out = h->info;
    return LBM_OK;
}

int lbm_set_staging(lbm_handle* h, int enable) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    h->stage = enable != 0;
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_handle* h, int rounds) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    h->spin = rounds < 0 ? STAGE_SPIN : rounds;
    return LBM_OK;
}

int lbm_wait_status(lbm_handle* h, int clear) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    if (!h->wait_status) return LBM_OK;
    CK(cudaSetDevice(h->device));
    int v = 0;
    CK(cudaMemcpyAsync(&v, h->wait_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (clear && v) CK(cudaMemsetAsync(h->wait_status, 0, sizeof(int), h->stream));
    if (v == LBM_ERR_TIMEOUT)
        return fail(LBM_ERR_TIMEOUT, "a bounded wait of the staged bulk kernel ran out (step results are invalid)");
    if (v) return fail(v, "the staged bulk kernel was launched for an odd nz (step results are invalid)");
    return LBM_OK;
}

int lbm_set_timing(lbm_handle* h, int enable) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    for (auto e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    h->timing = enable != 0;
    return LBM_OK;
}

int lbm_kernel_times(lbm_handle* h, double* bulk_ms, int64_t* bulk_launches, double* wall_ms,
                     int64_t* wall_launches) {
    if (!h) return fail(LBM_ERR_INVALID, "handle is NULL");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    double tb = 0, tw = 0;
    for (size_t i = 0; i + 3 < h->ev.size(); i += 4) {   // (bulk start, bulk end, wall start, wall end)
        float a = 0, b = 0;
        CK(cudaEventElapsedTime(&a, h->ev[i], h->ev[i + 1]));
        CK(cudaEventElapsedTime(&b, h->ev[i + 2], h->ev[i + 3]));
        tb += a;
        tw += b;
    }
    const int64_t n = (int64_t)(h->ev.size() / 4);
    if (bulk_ms) *bulk_ms = tb;
    if (bulk_launches) *bulk_launches = n;
    if (wall_ms) *wall_ms = tw;
    if (wall_launches) *wall_launches = n;
    return LBM_OK;
}

const char* lbm_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ----------------------------------------------- allocation-free residual --
// Scratch for lbm_field_residual_noalloc: LBM_NOALLOC_ROWS partial rows of RES_NV
// doubles (one per reduction block) and one result row, 49 KB in total.  Every GPU
// that loads this library holds the array until the process exits.  Host code only
// ever passes the address obtained from cudaGetSymbolAddress; the symbol itself is a
// host-side stand-in there.
constexpr int LBM_NOALLOC_ROWS = 1024;
static __device__ __align__(256) double g_noalloc_scratch[(LBM_NOALLOC_ROWS + 1) * RES_NV];

// cuMemGetAddressRange of the driver, reached through the runtime's entry-point query so
// that the library does not link libcuda itself; NULL when the driver does not offer it.
typedef CUresult (*addr_range_fn)(CUdeviceptr* base, size_t* size, CUdeviceptr ptr);
static addr_range_fn addr_range() {
    static std::once_flag once;
    static addr_range_fn fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (addr_range_fn)f;
        (void)cudaGetLastError();
    });
    return fn;
}

// A field-snapshot pointer must be device (or managed) memory of the current device
// whose allocation holds `bytes` from ptr on; checked without allocating anything.
static int check_field_ptr(const char* name, const float* ptr, int dev, size_t bytes) {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(LBM_ERR_INVALID, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(LBM_ERR_INVALID, "%s: host or unregistered memory; device memory required", name);
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return fail(LBM_ERR_INVALID, "%s: memory of device %d, current device %d", name, at.device, dev);
    if (addr_range_fn fn = addr_range()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)(uintptr_t)ptr) != CUDA_SUCCESS)
            return fail(LBM_ERR_INVALID, "%s: address range of the allocation unavailable", name);
        if ((uintptr_t)ptr + bytes > (uintptr_t)base + size)
            return fail(LBM_ERR_INVALID, "%s: its allocation ends %zu bytes after it, %zu needed", name,
                        (size_t)((uintptr_t)base + size - (uintptr_t)ptr), bytes);
    }
    return LBM_OK;
}

extern "C" int lbm_field_residual_noalloc(int32_t geometry, int32_t nr, int32_t nz, double r0, const float* cur,
                                          const float* prev, int64_t field_stride, double* res, double* mass,
                                          void* stream) {
    if (!cur || !prev || !res || !mass) return fail(LBM_ERR_INVALID, "NULL argument");
    if (geometry < 0 || geometry > 3) return fail(LBM_ERR_INVALID, "unknown geometry %d", geometry);
    if (nr < 3 || nz < 3 || nr > 65535 || nz > 65535 || (int64_t)nr * nz >= ((int64_t)1 << 31))
        return fail(LBM_ERR_INVALID, "grid %d x %d outside 3..65535 per side with nr*nz < 2^31", nr, nz);
    const int64_t N = (int64_t)nr * nz;
    if (field_stride < N || field_stride > ((int64_t)1 << 40))
        return fail(LBM_ERR_INVALID, "field_stride %lld outside [nr*nz, 2^40]", (long long)field_stride);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // both snapshots are read over their four planes: 3 * field_stride + nr * nz floats
    const size_t need = (size_t)(3 * field_stride + N) * sizeof(float);
    if (int rc = check_field_ptr("cur", cur, dev, need)) return rc;
    if (int rc = check_field_ptr("prev", prev, dev, need)) return rc;
    // the array's address in the current device's context, looked up on every call (a
    // lookup allocates nothing; an address kept from an earlier context could be stale)
    double* scratch = nullptr;
    CK(cudaGetSymbolAddress((void**)&scratch, g_noalloc_scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>(LBM_NOALLOC_ROWS, (N + 255) / 256);
    double* result = scratch + LBM_NOALLOC_ROWS * RES_NV;
    // every partial row the final sum reads is written by this call: nothing to clear
    k_resid_partial<<<blocks, 256, 0, s>>>(geometry, nr, nz, r0, cur, prev, field_stride, scratch);
    CK(cudaGetLastError());
    k_sum_rows<<<1, 256, 0, s>>>(scratch, blocks, result);
    CK(cudaGetLastError());
    double sum[RES_NV];
    CK(cudaMemcpyAsync(sum, result, sizeof(sum), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sum[5] > 0) return fail(LBM_ERR_DIVERGED, "%.0f nodes hold NaN or Inf", sum[5]);
    const double ru = sum[1] > 0 ? std::sqrt(sum[0] / sum[1]) : (sum[0] > 0 ? INFINITY : 0.0);
    const double rt = sum[3] > 0 ? std::sqrt(sum[2] / sum[3]) : (sum[2] > 0 ? INFINITY : 0.0);
    *res = ru > rt ? ru : rt;
    *mass = sum[4];
    return LBM_OK;
}

// ======================================================================= batch ==
// Many independent problems of uneven size advanced by the same launches.
//
// Layout: one pooled device allocation holds, per instance, state A, state B and the
// porosity plane (each instance's own nr*nz, plane stride padded to 64 elements), and
// a second pool holds two field snapshots (4 planes each) per instance.  A device
// table of InstDesc carries each instance's lattice constants and pool offsets.
// A step is two launches covering every active instance: k_batch_bulk over a
// flattened list of tiles (instance, first row, first column; block shape chosen by
// lbm_batch_tune) and k_batch_wall over the concatenated wall-node lists.  lbm_batch_run
// captures check_every steps (an even number, so every instance's A/B parity is the
// same at each check) in a CUDA graph and replays it; instances that reach the
// steady criterion leave the tile lists at the next check.
struct InstDesc {
    Consts<float> c;
    int64_t off_state[2];   // byte offsets of state buffers A and B in the state pool
    int64_t off_phi;        // byte offset of the porosity plane
    int64_t off_tref;       // byte offset of the reference-offset plane R(x) (FP16)
    int64_t off_fref;       // byte offset of the flow-reference plane Q(x) (16-bit storage)
    int64_t off_mac;        // float offset of the two field snapshots in the snapshot pool
    int64_t plane;          // elements per plane
    double r0, H, dTw;
};

template <int STO>
__device__ __forceinline__ Buf<STO> inst_buf(const InstDesc& d, char* pool, int which) {
    Buf<STO> b;
    b.f = (typename St<STO>::TF*)(pool + d.off_state[which]);
    b.g = (typename St<STO>::TG*)(pool + d.off_state[which] + 9 * d.plane * (int64_t)sizeof(typename St<STO>::TF));
    return b;
}

// Tile = (instance, first row, first column); block = (bz, rows); each thread updates
// RPT consecutive rows of its column (the instance descriptor is read once per thread).
// The per-node source is the single-problem kernel's (update_column); the two kernels
// agree to rounding (the compiler may fuse multiply-adds differently in each).
// Columns a thread of the bulk kernels covers: two with 16-bit storage (update_pair),
// one with FP32 storage.
template <int STO> __host__ __device__ constexpr int bulk_cols() { return has_fref<STO>() ? 2 : 1; }

#ifndef LBM_BATCH_DESC_SMEM
#define LBM_BATCH_DESC_SMEM 1
#endif
// VEC (16-bit storage): every tile of the launch belongs to an instance with even nz, so
// the pair update may use its vector loads; tiles of odd-nz instances go to a VEC = false
// launch (batch_rebuild orders them last).
template <int STO, int RPT, bool VEC>
__global__ void __launch_bounds__(256) k_batch_bulk(const InstDesc* __restrict__ desc, char* __restrict__ pool,
                                                    int parity, const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
#if LBM_BATCH_DESC_SMEM
    // every thread of a tile works on the same instance: its descriptor in shared memory,
    // read from there where the per-node code needs a constant (no register copy of it)
    __shared__ InstDesc sd;
    {
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int nw = (int)(sizeof(InstDesc) / sizeof(int));
        for (int w = tid; w < nw; w += blockDim.x * blockDim.y)
            reinterpret_cast<int*>(&sd)[w] = reinterpret_cast<const int*>(desc + t.x)[w];
        __syncthreads();
    }
    const InstDesc& d = sd;
    const Consts<float>& c = sd.c;
#else
    const InstDesc& d = desc[t.x];
    const Consts<float> c = d.c;
#endif
    const int kz = t.z + bulk_cols<STO>() * threadIdx.x;
    if (kz >= c.nz) return;
    const Buf<STO> A = inst_buf<STO>(d, pool, parity), B = inst_buf<STO>(d, pool, parity ^ 1);
    const typename St<STO>::P* phi = (const typename St<STO>::P*)(pool + d.off_phi);
    const int plane = (int)d.plane;
    if constexpr (has_fref<STO>()) {
        update_pair<STO, VEC>(c, A, B, phi, plane, t.y + threadIdx.y * RPT, RPT, kz);
    } else {
        update_column<STO, int>(c, A, B, phi, plane, t.y + threadIdx.y * RPT, RPT, kz);
    }
}

// 16-bit batches: the staged block (stage_block) over tiles (instance, first row, first
// column, rows) of BATCH_STAGE_NT column pairs of every active instance with even nz; the
// rows per tile (batch_stage_rows) are the same for all tiles of a batch.  On the sweep of 256 instances with Nr 64..512, 128-thread blocks at five
// per SM (the instance's pointers stay live: 102 registers allowed) measured 0.874 ms per
// step, 64-thread blocks 0.927 (ten per SM) and 0.969 (twelve, with spills), although
// 128-column tiles leave fewer thread slots idle on short rows (9 % against 17 %).
#ifndef LBM_BATCH_STAGE_NT
#define LBM_BATCH_STAGE_NT 128
#endif
#ifndef LBM_BATCH_STAGE_MIN_BLOCKS
#define LBM_BATCH_STAGE_MIN_BLOCKS 5
#endif
#ifndef LBM_BATCH_STAGE_MAX_ROWS
#define LBM_BATCH_STAGE_MAX_ROWS 16
#endif
constexpr int BATCH_STAGE_NT = LBM_BATCH_STAGE_NT;
template <int STO>
__global__ void __launch_bounds__(BATCH_STAGE_NT, LBM_BATCH_STAGE_MIN_BLOCKS) k_batch_stage(
    const InstDesc* __restrict__ desc, char* __restrict__ pool, int parity, const int4* __restrict__ tiles, int spin,
    int* __restrict__ status) {
    __shared__ PairStage<BATCH_STAGE_NT> sb;
    __shared__ InstDesc sd;   // the tile's instance: constants read from shared memory
    const int4 t = tiles[blockIdx.x];
    for (int w = threadIdx.x; w < (int)(sizeof(InstDesc) / sizeof(int)); w += BATCH_STAGE_NT)
        reinterpret_cast<int*>(&sd)[w] = reinterpret_cast<const int*>(desc + t.x)[w];
    __syncthreads();
    const Buf<STO> A = inst_buf<STO>(sd, pool, parity), B = inst_buf<STO>(sd, pool, parity ^ 1);
    stage_block<STO, BATCH_STAGE_NT, false>(sd.c, A, B, (const float*)(pool + sd.off_phi), (int)sd.plane, t.y, t.w, t.z,
                                            spin, status, sb);
}

// Flow reference refresh of every node the tiles cover (all nodes of the active instances),
// with the bulk kernels' tiles and block shape.
template <int STO, int RPT>
__global__ void __launch_bounds__(256) k_batch_rebase_flow(const InstDesc* __restrict__ desc, char* __restrict__ pool,
                                                           int parity, const int4* __restrict__ tiles) {
    if constexpr (has_fref<STO>()) {
        const int4 t = tiles[blockIdx.x];
        const InstDesc& d = desc[t.x];
        const Consts<float> c = d.c;
        const Buf<STO> S = inst_buf<STO>(d, pool, parity);
        uint2* fref = (uint2*)(pool + d.off_fref);
#pragma unroll 1
        for (int q = 0; q < RPT * bulk_cols<STO>(); ++q) {
            const int kr = t.y + threadIdx.y * RPT + q / bulk_cols<STO>();
            const int kz = t.z + bulk_cols<STO>() * threadIdx.x + q % bulk_cols<STO>();
            if (kr >= c.nr) break;
            if (kz >= c.nz) continue;
            rebase_16_node<STO, LAY_N, int>(c, S, (int)d.plane, kr, kz, kr * c.nz + kz, fref);
        }
    }
}

// Wall nodes of all active instances: prefix[k] = first wall thread of active instance k.
__device__ __forceinline__ int find_slot(const int* __restrict__ prefix, int n, int t) {
    int lo = 0, hi = n;   // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int STO>
__global__ void k_batch_wall(const InstDesc* __restrict__ desc, char* __restrict__ pool, int parity,
                             const int* __restrict__ active, const int* __restrict__ prefix, int nactive) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= prefix[nactive]) return;
    const int k = find_slot(prefix, nactive, t);
    const InstDesc& d = desc[active[k]];
    const Consts<float> c = d.c;
    int kr, kz;
    wall_node(c.geometry, c.nr, c.nz, t - prefix[k], kr, kz);
    const int cls = node_class(c.geometry, c.nr, c.nz, kr, kz);
    const Buf<STO> A = inst_buf<STO>(d, pool, parity), B = inst_buf<STO>(d, pool, parity ^ 1);
    const typename St<STO>::P* phi = (const typename St<STO>::P*)(pool + d.off_phi);
    float fh[9], gh[5], m0, rho, urb, uzb, dTb, refb;
    wall_state<STO>(c, A, phi, d.plane, cls, kr, kz, fh, gh, m0, rho, urb, uzb, dTb, refb);
    const int64_t n = (int64_t)kr * c.nz + kz;
    const float r = c.r0 + float(kr), ph = ldv(phi + n);
    float lin, nl, iph;
    porous(c, ph, lin, nl, iph);
    collide(c, r, rcp_acc(r), ph, lin, nl, iph, fh, gh, refb, m0, rho, urb, uzb, dTb);
    store<STO>(c, B, d.plane, kr, kz, n, fh, gh);
}

// Field snapshot `slot` (0 or 1) of every instance the tiles cover, all nodes.
template <int STO, int RPT>
__global__ void __launch_bounds__(256) k_batch_moments(const InstDesc* __restrict__ desc, char* __restrict__ pool,
                                                       float* __restrict__ macpool, int parity, int slot,
                                                       const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const InstDesc& d = desc[t.x];
    const Consts<float> c = d.c;
    const Buf<STO> A = inst_buf<STO>(d, pool, parity);
    const typename St<STO>::P* phi = (const typename St<STO>::P*)(pool + d.off_phi);
    float* m = macpool + d.off_mac + (int64_t)slot * 4 * d.plane;
#pragma unroll 1
    for (int q = 0; q < RPT * bulk_cols<STO>(); ++q) {
        const int j = q / bulk_cols<STO>();
        const int kz = t.z + bulk_cols<STO>() * threadIdx.x + q % bulk_cols<STO>();
        const int kr = t.y + threadIdx.y * RPT + j;
        if (kr >= c.nr) break;
        if (kz >= c.nz) continue;
        const int cls = node_class(c.geometry, c.nr, c.nz, kr, kz);
        const int64_t n = (int64_t)kr * c.nz + kz;
        float fh[9], gh[5], m0, rho, ur = 0.f, uz = 0.f, dT, ref;
        if (is_wall(cls)) {
            wall_state<STO>(c, A, phi, d.plane, cls, kr, kz, fh, gh, m0, rho, ur, uz, dT, ref);
        } else {
            pull<STO>(c, A, d.plane, kr, kz, fh, gh, ref);
            const float r = c.r0 + float(kr), ph = ldv(phi + n);
            float lin, nl, iph;
            porous(c, ph, lin, nl, iph);
            recover(c, r, rcp_acc(r), ph, lin, nl, fh, gh, ref, m0, rho, ur, uz, dT);
        }
        m[n] = rho;
        m[d.plane + n] = ur;
        m[2 * d.plane + n] = uz;
        m[3 * d.plane + n] = (c.T0 + ref) + dT;
    }
}

// Per-instance residual sums between the two snapshots (cur = slot `cur`): grid
// (RB, nactive); partial rows [k][block][RES_NV].
constexpr int BATCH_RB = 16;
__global__ void k_batch_resid(const InstDesc* __restrict__ desc, const float* __restrict__ macpool, int cur,
                              const int* __restrict__ active, double* __restrict__ partials) {
    const int k = blockIdx.y;
    const InstDesc& d = desc[active[k]];
    const int nr = d.c.nr, nz = d.c.nz, geometry = d.c.geometry;
    const float* C = macpool + d.off_mac + (int64_t)cur * 4 * d.plane;
    const float* P = macpool + d.off_mac + (int64_t)(cur ^ 1) * 4 * d.plane;
    const int64_t fs = d.plane;
    double v[RES_NV] = {0, 0, 0, 0, 0, 0};
    const int64_t N = (int64_t)nr * nz;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int kr = (int)(n / nz), kz = (int)(n - (int64_t)kr * nz);
        const float rho = C[n], ur = C[fs + n], uz = C[2 * fs + n], T = C[3 * fs + n];
        if (!isfinite(rho) || !isfinite(ur) || !isfinite(uz) || !isfinite(T)) v[5] += 1;
        v[4] += (d.r0 + kr) * (double)rho;
        if (is_wall(node_class(geometry, nr, nz, kr, kz))) continue;
        const double a = (double)ur - P[fs + n], b = (double)uz - P[2 * fs + n], e = (double)T - P[3 * fs + n];
        v[0] += a * a + b * b;
        v[1] += (double)ur * ur + (double)uz * uz;
        v[2] += e * e;
        v[3] += (double)T * T;
    }
    double out[RES_NV];
    block_sum<RES_NV>(v, out);
    if (threadIdx.x == 0)
        for (int j = 0; j < RES_NV; ++j) partials[((int64_t)k * gridDim.x + blockIdx.x) * RES_NV + j] = out[j];
}

__global__ void k_batch_resid_final(const double* __restrict__ partials, int rb, double* __restrict__ result) {
    const int k = blockIdx.x;
    double v[RES_NV] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < rb; b += blockDim.x)
        for (int j = 0; j < RES_NV; ++j) v[j] += partials[((int64_t)k * rb + b) * RES_NV + j];
    double out[RES_NV];
    block_sum<RES_NV>(v, out);
    if (threadIdx.x == 0)
        for (int j = 0; j < RES_NV; ++j) result[(int64_t)k * RES_NV + j] = out[j];
}

// Eq. 42 for every instance (one block each).
template <int STO>
__global__ void __launch_bounds__(256) k_batch_nusselt(const InstDesc* __restrict__ desc, char* __restrict__ pool,
                                                       const int* __restrict__ parity, double* __restrict__ result) {
    const InstDesc& d = desc[blockIdx.x];
    const Consts<float> c = d.c;
    const Buf<STO> A = inst_buf<STO>(d, pool, parity[blockIdx.x]);
    double v[2] = {0, 0};
    for (int kz = threadIdx.x; kz < c.nz; kz += blockDim.x) {
        const double wz = (kz == 0 || kz == c.nz - 1) ? 0.5 : 1.0;
        const double t0 = node_T<STO>(c, A, d.plane, 0, kz), t1 = node_T<STO>(c, A, d.plane, 1, kz);
        const double t2 = node_T<STO>(c, A, d.plane, 2, kz);
        const double u0 = node_T<STO>(c, A, d.plane, c.nr - 1, kz), u1 = node_T<STO>(c, A, d.plane, c.nr - 2, kz);
        const double u2 = node_T<STO>(c, A, d.plane, c.nr - 3, kz);
        v[0] += wz * (-3 * t0 + 4 * t1 - t2) * 0.5;
        v[1] += wz * (3 * u0 - 4 * u1 + u2) * 0.5;
    }
    double out[2];
    block_sum<2>(v, out);
    if (threadIdx.x == 0) {
        const double ro = d.r0 + (c.nr - 1);
        result[2 * blockIdx.x] = -d.r0 * out[0] / (d.H * d.dTw);
        result[2 * blockIdx.x + 1] = -ro * out[1] / (d.H * d.dTw);
    }
}

struct lbm_batch {
    int n = 0;
    int storage = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the wall kernel runs beside the bulk kernels on its own stream (fork / join per step)
    cudaStream_t wstream = nullptr;
    cudaEvent_t wfork = nullptr, wjoin = nullptr;
    std::vector<lbm_params> p;
    std::vector<lbm_info> info;
    std::vector<Consts<double>> cd;
    std::vector<InstDesc> desc;       // host copy
    InstDesc* d_desc = nullptr;
    char* pool = nullptr;
    float* macpool = nullptr;
    float* fstage = nullptr;          // largest instance: 3 planes (porosity or warm-start upload)
    int64_t max_plane = 0;
    int parity = 0;
    int64_t steps = 0;
    int64_t since_rebase = 0;         // steps since the last flow-reference refresh (16-bit)
    std::vector<char> active;         // 1 = still stepping
    // tiles and wall lists of the active set
    int bz = 128, rows = 1, rpt = 1;  // bulk block shape and rows per thread
    int4* d_tiles = nullptr;          // active instances, all rows
    int ntiles = 0;
    int ntiles_even = 0;              // leading tiles of instances with even nz
    int* d_active = nullptr;
    int* d_prefix = nullptr;
    int nactive = 0;
    int nwall = 0;
    size_t cap_tiles = 0;
    double* partials = nullptr;
    double* result = nullptr;
    std::vector<int> iparity;         // buffer holding the state of an instance that stopped
    int4* d_stiles = nullptr;         // 16-bit: staged tiles of the active instances with even nz
    int nstiles = 0;
    size_t cap_stiles = 0;
    int* wait_status = nullptr;       // 16-bit: LBM_ERR_TIMEOUT once a bounded wait of k_batch_stage ran out
    int spin = STAGE_SPIN;            // try_wait rounds of its per-row waits
    int stage = 1;                    // 16-bit: staged tiles for the even-nz instances (lbm_batch_set_staging)
    int sms = 0;                      // multiprocessors of the device
    cudaGraphExec_t graph = nullptr;
    int64_t graph_steps = 0;
    int graph_parity = 0;             // batch parity the graph was captured at
    bool graph_dirty = true;
    int cur_parity(int i) const { return active[i] ? parity : iparity[i]; }
};

static void batch_free_graph(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_dirty = true;
}

// Rebuild the tile list, the active list and the wall prefix for the current active
// set and block shape.
// Rows per staged tile: the most (of 16, 8, 4, 2) that still leave the tiles at least four
// waves of resident blocks, since a block overlaps only the copies of its own next row
// with its compute (the 256-instance sweep ran at 0.844 ms per step with 16 rows, 0.847
// with 8, 0.874 with 4 and 0.944 with 2; 16 small instances of 1 M nodes at 31.8 us with
// 8 rows, 27.8 with 4 and 26.5 with 2).
static int batch_stage_rows(const lbm_batch* b, const std::vector<int>& act) {
    const int64_t want = 4LL * LBM_BATCH_STAGE_MIN_BLOCKS * b->sms;
    for (int r = LBM_BATCH_STAGE_MAX_ROWS; r > 2; r /= 2) {
        int64_t n = 0;
        for (int i : act)
            if (!(b->p[i].nz & 1))
                n += (int64_t)((b->p[i].nr + r - 1) / r) * ((b->p[i].nz + 2 * BATCH_STAGE_NT - 1) / (2 * BATCH_STAGE_NT));
        if (n >= want) return r;
    }
    return 2;
}

static int batch_rebuild(lbm_batch* b) {
    std::vector<int4> tiles, odd;   // tiles of instances with odd nz last (k_batch_bulk's VEC)
    std::vector<int> act, prefix(1, 0);
    for (int i = 0; i < b->n; ++i) {
        if (!b->active[i]) continue;
        act.push_back(i);
        prefix.push_back(prefix.back() + wall_count(b->p[i].geometry, b->p[i].nr, b->p[i].nz));
        const int zstep = b->bz * (b->storage == LBM_F32 ? 1 : 2);   // columns of a tile (bulk_cols)
        std::vector<int4>& dst = (b->p[i].nz & 1) ? odd : tiles;
        for (int kr = 0; kr < b->p[i].nr; kr += b->rows * b->rpt)
            for (int z0 = 0; z0 < b->p[i].nz; z0 += zstep) dst.push_back(make_int4(i, kr, z0, 0));
    }
    b->ntiles_even = (int)tiles.size();
    tiles.insert(tiles.end(), odd.begin(), odd.end());
    std::vector<int4> st;
    if (b->storage != LBM_F32 && b->stage) {
        const int rpt = batch_stage_rows(b, act);
        for (int i : act)
            if (!(b->p[i].nz & 1))
                for (int kr = 0; kr < b->p[i].nr; kr += rpt)
                    for (int z0 = 0; z0 < b->p[i].nz; z0 += 2 * BATCH_STAGE_NT) st.push_back(make_int4(i, kr, z0, rpt));
    }
    b->nstiles = (int)st.size();
    if (st.size() > b->cap_stiles) {
        cudaFree(b->d_stiles);
        b->d_stiles = nullptr;
        CK(cudaMalloc((void**)&b->d_stiles, st.size() * sizeof(int4)));
        b->cap_stiles = st.size();
    }
    if (!st.empty())
        CK(cudaMemcpyAsync(b->d_stiles, st.data(), st.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    b->ntiles = (int)tiles.size();
    b->nactive = (int)act.size();
    b->nwall = prefix.back();
    if ((size_t)b->ntiles > b->cap_tiles) {
        cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        CK(cudaMalloc((void**)&b->d_tiles, tiles.size() * sizeof(int4)));
        b->cap_tiles = tiles.size();
    }
    if (b->ntiles)
        CK(cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    if (b->nactive) {
        CK(cudaMemcpyAsync(b->d_active, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    }
    CK(cudaMemcpyAsync(b->d_prefix, prefix.data(), prefix.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    batch_free_graph(b);
    return LBM_OK;
}

template <int STO> static Buf<STO> batch_buf(const lbm_batch* b, int i, int which) {
    const InstDesc& d = b->desc[i];
    Buf<STO> r;
    r.f = (typename St<STO>::TF*)(b->pool + d.off_state[which]);
    r.g = (typename St<STO>::TG*)(b->pool + d.off_state[which] + 9 * d.plane * (int64_t)sizeof(typename St<STO>::TF));
    return r;
}

// Flow-reference refresh of every active instance (16-bit storage), one launch.
static int batch_launch_rebase_flow(lbm_batch* b) {
    if (b->storage != LBM_F32 && b->nactive) {
        const dim3 blk(b->bz, b->rows);
        DISPATCH_STO16(b->storage, DISPATCH_RPT(b->rpt, k_batch_rebase_flow<S_, R_><<<b->ntiles, blk, 0, b->stream>>>(
                                                            b->d_desc, b->pool, b->parity, b->d_tiles)));
        CK(cudaGetLastError());
    }
    b->since_rebase = 0;
    return LBM_OK;
}

static int batch_launch_step(lbm_batch* b) {
    if (!b->nactive) return LBM_OK;
    // 16-bit storage: the refresh of lbm_step, every LBM_FREF_EVERY steps since the last
    if (b->storage != LBM_F32 && b->since_rebase >= LBM_FREF_EVERY)
        if (int rc = batch_launch_rebase_flow(b)) return rc;
    // the wall kernel reads only the pre-step states and writes only boundary nodes, which
    // the bulk kernels do not touch: it runs beside them on the wall stream
    CK(cudaEventRecord(b->wfork, b->stream));
    CK(cudaStreamWaitEvent(b->wstream, b->wfork, 0));
    DISPATCH_STO(b->storage, k_batch_wall<S_><<<(b->nwall + 127) / 128, 128, 0, b->wstream>>>(
                                 b->d_desc, b->pool, b->parity, b->d_active, b->d_prefix, b->nactive));
    CK(cudaGetLastError());
    const dim3 blk(b->bz, b->rows);
    if (b->storage == LBM_F32) {
        DISPATCH_RPT(b->rpt, k_batch_bulk<LBM_F32, R_, false><<<b->ntiles, blk, 0, b->stream>>>(
                                 b->d_desc, b->pool, b->parity, b->d_tiles));
    } else {
        const int ne = b->ntiles_even, no = b->ntiles - b->ntiles_even;
        if (b->stage) {   // even nz: staged tiles
            if (b->nstiles)
                DISPATCH_STO16(b->storage, k_batch_stage<S_><<<b->nstiles, BATCH_STAGE_NT, 0, b->stream>>>(
                                               b->d_desc, b->pool, b->parity, b->d_stiles, b->spin, b->wait_status));
        } else if (ne) {
            DISPATCH_STO16(b->storage, DISPATCH_RPT(b->rpt, k_batch_bulk<S_, R_, true><<<ne, blk, 0, b->stream>>>(
                                                                b->d_desc, b->pool, b->parity, b->d_tiles)));
        }
        if (no)
            DISPATCH_STO16(b->storage, DISPATCH_RPT(b->rpt, k_batch_bulk<S_, R_, false><<<no, blk, 0, b->stream>>>(
                                                                b->d_desc, b->pool, b->parity, b->d_tiles + ne)));
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(b->wjoin, b->wstream));
    CK(cudaStreamWaitEvent(b->stream, b->wjoin, 0));
    b->parity ^= 1;
    b->since_rebase += 1;
    return LBM_OK;
}

extern "C" {

int lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->wstream) {
        cudaStreamSynchronize(b->wstream);
        cudaStreamDestroy(b->wstream);
    }
    if (b->wfork) cudaEventDestroy(b->wfork);
    if (b->wjoin) cudaEventDestroy(b->wjoin);
    batch_free_graph(b);
    cudaFree(b->d_desc);
    cudaFree(b->pool);
    cudaFree(b->macpool);
    cudaFree(b->fstage);
    cudaFree(b->d_tiles);
    cudaFree(b->d_stiles);
    cudaFree(b->wait_status);
    cudaFree(b->d_active);
    cudaFree(b->d_prefix);
    cudaFree(b->partials);
    cudaFree(b->result);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

int lbm_batch_create(const lbm_params* p, int32_t n, lbm_batch** out) {
    if (!p || !out || n < 1) return fail(LBM_ERR_INVALID, "need params[n], n >= 1 and an output pointer");
    *out = nullptr;
    lbm_batch* b = new lbm_batch();
    b->n = n;
    b->storage = p[0].storage;
    b->p.assign(p, p + n);
    b->info.resize(n);
    b->cd.resize(n);
    b->desc.resize(n);
    int64_t state_off = 0, mac_off = 0;
    for (int i = 0; i < n; ++i) {
        int rc = derive(&p[i], &b->info[i], &b->cd[i]);
        if (rc) { delete b; return fail(rc, "instance %d: %s", i, g_err.c_str()); }
        if (p[i].storage != b->storage) { delete b; return fail(LBM_ERR_INVALID, "instance %d: storage differs", i); }
        if (p[i].inplace) { delete b; return fail(LBM_ERR_INVALID, "instance %d: in-place storage is for lbm_create", i); }
        const int64_t N = (int64_t)p[i].nr * p[i].nz, plane = (N + 63) / 64 * 64;
        if (14 * plane >= ((int64_t)1 << 31)) { delete b; return fail(LBM_ERR_INVALID, "instance %d too large", i); }
        InstDesc& d = b->desc[i];
        d.c = to_float(b->cd[i]);
        d.plane = plane;
        d.off_state[0] = state_off;
        state_off += (int64_t)state_bytes(b->storage, plane);
        d.off_state[1] = state_off;
        state_off += (int64_t)state_bytes(b->storage, plane);
        d.off_phi = state_off;
        state_off += (plane * (int64_t)phi_size(b->storage) + 255) / 256 * 256;
        d.off_tref = state_off;   // R(x) plane (FP32 storage) or reference words (16-bit storage)
        d.off_fref = state_off;
        state_off += (plane * (int64_t)(p[i].storage == LBM_F32 ? sizeof(__half) : sizeof(uint2)) + 255) / 256 * 256;
        d.off_mac = mac_off;
        mac_off += 8 * plane;
        d.r0 = b->info[i].r0;
        d.H = b->info[i].H;
        d.dTw = p[i].T_hot - p[i].T_cold;
        b->max_plane = std::max(b->max_plane, plane);
    }
    b->active.assign(n, 1);
    b->iparity.assign(n, 0);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->wstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->wfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->wjoin, cudaEventDisableTiming);
    b->own_stream = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->pool, state_off);
    if (e == cudaSuccess)
        for (int i = 0; i < n; ++i) {
            const __half* tr = b->storage == LBM_F32 ? (const __half*)(b->pool + b->desc[i].off_tref) : nullptr;
            b->desc[i].c.tref = tr;
            b->cd[i].tref = tr;
            const uint2* fr = b->storage == LBM_F32 ? nullptr : (const uint2*)(b->pool + b->desc[i].off_fref);
            b->desc[i].c.fref = fr;
            b->cd[i].fref = fr;
        }
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->macpool, mac_off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_desc, n * sizeof(InstDesc));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_active, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_prefix, (n + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->partials, (size_t)n * BATCH_RB * RES_NV * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->result, (size_t)n * RES_NV * sizeof(double));
    if (e == cudaSuccess && b->storage != LBM_F32) {
        e = cudaMalloc((void**)&b->wait_status, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->wait_status, 0, sizeof(int), b->stream);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(b->storage == LBM_F16 ? k_batch_stage<LBM_F16> : k_batch_stage<LBM_BF16>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_desc, b->desc.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice,
                                              b->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        lbm_batch_destroy(b);
        return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "batch allocation: %s",
                    cudaGetErrorString(e));
    }
    // uniform porosity and the cold start of every instance
    for (int i = 0; i < n; ++i) {
        const InstDesc& d = b->desc[i];
        const int64_t N = (int64_t)p[i].nr * p[i].nz;
        const dim3 g((unsigned)((p[i].nz + 127) / 128), (unsigned)p[i].nr);
        DISPATCH_STO(b->storage, {
            k_phi_fill<S_><<<(unsigned)((N + 255) / 256), 256, 0, b->stream>>>((PP<S_>*)(b->pool + d.off_phi), N,
                                                                                (float)p[i].eps_mean);
            k_init<S_><<<g, 128, 0, b->stream>>>(b->cd[i], batch_buf<S_>(b, i, 0), (const PP<S_>*)(b->pool + d.off_phi),
                                                 d.plane, nullptr, nullptr, nullptr, p[i].init_noise, p[i].seed,
                                                 (__half*)(b->pool + d.off_tref), (uint2*)b->cd[i].fref, 0);
        });
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return fail(LBM_ERR_CUDA, "batch initialisation: %s", cudaGetErrorString(e));
    }
    int rc = batch_rebuild(b);
    if (rc) { lbm_batch_destroy(b); return rc; }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch* b, void* stream) {
    if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
    if (!stream) return fail(LBM_ERR_INVALID, "a batch needs a created stream (graph capture)");
    CK(cudaSetDevice(b->device));
    CK(cudaStreamSynchronize(b->stream));
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->own_stream = false;
    b->stream = (cudaStream_t)stream;
    batch_free_graph(b);
    return LBM_OK;
}

static int batch_upload(lbm_batch* b, const float* src, int64_t N, int slot, const float** dev) {
    if (!b->fstage) CK(cudaMalloc((void**)&b->fstage, 3 * b->max_plane * sizeof(float)));
    CK(cudaMemcpyAsync(b->fstage + slot * b->max_plane, src, N * sizeof(float), cudaMemcpyHostToDevice, b->stream));
    *dev = b->fstage + slot * b->max_plane;
    return LBM_OK;
}

int lbm_batch_set_porosity(lbm_batch* b, int32_t i, const float* phi, int on_device) {
    if (!b || !phi || i < 0 || i >= b->n) return fail(LBM_ERR_INVALID, "bad batch, instance or pointer");
    CK(cudaSetDevice(b->device));
    const int64_t N = (int64_t)b->p[i].nr * b->p[i].nz;
    const float* src = phi;
    int rc;
    if (!on_device && (rc = batch_upload(b, phi, N, 0, &src))) return rc;
    unsigned int* bad = (unsigned int*)b->result;   // scratch word
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned int), b->stream));
    DISPATCH_STO(b->storage, k_phi<S_><<<phi_blocks(N), 256, 0, b->stream>>>(
                                 src, (PP<S_>*)(b->pool + b->desc[i].off_phi), N, aligned16(src), bad));
    CK(cudaGetLastError());
    unsigned int nb = 0;
    CK(cudaMemcpyAsync(&nb, bad, sizeof(nb), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (nb) return fail(LBM_ERR_INVALID, "instance %d: %u porosity values outside (0, 1]", i, nb);
    return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch* b, int32_t i, const float* ur, const float* uz, const float* T, int on_device) {
    if (!b || i < 0 || i >= b->n) return fail(LBM_ERR_INVALID, "bad batch or instance");
    if ((ur == nullptr) != (uz == nullptr)) return fail(LBM_ERR_INVALID, "give both u_r and u_z or neither");
    CK(cudaSetDevice(b->device));
    const int64_t N = (int64_t)b->p[i].nr * b->p[i].nz;
    const float *dur = ur, *duz = uz, *dT = T;
    int rc;
    if (!on_device) {
        if (ur && ((rc = batch_upload(b, ur, N, 0, &dur)) || (rc = batch_upload(b, uz, N, 1, &duz)))) return rc;
        if (T && (rc = batch_upload(b, T, N, 2, &dT))) return rc;
    }
    const InstDesc& d = b->desc[i];
    const dim3 g((unsigned)((b->p[i].nz + 127) / 128), (unsigned)b->p[i].nr);
    // the instance's current buffer is the batch parity
    DISPATCH_STO(b->storage, k_init<S_><<<g, 128, 0, b->stream>>>(b->cd[i], batch_buf<S_>(b, i, b->parity),
                                                                   (const PP<S_>*)(b->pool + d.off_phi), d.plane, dur,
                                                                   duz, dT, b->p[i].init_noise, b->p[i].seed,
                                                                   (__half*)(b->pool + d.off_tref), (uint2*)b->cd[i].fref,
                                                                   0));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(b->stream));
    if (!b->active[i]) {
        b->active[i] = 1;
        return batch_rebuild(b);
    }
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return fail(LBM_ERR_INVALID, "bad batch or nsteps");
    CK(cudaSetDevice(b->device));
    for (int64_t s = 0; s < nsteps; ++s) {
        int rc = batch_launch_step(b);
        if (rc) return rc;
    }
    b->steps += nsteps;
    return LBM_OK;
}

// Reference refresh of instance i (the kernel of lbm_rebase, on the instance's current
// buffer).
static int batch_rebase_one(lbm_batch* b, int i) {
    const InstDesc& d = b->desc[i];
    const int64_t N = (int64_t)b->p[i].nr * b->p[i].nz;
    const unsigned blocks = (unsigned)std::min<int64_t>((N + 255) / 256, 4096);
    if (b->storage == LBM_F32) {
        k_rebase<LBM_F32><<<blocks, 256, 0, b->stream>>>(d.c, batch_buf<LBM_F32>(b, i, b->cur_parity(i)), d.plane, N,
                                                         (__half*)(b->pool + d.off_tref));
    } else {
        DISPATCH_STO16(b->storage, k_rebase_16<S_><<<blocks, 256, 0, b->stream>>>(
                                       d.c, batch_buf<S_>(b, i, b->cur_parity(i)), d.plane, N,
                                       (uint2*)(b->pool + d.off_fref)));
    }
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_batch_rebase(lbm_batch* b) {
    if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
    CK(cudaSetDevice(b->device));
    for (int i = 0; i < b->n; ++i) {
        int rc = batch_rebase_one(b, i);
        if (rc) return rc;
    }
    b->since_rebase = 0;
    return LBM_OK;
}

// Snapshot `slot` of every active instance.
static int batch_snapshot(lbm_batch* b, int slot) {
    // moments use all rows of the active instances: the bulk tiles cover them
    const dim3 blk(b->bz, b->rows);
    DISPATCH_STO(b->storage, DISPATCH_RPT(b->rpt, k_batch_moments<S_, R_><<<b->ntiles, blk, 0, b->stream>>>(
                                                       b->d_desc, b->pool, b->macpool, b->parity, slot, b->d_tiles)));
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_batch_run(lbm_batch* b, int64_t max_steps, int64_t check_every, double tol, int64_t* steps_out,
                  double* res_out) {
    if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
    if (max_steps < 0 || check_every < 2 || (check_every & 1))
        return fail(LBM_ERR_INVALID, "max_steps >= 0 and an even check_every >= 2 required");
    CK(cudaSetDevice(b->device));
    std::vector<int64_t> done(b->n, 0);
    std::vector<double> res(b->n, INFINITY);
    int slot = 0;
    int rc = batch_snapshot(b, slot ^ 1);
    if (rc) return rc;
    int64_t total = 0;
    while (total < max_steps && b->nactive > 0) {
        const int64_t k = std::min(check_every, max_steps - total);
        // reference refresh before every check interval, as lbm_run does
        if (b->storage == LBM_F32) {
            for (int i = 0; i < b->n; ++i)
                if (b->active[i] && (rc = batch_rebase_one(b, i))) return rc;
        } else if ((rc = batch_launch_rebase_flow(b))) {
            return rc;
        }
        b->since_rebase = 0;
        if (k == check_every) {
            if (b->graph_dirty || b->graph_steps != k || b->graph_parity != b->parity) {
                batch_free_graph(b);
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                const int p0 = b->parity;
                for (int64_t s = 0; s < k; ++s) {
                    rc = batch_launch_step(b);
                    if (rc) break;
                }
                b->parity = p0;   // replays start from the same parity (k is even)
                cudaError_t e = cudaStreamEndCapture(b->stream, &g);
                if (rc) { if (g) cudaGraphDestroy(g); return rc; }
                if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
                e = cudaGraphInstantiate(&b->graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
                b->graph_steps = k;
                b->graph_parity = p0;
                b->graph_dirty = false;
            }
            CK(cudaGraphLaunch(b->graph, b->stream));
        } else {
            for (int64_t s = 0; s < k; ++s)
                if ((rc = batch_launch_step(b))) return rc;
            // an odd tail leaves the parity flipped, which the launches already track
        }
        total += k;
        b->steps += k;
        for (int i = 0; i < b->n; ++i)
            if (b->active[i]) done[i] += k;
        if ((rc = lbm_batch_wait_status(b, 0))) return rc;   // before the residual reads an invalid state
        if ((rc = batch_snapshot(b, slot))) return rc;
        const dim3 grid(BATCH_RB, b->nactive);
        k_batch_resid<<<grid, 256, 0, b->stream>>>(b->d_desc, b->macpool, slot, b->d_active, b->partials);
        CK(cudaGetLastError());
        k_batch_resid_final<<<b->nactive, 256, 0, b->stream>>>(b->partials, BATCH_RB, b->result);
        CK(cudaGetLastError());
        std::vector<double> s((size_t)b->nactive * RES_NV);
        CK(cudaMemcpyAsync(s.data(), b->result, s.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        std::vector<int> act;
        for (int i = 0; i < b->n; ++i)
            if (b->active[i]) act.push_back(i);
        bool changed = false;
        int diverged = -1;
        for (int j = 0; j < b->nactive; ++j) {
            const double* q = &s[(size_t)j * RES_NV];
            const int i = act[j];
            if (q[5] > 0) {
                diverged = i;
                b->active[i] = 0;
                b->iparity[i] = b->parity;
                changed = true;
                continue;
            }
            const double ru = q[1] > 0 ? std::sqrt(q[0] / q[1]) : (q[0] > 0 ? INFINITY : 0.0);
            const double rt = q[3] > 0 ? std::sqrt(q[2] / q[3]) : (q[2] > 0 ? INFINITY : 0.0);
            res[i] = (ru > rt ? ru : rt) / (double)k;
            if (res[i] <= tol) {
                b->active[i] = 0;
                b->iparity[i] = b->parity;
                changed = true;
            }
        }
        slot ^= 1;
        if (changed && (rc = batch_rebuild(b))) return rc;
        if (diverged >= 0) {
            if (steps_out) std::copy(done.begin(), done.end(), steps_out);
            if (res_out) std::copy(res.begin(), res.end(), res_out);
            return fail(LBM_ERR_DIVERGED, "instance %d holds NaN or Inf", diverged);
        }
    }
    if (steps_out) std::copy(done.begin(), done.end(), steps_out);
    if (res_out) std::copy(res.begin(), res.end(), res_out);
    return LBM_OK;
}

int lbm_batch_nusselt(lbm_batch* b, double* nu_inner, double* nu_outer) {
    if (!b || !nu_inner || !nu_outer) return fail(LBM_ERR_INVALID, "NULL argument");
    CK(cudaSetDevice(b->device));
    std::vector<int> par(b->n);
    for (int i = 0; i < b->n; ++i) par[i] = b->cur_parity(i);
    int* d_par = (int*)(b->partials);   // scratch: n ints fit in the partial rows
    CK(cudaMemcpyAsync(d_par, par.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    DISPATCH_STO(b->storage, k_batch_nusselt<S_><<<b->n, 256, 0, b->stream>>>(b->d_desc, b->pool, d_par, b->result));
    CK(cudaGetLastError());
    std::vector<double> r(2 * (size_t)b->n);
    CK(cudaMemcpyAsync(r.data(), b->result, r.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        const bool no_eq42 = b->p[i].geometry == LBM_PIPE_INFLOW || b->p[i].heater_len > 0;
        nu_inner[i] = b->p[i].geometry == LBM_PIPE_PERIODIC_Z || no_eq42 ? NAN : r[2 * i];
        nu_outer[i] = no_eq42 ? NAN : r[2 * i + 1];
    }
    return LBM_OK;
}

int lbm_batch_pipe_nusselt(lbm_batch* b, int32_t i, double* nu, int32_t nz) {
    if (!b || !nu || i < 0 || i >= b->n) return fail(LBM_ERR_INVALID, "bad batch, instance or pointer");
    if (b->p[i].geometry != LBM_PIPE_INFLOW) return fail(LBM_ERR_INVALID, "instance %d is not LBM_PIPE_INFLOW", i);
    if (nz != b->p[i].nz) return fail(LBM_ERR_INVALID, "nz = %d, instance %d has %d", nz, i, b->p[i].nz);
    CK(cudaSetDevice(b->device));
    const InstDesc& d = b->desc[i];
    float* m = b->macpool + d.off_mac;   // snapshot slot 0 of this instance as staging
    const dim3 g((unsigned)((nz + 127) / 128), (unsigned)b->p[i].nr);
    DISPATCH_STO(b->storage, k_moments<S_><<<g, 128, 0, b->stream>>>(d.c, batch_buf<S_>(b, i, b->cur_parity(i)),
                                                                      (const PP<S_>*)(b->pool + d.off_phi), d.plane,
                                                                      nullptr, nullptr, m + 2 * d.plane,
                                                                      m + 3 * d.plane));
    CK(cudaGetLastError());
    double* dn = nullptr;
    CK(cudaMallocAsync((void**)&dn, (size_t)nz * sizeof(double), b->stream));
    k_pipe_nusselt<<<(unsigned)((nz + 127) / 128), 128, 0, b->stream>>>(b->p[i].nr, nz, d.r0, m + 2 * d.plane,
                                                                        m + 3 * d.plane, dn);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(nu, dn, (size_t)nz * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    cudaFreeAsync(dn, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "batch pipe Nusselt: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch* b, int32_t i, float* rho, float* ur, float* uz, float* T, int on_device) {
    if (!b || i < 0 || i >= b->n) return fail(LBM_ERR_INVALID, "bad batch or instance");
    CK(cudaSetDevice(b->device));
    const InstDesc& d = b->desc[i];
    const int64_t N = (int64_t)b->p[i].nr * b->p[i].nz;
    float* m = b->macpool + d.off_mac;   // snapshot slot 0 of this instance as staging
    const dim3 g((unsigned)((b->p[i].nz + 127) / 128), (unsigned)b->p[i].nr);
    float* outs[4] = {rho, ur, uz, T};
    float* dst[4];
    for (int j = 0; j < 4; ++j) dst[j] = on_device ? outs[j] : (outs[j] ? m + j * d.plane : nullptr);
    DISPATCH_STO(b->storage, k_moments<S_><<<g, 128, 0, b->stream>>>(d.c, batch_buf<S_>(b, i, b->cur_parity(i)),
                                                                      (const PP<S_>*)(b->pool + d.off_phi), d.plane,
                                                                      dst[0], dst[1], dst[2], dst[3]));
    CK(cudaGetLastError());
    if (!on_device)
        for (int j = 0; j < 4; ++j)
            if (outs[j]) CK(cudaMemcpyAsync(outs[j], dst[j], N * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// Autotuner: time `steps` batched steps for each bulk tile shape (columns x rows per
// block x rows per thread, at most 256 threads) and keep the fastest.  Leaves the state
// advanced by the steps it ran (2 warm-up + `steps` per shape).
static const int kTuneShapes[][3] = {{64, 1, 1}, {128, 1, 1}, {256, 1, 1}, {64, 2, 1}, {128, 2, 1}, {64, 4, 1},
                                     {32, 8, 1}, {64, 1, 2}, {64, 1, 4}, {128, 1, 2}, {128, 1, 4}, {32, 4, 4}};

int lbm_batch_set_staging(lbm_batch* b, int enable) {
    if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
    b->stage = enable != 0;
    return batch_rebuild(b);   // the tile lists (and the captured graph) follow the choice
}

int lbm_batch_set_wait_limit(lbm_batch* b, int rounds) {
    if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
    b->spin = rounds < 0 ? STAGE_SPIN : rounds;
    b->graph_dirty = true;   // captured launches hold the old limit
    return LBM_OK;
}

int lbm_batch_wait_status(lbm_batch* b, int clear) {
    if (!b) return fail(LBM_ERR_INVALID, "batch is NULL");
    if (!b->wait_status) return LBM_OK;
    CK(cudaSetDevice(b->device));
    int v = 0;
    CK(cudaMemcpyAsync(&v, b->wait_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (clear && v) CK(cudaMemsetAsync(b->wait_status, 0, sizeof(int), b->stream));
    if (v == LBM_ERR_TIMEOUT)
        return fail(LBM_ERR_TIMEOUT, "a bounded wait of the staged batch kernel ran out (step results are invalid)");
    if (v) return fail(v, "the staged batch kernel was launched for an odd nz (step results are invalid)");
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int32_t steps, int32_t* bz_out, int32_t* rows_out, float* ms_out) {
    if (!b || steps < 1) return fail(LBM_ERR_INVALID, "bad batch or steps");
    CK(cudaSetDevice(b->device));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = INFINITY;
    int bb = b->bz, br = b->rows, bt = b->rpt;
    int rc = LBM_OK;
    for (const auto& s : kTuneShapes) {
        b->bz = s[0];
        b->rows = s[1];
        b->rpt = s[2];
        if ((rc = batch_rebuild(b))) break;
        if ((rc = lbm_batch_step(b, 2))) break;   // warm-up
        cudaEventRecord(e0, b->stream);
        if ((rc = lbm_batch_step(b, steps))) break;
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bb = s[0]; br = s[1]; bt = s[2]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->bz = bb;
    b->rows = br;
    b->rpt = bt;
    if ((rc = batch_rebuild(b))) return rc;
    if (bz_out) *bz_out = bb;
    if (rows_out) *rows_out = br * bt;
    if (ms_out) *ms_out = best / (float)steps;
    return LBM_OK;
}

int lbm_batch_get_info(lbm_batch* b, int32_t i, lbm_info* out) {
    if (!b || !out || i < 0 || i >= b->n) return fail(LBM_ERR_INVALID, "bad batch, instance or pointer");
    *out = b->info[i];
    out->steps = b->steps;
    return LBM_OK;
}

}  // extern "C"
