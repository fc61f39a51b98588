// fno_net.cu -- fused tensor-core kernels of the warm-start network (include/fno_net.h).
//
// The network's contractions all run on tcgen05.mma with BF16 operands in shared memory
// and FP32 accumulators in tensor memory; activations live in device memory as BF16.
// Every contraction over channels and every contraction over z of a channels-last tile
// reads the same shared-memory image (tc.cuh: K-major for the one, MN-major for the
// other), so nothing is transposed in software.  Kernels:
//   k_fwd   a group of 128 / C rows (all of z): pointwise mix + bias + inverse z
//           transform (one accumulator, 128 z x (rows, C)), GELU, the next layer's
//           forward z transform accumulated over the z tiles ((rows, C) x 2M);
//   k_proj  tiles of 128 pixels: projection forward, loss, projection backward with the
//           weight gradients accumulated in tensor memory over the CTA's tiles;
//   k_bwd   a group of rows: the layer's input gradient (dpre W^T + zDFT^T(dZ)), GELU',
//           the gradient's inverse-z-transform adjoint and the weight gradient of the
//           layer below (h^T dpre accumulated over all of the CTA's tiles);
//   k_r2k / k_k2r  the r transforms of one (batch, kz) spectrum;
//   k_mixf / k_mixb  per-mode complex channel mixing (CUDA cores: 8 x C x C per mode).
// The paper has no counterpart: the network only proposes an initial field; the lattice
// Boltzmann iteration always runs to convergence from it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/fno_net.h"
#include "tc.cuh"

using bf16 = __nv_bfloat16;

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

#define NCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            (void)cudaGetLastError();                                                              \
            return fail(FNO_NET_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                \
        }                                                                                          \
    } while (0)

constexpr int SPIN = 1 << 22;   // try_wait rounds of one bounded wait
__device__ int g_net_error;

// ------------------------------------------------------------------ helpers --
// Programmatic dependent launch: every kernel here is launched with the attribute that
// lets it start while the kernel before it in the stream finishes (launch_pdl); each one
// first lets its own successor be scheduled and then waits until its predecessor has
// completed and its writes are visible, before touching global or tensor memory.  The
// successor is scheduled only once every CTA of this grid has started, so a kernel of
// several waves is never short of SMs for its own CTAs.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ uint4 pack8(const float* v) {
    uint4 u;
    __nv_bfloat162 t;
    t = __floats2bfloat162_rn(v[0], v[1]);
    u.x = *reinterpret_cast<uint32_t*>(&t);
    t = __floats2bfloat162_rn(v[2], v[3]);
    u.y = *reinterpret_cast<uint32_t*>(&t);
    t = __floats2bfloat162_rn(v[4], v[5]);
    u.z = *reinterpret_cast<uint32_t*>(&t);
    t = __floats2bfloat162_rn(v[6], v[7]);
    u.w = *reinterpret_cast<uint32_t*>(&t);
    return u;
}

__device__ __forceinline__ void unpack8(uint4 u, float* v) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
        const float2 f = __bfloat1622float2(t);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

__device__ __forceinline__ void st16(uint8_t* p, uint4 u) { *reinterpret_cast<uint4*>(p) = u; }

// The standard normal's distribution function Phi(x) and density phi(x) from one
// exponential: erf(z) for z = |x| / sqrt 2 by Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (|error| <= 1.5e-7):
//     erf(z) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-z^2),  t = 1 / (1 + p z),
// whose exp(-z^2) = exp(-x^2 / 2) is also phi's.  The error is far below the BF16 rounding
// every activation of the network carries.
__device__ __forceinline__ void normal_cdf_pdf(float x, float& cdf, float& pdf) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float e = __expf(-z * z);
    const float t = __fdividef(1.f, fmaf(0.3275911f, z, 1.f));
    const float poly =
        t * (0.254829592f + t * (-0.284496736f + t * (1.421413741f + t * (-1.453152027f + t * 1.061405429f))));
    const float erfz = 1.f - poly * e;
    cdf = 0.5f + 0.5f * copysignf(erfz, x);
    pdf = 0.39894228040143268f * e;
}

// GELU in its exact form x Phi(x) and its derivative Phi(x) + x phi(x)
__device__ __forceinline__ float gelu(float x) {
    float c, d;
    normal_cdf_pdf(x, c, d);
    return x * c;
}
__device__ __forceinline__ float gelu_d(float x) {
    float c, d;
    normal_cdf_pdf(x, c, d);
    return fmaf(x, d, c);
}

// A bounded wait that the whole block agrees on (every thread calls it).
__device__ __forceinline__ bool block_wait(uint32_t mbar, uint32_t phase) {
    return __syncthreads_and(tc::wait(mbar, phase, SPIN) ? 1 : 0) != 0;
}

__device__ __forceinline__ tc::Opnd opnd(const void* base, int inner, int m0, int k0, bool mn) {
    return tc::Opnd{tc::smem_u32(base), inner, m0, k0, mn};
}

// flat 16-byte copy of `bytes` (a multiple of 16) into shared memory
__device__ __forceinline__ void cp_flat(uint8_t* dst, const void* src, int bytes, int tid, int nthr) {
    const uint8_t* s = reinterpret_cast<const uint8_t*>(src);
    for (int i = tid; i < bytes / 16; i += nthr) tc::cp16(tc::smem_u32(dst + 16 * i), s + 16 * i);
}

// Recovery after a wait ran out: one more bounded wait on each barrier whose commit is
// outstanding (so that no MMA still runs when the tensor memory is freed), then the
// error flag (1: those waits completed, 2: one of them ran out too).
__device__ __forceinline__ void recover(const uint64_t* mbar, const uint32_t* phase, const bool* pend, int n) {
    bool clean = true;
    for (int i = 0; i < n; ++i)
        if (pend[i]) clean = tc::wait(tc::smem_u32(&mbar[i]), phase[i], SPIN) && clean;
    clean = __syncthreads_and(clean ? 1 : 0) != 0;
    if (threadIdx.x == 0) atomicMax(&g_net_error, clean ? 1 : 2);
}

// ------------------------------------------------------------------- pack --
__global__ void k_pack(const float* __restrict__ src, int64_t so, int64_t si, int O, int I, bf16* __restrict__ dst,
                       int Opad, int Ipad) {
    pdl_enter();
    const int64_t n = (int64_t)Opad * Ipad;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(idx / Ipad), i = (int)(idx % Ipad);
        const float v = (o < O && i < I) ? src[o * so + i * si] : 0.f;
        dst[tc::img_off(i, o, Ipad) >> 1] = __float2bfloat16_rn(v);
    }
}

// Up to FNO_NET_PACK_MAX images in one launch (blockIdx.y = the job), jobs passed by value.
struct PackJobs {
    fno_net_pack_job j[FNO_NET_PACK_MAX];
};

__global__ void k_pack_many(const PackJobs jobs) {
    pdl_enter();
    const fno_net_pack_job& jb = jobs.j[blockIdx.y];
    const int64_t n = (int64_t)jb.Opad * jb.Ipad;
    const float* src = jb.src;
    bf16* dst = (bf16*)jb.dst;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(idx / jb.Ipad), i = (int)(idx % jb.Ipad);
        const float v = (o < jb.O && i < jb.I) ? src[o * jb.so + i * jb.si] : 0.f;
        dst[tc::img_off(i, o, jb.Ipad) >> 1] = __float2bfloat16_rn(v);
    }
}

// --------------------------------------------------------------- forward --
struct FwdP {
    int nrows, nr, nz, ci;
    const float* x;
    const bf16* h;
    const bf16* w;
    const float* bias;
    const bf16* gzt;
    const bf16* fz;
    const bf16* V;
    bf16* out;
    bf16* hout;
    bf16* Z;
};

template <int C, int KZ2, int MODE>
struct FwdSmem {
    static constexpr int G = 128 / C;
    static constexpr int KIN = MODE == 0 ? 16 : C;
    static constexpr int HIN = G * KIN;
    static constexpr bool IZ = MODE != 0, ZF = MODE != 2;
    static size_t bytes(int nz) {
        return (size_t)C * KIN * 2 + (IZ ? (size_t)nz * KZ2 * 2 : 0) + (ZF ? (size_t)nz * KZ2 * 2 : 0) +
               (size_t)128 * HIN * 2 + (IZ ? (size_t)G * KZ2 * C * 2 : 0) + (ZF ? (size_t)128 * 128 * 2 : 0) +
               (size_t)C * 4 + 1024;
    }
};

template <int C, int KZ2, int MODE>
__global__ void __launch_bounds__(256) k_fwd(const FwdP a) {
    pdl_enter();
    using S = FwdSmem<C, KZ2, MODE>;
    constexpr int G = S::G, KIN = S::KIN, HIN = S::HIN;
    constexpr bool IZ = S::IZ, ZF = S::ZF;
    constexpr int M = KZ2 / 2;
    extern __shared__ uint8_t dsm[];
    uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    uint8_t* sW = sm;
    uint8_t* sG = sW + C * KIN * 2;
    uint8_t* sF = sG + (IZ ? a.nz * KZ2 * 2 : 0);
    uint8_t* sH = sF + (ZF ? a.nz * KZ2 * 2 : 0);
    uint8_t* sV = sH + 128 * HIN * 2;
    uint8_t* sZ = sV + (IZ ? G * KZ2 * C * 2 : 0);
    float* sb = reinterpret_cast<float*>(sZ + (ZF ? 128 * 128 * 2 : 0));
    __shared__ __align__(8) uint64_t mbar[2];   // [0] main accumulator, [1] z transform
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;

    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cp_flat(sW, a.w, C * KIN * 2, tid, 256);
    if (IZ) cp_flat(sG, a.gzt, a.nz * KZ2 * 2, tid, 256);
    if (ZF) cp_flat(sF, a.fz, a.nz * KZ2 * 2, tid, 256);
    for (int i = tid; i < C; i += 256) sb[i] = a.bias[i];
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    const uint32_t mb0 = tc::smem_u32(&mbar[0]), mb1 = tc::smem_u32(&mbar[1]);
    uint32_t phase[2] = {0, 0};
    bool pend[2] = {false, false};
    bool ok = true;
    const int ngroups = a.nrows / G, ntz = a.nz / 128;

    for (int g = blockIdx.x; g < ngroups && ok; g += gridDim.x) {
        const int R0 = g * G, b = R0 / a.nr, r0 = R0 % a.nr;
        if (IZ) {   // V rows of the group: (n = c inner, k = kz2 outer) per row
            for (int i = tid; i < G * KZ2 * (C / 8); i += 256) {
                const int c8 = i % (C / 8), t2 = i / (C / 8), kz2 = t2 % KZ2, rl = t2 / KZ2;
                const int part = kz2 / M, kz = kz2 % M;
                const bf16* src = a.V + ((((int64_t)b * M + kz) * 2 + part) * a.nr + r0 + rl) * C + c8 * 8;
                tc::cp16(tc::smem_u32(sV + rl * (KZ2 * C * 2) + tc::img_off(c8 * 8, kz2, C)), src);
            }
        }
        for (int t = 0; t < ntz && ok; ++t) {
            const int z0 = t * 128;
            if (MODE == 0) {   // x (FP32, ci <= 16 channels) rounded into the image
                for (int i = tid; i < 128 * G; i += 256) {
                    const int z = i % 128, rl = i / 128;
                    const float* src = a.x + ((int64_t)(R0 + rl) * a.nz + z0 + z) * a.ci;
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = j < a.ci ? src[j] : 0.f;
                    st16(sH + tc::img_off(rl * 16, z, HIN), pack8(v));
                    st16(sH + tc::img_off(rl * 16 + 8, z, HIN), pack8(v + 8));
                }
            } else {
                for (int i = tid; i < 128 * G * (C / 8); i += 256) {
                    const int c8 = i % (C / 8), t2 = i / (C / 8), z = t2 % 128, rl = t2 / 128;
                    const bf16* src = a.h + ((int64_t)(R0 + rl) * a.nz + z0 + z) * C + c8 * 8;
                    tc::cp16(tc::smem_u32(sH + tc::img_off(rl * C + c8 * 8, z, HIN)), src);
                }
            }
            tc::cp_wait_all();
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
                for (int rl = 0; rl < G; ++rl) {
                    const uint32_t d = tmem + rl * C;
                    tc::mma(d, opnd(sH, HIN, 0, rl * KIN, false), opnd(sW, KIN, 0, 0, false), C, KIN, false);
                    if (IZ)
                        tc::mma(d, opnd(sG, KZ2, z0, 0, false), opnd(sV + rl * (KZ2 * C * 2), C, 0, 0, true), C, KZ2,
                                true);
                }
                tc::commit(mb0);
            }
            pend[0] = true;
            if (!(ok = block_wait(mb0, phase[0]))) break;
            phase[0] ^= 1;
            pend[0] = false;
            if (ZF && pend[1]) {   // the previous tile's z transform has read sZ
                if (!(ok = block_wait(mb1, phase[1]))) break;
                phase[1] ^= 1;
                pend[1] = false;
            }
            tc::fence_after();
            // epilogue: thread = z (lane quadrant q), columns 64 hh .. 64 hh + 63 = (row, c)
#pragma unroll 1
            for (int jc = 0; jc < 2; ++jc) {
                const int col0 = 64 * hh + 32 * jc, rl = col0 / C, c0 = col0 % C;
                const int z = 32 * q + lane;
                float v[32];
                tc::ld32(tc::taddr(tmem, q, col0), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] += sb[c0 + i];
                const int64_t pix = (int64_t)(R0 + rl) * a.nz + z0 + z;
                uint4* o = reinterpret_cast<uint4*>(a.out + pix * C + c0);
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] = pack8(v + 8 * k);
                if (MODE == 1) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = gelu(v[i]);
                    uint4* ho = reinterpret_cast<uint4*>(a.hout + pix * C + c0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) ho[k] = pack8(v + 8 * k);
                }
                if (ZF) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) st16(sZ + tc::img_off(rl * C + c0 + 8 * k, z, 128), pack8(v + 8 * k));
                }
            }
            tc::fence_async_smem();
            tc::fence_before();
            __syncthreads();
            if (ZF) {
                if (tid == 0) {
                    tc::fence_after();
                    tc::mma(tmem + 128, opnd(sZ, 128, 0, 0, true), opnd(sF, KZ2, 0, z0, true), KZ2, 128, t > 0);
                    tc::commit(mb1);
                }
                pend[1] = true;
            }
        }
        if (!ok) break;
        if (ZF) {   // Z of the group: thread = (row, c), kz2 columns split over the warp pair
            if (!(ok = block_wait(mb1, phase[1]))) break;
            phase[1] ^= 1;
            pend[1] = false;
            tc::fence_after();
            const int m = 32 * q + lane, rl = m / C, c = m % C;
            if (hh * 16 < KZ2) {
                float v[16];
                tc::ld16(tc::taddr(tmem, q, 128 + 16 * hh), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int kz2 = 16 * hh + i, part = kz2 / M, kz = kz2 % M;
                    a.Z[((((int64_t)b * M + kz) * 2 + part) * a.nr + r0 + rl) * C + c] = __float2bfloat16_rn(v[i]);
                }
            }
        }
        tc::fence_before();
        __syncthreads();
    }
    if (!ok) recover(mbar, phase, pend, 2);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 256);
}

// ------------------------------------------------------------ projection --
struct ProjP {
    int P, CO;
    float inv_n2;   // 2 / (P CO)
    const bf16* hL;
    const bf16* q1w;
    const bf16* q1n;
    const float* q1;
    const bf16* q2w;
    const bf16* q2n;
    const float* q2;
    const float* t;
    float* y;
    bf16* dhL;
    double* loss;
    float* gQ1;   // dL/dQ1 [C][H], added to
    float* gq1;
    float* gQ2;   // dL/dQ2 [H][CO]
    float* gq2;
};

template <int C>
struct ProjSmem {
    static constexpr int H = 128, HI = C + 16;
    static constexpr size_t bytes = (size_t)H * C * 2 * 2 + 16 * H * 2 * 2 + 128 * HI * 2 + 128 * H * 2 * 2 +
                                    128 * 16 * 2 + (H + 16) * 4 + 16 * 4 + 1024;
};

// Tensor-memory columns of k_proj: q_pre, then (same columns) the raw dq; y; dQ2; dh;
// [dQ1^T | dq1].  Width 32 fits 256 columns (two CTAs per SM), width 64 takes 512.
template <int C>
struct ProjCols {
    static constexpr int TCOLS = C == 32 ? 256 : 512;
    static constexpr int D1 = 0, D3 = 0, D2 = 128, D6 = 144, D4 = 160, D5 = C == 32 ? 192 : 256;
};

template <int C, bool TRAIN>
__global__ void __launch_bounds__(256, C == 32 ? 2 : 1) k_proj(const ProjP a) {
    pdl_enter();
    constexpr int H = 128, HI = ProjSmem<C>::HI;
    extern __shared__ uint8_t dsm[];
    uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    uint8_t* sQ1W = sm;                 // outer j (H), inner c
    uint8_t* sQ1N = sQ1W + H * C * 2;   // outer c, inner j
    uint8_t* sQ2W = sQ1N + H * C * 2;   // outer o (16), inner j
    uint8_t* sQ2N = sQ2W + 16 * H * 2;  // outer j, inner o (16)
    uint8_t* sHH = sQ2N + 16 * H * 2;   // outer p, inner c (+ ones, zeros)
    uint8_t* sQI = sHH + 128 * HI * 2;  // outer p, inner j: q
    uint8_t* sDQ = sQI + 128 * H * 2;   // outer p, inner j: dq
    uint8_t* sDY = sDQ + 128 * H * 2;   // outer p, inner o (16): dy
    float* sq1 = reinterpret_cast<float*>(sDY + 128 * 16 * 2);
    float* sq2 = sq1 + H;
    float* sdq2 = sq2 + 16;
    __shared__ __align__(8) uint64_t mbar[1];
    __shared__ uint32_t tslot;
    __shared__ double sloss;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;
    using TC = ProjCols<C>;
    constexpr int D1 = TC::D1, D2 = TC::D2, D3 = TC::D3, D4 = TC::D4, D5 = TC::D5, D6 = TC::D6;

    if (warp == 0) tc::tmem_alloc(&tslot, TC::TCOLS);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sloss = 0.0;
    }
    cp_flat(sQ1W, a.q1w, H * C * 2, tid, 256);
    cp_flat(sQ2W, a.q2w, 16 * H * 2, tid, 256);
    if (TRAIN) {   // the backward's images (NULL without targets)
        cp_flat(sQ1N, a.q1n, H * C * 2, tid, 256);
        cp_flat(sQ2N, a.q2n, 16 * H * 2, tid, 256);
    }
    for (int i = tid; i < H; i += 256) sq1[i] = a.q1[i];
    for (int i = tid; i < 16; i += 256) {
        sq2[i] = i < a.CO ? a.q2[i] : 0.f;
        sdq2[i] = 0.f;
    }
    for (int p = tid; p < 128; p += 256) {   // the ones column (index C) and its zero neighbours
        float one[8], zero[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            one[i] = 1.f;
            zero[i] = 0.f;
        }
        st16(sHH + tc::img_off(C, p, HI), pack8(one));
        st16(sHH + tc::img_off(C + 8, p, HI), pack8(zero));
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot, mb = tc::smem_u32(&mbar[0]);
    uint32_t phase[1] = {0};
    bool pend[1] = {false};
    bool ok = true, first = true;
    float lacc = 0.f, dq2acc[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) dq2acc[o] = 0.f;
    const int ntiles = a.P / 128;

    auto issue_wait = [&](auto&& body) -> bool {
        if (tid == 0) {
            tc::fence_after();
            body();
            tc::commit(mb);
        }
        pend[0] = true;
        if (!block_wait(mb, phase[0])) return false;
        phase[0] ^= 1;
        pend[0] = false;
        tc::fence_after();
        return true;
    };

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t p0 = (int64_t)tile * 128;
        for (int i = tid; i < 128 * (C / 8); i += 256) {
            const int c8 = i % (C / 8), p = i / (C / 8);
            tc::cp16(tc::smem_u32(sHH + tc::img_off(c8 * 8, p, HI)), a.hL + (p0 + p) * C + c8 * 8);
        }
        tc::cp_wait_all();
        tc::fence_async_smem();
        __syncthreads();
        if (!(ok = issue_wait([&] { tc::mma(tmem + D1, opnd(sHH, HI, 0, 0, false), opnd(sQ1W, C, 0, 0, false), H, C, false); })))
            break;
        const int p = 32 * q + lane;
#pragma unroll 1
        for (int jc = 0; jc < 2; ++jc) {   // q = GELU(q_pre) into sQI; GELU'(q_pre) into sDQ
            const int col0 = 64 * hh + 32 * jc;
            float v[32];
            tc::ld32(tc::taddr(tmem, q, D1 + col0), v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float gq[8], gd[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float x = v[8 * k + i] + sq1[col0 + 8 * k + i];
                    float c, d;
                    normal_cdf_pdf(x, c, d);
                    gq[i] = x * c;
                    gd[i] = fmaf(x, d, c);
                }
                st16(sQI + tc::img_off(col0 + 8 * k, p, H), pack8(gq));
                if (TRAIN) st16(sDQ + tc::img_off(col0 + 8 * k, p, H), pack8(gd));
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (!(ok = issue_wait([&] { tc::mma(tmem + D2, opnd(sQI, H, 0, 0, false), opnd(sQ2W, H, 0, 0, false), 16, H, false); })))
            break;
        if (hh == 0) {   // y, loss, dy
            float v[16];
            tc::ld16(tc::taddr(tmem, q, D2), v);
            float dy[16];
#pragma unroll
            for (int o = 0; o < 16; ++o) {
                dy[o] = 0.f;
                if (o < a.CO) {
                    const float yv = v[o] + sq2[o];
                    a.y[(p0 + p) * a.CO + o] = yv;
                    if (TRAIN) {
                        const float d = yv - a.t[(p0 + p) * a.CO + o];
                        lacc += d * d;
                        dy[o] = d * a.inv_n2;
                        dq2acc[o] += dy[o];
                    }
                }
            }
            if (TRAIN) {
                st16(sDY + tc::img_off(0, p, 16), pack8(dy));
                st16(sDY + tc::img_off(8, p, 16), pack8(dy + 8));
            }
        }
        if (!TRAIN) {
            tc::fence_before();
            __syncthreads();
            continue;
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        const bool acc_w = !first;
        if (!(ok = issue_wait([&] {
                  tc::mma(tmem + D3, opnd(sDY, 16, 0, 0, false), opnd(sQ2N, 16, 0, 0, false), H, 16, false);
                  tc::mma(tmem + D6, opnd(sQI, H, 0, 0, true), opnd(sDY, 16, 0, 0, true), 16, 128, acc_w);
              })))
            break;
#pragma unroll 1
        for (int jc = 0; jc < 2; ++jc) {   // dq = (dy Q2^T) GELU'(q_pre), in place of GELU'
            const int col0 = 64 * hh + 32 * jc;
            float g[32];
            tc::ld32(tc::taddr(tmem, q, D3 + col0), g);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint8_t* at = sDQ + tc::img_off(col0 + 8 * k, p, H);
                float gd[8];
                unpack8(*reinterpret_cast<const uint4*>(at), gd);
#pragma unroll
                for (int i = 0; i < 8; ++i) gd[i] *= g[8 * k + i];
                st16(at, pack8(gd));
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (!(ok = issue_wait([&] {
                  tc::mma(tmem + D4, opnd(sDQ, H, 0, 0, false), opnd(sQ1N, H, 0, 0, false), C, H, false);
                  tc::mma(tmem + D5, opnd(sDQ, H, 0, 0, true), opnd(sHH, HI, 0, 0, true), HI, 128, acc_w);
              })))
            break;
        first = false;
        if (hh * 32 < C) {   // dh = dq Q1^T
            float v[32];
            tc::ld32(tc::taddr(tmem, q, D4 + 32 * hh), v);
            uint4* o = reinterpret_cast<uint4*>(a.dhL + (p0 + p) * C + 32 * hh);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = pack8(v + 8 * k);
        }
        tc::fence_before();
        __syncthreads();
    }
    if (!ok) {
        recover(mbar, phase, pend, 1);
    } else if (TRAIN && !first) {
        // this CTA's sums over its tiles, added to the gradients (FP32 atomics)
        const int j = 32 * q + lane;
        for (int c0 = 32 * hh; c0 < HI; c0 += 64) {
            float v[32];
            tc::ld32(tc::taddr(tmem, q, D5 + c0), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int c = c0 + i;
                if (c < C) atomicAdd(&a.gQ1[(int64_t)c * H + j], v[i]);   // D5 holds dQ1^T
                else if (c == C) atomicAdd(&a.gq1[j], v[i]);
            }
        }
        if (hh == 0) {
            float v[16];
            tc::ld16(tc::taddr(tmem, q, D6), v);
#pragma unroll
            for (int o = 0; o < 16; ++o)
                if (o < a.CO) atomicAdd(&a.gQ2[(int64_t)j * a.CO + o], v[o]);
        }
#pragma unroll
        for (int o = 0; o < 16; ++o) {
            float s = dq2acc[o];
            for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
            if (lane == 0 && hh == 0) atomicAdd(&sdq2[o], s);
        }
        float l = lacc;
        for (int w = 16; w > 0; w >>= 1) l += __shfl_xor_sync(0xffffffffu, l, w);
        if (lane == 0) atomicAdd(&sloss, (double)l);
        __syncthreads();
        if (tid < a.CO) atomicAdd(&a.gq2[tid], sdq2[tid]);
        if (tid == 0) atomicAdd(a.loss, sloss / ((double)a.P * a.CO));
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, TC::TCOLS);
}

// -------------------------------------------------------------- backward --
struct BwdP {
    int nrows, nr, nz, ci;
    float db_scale;   // nr nz: the kz = 0 coefficient of Gz is 1 / (nr nz)
    const bf16* dpre_in;
    const bf16* dZ;
    const bf16* wn;
    const bf16* fz;
    const bf16* pre;
    const bf16* h;
    const float* x;
    const bf16* gzt;
    bf16* dpre_out;
    bf16* dV;
    float* gW;   // dL/dW [C][C] (dL/dP [ci][C] for the lift), added to
    float* gb;
};

template <int C, int KZ2, int MODE>
struct BwdSmem {
    static constexpr int G = 128 / C;
    static constexpr bool HB = MODE != 0, HA = MODE != 2;
    static constexpr size_t TILE = 128 * 128 * 2;
    // the gradient tile (dpre_in, overwritten by the next dpre), W, Fz, dZ rows, the h (x)
    // tile, Gz^T, the CTA's sums
    static size_t bytes(int nz) {
        return TILE + (HB ? C * C * 2 + (size_t)nz * KZ2 * 2 + (size_t)G * KZ2 * C * 2 : 0) + TILE +
               (HA ? (size_t)nz * KZ2 * 2 : 0) + (size_t)C * C * 4 + C * 4 + 1024;
    }
};

// Two CTAs per SM (256 tensor-memory columns each): columns 0..127 hold the layer's input
// gradient dh (B part) and then, per tile, the weight-gradient product whose diagonal
// blocks each thread adds to 32 registers; columns 128.. the dV accumulator of the group.
template <int C, int KZ2, int MODE>
__global__ void __launch_bounds__(256, 2) k_bwd(const BwdP a) {
    pdl_enter();
    using S = BwdSmem<C, KZ2, MODE>;
    constexpr int G = S::G;
    constexpr bool HB = S::HB, HA = S::HA;
    constexpr int M = KZ2 / 2;
    constexpr int TILE = (int)S::TILE;
    extern __shared__ uint8_t dsm[];
    uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    uint8_t* sD2 = sm;                                        // dpre_l (B part), then the gradient the A part uses
    uint8_t* sWN = sD2 + TILE;
    uint8_t* sF = sWN + (HB ? C * C * 2 : 0);
    uint8_t* sdZ = sF + (HB ? a.nz * KZ2 * 2 : 0);
    uint8_t* sH = sdZ + (HB ? G * KZ2 * C * 2 : 0);           // h_{l-1} tile, or x with ones
    uint8_t* sG = sH + TILE;
    float* sacc = reinterpret_cast<float*>(sG + (HA ? a.nz * KZ2 * 2 : 0));   // C x C
    float* sdb = sacc + C * C;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2;
    constexpr int DB = 0, DW = 0, DV = 128;

    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (HB) {
        cp_flat(sWN, a.wn, C * C * 2, tid, 256);
        cp_flat(sF, a.fz, a.nz * KZ2 * 2, tid, 256);
    }
    if (HA) cp_flat(sG, a.gzt, a.nz * KZ2 * 2, tid, 256);
    for (int i = tid; i < C * C; i += 256) sacc[i] = 0.f;
    for (int i = tid; i < C; i += 256) sdb[i] = 0.f;
    if (MODE == 2) {   // per row block of the x image: x (16) | ones (8) | zeros
        for (int i = tid; i < 128 * G; i += 256) {
            const int z = i % 128, rl = i / 128;
            float one[8], zero[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                one[k] = 1.f;
                zero[k] = 0.f;
            }
            st16(sH + tc::img_off(rl * C + 16, z, 128), pack8(one));
            for (int c = 24; c < C; c += 8) st16(sH + tc::img_off(rl * C + c, z, 128), pack8(zero));
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot;
    const uint32_t mb0 = tc::smem_u32(&mbar[0]), mb1 = tc::smem_u32(&mbar[1]);
    uint32_t phase[2] = {0, 0};
    bool pend[2] = {false, false};
    bool ok = true, any = false;
    float dbacc = 0.f, wacc[32];   // this thread's diagonal row: (rl, c_in) x 32 columns c
#pragma unroll
    for (int i = 0; i < 32; ++i) wacc[i] = 0.f;
    const int ngroups = a.nrows / G, ntz = a.nz / 128;
    const int m = 32 * q + lane, mrl = m / C, mci = m % C;
    const int wc0 = 32 * hh;                // this warp's 32 diagonal columns (C = 32: warps 0..3 only)
    const bool wdiag = wc0 < C;

    for (int g = blockIdx.x; g < ngroups && ok; g += gridDim.x) {
        const int R0 = g * G, b = R0 / a.nr, r0 = R0 % a.nr;
        if (HB) {
            for (int i = tid; i < G * KZ2 * (C / 8); i += 256) {
                const int c8 = i % (C / 8), t2 = i / (C / 8), kz2 = t2 % KZ2, rl = t2 / KZ2;
                const int part = kz2 / M, kz = kz2 % M;
                const bf16* src = a.dZ + ((((int64_t)b * M + kz) * 2 + part) * a.nr + r0 + rl) * C + c8 * 8;
                tc::cp16(tc::smem_u32(sdZ + rl * (KZ2 * C * 2) + tc::img_off(c8 * 8, kz2, C)), src);
            }
        }
        for (int t = 0; t < ntz && ok; ++t) {
            const int z0 = t * 128;
            for (int i = tid; i < 128 * G * (C / 8); i += 256) {
                const int c8 = i % (C / 8), t2 = i / (C / 8), z = t2 % 128, rl = t2 / 128;
                const int64_t off = ((int64_t)(R0 + rl) * a.nz + z0 + z) * C + c8 * 8;
                const uint32_t so = tc::img_off(rl * C + c8 * 8, z, 128);
                tc::cp16(tc::smem_u32(sD2 + so), a.dpre_in + off);
                if (HA) tc::cp16(tc::smem_u32(sH + so), a.h + off);
            }
            if (MODE == 2) {
                for (int i = tid; i < 128 * G; i += 256) {
                    const int z = i % 128, rl = i / 128;
                    const float* src = a.x + ((int64_t)(R0 + rl) * a.nz + z0 + z) * a.ci;
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = j < a.ci ? src[j] : 0.f;
                    st16(sH + tc::img_off(rl * C, z, 128), pack8(v));
                    st16(sH + tc::img_off(rl * C + 8, z, 128), pack8(v + 8));
                }
            }
            tc::cp_wait_all();
            tc::fence_async_smem();
            __syncthreads();
            if (HB) {
                if (tid == 0) {
                    tc::fence_after();
                    for (int rl = 0; rl < G; ++rl) {
                        const uint32_t d = tmem + DB + rl * C;
                        tc::mma(d, opnd(sD2, 128, 0, rl * C, false), opnd(sWN, C, 0, 0, false), C, C, false);
                        tc::mma(d, opnd(sF, KZ2, z0, 0, false), opnd(sdZ + rl * (KZ2 * C * 2), C, 0, 0, true), C,
                                KZ2, true);
                    }
                    tc::commit(mb0);
                }
                pend[0] = true;
                if (!(ok = block_wait(mb0, phase[0]))) break;
                phase[0] ^= 1;
                pend[0] = false;
                tc::fence_after();
                // dh -> (MODE 1) dpre_{l-1} = dh GELU'(pre_{l-1}); written over dpre_l in sD2,
                // which the MMAs above have finished reading
                const int z = 32 * q + lane;
#pragma unroll 1
                for (int jc = 0; jc < 4; ++jc) {   // 16 columns at a time (the 32 wacc registers stay live)
                    const int col0 = 64 * hh + 16 * jc, rl = col0 / C, c0 = col0 % C;
                    const int64_t pix = (int64_t)(R0 + rl) * a.nz + z0 + z;
                    uint4 pr[2];
                    if (MODE == 1) {
                        const uint4* pp = reinterpret_cast<const uint4*>(a.pre + pix * C + c0);
                        pr[0] = pp[0];
                        pr[1] = pp[1];
                    }
                    float v[16];
                    tc::ld16(tc::taddr(tmem, q, DB + col0), v);
                    if (MODE == 1) {
                        uint4* po = reinterpret_cast<uint4*>(a.dpre_out + pix * C + c0);
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            float pv[8];
                            unpack8(pr[k], pv);
#pragma unroll
                            for (int i = 0; i < 8; ++i) v[8 * k + i] *= gelu_d(pv[i]);
                            po[k] = pack8(v + 8 * k);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) st16(sD2 + tc::img_off(rl * C + c0 + 8 * k, z, 128), pack8(v + 8 * k));
                }
                tc::fence_async_smem();
                tc::fence_before();
                __syncthreads();
            }
            if (tid == 0) {
                tc::fence_after();
                if (HA) tc::mma(tmem + DV, opnd(sD2, 128, 0, 0, true), opnd(sG, KZ2, 0, z0, true), KZ2, 128, t > 0);
                tc::mma(tmem + DW, opnd(sH, 128, 0, 0, true), opnd(sD2, 128, 0, 0, true), 128, 128, false);
                tc::commit(mb1);
            }
            pend[1] = true;
            if (!(ok = block_wait(mb1, phase[1]))) break;
            phase[1] ^= 1;
            pend[1] = false;
            tc::fence_after();
            if (wdiag) {   // the diagonal block of this tile's (rows, c_in) x (rows, c) product
                float v[32];
                tc::ld32(tc::taddr(tmem, q, DW + mrl * C + wc0), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) wacc[i] += v[i];
            }
            any = true;
            if (HA && t == ntz - 1) {   // dV of the group; db from its kz = 0 cosine coefficient
                const int rl = mrl, c = mci;
                if (hh * 16 < KZ2) {
                    float v[16];
                    tc::ld16(tc::taddr(tmem, q, DV + 16 * hh), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int kz2 = 16 * hh + i, part = kz2 / M, kz = kz2 % M;
                        a.dV[((((int64_t)b * M + kz) * 2 + part) * a.nr + r0 + rl) * C + c] =
                            __float2bfloat16_rn(v[i]);
                    }
                    if (hh == 0) dbacc += v[0];
                }
            }
            tc::fence_before();
            __syncthreads();   // tensor memory read before the next tile's MMAs overwrite it
        }
    }
    if (!ok) {
        recover(mbar, phase, pend, 2);
    } else if (any) {
        // this CTA's sums, added to the gradients (FP32 atomics): dL/dW[c_in][c] from every
        // diagonal row, or for the lift dL/dP[ci][c] (rows ci < in_ch of each x block) and
        // dL/dp (its first ones row)
        if (wdiag) {
            if (MODE == 2 && mci == 16) {
#pragma unroll
                for (int i = 0; i < 32; ++i) atomicAdd(&sdb[wc0 + i], wacc[i]);
            } else if (MODE != 2 || mci < a.ci) {
#pragma unroll
                for (int i = 0; i < 32; ++i) atomicAdd(&sacc[mci * C + wc0 + i], wacc[i]);
            }
        }
        if (HA && hh == 0) atomicAdd(&sdb[mci], dbacc * a.db_scale);
        __syncthreads();
        const int rows = MODE == 2 ? a.ci : C;
        for (int i = tid; i < rows * C; i += 256) atomicAdd(&a.gW[i], sacc[i]);
        for (int i = tid; i < C; i += 256) atomicAdd(&a.gb[i], sdb[i]);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 256);
}

// ------------------------------------------------------- r transforms --
// k_r2k: CTA (b, kz): out[kz][kr][part][b][:] = F2 [Z_re; Z_im], F2 (4M x 2 nr) padded to
// 128 rows.  k_k2r: CTA (b, kz, row tile): out[b][kz][part][r][:] = F2i [Y_re; Y_im].
template <int C>
__global__ void __launch_bounds__(128) k_r2k(const bf16* __restrict__ in, const bf16* __restrict__ f2,
                                             float* __restrict__ out, int B, int nr, int M) {
    pdl_enter();
    const int K = 2 * nr, kz = blockIdx.x % M, b = blockIdx.x / M;
    extern __shared__ uint8_t dsm[];
    uint8_t* sA = reinterpret_cast<uint8_t*>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = sA + 128 * K * 2;
    __shared__ __align__(8) uint64_t mbar[1];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tslot, C);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cp_flat(sA, f2, 128 * K * 2, tid, 128);
    const bf16* src = in + (int64_t)(b * M + kz) * K * C;
    for (int i = tid; i < K * (C / 8); i += 128) {
        const int k = i / (C / 8), c8 = i % (C / 8);
        tc::cp16(tc::smem_u32(sB + tc::img_off(c8 * 8, k, C)), src + (int64_t)k * C + c8 * 8);
    }
    tc::cp_wait_all();
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot, mb = tc::smem_u32(&mbar[0]);
    if (tid == 0) {
        tc::fence_after();
        tc::mma(tmem, opnd(sA, K, 0, 0, false), opnd(sB, C, 0, 0, true), C, K, false);
        tc::commit(mb);
    }
    uint32_t phase[1] = {0};
    bool pend[1] = {true};
    if (block_wait(mb, 0)) {
        tc::fence_after();
        const int m = 32 * warp + lane;
        if (32 * warp < 4 * M) {
            for (int c0 = 0; c0 < C; c0 += 32) {
                float v[32];
                tc::ld32(tc::taddr(tmem, warp, c0), v);
                if (m < 4 * M) {
                    const int part = m / (2 * M), kr = m % (2 * M);
                    float4* o = reinterpret_cast<float4*>(out + ((((int64_t)kz * 2 * M + kr) * 2 + part) * B + b) * C + c0);
#pragma unroll
                    for (int k = 0; k < 8; ++k) o[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                }
            }
        }
    } else {
        recover(mbar, phase, pend, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, C);
}

template <int C>
__global__ void __launch_bounds__(128) k_k2r(const float* __restrict__ in, const bf16* __restrict__ f2i,
                                             bf16* __restrict__ out, int B, int nr, int M) {
    pdl_enter();
    const int K = 4 * M, ntm = 2 * nr / 128;
    const int mt = blockIdx.x % ntm, kz = (blockIdx.x / ntm) % M, b = blockIdx.x / (ntm * M);
    extern __shared__ uint8_t dsm[];
    uint8_t* sA = reinterpret_cast<uint8_t*>(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = sA + 128 * K * 2;
    __shared__ __align__(8) uint64_t mbar[1];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tslot, C);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // rows mt*128 .. of the F2i image: 16 outer groups, contiguous
    cp_flat(sA, reinterpret_cast<const uint8_t*>(f2i) + (size_t)mt * 128 * K * 2, 128 * K * 2, tid, 128);
    for (int i = tid; i < K * (C / 8); i += 128) {   // k = (part, kr), 8 channels, FP32 -> BF16
        const int k = i / (C / 8), c8 = i % (C / 8);
        const int part = k / (2 * M), kr = k % (2 * M);
        const float4* s = reinterpret_cast<const float4*>(in + ((((int64_t)kz * 2 * M + kr) * 2 + part) * B + b) * C + c8 * 8);
        const float4 u = s[0], w = s[1];
        const float v[8] = {u.x, u.y, u.z, u.w, w.x, w.y, w.z, w.w};
        st16(sB + tc::img_off(c8 * 8, k, C), pack8(v));
    }
    tc::cp_wait_all();
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tslot, mb = tc::smem_u32(&mbar[0]);
    if (tid == 0) {
        tc::fence_after();
        tc::mma(tmem, opnd(sA, K, 0, 0, false), opnd(sB, C, 0, 0, true), C, K, false);
        tc::commit(mb);
    }
    uint32_t phase[1] = {0};
    bool pend[1] = {true};
    if (block_wait(mb, 0)) {
        tc::fence_after();
        const int row = mt * 128 + 32 * warp + lane, part = row / nr, r = row % nr;
        for (int c0 = 0; c0 < C; c0 += 32) {
            float v[32];
            tc::ld32(tc::taddr(tmem, warp, c0), v);
            uint4* o = reinterpret_cast<uint4*>(out + ((((int64_t)b * M + kz) * 2 + part) * nr + r) * C + c0);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = pack8(v + 8 * k);
        }
    } else {
        recover(mbar, phase, pend, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, C);
}

// ---------------------------------------------------------- mode mixing --
// CTA (kz, kr): the mode's weights R[kr][kz] (C x C complex) and the batch's coefficients.
__global__ void k_mixf(const float* __restrict__ W, const float* __restrict__ R, float* __restrict__ Y, int B, int C,
                       int M) {
    pdl_enter();
    extern __shared__ float s[];
    float* sR = s;                 // C x C x 2
    float* sW = sR + 2 * C * C;    // [part][b][c]
    const int kz = blockIdx.x / (2 * M), kr = blockIdx.x % (2 * M);
    const float* Rm = R + ((int64_t)kr * M + kz) * C * C * 2;
    const float* Wm = W + ((int64_t)kz * 2 * M + kr) * 2 * B * C;
    for (int i = threadIdx.x; i < 2 * C * C; i += blockDim.x) sR[i] = Rm[i];
    for (int i = threadIdx.x; i < 2 * B * C; i += blockDim.x) sW[i] = Wm[i];
    __syncthreads();
    float* Ym = Y + ((int64_t)kz * 2 * M + kr) * 2 * B * C;
    for (int i = threadIdx.x; i < B * C; i += blockDim.x) {
        const int bb = i / C, o = i % C;
        float re = 0.f, im = 0.f;
        for (int c = 0; c < C; ++c) {
            const float xr = sW[bb * C + c], xi = sW[(B + bb) * C + c];
            const float rr = sR[(c * C + o) * 2], ri = sR[(c * C + o) * 2 + 1];
            re += xr * rr - xi * ri;
            im += xr * ri + xi * rr;
        }
        Ym[bb * C + o] = re;
        Ym[(B + bb) * C + o] = im;
    }
}

__global__ void k_mixb(const float* __restrict__ W, const float* __restrict__ R, const float* __restrict__ dY,
                       float* __restrict__ dW, float* __restrict__ dR, int B, int C, int M, int accumulate) {
    pdl_enter();
    extern __shared__ float s[];
    float* sR = s;
    float* sW = sR + 2 * C * C;
    float* sY = sW + 2 * B * C;
    const int kz = blockIdx.x / (2 * M), kr = blockIdx.x % (2 * M);
    const int64_t mode = (int64_t)kr * M + kz, slab = ((int64_t)kz * 2 * M + kr) * 2 * B * C;
    // R[c][o] kept as [o][c]: the dW sums run over o with c across the threads
    for (int i = threadIdx.x; i < 2 * C * C; i += blockDim.x) {
        const int part = i & 1, co = i >> 1, c = co / C, o = co % C;
        sR[(o * C + c) * 2 + part] = R[mode * C * C * 2 + i];
    }
    for (int i = threadIdx.x; i < 2 * B * C; i += blockDim.x) {
        sW[i] = W[slab + i];
        sY[i] = dY[slab + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < B * C; i += blockDim.x) {   // dW = dY R^H
        const int bb = i / C, c = i % C;
        float gr = 0.f, gi = 0.f;
        for (int o = 0; o < C; ++o) {
            const float yr = sY[bb * C + o], yi = sY[(B + bb) * C + o];
            const float rr = sR[(o * C + c) * 2], ri = sR[(o * C + c) * 2 + 1];
            gr += yr * rr + yi * ri;
            gi += -yr * ri + yi * rr;
        }
        dW[slab + bb * C + c] = gr;
        dW[slab + (B + bb) * C + c] = gi;
    }
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) {   // dR = W^H dY
        const int c = i / C, o = i % C;
        float gr = 0.f, gi = 0.f;
        for (int bb = 0; bb < B; ++bb) {
            const float xr = sW[bb * C + c], xi = sW[(B + bb) * C + c];
            const float yr = sY[bb * C + o], yi = sY[(B + bb) * C + o];
            gr += yr * xr + yi * xi;
            gi += -yr * xi + yi * xr;
        }
        float* d = dR + (mode * C * C + i) * 2;
        d[0] = accumulate ? d[0] + gr : gr;
        d[1] = accumulate ? d[1] + gi : gi;
    }
}

// --------------------------------------------------------------- host --
static int g_sms = 0;

static int sms() {
    if (!g_sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            g_sms = 0;
    }
    return g_sms;
}

// Launch with programmatic stream serialization allowed (see pdl_enter).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

static bool dims_ok(const fno_net_dims* d, std::string* why) {
    auto no = [&](const char* m) {
        if (why) *why = m;
        return false;
    };
    if (!d) return no("dims is NULL");
    if (d->width != 32 && d->width != 64) return no("width must be 32 or 64");
    if (d->batch < 1 || d->nr < 1 || d->nz < 128 || d->nz % 128 || d->nz > 512)
        return no("nz must be a multiple of 128, at most 512");
    if (d->nr % (128 / d->width)) return no("nr must be a multiple of 128 / width");
    if (2 * d->modes != 16 && 2 * d->modes != 32) return no("2 * modes must be 16 or 32");
    if (2 * d->modes > d->nr || d->modes > d->nz / 2) return no("too many modes for the grid");
    if (2 * d->nr % 128) return no("2 * nr must be a multiple of 128 (inverse r transform tiles)");
    if (d->nr > 256) return no("nr <= 256 (r transform operand in shared memory)");
    if (d->hidden != 128) return no("hidden must be 128");
    if (d->in_ch < 1 || d->in_ch > 16 || d->out_ch < 1 || d->out_ch > 16) return no("in_ch, out_ch in [1, 16]");
    return true;
}

template <typename K>
static int set_smem(K kernel, size_t bytes) {
    NCK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return FNO_NET_OK;
}

extern "C" {

int fno_net_supported(const fno_net_dims* d) { return dims_ok(d, nullptr) ? 1 : 0; }

int fno_net_pack(const float* src, int64_t so, int64_t si, int O, int I, void* dst, int Opad, int Ipad, void* stream) {
    if (!src || !dst || O < 0 || I < 0 || O > Opad || I > Ipad || Opad % 8 || Ipad % 8)
        return fail(FNO_NET_ERR_INVALID, "fno_net_pack: bad arguments");
    const int64_t n = (int64_t)Opad * Ipad;
    if (n == 0) return FNO_NET_OK;
    NCK(launch_pdl(k_pack, dim3((unsigned)std::min<int64_t>((n + 255) / 256, 4096)), dim3(256), 0, (cudaStream_t)stream, 
        src, so, si, O, I, (bf16*)dst, Opad, Ipad));
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

// Dynamic shared memory is padded so that no more CTAs share an SM than its 512
// tensor-memory columns serve: a CTA whose allocation cannot be met would wait in
// tcgen05.alloc until another one on the SM finishes.  k_fwd: 256 columns, at most two CTAs
// per SM; k_proj: 256 columns at width 32 (two per SM), else 512 (one); k_bwd: 256
// columns, two; k_k2r: up to 64 columns, at most seven.
constexpr size_t SMEM_2_PER_SM = 80 * 1024, SMEM_1_PER_SM = 120 * 1024, SMEM_7_PER_SM = 32 * 1024;

int fno_net_pack_many(const fno_net_pack_job* jobs, int n, void* stream) {
    if (!jobs || n < 1 || n > FNO_NET_PACK_MAX) return fail(FNO_NET_ERR_INVALID, "fno_net_pack_many: 1 <= n <= %d", FNO_NET_PACK_MAX);
    PackJobs pj{};
    int64_t most = 0;
    for (int k = 0; k < n; ++k) {
        const fno_net_pack_job& j = jobs[k];
        if (!j.src || !j.dst || j.O < 0 || j.I < 0 || j.O > j.Opad || j.I > j.Ipad || j.Opad % 8 || j.Ipad % 8)
            return fail(FNO_NET_ERR_INVALID, "fno_net_pack_many: bad job %d", k);
        pj.j[k] = j;
        most = std::max(most, (int64_t)j.Opad * j.Ipad);
    }
    if (most == 0) return FNO_NET_OK;
    const dim3 grid((unsigned)std::min<int64_t>((most + 255) / 256, 256), (unsigned)n);
    NCK(launch_pdl(k_pack_many, dim3(grid), dim3(256), 0, (cudaStream_t)stream, pj));
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

#define FWD_CASE(C_, K_, MODE_)                                                                         \
    if (d->width == C_ && 2 * d->modes == K_ && mode == MODE_) {                                       \
        const size_t sb = std::max(FwdSmem<C_, K_, MODE_>::bytes(d->nz), SMEM_2_PER_SM);               \
        if (int rc = set_smem(k_fwd<C_, K_, MODE_>, sb)) return rc;                                    \
        NCK(launch_pdl(k_fwd<C_, K_, MODE_>, dim3(grid), dim3(256), sb, s, p));                                                  \
        launched = true;                                                                              \
    }

int fno_net_fwd(int mode, const fno_net_dims* d, const float* x, const void* h, const void* w_img, const float* bias,
                const void* gzt_img, const void* fz_img, const void* V, void* out, void* hout, void* Z, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_fwd: %s", why.c_str());
    if (mode < 0 || mode > 2 || !w_img || !bias || !out || (mode == 0 && !x) || (mode != 0 && (!h || !gzt_img || !V)) ||
        (mode != 2 && (!fz_img || !Z)) || (mode == 1 && !hout))
        return fail(FNO_NET_ERR_INVALID, "fno_net_fwd: missing argument for mode %d", mode);
    FwdP p{d->batch * d->nr, d->nr, d->nz, d->in_ch, x, (const bf16*)h, (const bf16*)w_img, bias,
           (const bf16*)gzt_img, (const bf16*)fz_img, (const bf16*)V, (bf16*)out, (bf16*)hout, (bf16*)Z};
    const int groups = p.nrows / (128 / d->width);
    const unsigned grid = (unsigned)std::min(groups, std::max(1, 2 * sms()));
    cudaStream_t s = (cudaStream_t)stream;
    bool launched = false;
    FWD_CASE(32, 32, 0) FWD_CASE(32, 32, 1) FWD_CASE(32, 32, 2)
    FWD_CASE(32, 16, 0) FWD_CASE(32, 16, 1) FWD_CASE(32, 16, 2)
    FWD_CASE(64, 32, 0) FWD_CASE(64, 32, 1) FWD_CASE(64, 32, 2)
    FWD_CASE(64, 16, 0) FWD_CASE(64, 16, 1) FWD_CASE(64, 16, 2)
    if (!launched) return fail(FNO_NET_ERR_INVALID, "fno_net_fwd: no kernel for these sizes");
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

int fno_net_proj(const fno_net_dims* d, const void* hL, const void* q1w, const void* q1n, const float* q1,
                 const void* q2w, const void* q2n, const float* q2, const float* t, float* y, void* dhL, double* loss,
                 float* dQ1, float* dq1, float* dQ2, float* dq2, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_proj: %s", why.c_str());
    if (!hL || !q1w || !q1 || !q2w || !q2 || !y ||
        (t && (!q1n || !q2n || !dhL || !loss || !dQ1 || !dq1 || !dQ2 || !dq2)))
        return fail(FNO_NET_ERR_INVALID, "fno_net_proj: missing argument");
    const int64_t P = (int64_t)d->batch * d->nr * d->nz;
    ProjP p{(int)P, d->out_ch, (float)(2.0 / ((double)P * d->out_ch)), (const bf16*)hL, (const bf16*)q1w,
            (const bf16*)q1n, q1, (const bf16*)q2w, (const bf16*)q2n, q2, t, y, (bf16*)dhL, loss,
            dQ1, dq1, dQ2, dq2};
    const int per_sm = d->width == 32 ? 2 : 1;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(P / 128, (int64_t)per_sm * sms()));
    cudaStream_t s = (cudaStream_t)stream;
    if (d->width == 32) {
        const size_t sb = std::max(ProjSmem<32>::bytes, SMEM_2_PER_SM);
        if (t) {
            if (int rc = set_smem(k_proj<32, true>, sb)) return rc;
            NCK(launch_pdl(k_proj<32, true>, dim3(grid), dim3(256), sb, s, p));
        } else {
            if (int rc = set_smem(k_proj<32, false>, sb)) return rc;
            NCK(launch_pdl(k_proj<32, false>, dim3(grid), dim3(256), sb, s, p));
        }
    } else {
        const size_t sb = std::max(ProjSmem<64>::bytes, SMEM_1_PER_SM);
        if (t) {
            if (int rc = set_smem(k_proj<64, true>, sb)) return rc;
            NCK(launch_pdl(k_proj<64, true>, dim3(grid), dim3(256), sb, s, p));
        } else {
            if (int rc = set_smem(k_proj<64, false>, sb)) return rc;
            NCK(launch_pdl(k_proj<64, false>, dim3(grid), dim3(256), sb, s, p));
        }
    }
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

#define BWD_CASE(C_, K_, MODE_)                                                                         \
    if (d->width == C_ && 2 * d->modes == K_ && mode == MODE_) {                                       \
        const size_t sb = std::max(BwdSmem<C_, K_, MODE_>::bytes(d->nz), SMEM_2_PER_SM);               \
        if (int rc = set_smem(k_bwd<C_, K_, MODE_>, sb)) return rc;                                    \
        NCK(launch_pdl(k_bwd<C_, K_, MODE_>, dim3(grid), dim3(256), sb, s, p));                                                  \
        launched = true;                                                                              \
    }

int fno_net_bwd(int mode, const fno_net_dims* d, const void* dpre_in, const void* dZ, const void* wn_img,
                const void* fz_img, const void* pre, const void* h, const float* x, const void* gzt_img, void* dpre_out,
                void* dV, float* dW, float* db, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_bwd: %s", why.c_str());
    if (mode < 0 || mode > 2 || !dpre_in || !dW || !db || (mode != 0 && (!dZ || !wn_img || !fz_img)) ||
        (mode == 1 && (!pre || !dpre_out)) || (mode != 2 && (!h || !gzt_img || !dV)) || (mode == 2 && !x))
        return fail(FNO_NET_ERR_INVALID, "fno_net_bwd: missing argument for mode %d", mode);
    BwdP p{d->batch * d->nr, d->nr, d->nz, d->in_ch, (float)((double)d->nr * d->nz), (const bf16*)dpre_in,
           (const bf16*)dZ, (const bf16*)wn_img, (const bf16*)fz_img, (const bf16*)pre, (const bf16*)h, x,
           (const bf16*)gzt_img, (bf16*)dpre_out, (bf16*)dV, dW, db};
    const unsigned grid = (unsigned)std::max(1, std::min(p.nrows / (128 / d->width), 2 * sms()));
    cudaStream_t s = (cudaStream_t)stream;
    bool launched = false;
    BWD_CASE(32, 32, 0) BWD_CASE(32, 32, 1) BWD_CASE(32, 32, 2)
    BWD_CASE(32, 16, 0) BWD_CASE(32, 16, 1) BWD_CASE(32, 16, 2)
    BWD_CASE(64, 32, 0) BWD_CASE(64, 32, 1) BWD_CASE(64, 32, 2)
    BWD_CASE(64, 16, 0) BWD_CASE(64, 16, 1) BWD_CASE(64, 16, 2)
    if (!launched) return fail(FNO_NET_ERR_INVALID, "fno_net_bwd: no kernel for these sizes");
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

int fno_net_r2k(const fno_net_dims* d, const void* in, const void* f2_img, float* out, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_r2k: %s", why.c_str());
    if (!in || !f2_img || !out) return fail(FNO_NET_ERR_INVALID, "fno_net_r2k: NULL argument");
    const size_t sb = (size_t)128 * 2 * d->nr * 2 + (size_t)2 * d->nr * d->width * 2 + 1024;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)(d->batch * d->modes);
    if (d->width == 32) {
        if (int rc = set_smem(k_r2k<32>, sb)) return rc;
        NCK(launch_pdl(k_r2k<32>, dim3(grid), dim3(128), sb, s, (const bf16*)in, (const bf16*)f2_img, out, d->batch, d->nr, d->modes));
    } else {
        if (int rc = set_smem(k_r2k<64>, sb)) return rc;
        NCK(launch_pdl(k_r2k<64>, dim3(grid), dim3(128), sb, s, (const bf16*)in, (const bf16*)f2_img, out, d->batch, d->nr, d->modes));
    }
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

int fno_net_k2r(const fno_net_dims* d, const float* in, const void* f2i_img, void* out, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_k2r: %s", why.c_str());
    if (!in || !f2i_img || !out) return fail(FNO_NET_ERR_INVALID, "fno_net_k2r: NULL argument");
    const size_t sb = std::max((size_t)128 * 4 * d->modes * 2 + (size_t)4 * d->modes * d->width * 2 + 1024,
                               SMEM_7_PER_SM);
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)(d->batch * d->modes * (2 * d->nr / 128));
    if (d->width == 32) {
        if (int rc = set_smem(k_k2r<32>, sb)) return rc;
        NCK(launch_pdl(k_k2r<32>, dim3(grid), dim3(128), sb, s, in, (const bf16*)f2i_img, (bf16*)out, d->batch, d->nr, d->modes));
    } else {
        if (int rc = set_smem(k_k2r<64>, sb)) return rc;
        NCK(launch_pdl(k_k2r<64>, dim3(grid), dim3(128), sb, s, in, (const bf16*)f2i_img, (bf16*)out, d->batch, d->nr, d->modes));
    }
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

int fno_net_mix_fwd(const fno_net_dims* d, const float* W, const float* R, float* Y, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_mix_fwd: %s", why.c_str());
    if (!W || !R || !Y) return fail(FNO_NET_ERR_INVALID, "fno_net_mix_fwd: NULL argument");
    const int C = d->width, B = d->batch;
    const size_t sb = (size_t)(2 * C * C + 2 * B * C) * 4;
    if (sb > 200 * 1024) return fail(FNO_NET_ERR_INVALID, "fno_net_mix_fwd: batch too large");
    if (int rc = set_smem(k_mixf, sb)) return rc;
    NCK(launch_pdl(k_mixf, dim3((unsigned)(2 * d->modes * d->modes)), dim3(256), sb, (cudaStream_t)stream, W, R, Y, B, C, d->modes));
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

int fno_net_mix_bwd(const fno_net_dims* d, const float* W, const float* R, const float* dY, float* dW, float* dR,
                    int accumulate, void* stream) {
    std::string why;
    if (!dims_ok(d, &why)) return fail(FNO_NET_ERR_INVALID, "fno_net_mix_bwd: %s", why.c_str());
    if (!W || !R || !dY || !dW || !dR) return fail(FNO_NET_ERR_INVALID, "fno_net_mix_bwd: NULL argument");
    const int C = d->width, B = d->batch;
    const size_t sb = (size_t)(2 * C * C + 4 * B * C) * 4;
    if (sb > 200 * 1024) return fail(FNO_NET_ERR_INVALID, "fno_net_mix_bwd: batch too large");
    if (int rc = set_smem(k_mixb, sb)) return rc;
    NCK(launch_pdl(k_mixb, dim3((unsigned)(2 * d->modes * d->modes)), dim3(256), sb, (cudaStream_t)stream, W, R, dY, dW, dR, B, C, d->modes,
                                                                                     accumulate));
    NCK(cudaGetLastError());
    return FNO_NET_OK;
}

int fno_net_status(int clear) {
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(&v, g_net_error, sizeof(int)) != cudaSuccess) return -1;
    if (clear) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_net_error, &z, sizeof(int)) != cudaSuccess) return -1;
    }
    return v;
}

const char* fno_net_last_error(void) { return g_err.c_str(); }

}  // extern "C"
