// fno.cu -- kernels of the learned warm start (Fourier neural operator) behind the C
// ABI of include/fno.h.  BF16 tensor-core GEMM with FP32 accumulation (mma.sync
// m16n8k16), per-mode complex channel mixing, GELU, column sums, MSE and Adam.
// The paper has no counterpart: the network only proposes an initial field; the
// lattice Boltzmann iteration always runs to convergence from it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/fno.h"

static thread_local std::string g_fno_err;

static int fno_fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_fno_err = buf;
    return code;
}

#define FCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            (void)cudaGetLastError();                                                              \
            return fno_fail(FNO_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                \
        }                                                                                          \
    } while (0)

// ------------------------------------------------------------------- GEMM --
// Block tile 64 x 64 x 32, four warps (2 x 2), each warp 32 x 32 = 2 x 4 tiles of the
// m16n8k16 BF16 MMA.  Operands are read from FP32 global memory (any transposition,
// bounds-checked, zero-filled) and rounded to BF16 into shared memory: A as [m][k],
// B as [n][k] (the "col" operand of the MMA).  Rows padded to 40 elements so that the
// fragment loads of a warp hit 32 different banks.
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 40;

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, float alpha, const float* __restrict__ A,
                                              int64_t lda, int64_t sA, const float* __restrict__ B, int64_t ldb,
                                              int64_t sB, float beta, float* __restrict__ C, int64_t ldc, int64_t sC,
                                              const float* __restrict__ bias) {
    __shared__ __align__(16) __nv_bfloat16 As[GBM][GPAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    A += (int64_t)blockIdx.z * sA;
    B += (int64_t)blockIdx.z * sB;
    C += (int64_t)blockIdx.z * sC;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
        for (int i = 0; i < (GBM * GBK) / 128; ++i) {
            const int idx = tid + 128 * i;
            int m, k;
            if (TA) { k = idx / GBM; m = idx % GBM; } else { m = idx / GBK; k = idx % GBK; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.f;
            if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[m][k] = __float2bfloat16_rn(v);
        }
#pragma unroll
        for (int i = 0; i < (GBN * GBK) / 128; ++i) {
            const int idx = tid + 128 * i;
            int n, k;
            if (TB) { n = idx / GBK; k = idx % GBK; } else { k = idx / GBN; n = idx % GBN; }
            const int gn = n0 + n, gk = k0 + k;
            float v = 0.f;
            if (gn < N && gk < K) v = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
            Bs[n][k] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + g;
                af[i][0] = ld_pair(&As[r][kk + 2 * t]);
                af[i][1] = ld_pair(&As[r + 8][kk + 2 * t]);
                af[i][2] = ld_pair(&As[r][kk + 2 * t + 8]);
                af[i][3] = ld_pair(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + g;
                bf[j][0] = ld_pair(&Bs[c][kk + 2 * t]);
                bf[j][1] = ld_pair(&Bs[c][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + wm + 16 * i + g + (e >= 2 ? 8 : 0);
                const int col = n0 + wn + 8 * j + 2 * t + (e & 1);
                if (row < M && col < N) {
                    float* c = C + (int64_t)row * ldc + col;
                    float v = alpha * acc[i][j][e];
                    if (beta != 0.f) v += beta * *c;
                    if (bias) v += bias[col];
                    *c = v;
                }
            }
}


// ------------------------------------------------------- tcgen05 GEMM path --
// Persistent CTAs (four warps) on the 5th-generation tensor cores.  Each CTA allocates
// its tensor-memory accumulator (128 lanes x ncols FP32 columns) once and walks a
// strided list of steps: (tile, K chunk) pairs, a tile being 128 x ntile of C (ntile <=
// 256, a multiple of 16) of one batch entry and a chunk 64 of K.  Operands are staged
// from FP32 global memory as BF16 into shared memory in the canonical K-major layout
// without swizzle (core matrices of 8 rows x 16 bytes; LBO = 128 B between core
// matrices along K, SBO = 1024 B between 8-row groups), with 16-byte loads where the
// layout allows; two stage buffers let the next chunk be staged while thread 0's four
// tcgen05.mma (K = 16 each) on the current one run.  Each buffer has an mbarrier that
// tcgen05.commit arrives on.  After a tile's last chunk each warp reads its 32
// accumulator lanes back with tcgen05.ld and writes C (16-byte stores where aligned).
// Every wait is bounded: on timeout the kernel stops issuing work, waits once more
// (bounded) for each buffer whose commit it has not seen complete, records an error
// (1: those waits completed, so no MMA was outstanding when the tensor memory was
// freed; 2: one of them ran out too), frees its tensor memory and returns.
constexpr int TC_BM = 128, TC_BK = 64;
constexpr int TC_SPIN = 1 << 22;        // try_wait rounds of a normal wait
constexpr int TC_TEST_SPIN = 1 << 12;   // rounds of the test wait (fno_test_wait_timeout)
__device__ int g_tc_error;
// Test hook: when set, the main loop's first wait for a commit is replaced by a wait on
// a barrier nothing arrives at, with a short bound, so that the timeout path runs.
__device__ int g_tc_wait_test;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start address, leading-dimension byte
// offset (LBO) and stride-dimension byte offset (SBO).  Tiles are kept in the canonical
// layout of 8 x 16-byte core matrices, each 128 contiguous bytes.  Without swizzling LBO is
// the stride between core matrices adjacent along K and SBO the stride between those
// adjacent along M (N), whether the operand is K-major (8 consecutive k per 16-byte row)
// or MN-major (8 consecutive m (n) per 16-byte row, the 8 rows being 8 consecutive k).
__device__ __forceinline__ uint64_t tc_desc_raw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// K-major tile whose rows hold BK elements: LBO = 128 B, SBO = BK / 8 x 128 B.
template <int BK>
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return tc_desc_raw(saddr, 128, (BK / 8) * 128);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase, int spin = TC_SPIN) {
    for (int i = 0; i < spin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// byte offset of element (row, k) of a [rows x BK] K-major tile in the canonical layout
template <int BK>
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
    return (uint32_t)((((row >> 3) * (BK / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// byte offset of element (row, k) of a [rows x BK] MN-major tile (rows contiguous within a
// 16-byte core-matrix row): core matrices adjacent along the rows 128 B apart, groups of 8
// k rows / 8 x 128 B apart
__device__ __forceinline__ uint32_t tc_off_mn(int rows, int row, int k) {
    return (uint32_t)((((k >> 3) * (rows >> 3) + (row >> 3)) << 7) + ((k & 7) << 4) + ((row & 7) << 1));
}

__device__ __forceinline__ void st_bf16x4(uint8_t* p, float a, float b, float c, float d) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t*>(&lo);
    v.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(p) = v;
}

// Stage the rows x 64 chunk starting at (r0, k0) of an operand X whose element (row, k)
// is at X[row * ld + k] (kmajor) or X[k * ld + row] (!kmajor) into tile T, as BF16,
// zero outside [0, R) x [0, K).  vec: ld and X allow 16-byte loads along the contiguous
// direction.
template <bool KMAJOR, int BK>
__device__ __forceinline__ void tc_stage(uint8_t* T, const float* __restrict__ X, int64_t ld, int rows, int r0,
                                         int R, int k0, int K, bool vec) {
    const int tid = threadIdx.x;
    constexpr int KQ = BK / 4;   // float4 per row along k
    if (KMAJOR) {
        for (int f = tid; f < rows * KQ; f += 128) {
            const int r = f / KQ, kq = (f % KQ) << 2;
            const int gr = r0 + r, gk = k0 + kq;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (gr < R) {
                const float* src = X + (int64_t)gr * ld + gk;
                if (vec && gk + 3 < K) {
                    const float4 q = *reinterpret_cast<const float4*>(src);
                    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (gk + i < K) v[i] = src[i];
                }
            }
            st_bf16x4(T + tc_off<BK>(r, kq), v[0], v[1], v[2], v[3]);
        }
    } else {        // MN-major tile: rows / 4 float4 along the row index per k, 8-byte stores
        const int rq = rows >> 2;
        for (int f = tid; f < rq * BK; f += 128) {
            const int k = f / rq, r = (f - k * rq) << 2;
            const int gr = r0 + r, gk = k0 + k;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (gk < K) {
                const float* src = X + (int64_t)gk * ld + gr;
                if (vec && gr + 3 < R) {
                    const float4 q = *reinterpret_cast<const float4*>(src);
                    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (gr + i < R) v[i] = src[i];
                }
            }
            st_bf16x4(T + tc_off_mn(rows, r, k), v[0], v[1], v[2], v[3]);
        }
    }
}

template <bool TA, bool TB, int BK>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, int ntile, int ntm, int ntn, int batch,
                                                 float alpha, const float* __restrict__ A, int64_t lda, int64_t sA,
                                                 const float* __restrict__ B, int64_t ldb, int64_t sB, float beta,
                                                 float* __restrict__ C, int64_t ldc, int64_t sC,
                                                 const float* __restrict__ bias, int vecA, int vecB, int vecC) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ __align__(8) uint64_t mbar[3];   // two stage buffers; [2] never arrived at (test hook)
    __shared__ uint32_t tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t abytes = TC_BM * BK * 2, stage_bytes = abytes + (uint32_t)ntile * BK * 2;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)ntile) ncols <<= 1;
    const uint32_t mb0 = smem_u32(&mbar[0]);   // buffer b's barrier at mb0 + 8 b
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 16) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_sh;
    // kind::f16 instruction descriptor: D F32, A and B BF16, N, M = 128; an operand stored
    // with its M (N) index contiguous (A transposed, B not) is staged MN-major (bits 15, 16)
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (TA ? (1u << 15) : 0u) | (TB ? 0u : (1u << 16)) |
                           ((uint32_t)(ntile >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
    const int nk = (K + BK - 1) / BK;
    const int64_t ntiles = (int64_t)ntm * ntn * batch;
    // this CTA's steps: tiles t = blockIdx.x + j gridDim.x, each in nk chunks of K
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nsteps = my_tiles * nk;
    uint32_t phase_bits = 0, pend_bits = 0;   // per stage buffer: mbarrier phase, commit outstanding
    bool ok = true;
    bool test_wait = *(volatile int*)&g_tc_wait_test != 0;
    auto step_tile = [&](int64_t st, int& tb, int& tm, int& tn, int& kc) {
        const int64_t t = blockIdx.x + (st / nk) * (int64_t)gridDim.x;
        kc = (int)(st % nk);
        tb = (int)(t / ((int64_t)ntm * ntn));
        const int64_t rem = t - (int64_t)tb * ntm * ntn;
        tm = (int)(rem / ntn);
        tn = (int)(rem - (int64_t)tm * ntn);
    };
    auto stage = [&](int64_t st, int buf) {
        int tb, tm, tn, kc;
        step_tile(st, tb, tm, tn, kc);
        uint8_t* As = tc_smem + buf * stage_bytes;
        tc_stage<!TA, BK>(As, A + (int64_t)tb * sA, lda, TC_BM, tm * TC_BM, M, kc * BK, K, vecA != 0);
        tc_stage<TB, BK>(As + abytes, B + (int64_t)tb * sB, ldb, ntile, tn * ntile, N, kc * BK, K, vecB != 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };
    auto issue = [&](int64_t st, int buf) {   // all threads call it (state stays uniform)
        if (tid == 0) {
            const int kc = (int)(st % nk);
            const uint32_t a0 = smem_u32(tc_smem + buf * stage_bytes);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) {
                // K step j (16 k): K-major tiles advance two core matrices along K (256 B),
                // MN-major tiles two groups of 8 k rows (2 x rows / 8 x 128 B)
                const uint64_t ad = TA ? tc_desc_raw(a0 + j * 2 * TC_BM * 16, TC_BM * 16, 128)
                                       : tc_desc<BK>(a0 + j * 256);
                const uint64_t bd = TB ? tc_desc<BK>(a0 + abytes + j * 256)
                                       : tc_desc_raw(a0 + abytes + j * 2 * ntile * 16, ntile * 16, 128);
                const uint32_t acc = (kc > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             mb0 + 8 * buf)
                         : "memory");
        }
        pend_bits |= 1u << buf;
    };
    // wait for the commit on buf, if one is outstanding; every thread reaches each call,
    // and the block agrees on the outcome (a lone timeout must not split the barriers).
    // The commit counts as consumed only when every thread saw it complete; otherwise it
    // stays outstanding for the recovery wait below.
    auto drain = [&](int buf) {
        if (pend_bits & (1u << buf)) {
            const bool got = test_wait ? tc_wait(mb0 + 16, 0u, TC_TEST_SPIN)
                                       : tc_wait(mb0 + 8 * buf, (phase_bits >> buf) & 1u);
            test_wait = false;
            const bool all = __syncthreads_and(got) != 0;
            if (all) {
                phase_bits ^= 1u << buf;
                pend_bits &= ~(1u << buf);
            }
            ok = ok && all;
        }
    };
    if (nsteps > 0) {
        stage(0, 0);
        __syncthreads();
        issue(0, 0);
    }
    for (int64_t st = 0; st < nsteps && ok; ++st) {
        const int buf = (int)(st & 1), nb = buf ^ 1;
        if (st + 1 < nsteps) {
            drain(nb);                 // the MMA that read buffer nb (step st - 1) is done
            if (!ok) break;
            stage(st + 1, nb);         // overlaps the MMA of step st
        }
        int tb, tm, tn, kc;
        step_tile(st, tb, tm, tn, kc);
        if (kc == nk - 1) {            // last chunk of the tile: epilogue
            drain(buf);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = tm * TC_BM + warp * 32 + lane;
            float* Cb = C + (int64_t)tb * sC;
            for (int c = 0; c < ntile; c += 8) {
                uint32_t r[8];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(taddr)
                             : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int col0 = tn * ntile + c;
                if (row < M) {
                    float* cp = Cb + (int64_t)row * ldc + col0;
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        v[q] = alpha * __uint_as_float(r[q]);
                        if (bias && col0 + q < N) v[q] += bias[col0 + q];
                    }
                    if (vecC && beta == 0.f && col0 + 7 < N && c + 7 < ntile) {
                        *reinterpret_cast<float4*>(cp) = make_float4(v[0], v[1], v[2], v[3]);
                        *reinterpret_cast<float4*>(cp + 4) = make_float4(v[4], v[5], v[6], v[7]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (col0 + q < N && c + q < ntile) cp[q] = beta != 0.f ? v[q] + beta * cp[q] : v[q];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        __syncthreads();               // staging of st + 1 complete; accumulator free after an epilogue
        if (st + 1 < nsteps) issue(st + 1, nb);
    }
    if (ok) {                          // consume any commit left (complete: they finish in order)
        drain(0);
        drain(1);
    } else {
        // one more bounded wait for every commit not yet seen complete, before the tensor
        // memory is freed; error 2 if one of them runs out as well
        bool clean = true;
        for (int b = 0; b < 2; ++b)
            if (pend_bits & (1u << b)) clean = tc_wait(mb0 + 8 * b, (phase_bits >> b) & 1u) && clean;
        clean = __syncthreads_and(clean) != 0;
        if (tid == 0) atomicMax(&g_tc_error, clean ? 1 : 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

static int g_tc_path = 0;          // 1: route fno_gemm through the tcgen05 kernel
static bool g_tc_poisoned = false; // a recovery wait ran out: the tcgen05 path stays off
static int g_num_sms = 0;

static bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

static int gemm_tc(int transA, int transB, int M, int N, int K, float alpha, const float* A, int64_t lda,
                   int64_t strideA, const float* B, int64_t ldb, int64_t strideB, float beta, float* C, int64_t ldc,
                   int64_t strideC, int batch, const float* bias, cudaStream_t s) {
    if (!g_num_sms) {
        int dev = 0;
        FCK(cudaGetDevice(&dev));
        FCK(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // tile width: the widest (<= 256, a multiple of 16, not wider than N needs) that still
    // gives four tiles per SM; small GEMMs take narrower tiles to fill the machine
    const int ntm = (M + TC_BM - 1) / TC_BM;
    int ntile = std::min(256, ((N + 15) / 16) * 16);
    while (ntile > 16 && (int64_t)ntm * ((N + ntile - 1) / ntile) * batch < 4LL * g_num_sms)
        ntile = std::max(16, ((ntile / 2 + 15) / 16) * 16);
    const int ntn = (N + ntile - 1) / ntile;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)ntile) ncols <<= 1;
    // resident CTAs per SM whose accumulators fit the 512 tensor-memory columns
    const int64_t per_sm = std::max<int64_t>(1, std::min<int64_t>(4, 512 / ncols));
    const int64_t ntiles = (int64_t)ntm * ntn * batch;
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, per_sm * g_num_sms);
    // K chunk: 32 when K fits in it (half the staging of a padded 64-wide chunk), else 64
    const int bk = K <= 32 ? 32 : TC_BK;
    const size_t smem = 2 * (size_t)(TC_BM + ntile) * bk * 2;
    static bool attr_done = false;
    if (!attr_done) {
        const int lim = 2 * (TC_BM + 256) * TC_BK * 2;
        FCK(cudaFuncSetAttribute(k_gemm_tc<false, false, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<false, true, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<true, false, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<true, true, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<false, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<false, true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<true, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<true, true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        attr_done = true;
    }
    // 16-byte loads along the contiguous direction: base, leading dimension and batch stride
    // aligned, the row length in that direction a multiple of 4
    const int vecA = al16(A) && lda % 4 == 0 && strideA % 4 == 0;
    const int vecB = al16(B) && ldb % 4 == 0 && strideB % 4 == 0;
    const int vecC = al16(C) && ldc % 4 == 0 && strideC % 4 == 0 && ntile % 8 == 0;
#define TC_LAUNCH(TA_, TB_)                                                                                      \
    do {                                                                                                         \
        if (bk == 32)                                                                                            \
            k_gemm_tc<TA_, TB_, 32><<<grid, 128, smem, s>>>(M, N, K, ntile, ntm, ntn, batch, alpha, A, lda,     \
                                                            strideA, B, ldb, strideB, beta, C, ldc, strideC,    \
                                                            bias, vecA, vecB, vecC);                            \
        else                                                                                                     \
            k_gemm_tc<TA_, TB_, 64><<<grid, 128, smem, s>>>(M, N, K, ntile, ntm, ntn, batch, alpha, A, lda,     \
                                                            strideA, B, ldb, strideB, beta, C, ldc, strideC,    \
                                                            bias, vecA, vecB, vecC);                            \
    } while (0)
    if (!transA && !transB) TC_LAUNCH(false, false);
    else if (!transA && transB) TC_LAUNCH(false, true);
    else if (transA && !transB) TC_LAUNCH(true, false);
    else TC_LAUNCH(true, true);
#undef TC_LAUNCH
    FCK(cudaGetLastError());
    return FNO_OK;
}

// ---------------------------------------------------------------- elementwise --
__global__ void k_gelu_fwd(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        y[i] = 0.5f * v * (1.0f + erff(v * 0.70710678118654752f));
    }
}

__global__ void k_gelu_bwd(const float* __restrict__ x, const float* __restrict__ dy, float* __restrict__ dx, int64_t n,
                           int accumulate) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        const float d = 0.5f * (1.0f + erff(v * 0.70710678118654752f)) + v * 0.39894228040143268f * expf(-0.5f * v * v);
        const float r = d * dy[i];
        dx[i] = accumulate ? dx[i] + r : r;
    }
}

// ------------------------------------------------------------- spectral mix --
// X offset of (b, kr, kz2, c) with kz2 in [0, 2 nkz): real parts at kz2 = kz,
// imaginary parts at kz2 = nkz + kz.
__device__ __forceinline__ int64_t xoff(int b, int kr, int kz2, int c, int nkr, int nkz, int C) {
    return (((int64_t)b * nkr + kr) * (2 * nkz) + kz2) * C + c;
}

__global__ void k_mix_fwd(const float* __restrict__ X, const float* __restrict__ R, float* __restrict__ Y, int nkr,
                          int nkz, int C, int O) {
    extern __shared__ float sx[];   // 2 C
    const int mode = blockIdx.x, b = blockIdx.y;
    const int kr = mode / nkz, kz = mode % nkz;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        sx[c] = X[xoff(b, kr, kz, c, nkr, nkz, C)];
        sx[C + c] = X[xoff(b, kr, nkz + kz, c, nkr, nkz, C)];
    }
    __syncthreads();
    const float* Rm = R + (int64_t)mode * C * O * 2;
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int c = 0; c < C; ++c) {
            const float xr = sx[c], xi = sx[C + c];
            const float rr = Rm[((int64_t)c * O + o) * 2], ri = Rm[((int64_t)c * O + o) * 2 + 1];
            re += xr * rr - xi * ri;
            im += xr * ri + xi * rr;
        }
        Y[xoff(b, kr, kz, o, nkr, nkz, O)] = re;
        Y[xoff(b, kr, nkz + kz, o, nkr, nkz, O)] = im;
    }
}

__global__ void k_mix_bwd_x(const float* __restrict__ R, const float* __restrict__ dY, float* __restrict__ dX, int nkr,
                            int nkz, int C, int O) {
    extern __shared__ float sy[];   // 2 O
    const int mode = blockIdx.x, b = blockIdx.y;
    const int kr = mode / nkz, kz = mode % nkz;
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        sy[o] = dY[xoff(b, kr, kz, o, nkr, nkz, O)];
        sy[O + o] = dY[xoff(b, kr, nkz + kz, o, nkr, nkz, O)];
    }
    __syncthreads();
    const float* Rm = R + (int64_t)mode * C * O * 2;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float gr = 0.f, gi = 0.f;
        for (int o = 0; o < O; ++o) {
            const float yr = sy[o], yi = sy[O + o];
            const float rr = Rm[((int64_t)c * O + o) * 2], ri = Rm[((int64_t)c * O + o) * 2 + 1];
            gr += yr * rr + yi * ri;
            gi += -yr * ri + yi * rr;
        }
        dX[xoff(b, kr, kz, c, nkr, nkz, C)] = gr;
        dX[xoff(b, kr, nkz + kz, c, nkr, nkz, C)] = gi;
    }
}

__global__ void k_mix_bwd_r(const float* __restrict__ X, const float* __restrict__ dY, float* __restrict__ dR, int batch,
                            int nkr, int nkz, int C, int O, int accumulate) {
    const int mode = blockIdx.x;
    const int kr = mode / nkz, kz = mode % nkz;
    for (int co = threadIdx.x; co < C * O; co += blockDim.x) {
        const int c = co / O, o = co % O;
        float gr = 0.f, gi = 0.f;
        for (int b = 0; b < batch; ++b) {
            const float xr = X[xoff(b, kr, kz, c, nkr, nkz, C)], xi = X[xoff(b, kr, nkz + kz, c, nkr, nkz, C)];
            const float yr = dY[xoff(b, kr, kz, o, nkr, nkz, O)], yi = dY[xoff(b, kr, nkz + kz, o, nkr, nkz, O)];
            gr += yr * xr + yi * xi;
            gi += -yr * xi + yi * xr;
        }
        float* d = dR + (((int64_t)mode * C + c) * O + o) * 2;
        d[0] = accumulate ? d[0] + gr : gr;
        d[1] = accumulate ? d[1] + gi : gi;
    }
}

// ------------------------------------------------------------- reductions --
__global__ void k_colsum(const float* __restrict__ X, int64_t rows, int N, int64_t ldx, float* __restrict__ out) {
    __shared__ float s[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.f;
    if (n < N)
        for (int64_t r = (int64_t)blockIdx.y * 8 + threadIdx.y; r < rows; r += (int64_t)gridDim.y * 8)
            acc += X[r * ldx + n];
    s[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float v = 0.f;
        for (int j = 0; j < 8; ++j) v += s[j][threadIdx.x];
        atomicAdd(out + n, v);
    }
}

__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy, double* loss,
                      int64_t n) {
    __shared__ double s[32];
    double acc = 0.0;
    const float sc = 2.0f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        acc += (double)d * d;
        dy[i] = sc * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(loss, v / (double)n);
    }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static unsigned grid1d(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

extern "C" {

int fno_gemm(int transA, int transB, int M, int N, int K, float alpha, const float* A, int64_t lda, int64_t strideA,
             const float* B, int64_t ldb, int64_t strideB, float beta, float* C, int64_t ldc, int64_t strideC,
             int batch, const float* bias, void* stream) {
    if (M < 0 || N < 0 || K < 0 || batch < 0 || !A || !B || !C) return fno_fail(FNO_ERR_INVALID, "bad GEMM argument");
    if (M == 0 || N == 0 || batch == 0) return FNO_OK;
    if (batch > 65535 || (M + GBM - 1) / GBM > 65535) return fno_fail(FNO_ERR_INVALID, "GEMM grid too large");
    if (g_tc_path)
        return gemm_tc(transA, transB, M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, batch,
                       bias, (cudaStream_t)stream);
    const dim3 grid((unsigned)((N + GBN - 1) / GBN), (unsigned)((M + GBM - 1) / GBM), (unsigned)batch);
    cudaStream_t s = (cudaStream_t)stream;
    if (!transA && !transB)
        k_gemm<false, false><<<grid, 128, 0, s>>>(M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    else if (!transA && transB)
        k_gemm<false, true><<<grid, 128, 0, s>>>(M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    else if (transA && !transB)
        k_gemm<true, false><<<grid, 128, 0, s>>>(M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    else
        k_gemm<true, true><<<grid, 128, 0, s>>>(M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_gelu_fwd(const float* x, float* y, int64_t n, void* stream) {
    if (!x || !y || n < 0) return fno_fail(FNO_ERR_INVALID, "bad GELU argument");
    if (n == 0) return FNO_OK;
    k_gelu_fwd<<<grid1d(n, 256), 256, 0, (cudaStream_t)stream>>>(x, y, n);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_gelu_bwd(const float* x, const float* dy, float* dx, int64_t n, int accumulate, void* stream) {
    if (!x || !dy || !dx || n < 0) return fno_fail(FNO_ERR_INVALID, "bad GELU argument");
    if (n == 0) return FNO_OK;
    k_gelu_bwd<<<grid1d(n, 256), 256, 0, (cudaStream_t)stream>>>(x, dy, dx, n, accumulate);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_mix_fwd(const float* X, const float* R, float* Y, int batch, int nkr, int nkz, int C, int O, void* stream) {
    if (!X || !R || !Y || batch < 1 || nkr < 1 || nkz < 1 || C < 1 || O < 1 || batch > 65535 || C > 4096 || O > 4096)
        return fno_fail(FNO_ERR_INVALID, "bad mixing argument");
    k_mix_fwd<<<dim3(nkr * nkz, batch), 128, 2 * C * sizeof(float), (cudaStream_t)stream>>>(X, R, Y, nkr, nkz, C, O);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_mix_bwd(const float* X, const float* R, const float* dY, float* dX, float* dR, int batch, int nkr, int nkz,
                int C, int O, int accumulate, void* stream) {
    if (!X || !R || !dY || !dX || !dR || batch < 1 || nkr < 1 || nkz < 1 || C < 1 || O < 1 || batch > 65535 ||
        C > 4096 || O > 4096)
        return fno_fail(FNO_ERR_INVALID, "bad mixing argument");
    cudaStream_t s = (cudaStream_t)stream;
    k_mix_bwd_x<<<dim3(nkr * nkz, batch), 128, 2 * O * sizeof(float), s>>>(R, dY, dX, nkr, nkz, C, O);
    FCK(cudaGetLastError());
    k_mix_bwd_r<<<nkr * nkz, 256, 0, s>>>(X, dY, dR, batch, nkr, nkz, C, O, accumulate);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_colsum(const float* X, int64_t rows, int N, int64_t ldx, float* out, int accumulate, void* stream) {
    if (!X || !out || rows < 0 || N < 1) return fno_fail(FNO_ERR_INVALID, "bad colsum argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!accumulate) FCK(cudaMemsetAsync(out, 0, N * sizeof(float), s));
    if (rows == 0) return FNO_OK;
    const int64_t chunks = (rows + 1023) / 1024;
    const dim3 grid((unsigned)((N + 31) / 32), (unsigned)(chunks < 512 ? chunks : 512));
    k_colsum<<<grid, dim3(32, 8), 0, s>>>(X, rows, N, ldx, out);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_mse(const float* y, const float* t, float* dy, double* loss, int64_t n, void* stream) {
    if (!y || !t || !dy || !loss || n < 1) return fno_fail(FNO_ERR_INVALID, "bad MSE argument");
    k_mse<<<grid1d(n, 256), 256, 0, (cudaStream_t)stream>>>(y, t, dy, loss, n);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2, float eps,
             int t, void* stream) {
    if (!w || !g || !m || !v || n < 0 || t < 1) return fno_fail(FNO_ERR_INVALID, "bad Adam argument");
    if (n == 0) return FNO_OK;
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_adam<<<grid1d(n, 256), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    FCK(cudaGetLastError());
    return FNO_OK;
}

int fno_set_tensor_path(int path) {
    if (path != 0 && path != 1) return fno_fail(FNO_ERR_INVALID, "path must be 0 (mma.sync) or 1 (tcgen05)");
    if (path == 1 && g_tc_poisoned)
        return fno_fail(FNO_ERR_CUDA, "the tcgen05 path is disabled for this process (a recovery wait ran out)");
    g_tc_path = path;
    return FNO_OK;
}

int fno_tensor_path_status(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
    if (v >= 2 && !g_tc_poisoned) {
        // tensor memory may have been freed under an MMA still in flight: results of
        // later tcgen05 GEMMs could be wrong without any report, so the path stays off
        g_tc_poisoned = true;
        g_tc_path = 0;
    }
    if (clear) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int)) != cudaSuccess) return -1;
    }
    return g_tc_poisoned ? 2 : v;
}

int fno_test_wait_timeout(int enable) {
    const int v = enable ? 1 : 0;
    FCK(cudaMemcpyToSymbol(g_tc_wait_test, &v, sizeof(int)));
    return FNO_OK;
}

int fno_test_set_tc_error(int value) {
    if (value < 0 || value > 2) return fno_fail(FNO_ERR_INVALID, "value must be 0, 1 or 2");
    FCK(cudaMemcpyToSymbol(g_tc_error, &value, sizeof(int)));
    return FNO_OK;
}

const char* fno_last_error(void) { return g_fno_err.c_str(); }

}  // extern "C"
