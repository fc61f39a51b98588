// fno.cu -- kernels of the learned warm start (Fourier neural operator) behind the C
// ABI of include/fno.h.  BF16 tensor-core GEMM with FP32 accumulation (mma.sync
// m16n8k16), per-mode complex channel mixing, GELU, column sums, MSE and Adam.
// The paper has no counterpart: the network only proposes an initial field; the
// lattice Boltzmann iteration always runs to convergence from it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

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
// One CTA (four warps) computes a 128 x ntile tile of C (ntile <= 256, a multiple of
// 16) on the 5th-generation tensor cores: operands are staged from FP32 global memory
// as BF16 into shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes; LBO = 128 B between core matrices along K, SBO =
// 1024 B between 8-row groups for a 64-wide K chunk), thread 0 issues four
// tcgen05.mma (K = 16 each) per chunk into an FP32 accumulator in tensor memory and
// commits them to an mbarrier, and each warp reads its 32 accumulator lanes back with
// tcgen05.ld.  Every wait is bounded: on timeout the kernel records an error, waits
// once more (bounded) for the tensor core, frees its tensor memory and returns.
constexpr int TC_BM = 128, TC_BK = 64;
__device__ int g_tc_error;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    const uint64_t lbo = 128, sbo = 1024;
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
    for (int i = 0; i < (1 << 22); ++i) {
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

// byte offset of element (row, k) of a [rows x 64] K-major tile in the canonical layout
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
    return (uint32_t)((((row >> 3) * 8 + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, int ntile, float alpha,
                                                 const float* __restrict__ A, int64_t lda, int64_t sA,
                                                 const float* __restrict__ B, int64_t ldb, int64_t sB, float beta,
                                                 float* __restrict__ C, int64_t ldc, int64_t sC,
                                                 const float* __restrict__ bias) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_sh;
    uint8_t* As = tc_smem;
    uint8_t* Bs = tc_smem + TC_BM * TC_BK * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * ntile;
    A += (int64_t)blockIdx.z * sA;
    B += (int64_t)blockIdx.z * sB;
    C += (int64_t)blockIdx.z * sC;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)ntile) ncols <<= 1;
    const uint32_t mbar_a = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_sh;
    // kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, N, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ntile >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K && ok; k0 += TC_BK) {
        for (int i = tid; i < TC_BM * TC_BK; i += 128) {
            int m, k;
            if (TA) { k = i / TC_BM; m = i % TC_BM; } else { m = i / TC_BK; k = i % TC_BK; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.f;
            if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            *reinterpret_cast<__nv_bfloat16*>(As + tc_off(m, k)) = __float2bfloat16_rn(v);
        }
        for (int i = tid; i < ntile * TC_BK; i += 128) {
            int n, k;
            if (TB) { n = i / TC_BK; k = i % TC_BK; } else { k = i / ntile; n = i % ntile; }
            const int gn = n0 + n, gk = k0 + k;
            float v = 0.f;
            if (gn < N && gk < K) v = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
            *reinterpret_cast<__nv_bfloat16*>(Bs + tc_off(n, k)) = __float2bfloat16_rn(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j) {
                const uint64_t ad = tc_desc(smem_u32(As) + j * 256), bd = tc_desc(smem_u32(Bs) + j * 256);
                const uint32_t acc = (k0 > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                         : "memory");
        }
        ok = tc_wait(mbar_a, phase);
        phase ^= 1;
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicExch(&g_tc_error, 1);
        tc_wait(mbar_a, phase ^ 1);   // one more bounded wait for the tensor core
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + warp * 32 + lane;
        for (int c = 0; c < ntile; c += 8) {
            uint32_t r[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = n0 + c + q;
                    if (col < N && c + q < ntile) {
                        float* cp = C + (int64_t)row * ldc + col;
                        float v = alpha * __uint_as_float(r[q]);
                        if (beta != 0.f) v += beta * *cp;
                        if (bias) v += bias[col];
                        *cp = v;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

static int g_tc_path = 0;   // 1: route fno_gemm through the tcgen05 kernel

static int gemm_tc(int transA, int transB, int M, int N, int K, float alpha, const float* A, int64_t lda,
                   int64_t strideA, const float* B, int64_t ldb, int64_t strideB, float beta, float* C, int64_t ldc,
                   int64_t strideC, int batch, const float* bias, cudaStream_t s) {
    int ntile = ((N + 15) / 16) * 16;
    if (ntile > 256) ntile = 256;
    const dim3 grid((unsigned)((N + ntile - 1) / ntile), (unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)batch);
    if (grid.y > 65535) return fno_fail(FNO_ERR_INVALID, "GEMM grid too large");
    const size_t smem = (size_t)(TC_BM + ntile) * TC_BK * 2;
    static bool attr_done = false;
    if (!attr_done) {
        const int lim = (TC_BM + 256) * TC_BK * 2;
        FCK(cudaFuncSetAttribute(k_gemm_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        FCK(cudaFuncSetAttribute(k_gemm_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        attr_done = true;
    }
    if (!transA && !transB)
        k_gemm_tc<false, false><<<grid, 128, smem, s>>>(M, N, K, ntile, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    else if (!transA && transB)
        k_gemm_tc<false, true><<<grid, 128, smem, s>>>(M, N, K, ntile, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    else if (transA && !transB)
        k_gemm_tc<true, false><<<grid, 128, smem, s>>>(M, N, K, ntile, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
    else
        k_gemm_tc<true, true><<<grid, 128, smem, s>>>(M, N, K, ntile, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC, bias);
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
    g_tc_path = path;
    return FNO_OK;
}

int fno_tensor_path_status(int clear) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
    if (clear) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int)) != cudaSuccess) return -1;
    }
    return v;
}

const char* fno_last_error(void) { return g_fno_err.c_str(); }

}  // extern "C"
