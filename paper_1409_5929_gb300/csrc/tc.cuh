// tc.cuh -- 5th-generation tensor-core (tcgen05) building blocks shared by the fused
// kernels of the warm-start network: shared-memory operand images, matrix and
// instruction descriptors, MMA issue and commit, bounded mbarrier waits, tensor-memory
// allocation and loads.  Inline PTX for sm_103a.
//
// Operand images.  Every BF16 operand tile in shared memory is kept in the canonical
// no-swizzle layout of core matrices: 8 rows of 16 bytes (8 consecutive elements along
// the "inner" dimension), each core matrix 128 contiguous bytes.  An image with INNER
// elements along the inner dimension places element (inner, outer) at
//     ((outer / 8) * (INNER / 8) + inner / 8) * 128 + (outer % 8) * 16 + (inner % 8) * 2,
// so core matrices adjacent along the inner dimension are 128 B apart and groups of 8
// outer rows INNER * 16 B apart.  The same bytes serve as a K-major operand (inner = K,
// outer = M or N) and as an MN-major operand (inner = M or N, outer = K); only the
// descriptor's strides (desc) and the major-ness bit of the instruction descriptor
// differ.  A tile stored with channels contiguous (pixels x
// channels) is therefore both "pixels x channels" for a contraction over channels and
// "channels x pixels" for a contraction over pixels, without any transposition.
#pragma once
#include <cstdint>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__host__ __device__ constexpr uint32_t img_off(int inner, int outer, int INNER) {
    return (uint32_t)((((outer >> 3) * (INNER >> 3) + (inner >> 3)) << 7) + ((outer & 7) << 4) + ((inner & 7) << 1));
}

// Matrix descriptor (no swizzle, version bit 46): start address, leading-dimension byte
// offset LBO and stride-dimension byte offset SBO.  Without swizzling, LBO is the stride
// between core matrices adjacent along K and SBO the stride between core matrices adjacent
// along M (N), for either major-ness.
__device__ __forceinline__ uint64_t desc_raw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Descriptor of an operand read from an image with INNER elements along the inner
// dimension, starting at byte saddr.  K-major (K along inner): K groups 128 B apart, M (N)
// groups INNER * 16 B apart; MN-major (M or N along inner): the reverse.
__device__ __forceinline__ uint64_t desc(uint32_t saddr, int INNER, bool mn) {
    const uint32_t inner_stride = 128, outer_stride = (uint32_t)INNER * 16;
    return mn ? desc_raw(saddr, outer_stride, inner_stride) : desc_raw(saddr, inner_stride, outer_stride);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, M x N, each operand
// K-major (false) or MN-major (true).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? (1u << 15) : 0u) | (b_mn ? (1u << 16) : 0u) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// An operand: image base (shared address), its INNER extent, whether the MMA reads it
// MN-major, and the offsets of the first row along M (N) and along K.
struct Opnd {
    uint32_t base;
    int inner, m0, k0;
    bool mn;
};

// Byte address of the 16-wide K step kk of operand o.
__device__ __forceinline__ uint32_t op_addr(const Opnd& o, int kk) {
    return o.mn ? o.base + img_off(o.m0, o.k0 + kk, o.inner) : o.base + img_off(o.k0 + kk, o.m0, o.inner);
}

// D[tmem] (+)= A B over K (a multiple of 16), M = 128, N given; issued by one thread.
// acc0 = 0 overwrites D with the first product.
__device__ __forceinline__ void mma(uint32_t tmem_d, const Opnd& a, const Opnd& b, int N, int K, bool acc0) {
    const uint32_t id = idesc_bf16(128, N, a.mn, b.mn);
    for (int kk = 0; kk < K; kk += 16) {
        const uint64_t ad = desc(op_addr(a, kk), a.inner, a.mn), bd = desc(op_addr(b, kk), b.inner, b.mn);
        const uint32_t acc = (acc0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// Bounded wait for phase `phase` of an mbarrier: false if `spin` rounds pass first.
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t phase, int spin) {
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

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory (st.shared, cp.async) made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor-memory allocation by one whole warp; the address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of the warp's 32 lanes (lane quadrant of warp % 4).
__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tensor-memory address of lane quadrant q (lanes 32 q ..), column col.
__device__ __forceinline__ uint32_t taddr(uint32_t tmem, int q, int col) {
    return tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col;
}

// 16-byte asynchronous global -> shared copy (L2 only) and its completion.
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace tc
