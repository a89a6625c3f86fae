// tcgen05 BF16 GEMM (see tc_gemm.cuh).
#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace die {

namespace {

constexpr int kBM = 128, kBK = 64, kThreads = 128;
// Shared memory per operand region.  An operand tile takes R * 64 * 2 bytes (16 KB for
// R = 128); the region is sized so that the addresses the tensor cores may form from a
// descriptor of the tile stay inside it for every reading of its two offsets.
constexpr int kRegion = 48 * 1024;
constexpr long kWaitLimit = 1L << 26;    // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address, leading-
// dimension byte offset (core matrices adjacent in K), stride byte offset (8-row groups
// adjacent in M or N), all in 16-byte units; bits 46-47 hold the descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase `parity` of the barrier to complete; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long i = 0; i < kWaitLimit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 16 consecutive accumulator columns of this thread's TMEM lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Copy rows [r0, r0 + R) x k [k0, k0 + 64) of X(r, k) = X[r * sr + k * sk] into the
// canonical layout at `tile` as BF16, zeros outside [0, rows) x [0, K).  Element (r, k)
// of the tile goes to byte (k / 8) (R 16) + (r / 8) 128 + (r % 8) 16 + (k % 8) 2.  The
// loop runs along whichever index has unit stride, so global reads are coalesced.
template <int R>
__device__ __forceinline__ void stage_tile(unsigned char* tile, const float* __restrict__ X, long sr, long sk,
                                           int r0, int k0, int rows, int K) {
    const bool k_inner = sk == 1 || sr != 1;
    for (int e = threadIdx.x; e < R * kBK; e += kThreads) {
        const int r = k_inner ? e / kBK : e % R;
        const int k = k_inner ? e % kBK : e / R;
        const int gr = r0 + r, gk = k0 + k;
        const float v = (gr < rows && gk < K) ? X[(long)gr * sr + (long)gk * sk] : 0.f;
        const uint32_t off = (uint32_t)((k >> 3) * (R * 16) + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
        *reinterpret_cast<__nv_bfloat16*>(tile + off) = __float2bfloat16_rn(v);
    }
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + kRegion;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kRegion);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kRegion + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN, b = blockIdx.z;
    const float* A = g.A + (long)b * g.sab;
    const float* B = g.B + (long)b * g.sbb;
    float* C = g.C + (long)b * g.scb;
    const uint32_t bar_a = smem_u32(bar);
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), BN);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) mbar_init(bar_a, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < g.K; k0 += kBK) {
        stage_tile<kBM>(sA, A, g.sam, g.sak, m0, k0, g.M, g.K);
        stage_tile<BN>(sB, B, g.sbn, g.sbk, n0, k0, g.N, g.K);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int i = 0; i < kBK / 16; i++) {
                const uint64_t ad = smem_desc(a0 + i * 2 * kBM * 16, kBM * 16, 128);
                const uint64_t bd = smem_desc(b0 + i * 2 * BN * 16, BN * 16, 128);
                mma_bf16(tmem, ad, bd, idesc, (k0 > 0 || i > 0) ? 1u : 0u);
            }
            mma_commit(bar_a);
        }
        ok = mbar_wait(bar_a, phase) && ok;   // the tiles are read by the tensor cores until then
        phase ^= 1;
        if (!ok) break;
        __syncthreads();
    }
    tc_fence_after();
    if (!ok) {
        if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
        mbar_wait(bar_a, phase ^ 1);       // one more bounded wait for the MMAs in flight
    } else {
        const int m = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            if (g.K > 0) {
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int i = 0; i < 16; i++) v[i] = 0.f;
            }
            if (m < g.M) {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int n = n0 + c0 + i;
                    if (n < g.N) {
                        float* cp = C + (long)m * g.scm + (long)n * g.scn;
                        float out = g.alpha * v[i];
                        if (g.bias) out += g.bias[n];
                        if (g.beta != 0.f) out += g.beta * *cp;
                        *cp = out;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

}  // namespace

die_status tc_gemm(const GemmArgs& g, cudaStream_t st) {
    if (g.M < 0 || g.N < 0 || g.K < 0 || g.batch < 1 || g.batch > 65535) return DIE_EINVAL;
    if (g.M == 0 || g.N == 0) return DIE_OK;
    if (!g.A || !g.B || !g.C) return DIE_EINVAL;
    const size_t smem = 2 * kRegion + 16;
    const dim3 block(kThreads);
    // the shared-memory limit is raised on every call (a host-side attribute, cheap, and
    // correct on whichever device is current)
    if (g.N <= 64) {
        DIE_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const dim3 grid((g.M + kBM - 1) / kBM, (g.N + 63) / 64, g.batch);
        tc_gemm_kernel<64><<<grid, block, smem, st>>>(g);
    } else {
        DIE_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const dim3 grid((g.M + kBM - 1) / kBM, (g.N + 127) / 128, g.batch);
        tc_gemm_kernel<128><<<grid, block, smem, st>>>(g);
    }
    DIE_LAUNCH_CHECK();
    return DIE_OK;
}

}  // namespace die
