// Tensor-core (tcgen05) network of the learned per-atom surrogate: energy and input gradient
// of 128-atom tiles with BF16 operands and FP32 accumulation in tensor memory.
//
// Per tile (x: 128 x 32 standardised descriptors, bf16, written by the descriptor kernel in the
// layout below and brought in by one bulk TMA copy), four MMAs of M = 128 rows, one per layer,
// each followed by an epilogue in which the two warpgroups of the CTA each take half of the
// accumulator's columns: thread t of a warpgroup reads row t from TMEM (tcgen05.ld 32x32b),
// applies bias and SiLU in FP32 and writes the next operand to shared memory as bf16:
//   D0 [TMEM cols 0..63]   = x  W1^T           z1 = D0 + b1,  a1 = s(z1)            -> act
//   D1 [cols 64..127]      = a1 W2^T           z2 = D1 + b2,  E = w3 . s(z2) + b3,
//                                              d2 = w3 s'(z2)                       -> act
//   D1 [cols 64..127]      = d2 W2             d1 = D1 s'(z1)  (z1 from D0)          -> act
//   D0 [cols 0..31]        = d1 W1             dE/dG = D0 * ginv                    -> global
// Shared-memory operands use the no-swizzle K-major core-matrix layout: 8 rows x 16 bytes per
// core matrix (128 contiguous bytes), core matrices adjacent along K 128 bytes apart (leading
// byte offset), 8-row groups K/8 * 128 bytes apart (stride byte offset).  One thread issues the
// MMAs and commits them to an mbarrier; every wait on it is bounded and ends the kernel with
// FLAG_TIMEOUT (TMEM freed) if the MMAs do not complete.  The sigmoid of SiLU is taken as
// (1 + tanh(z/2)) / 2 with the hardware tanh (tanh.approx.f32, relative error ~2^-11, below the
// bf16 rounding of the activations).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

constexpr int kTcThreads = 256;   // two warpgroups
constexpr int kTmemCols = 128;
constexpr unsigned kWaitPolls = 4000000u;   // x >= 32 ns each: > 0.1 s before giving up
// shared memory layout (bytes)
constexpr int kSmImg = 0;                       // weights image, kSurImgBytes
constexpr int kSmG = kSmImg + kSurImgBytes;     // x tile, kSurTileBytes
constexpr int kSmAct = kSmG + kSurTileBytes;    // 128 x 64 bf16 activations (16 KB)
constexpr int kSmPar = kSmAct + 16384;          // b1, b2, w3, ginv (64+64+64+32 floats), b3
constexpr int kSmE = kSmPar + 1024;             // energy partials of warpgroup 1 (128 floats)
constexpr int kSmBar = kSmE + 512;              // MMA mbarrier, TMA mbarrier (8 B each), TMEM address
constexpr int kSmBytes = kSmBar + 32;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 in bits 0-13, leading byte offset >> 4 in 16-29,
// stride byte offset >> 4 in 32-45, descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B bf16 (bits 7-9
// and 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_smem_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk (untiled) TMA copy global -> shared, completion counted on the mbarrier.  Both addresses
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (unsigned it = 0; it < kWaitPolls; ++it) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (load and wait in one statement, so
// that no use of the registers can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Row `row` of a 128 x 64 bf16 K-major operand: 16 columns c0..c0+15 -> two core-matrix rows.
__device__ __forceinline__ void put_row16(unsigned char *act, int row, int c0, const float (&v)[16]) {
    unsigned char *base = act + (row >> 3) * 1024 + (c0 >> 3) * 128 + (row & 7) * 16;
    *reinterpret_cast<uint4 *>(base) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    *reinterpret_cast<uint4 *>(base + 128) = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]),
                                                        pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
}

__device__ __forceinline__ float sigm(float z) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    return fmaf(0.5f, t, 0.5f);
}

__global__ void __launch_bounds__(kTcThreads, 4) k_sur_net_tc(Atoms A, SurNet S, int ntiles) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *img = sm + kSmImg, *gt = sm + kSmG, *act = sm + kSmAct;
    float *b1 = reinterpret_cast<float *>(sm + kSmPar), *b2 = b1 + 64, *w3 = b2 + 64, *ginv = w3 + 64, *b3 = ginv + 32;
    float *epart = reinterpret_cast<float *>(sm + kSmE);
    uint64_t *bar_p = reinterpret_cast<uint64_t *>(sm + kSmBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kSmBar + 16);
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid >> 7, row = tid & 127;
    const uint32_t bar = smem_addr(bar_p), bar_g = smem_addr(bar_p + 1);

    // weights (bf16 image) and FP32 biases
    for (int q = tid; q < kSurImgBytes / 16; q += kTcThreads)
        reinterpret_cast<uint4 *>(img)[q] = reinterpret_cast<const uint4 *>(S.img)[q];
    const float *th = S.theta;
    if (tid < 64) {
        b1[tid] = th[kSurH1 * kSurNb + tid];
        b2[tid] = th[kSurH1 * kSurNb + kSurH1 + kSurH2 * kSurH1 + tid];
        w3[tid] = th[kSurH1 * kSurNb + kSurH1 + kSurH2 * kSurH1 + kSurH2 + tid];
    }
    if (tid < 32) ginv[tid] = S.ginv[tid];
    if (tid == 0) {
        *b3 = th[kSurParams - 1];
        mbar_init(bar, 1);
        mbar_init(bar_g, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    async_smem_fence();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;   // this warp's 32 TMEM lanes
    const uint32_t a_g = smem_addr(gt), a_act = smem_addr(act), a_img = smem_addr(img);
    const int cA = 32 * grp;   // this warpgroup's columns of a 64-column accumulator
    const int cB = 16 * grp;   // ... and of the 32-column input gradient
    uint32_t phase = 0, phase_g = 0;
    bool ok = true;

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int atom = tile * kSurTile + row;
        const bool live = atom < A.n;
        if (tid == 0) {
            mbar_expect_tx(bar_g, kSurTileBytes);
            bulk_g2s(a_g, S.Gt + (size_t)tile * kSurTileBytes, kSurTileBytes, bar_g);
        }
        ok = __syncthreads_and(mbar_wait(bar_g, phase_g));
        phase_g ^= 1;
        if (!ok) break;
        // layer 1: D0 = x W1^T  (K = 32: 2 MMAs of K = 16)
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < 2; ks++)
                mma_bf16(tmem, sdesc(a_g + ks * 256, 128, 512), sdesc(a_img + kSurImgW1 + ks * 256, 128, 512),
                         idesc_bf16(128, 64), ks > 0);
            mma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_after();
        // epilogue 1: a1 = s(D0 + b1)
#pragma unroll
        for (int c0 = cA; c0 < cA + 32; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_off + c0, v);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const float z = v[i] + b1[c0 + i];
                v[i] = z * sigm(z);
            }
            put_row16(act, row, c0, v);
        }
        async_smem_fence();
        tc_before();
        __syncthreads();
        // layer 2: D1 = a1 W2^T  (K = 64)
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                mma_bf16(tmem + 64, sdesc(a_act + ks * 256, 128, 1024), sdesc(a_img + kSurImgW2 + ks * 256, 128, 1024),
                         idesc_bf16(128, 64), ks > 0);
            mma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_after();
        // epilogue 2: E and d2 = w3 s'(z2)
        float e = 0.f;
#pragma unroll
        for (int c0 = cA; c0 < cA + 32; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_off + 64 + c0, v);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const float z = v[i] + b2[c0 + i];
                const float sg = sigm(z);
                e = fmaf(w3[c0 + i], z * sg, e);
                v[i] = w3[c0 + i] * sg * fmaf(z, 1.f - sg, 1.f);
            }
            put_row16(act, row, c0, v);
        }
        if (grp == 1) epart[row] = e;
        async_smem_fence();
        tc_before();
        __syncthreads();
        // backward 2: D1 = d2 W2  (B = W2^T image: N = p, K = q)
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                mma_bf16(tmem + 64, sdesc(a_act + ks * 256, 128, 1024),
                         sdesc(a_img + kSurImgW2T + ks * 256, 128, 1024), idesc_bf16(128, 64), ks > 0);
            mma_commit(bar);
        }
        if (grp == 0 && live) A.e_atom[atom] = (double)(e + epart[row] + *b3);
        ok = __syncthreads_and(mbar_wait(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_after();
        // epilogue 3: d1 = D1 s'(z1), z1 = D0 + b1
#pragma unroll
        for (int c0 = cA; c0 < cA + 32; c0 += 16) {
            float v[16], z1[16];
            tmem_ld16(tmem + lane_off + 64 + c0, v);
            tmem_ld16(tmem + lane_off + c0, z1);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const float z = z1[i] + b1[c0 + i];
                const float sg = sigm(z);
                v[i] *= sg * fmaf(z, 1.f - sg, 1.f);
            }
            put_row16(act, row, c0, v);
        }
        async_smem_fence();
        tc_before();
        __syncthreads();
        // backward 1: D0[0..31] = d1 W1  (B = W1^T image: N = 32 (k), K = 64 (p))
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < 4; ks++)
                mma_bf16(tmem, sdesc(a_act + ks * 256, 128, 1024), sdesc(a_img + kSurImgW1T + ks * 256, 128, 1024),
                         idesc_bf16(128, 32), ks > 0);
            mma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, phase));
        phase ^= 1;
        if (!ok) break;
        tc_after();
        // epilogue 4: dE/dG = D0 * ginv (16 columns per warpgroup)
        {
            float v[16];
            tmem_ld16(tmem + lane_off + cB, v);
            if (live) {
                float4 *dst = reinterpret_cast<float4 *>(S.g + (size_t)atom * kSurNb + cB);
#pragma unroll
                for (int q = 0; q < 4; q++)
                    dst[q] = make_float4(v[4 * q] * ginv[cB + 4 * q], v[4 * q + 1] * ginv[cB + 4 * q + 1],
                                         v[4 * q + 2] * ginv[cB + 4 * q + 2], v[4 * q + 3] * ginv[cB + 4 * q + 3]);
            }
        }
        tc_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(&A.flags->error, FLAG_TIMEOUT);
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

int tc_blocks(int ntiles) {
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    return std::max(1, std::min(ntiles, 4 * n_sm));   // 4 x 128 TMEM columns per SM
}

}  // namespace

cudaError_t launch_sur_net_tc(const Atoms &A, const SurNet &S, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sur_net_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = (A.n + kSurTile - 1) / kSurTile;
    k_sur_net_tc<<<tc_blocks(ntiles), kTcThreads, kSmBytes, s>>>(A, S, ntiles);
    return cudaGetLastError();
}

}  // namespace mdk
