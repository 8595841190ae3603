// FP32 network of the learned per-atom surrogate on tiles of 64 atoms (CUDA cores), its
// training pass, the Adam update and the bf16 operand image of the tensor-core network.
//
// Network (one atom; x = standardised descriptors, s = SiLU, s(z) = z sigmoid(z)):
//   z1 = W1 x + b1, a1 = s(z1);  z2 = W2 a1 + b2, a2 = s(z2);  E = w3 . a2 + b3.
// Input gradient (the forces need dE/dG = dE/dx * ginv):
//   d2 = w3 s'(z2);  d1 = (W2^T d2) s'(z1);  dE/dx = W1^T d1.
// Training pass.  Each atom contributes the parameter gradient of J = c E - (tangent of E along
// v), where c = dL/dE_i of its replica and v = the standardised tangent u_i of its descriptors
// (the force term of the loss, see k_sur_u).  Forward with tangents:
//   t1 = W1 v, ta1 = s'(z1) t1;  t2 = W2 ta1, ta2 = s'(z2) t2;  tangent of E = w3 . ta2,
// then reverse through both:
//   gw3 += c a2 - ta2,  gb3 += c,
//   bz2 = w3 (c s'(z2) - s''(z2) t2),  btz2 = -w3 s'(z2),  gW2 += bz2 a1^T + btz2 ta1^T,  gb2 += bz2,
//   ba1 = W2^T bz2, bta1 = W2^T btz2,  bz1 = ba1 s'(z1) + bta1 s''(z1) t1,  btz1 = bta1 s'(z1),
//   gW1 += bz1 x^T + btz1 v^T,  gb1 += bz1.
// Over a tile the per-atom products are small matrix products, done in shared memory with 4x4
// register blocks per thread.  Each block sums its tiles' gradients in shared memory and writes
// one row of per-block partials; the update kernel adds the rows in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

constexpr int BM = 64;    // atoms per tile
constexpr int NT = 256;   // threads per block
constexpr int H1 = kSurH1, H2 = kSurH2, NB = kSurNb;
// parameter offsets in theta
constexpr int oW1 = 0, oB1 = H1 * NB, oW2 = oB1 + H1, oB2 = oW2 + H2 * H1, oW3 = oB2 + H2, oB3 = oW3 + H2;

struct Smem {
    float W1[H1 * NB];    // [p][k]
    float W1T[NB * H1];   // [k][p]
    float W2[H2 * H1];    // [q][p]
    float W2T[H1 * H2];   // [p][q]
    float b1[H1], b2[H2], w3[H2], gmu[NB], ginv[NB];
    float b3, pad[3];
    float X[BM * NB], V[BM * NB];
    float Z1[BM * H1], T1[BM * H1], A1[BM * H1], TA1[BM * H1], Z2[BM * H2], T2[BM * H2];
    float c[BM];
    float red[4][H1];
    float gacc[kSurParams + 3];
};

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + __expf(-z)); }

// C[M][N] (row stride ldc) = [C +] sum_k A(m,k) B(k,n); A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];
// B(k,n) = B[k*ldb + n].  4x4 outputs per thread; all threads of the block take part.
template <int M, int N, int K, bool TA, bool ACC>
__device__ __forceinline__ void mm(float *C, int ldc, const float *A, int lda, const float *B, int ldb) {
    constexpr int TN = N / 4, TILES = (M / 4) * TN;
    for (int t = threadIdx.x; t < TILES; t += NT) {
        const int m0 = (t / TN) * 4, n0 = (t % TN) * 4;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[r][q] = 0.f;
#pragma unroll 4
        for (int k = 0; k < K; k++) {
            const float4 b = *reinterpret_cast<const float4 *>(B + k * ldb + n0);
            float a[4];
            if (TA) {
                const float4 av = *reinterpret_cast<const float4 *>(A + k * lda + m0);
                a[0] = av.x; a[1] = av.y; a[2] = av.z; a[3] = av.w;
            } else {
#pragma unroll
                for (int r = 0; r < 4; r++) a[r] = A[(m0 + r) * lda + k];
            }
#pragma unroll
            for (int r = 0; r < 4; r++) {
                acc[r][0] = fmaf(a[r], b.x, acc[r][0]);
                acc[r][1] = fmaf(a[r], b.y, acc[r][1]);
                acc[r][2] = fmaf(a[r], b.z, acc[r][2]);
                acc[r][3] = fmaf(a[r], b.w, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            float4 *o = reinterpret_cast<float4 *>(C + (m0 + r) * ldc + n0);
            float4 v = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            if (ACC) {
                const float4 p = *o;
                v.x += p.x; v.y += p.y; v.z += p.z; v.w += p.w;
            }
            *o = v;
        }
    }
}

// Column sums of per-thread partials: thread t holds column t % 64 of rows t/64, t/64 + 4, ...;
// the 4 partials of a column are added in a fixed order into dst[col].
__device__ __forceinline__ void col_reduce(Smem &sm, float part, float *dst) {
    sm.red[threadIdx.x / H1][threadIdx.x % H1] = part;
    __syncthreads();
    if (threadIdx.x < H1)
        dst[threadIdx.x] += (sm.red[0][threadIdx.x] + sm.red[1][threadIdx.x]) +
                            (sm.red[2][threadIdx.x] + sm.red[3][threadIdx.x]);
    __syncthreads();
}

__device__ void load_weights(Smem &sm, const SurNet &S) {
    const float *th = S.theta;
    for (int e = threadIdx.x; e < H1 * NB; e += NT) {
        const int p = e / NB, k = e % NB;
        sm.W1[e] = th[oW1 + e];
        sm.W1T[k * H1 + p] = th[oW1 + e];
    }
    for (int e = threadIdx.x; e < H2 * H1; e += NT) {
        const int q = e / H1, p = e % H1;
        sm.W2[e] = th[oW2 + e];
        sm.W2T[p * H2 + q] = th[oW2 + e];
    }
    if (threadIdx.x < H1) {
        sm.b1[threadIdx.x] = th[oB1 + threadIdx.x];
        sm.b2[threadIdx.x] = th[oB2 + threadIdx.x];
        sm.w3[threadIdx.x] = th[oW3 + threadIdx.x];
    }
    if (threadIdx.x < NB) {
        sm.gmu[threadIdx.x] = S.gmu[threadIdx.x];
        sm.ginv[threadIdx.x] = S.ginv[threadIdx.x];
    }
    if (threadIdx.x == 0) sm.b3 = th[oB3];
}

// MODE 0: E_i -> A.e_atom, dE/dG -> S.g.  MODE 1: parameter-gradient partials -> S.gpart.
template <int MODE>
__global__ void __launch_bounds__(NT, 1) k_sur_net32(Atoms A, SurNet S, int a0, int a1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    load_weights(sm, S);
    if (MODE == 1)
        for (int e = threadIdx.x; e < kSurParams; e += NT) sm.gacc[e] = 0.f;
    __syncthreads();
    const int ntiles = (a1 - a0 + BM - 1) / BM;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int t0 = a0 + tile * BM;
        // inputs: standardised descriptors (and tangents, replica energy weights)
        for (int e = threadIdx.x; e < BM * NB; e += NT) {
            const int a = t0 + e / NB, k = e % NB;
            const bool live = a < a1;
            sm.X[e] = live ? (S.G[(size_t)a * NB + k] - sm.gmu[k]) * sm.ginv[k] : 0.f;
            if (MODE == 1) sm.V[e] = live ? S.u[(size_t)a * NB + k] : 0.f;
        }
        if (MODE == 1 && threadIdx.x < BM) {
            const int a = t0 + threadIdx.x;
            sm.c[threadIdx.x] = a < a1 ? (float)S.ce[2 * (A.rep ? A.rep[a] : 0)] : 0.f;
        }
        __syncthreads();
        mm<BM, H1, NB, false, false>(sm.Z1, H1, sm.X, NB, sm.W1T, H1);
        if (MODE == 1) mm<BM, H1, NB, false, false>(sm.T1, H1, sm.V, NB, sm.W1T, H1);
        __syncthreads();
        for (int e = threadIdx.x; e < BM * H1; e += NT) {
            const float z = sm.Z1[e] + sm.b1[e % H1];
            const float sg = sigm(z);
            sm.Z1[e] = z;
            sm.A1[e] = z * sg;
            if (MODE == 1) sm.TA1[e] = sg * fmaf(z, 1.f - sg, 1.f) * sm.T1[e];
        }
        __syncthreads();
        mm<BM, H2, H1, false, false>(sm.Z2, H2, sm.A1, H1, sm.W2T, H2);
        if (MODE == 1) mm<BM, H2, H1, false, false>(sm.T2, H2, sm.TA1, H1, sm.W2T, H2);
        __syncthreads();
        if (MODE == 0) {
            // E per atom (4 threads per atom, 16 columns each) and d2 = w3 s'(z2) into Z2
            const int a = threadIdx.x >> 2, part = threadIdx.x & 3;
            float e = 0.f;
            for (int q = part * 16; q < part * 16 + 16; q++) {
                const float z = sm.Z2[a * H2 + q] + sm.b2[q];
                const float sg = sigm(z);
                e = fmaf(sm.w3[q], z * sg, e);
                sm.Z2[a * H2 + q] = sm.w3[q] * sg * fmaf(z, 1.f - sg, 1.f);
            }
            e += __shfl_xor_sync(0xffffffffu, e, 1);
            e += __shfl_xor_sync(0xffffffffu, e, 2);
            if (part == 0 && t0 + a < a1) A.e_atom[t0 + a] = (double)(e + sm.b3);
            __syncthreads();
            mm<BM, H1, H2, false, false>(sm.A1, H1, sm.Z2, H2, sm.W2, H1);   // W2^T d2
            __syncthreads();
            for (int e2 = threadIdx.x; e2 < BM * H1; e2 += NT) {
                const float z = sm.Z1[e2], sg = sigm(z);
                sm.A1[e2] *= sg * fmaf(z, 1.f - sg, 1.f);
            }
            __syncthreads();
            mm<BM, NB, H1, false, false>(sm.X, NB, sm.A1, H1, sm.W1, NB);    // W1^T d1
            __syncthreads();
            for (int e2 = threadIdx.x; e2 < BM * NB; e2 += NT) {
                const int a2 = t0 + e2 / NB, k = e2 % NB;
                if (a2 < a1) S.g[(size_t)a2 * NB + k] = sm.X[e2] * sm.ginv[k];
            }
            __syncthreads();
        } else {
            // elementwise backward through layer 2 (thread t: column t % 64)
            float pw3 = 0.f, pb2 = 0.f;
            for (int e = threadIdx.x; e < BM * H2; e += NT) {
                const int a = e / H2, q = e % H2;
                const float z = sm.Z2[e] + sm.b2[q];
                const float sg = sigm(z);
                const float ds = sg * fmaf(z, 1.f - sg, 1.f);
                const float dds = sg * (1.f - sg) * fmaf(z, 1.f - 2.f * sg, 2.f);
                const float t2 = sm.T2[e];
                const float c = sm.c[a];
                pw3 += c * (z * sg) - ds * t2;
                const float bz2 = sm.w3[q] * (c * ds - dds * t2);
                pb2 += bz2;
                sm.Z2[e] = bz2;
                sm.T2[e] = -sm.w3[q] * ds;
            }
            col_reduce(sm, pw3, sm.gacc + oW3);
            col_reduce(sm, pb2, sm.gacc + oB2);
            if (threadIdx.x == 0) {
                float s = 0.f;
                for (int a = 0; a < BM; a++) s += sm.c[a];
                sm.gacc[oB3] += s;
            }
            // gW2 += bz2^T a1 + btz2^T ta1
            mm<H2, H1, BM, true, true>(sm.gacc + oW2, H1, sm.Z2, H2, sm.A1, H1);
            __syncthreads();
            mm<H2, H1, BM, true, true>(sm.gacc + oW2, H1, sm.T2, H2, sm.TA1, H1);
            __syncthreads();
            // ba1 = W2^T bz2 -> A1, bta1 = W2^T btz2 -> TA1
            mm<BM, H1, H2, false, false>(sm.A1, H1, sm.Z2, H2, sm.W2, H1);
            mm<BM, H1, H2, false, false>(sm.TA1, H1, sm.T2, H2, sm.W2, H1);
            __syncthreads();
            float pb1 = 0.f;
            for (int e = threadIdx.x; e < BM * H1; e += NT) {
                const float z = sm.Z1[e], sg = sigm(z);
                const float ds = sg * fmaf(z, 1.f - sg, 1.f);
                const float dds = sg * (1.f - sg) * fmaf(z, 1.f - 2.f * sg, 2.f);
                const float ba = sm.A1[e], bta = sm.TA1[e];
                const float bz1 = fmaf(ba, ds, bta * dds * sm.T1[e]);
                pb1 += bz1;
                sm.A1[e] = bz1;
                sm.TA1[e] = bta * ds;
            }
            col_reduce(sm, pb1, sm.gacc + oB1);
            // gW1 += bz1^T x + btz1^T v
            mm<H1, NB, BM, true, true>(sm.gacc + oW1, NB, sm.A1, H1, sm.X, NB);
            __syncthreads();
            mm<H1, NB, BM, true, true>(sm.gacc + oW1, NB, sm.TA1, H1, sm.V, NB);
            __syncthreads();
        }
    }
    if (MODE == 1) {
        __syncthreads();
        for (int e = threadIdx.x; e < kSurParams; e += NT) S.gpart[(size_t)blockIdx.x * kSurParams + e] = sm.gacc[e];
    }
}

// Sum of the per-block gradient rows (fixed order), then one Adam step (Kingma & Ba) on theta.
// lr <= 0: only the summed gradient is written (grad_out).
__global__ void k_sur_update(const float *gpart, int blocks, float *theta, float *m, float *v, float *grad_out,
                             int t, float lr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kSurParams) return;
    float g = 0.f;
    for (int b = 0; b < blocks; b++) g += gpart[(size_t)b * kSurParams + p];
    if (grad_out) grad_out[p] = g;
    if (!(lr > 0.f)) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mm_ = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm_;
    v[p] = vv;
    const float mh = mm_ / (1.f - powf(b1, (float)t));
    const float vh = vv / (1.f - powf(b2, (float)t));
    theta[p] -= lr * mh / (sqrtf(vh) + eps);
}

// bf16 operand image (see kSurImg*): matrix N x K, element (n, k) at
// (n/8) * (K/8 * 128) + (k/8) * 128 + (n%8) * 16 + (k%8) * 2 bytes.
__device__ __forceinline__ void put(unsigned char *img, int base, int K, int n, int k, float x) {
    const int off = base + (n >> 3) * (K / 8 * 128) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16 *>(img + off) = __float2bfloat16_rn(x);
}

__global__ void k_sur_pack(const float *theta, unsigned char *img) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < H1 * NB) {
        const int p = e / NB, k = e % NB;
        put(img, kSurImgW1, NB, p, k, theta[oW1 + e]);    // W1: N = p, K = k
        put(img, kSurImgW1T, H1, k, p, theta[oW1 + e]);   // W1^T: N = k, K = p
    }
    if (e < H2 * H1) {
        const int q = e / H1, p = e % H1;
        put(img, kSurImgW2, H1, q, p, theta[oW2 + e]);    // W2: N = q, K = p
        put(img, kSurImgW2T, H2, p, q, theta[oW2 + e]);   // W2^T: N = p, K = q
    }
}

template <int MODE>
cudaError_t net32(const Atoms &A, const SurNet &S, int a0, int a1, int blocks, cudaStream_t s) {
    const size_t bytes = sizeof(Smem);
    static bool attr = false;   // one-time opt-in to the large shared-memory carve-out
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sur_net32<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_sur_net32<MODE><<<blocks, NT, bytes, s>>>(A, S, a0, a1);
    return cudaGetLastError();
}

int n_sm() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
    }
    return v;
}

}  // namespace

int sur_net32_blocks(int n_atoms) {
    const int tiles = (n_atoms + BM - 1) / BM;
    return std::max(1, std::min(tiles, n_sm()));
}

cudaError_t launch_sur_net32(const Atoms &A, const SurNet &S, int a0, int a1, cudaStream_t s) {
    if (a1 <= a0) return cudaSuccess;
    return net32<0>(A, S, a0, a1, sur_net32_blocks(a1 - a0), s);
}

cudaError_t launch_sur_train_tiles(const Atoms &A, const SurNet &S, int a0, int a1, int *blocks_out,
                                   cudaStream_t s) {
    const int blocks = sur_net32_blocks(std::max(a1 - a0, 1));
    *blocks_out = blocks;
    if (a1 <= a0) return cudaSuccess;
    return net32<1>(A, S, a0, a1, blocks, s);
}

cudaError_t launch_sur_update(const SurNet &S, float *theta, float *adam_m, float *adam_v, float *grad_out,
                              int blocks, int t, float lr, cudaStream_t s) {
    k_sur_update<<<blocks_for(kSurParams, 256), 256, 0, s>>>(S.gpart, blocks, theta, adam_m, adam_v, grad_out, t, lr);
    return cudaGetLastError();
}

cudaError_t launch_sur_pack(const float *theta, unsigned char *img, cudaStream_t s) {
    k_sur_pack<<<blocks_for(H2 * H1, 256), 256, 0, s>>>(theta, img);
    return cudaGetLastError();
}

}  // namespace mdk
