// md_neighbours_noalloc: the link-cell neighbour list for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's memory
// pool or allocator hooks, code that must not grow the device footprint after start-up,
// and code on paths where an allocation could block or fail at the wrong moment.  This
// entry point takes the caller's device arrays for input and output and keeps all of its
// own working memory in one file-scope __device__ array of fixed size, which every GPU that
// loads the library holds until the process exits.  It makes no cudaMalloc or cudaFree call
// and calls no allocating library routine.
//
// The scratch array is shared by every call: calls that overlap on the GPU (two streams, two
// host threads) race on it.  Each call first clears what must start at zero.
#include <cuda_runtime.h>

#include <mutex>

#include "md_internal.cuh"

namespace mdk {
namespace {

constexpr int kNaMaxAtoms = MD_NOALLOC_MAX_ATOMS;
constexpr int kNaMaxCells = MD_NOALLOC_MAX_CELLS;
constexpr int kNaScanThreads = 1024;

struct NoallocScratch {
    int32_t cell_count[kNaMaxCells];
    int32_t cell_start[kNaMaxCells + 8];
    int32_t cell_of[kNaMaxAtoms];
    int32_t slot[kNaMaxAtoms];
    int32_t order[kNaMaxAtoms];
    double spos[kNaMaxAtoms * 3];
    int32_t overflow;
    int32_t pad[63];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Link cells of width >= r_list along an edge of length L; kNaMaxCells + 1 stands for "more
// than the scratch holds" (L / r_list is range-checked before the integer conversion).
int na_cells_along(double L, double r_list) {
    const double q = floor(L / r_list);
    if (!(q <= (double)kNaMaxCells)) return kNaMaxCells + 1;
    int nc = (int)q;
    while (nc > 0 && L / nc < r_list * (1.0 + 1e-12)) nc--;
    return nc;
}

struct NaGeom {
    double L[3], invL[3];
    int nc[3];
    int ncell;
    double rl2;
};

__device__ __forceinline__ int na_cell_coord(double x, double invL, int nc) {
    double s = x * invL;
    s = s - floor(s);
    int c = (int)(s * (double)nc);
    return min(max(c, 0), nc - 1);
}

__device__ __forceinline__ double na_mi(double d, double L, double invL) {
    return __dsub_rn(d, __dmul_rn(L, rint(__dmul_rn(d, invL))));
}

__global__ void k_na_clear(NoallocScratch *S, int ncell) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
        S->cell_count[c] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) S->overflow = 0;
}

__global__ void k_na_bin(NoallocScratch *S, const double *__restrict__ pos, int n, NaGeom G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cx = na_cell_coord(pos[3 * i], G.invL[0], G.nc[0]);
    const int cy = na_cell_coord(pos[3 * i + 1], G.invL[1], G.nc[1]);
    const int cz = na_cell_coord(pos[3 * i + 2], G.invL[2], G.nc[2]);
    const int c = (cz * G.nc[1] + cy) * G.nc[0] + cx;
    S->cell_of[i] = c;
    S->slot[i] = atomicAdd(&S->cell_count[c], 1);
}

// Single-block exclusive scan of the cell counts (ncell <= kNaMaxCells).
__global__ void k_na_scan(NoallocScratch *S, int ncell) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += kNaScanThreads) {
        const int c = base + threadIdx.x;
        const int v = c < ncell ? S->cell_count[c] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (w > 0 ? warp_sums[w - 1] : 0) + x - v;
        if (c < ncell) S->cell_start[c] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) S->cell_start[ncell] = carry;
}

__global__ void k_na_scatter(NoallocScratch *S, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    S->order[S->cell_start[S->cell_of[i]] + S->slot[i]] = i;
}

// Ascending caller index inside each cell (independent of the counter order of k_na_bin),
// then the positions in cell order.  The coordinates are copied as the caller gave them,
// unwrapped: the exact test forms d = r_j - r_i from them and takes the minimum image of d,
// the operations md_build_neighbours applies to the same unwrapped coordinates, so both
// decide every pair alike.
__global__ void k_na_cell_sort(NoallocScratch *S, const double *__restrict__ pos, int ncell) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int s = S->cell_start[c], e = S->cell_start[c + 1];
    for (int a = s + 1; a < e; a++) {
        const int v = S->order[a];
        int b = a - 1;
        while (b >= s && S->order[b] > v) {
            S->order[b + 1] = S->order[b];
            b--;
        }
        S->order[b + 1] = v;
    }
    for (int a = s; a < e; a++) {
        const int i = S->order[a];
        S->spos[3 * a] = pos[3 * i];
        S->spos[3 * a + 1] = pos[3 * i + 1];
        S->spos[3 * a + 2] = pos[3 * i + 2];
    }
}

// One thread per atom in cell order; the exact FP64 test (the same IEEE operations as the
// library's list build); the output row of caller atom i lists caller ids, -1 after the end.
__global__ void k_na_list(NoallocScratch *S, int n, NaGeom G, int k_max, int32_t *count, int32_t *list) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const double px = S->spos[3 * a], py = S->spos[3 * a + 1], pz = S->spos[3 * a + 2];
    const int cx = na_cell_coord(px, G.invL[0], G.nc[0]);
    const int cy = na_cell_coord(py, G.invL[1], G.nc[1]);
    const int cz = na_cell_coord(pz, G.invL[2], G.nc[2]);
    const int self = S->order[a];
    int32_t *row = list + (size_t)self * k_max;
    int cnt = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int x = (cx + dx + G.nc[0]) % G.nc[0];
                const int y = (cy + dy + G.nc[1]) % G.nc[1];
                const int z = (cz + dz + G.nc[2]) % G.nc[2];
                const int c = (z * G.nc[1] + y) * G.nc[0] + x;
                for (int b = S->cell_start[c]; b < S->cell_start[c + 1]; b++) {
                    if (b == a) continue;
                    const double ex = na_mi(__dsub_rn(S->spos[3 * b], px), G.L[0], G.invL[0]);
                    const double ey = na_mi(__dsub_rn(S->spos[3 * b + 1], py), G.L[1], G.invL[1]);
                    const double ez = na_mi(__dsub_rn(S->spos[3 * b + 2], pz), G.L[2], G.invL[2]);
                    const double r2 =
                        __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    if (r2 < G.rl2) {
                        if (cnt < k_max) row[cnt] = S->order[b];
                        cnt++;
                    }
                }
            }
    for (int k = cnt; k < k_max; k++) row[k] = -1;
    count[self] = cnt;
    if (cnt > k_max) atomicOr(&S->overflow, 1);
}

// Device address of the scratch array, looked up once per device with that device current.
std::mutex g_na_mutex;
void *g_na_ptr[64] = {nullptr};

cudaError_t na_scratch(NoallocScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = static_cast<NoallocScratch *>(g_na_ptr[dev]);
    return cudaSuccess;
}

}  // namespace
}  // namespace mdk

extern "C" md_status md_neighbours_noalloc(const double *pos, int64_t n_atoms, const double *box,
                                           double r_list, int32_t k_max, int32_t *count, int32_t *list,
                                           void *stream) {
    using namespace mdk;
    if (n_atoms < 0 || !box || k_max < 1 || !(r_list > 0.0)) return MD_ERR_ARG;
    if (n_atoms > kNaMaxAtoms) return MD_ERR_CAPACITY;
    NaGeom G;
    long long ncell = 1;
    for (int k = 0; k < 3; k++) {
        if (!(box[k] > 0.0) || !(box[k] < INFINITY)) return MD_ERR_BOX;
        G.L[k] = box[k];
        G.invL[k] = 1.0 / box[k];
        G.nc[k] = na_cells_along(box[k], r_list);
        if (G.nc[k] < 3) return MD_ERR_BOX;
    }
    for (int k = 0; k < 3; k++) {
        // each factor is at most kNaMaxCells + 1, so the running product fits in 64 bits
        ncell *= G.nc[k];
        if (ncell > kNaMaxCells) return MD_ERR_CAPACITY;
    }
    G.ncell = (int)ncell;
    G.rl2 = r_list * r_list;
    if (n_atoms == 0) return MD_OK;
    if (!pos || !count || !list) return MD_ERR_ARG;
    NoallocScratch *S = nullptr;
    if (na_scratch(&S) != cudaSuccess) return MD_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // An error left on this thread by an earlier, unrelated call must not be taken for one of
    // these launches: clear it first (a sticky error shows again at the synchronisation below).
    (void)cudaGetLastError();
    const int n = (int)n_atoms;
    const int nb = (n + kThreads - 1) / kThreads;
    k_na_clear<<<(G.ncell + 255) / 256, 256, 0, s>>>(S, G.ncell);
    k_na_bin<<<nb, kThreads, 0, s>>>(S, pos, n, G);
    k_na_scan<<<1, kNaScanThreads, 0, s>>>(S, G.ncell);
    k_na_scatter<<<nb, kThreads, 0, s>>>(S, n);
    k_na_cell_sort<<<(G.ncell + kThreads - 1) / kThreads, kThreads, 0, s>>>(S, pos, G.ncell);
    k_na_list<<<nb, kThreads, 0, s>>>(S, n, G, k_max, count, list);
    if (cudaGetLastError() != cudaSuccess) return MD_ERR_CUDA;
    int32_t overflow = 0;
    if (cudaMemcpyAsync(&overflow, &S->overflow, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MD_ERR_CUDA;
    return overflow ? MD_ERR_NBR_OVERFLOW : MD_OK;
}
