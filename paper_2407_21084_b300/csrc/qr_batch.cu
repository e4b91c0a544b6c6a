// qr_batch.cu -- many QRMC problem instances of uneven d, |Gamma|, N and M
// advanced by one Picard iteration together.
//
// The path-and-series phase of all instances is ONE persistent kernel: every
// CTA takes work items (instance, time index i, run of path tiles) from a
// global counter. Items are ordered class by class (the class with the most
// work first) and longest first (work ~ N - i) within a class, so that the
// CTAs running at any time mostly execute the same body (shared instruction
// caches) and the short rows fill each class's tail. Each item runs the
// compile-time chain-tree body of its instance's index-set class (a switch
// over the compiled classes; the class is uniform per item). Coefficient
// rows are staged in a double buffer sized for the largest row; mbarrier
// phases carry over from item to item.
//
// Projection and reduction reuse the single-instance kernels, one launch per
// instance, and the whole iteration (counter resets, the persistent kernel,
// the projections and reductions) is captured in one CUDA graph. The items
// per claim (tiles per item) and the grid of the persistent kernel are chosen
// by timing candidates on the first iteration (autotuner).
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "qr_batch.h"
#include "qr_tree.cuh"

namespace qr {

// compiled index-set classes of the engine: (class id, kind, d, n)
#define QR_BATCH_CLASSES(X) \
    X(0, QR_G_LINF, 2, 4)   \
    X(1, QR_G_L1, 3, 5)     \
    X(2, QR_G_L1, 4, 4)     \
    X(3, QR_G_L1, 5, 4)     \
    X(4, QR_G_L1, 6, 3)     \
    X(5, QR_G_L1, 6, 4)     \
    X(6, QR_G_L1, 7, 3)     \
    X(7, QR_G_L1, 8, 3)

int batch_class(int kind, int d, int n)
{
#define QR_X(C, K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return C;
    QR_BATCH_CLASSES(QR_X)
#undef QR_X
    return -1;
}

constexpr int kBatchBS = 128, kBatchP = 2;

// resident CTAs per SM the register allocation is held to (3: 168 registers,
// a few hundred bytes of spills, still 17% faster than 255 registers at 2 CTAs)
#ifndef QR_BATCH_MINB
#define QR_BATCH_MINB 3
#endif

__global__ void __launch_bounds__(kBatchBS, QR_BATCH_MINB) k_paths_batch(const BatchInst* __restrict__ inst,
                                                          const BatchItem* __restrict__ items, int n_items,
                                                          unsigned* __restrict__ next_item, uint32_t max_rowbytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2* const abuf[2] = {reinterpret_cast<float2*>(smem), reinterpret_cast<float2*>(smem + max_rowbytes)};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * (size_t)max_rowbytes);
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) return;
        const BatchItem item = items[it];
        const BatchInst& I = inst[item.inst];
        const float2* tree = static_cast<const float2*>(I.tree);
        float* S = static_cast<float*>(I.S);
        for (int t = 0; t < item.ntiles; ++t) {
            const long long m0 = (long long)(item.tile0 + t) * (kBatchBS * kBatchP) + threadIdx.x;
            bool ok = true;
            switch (I.cls) {
#define QR_X(C, K, DD, NNN)                                                                                     \
    case C:                                                                                                     \
        ok = path_item<float, DD, NNN, K, kBatchP, kBatchBS>(I.P, tree, I.tree_stride, S, item.i, 0, m0, abuf, \
                                                               bars, phase, I.counters, I.status);             \
        break;
                QR_BATCH_CLASSES(QR_X)
#undef QR_X
            default:
                break;
            }
            if (!ok) return;
        }
    }
}

size_t batch_smem(size_t max_rowbytes) { return 2 * max_rowbytes + 16; }

cudaError_t launch_paths_batch(const BatchInst* inst, const BatchItem* items, int n_items, unsigned* next_item,
                               size_t max_rowbytes, int grid, cudaStream_t st)
{
    const size_t sm = batch_smem(max_rowbytes);
    if (sm > 227 * 1024 || max_rowbytes % 16) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_paths_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    k_paths_batch<<<grid, kBatchBS, sm, st>>>(inst, items, n_items, next_item, (uint32_t)max_rowbytes);
    return cudaGetLastError();
}

int batch_blocks_per_sm(size_t max_rowbytes)
{
    const size_t sm = batch_smem(max_rowbytes);
    cudaFuncSetAttribute(k_paths_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_paths_batch, kBatchBS, sm);
    return n;
}

int batch_tile_paths() { return kBatchBS * kBatchP; }

}  // namespace qr
