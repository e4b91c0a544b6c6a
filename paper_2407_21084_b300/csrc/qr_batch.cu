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
// Projection, reduction and repacks of every instance are ONE more launch
// (k_finish_batch): a block per (instance, row, chunk of paths), ordered
// class by class, projects its chunk with the instance's compiled tiled
// projection; the last chunk of a row to finish (an arrival counter per row)
// reduces the row -- the same fixed-order two-level chunk sum as a single
// run, so the coefficients are bit-identical -- and rebuilds the row's tree
// layout, and the last member of a shared-point group to finish a row
// repacks the group's tensor-core coefficient blocks of that row. The whole
// iteration (counter resets, the persistent path kernel, the shared-point
// kernels, the finishing kernel) is captured in one CUDA graph. The items
// per claim (tiles per item) and the grid of the persistent kernel are chosen
// by timing candidates on the first iteration (autotuner).
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "qr_batch.h"
#include "qr_groupdev.cuh"
#include "qr_ptree.cuh"
#include "qr_reduce.cuh"
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

// resident CTAs per SM the register allocation is held to (4: 128 registers
// and about 1 KB of spills, 0.770 s per 256-instance iteration against 0.831
// at 3 CTAs with 168 registers; 2 CTAs without a cap were slower still)
#ifndef QR_BATCH_MINB
#define QR_BATCH_MINB 4
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

// ---------------------------------------------------------------- finishing
constexpr int kFinBS = 128, kFinSC = 1024;  // as the single-instance FP32 tiled projection

#define QR_GROUP_CLASSES(X) \
    X(0, QR_G_LINF, 2, 4)   \
    X(1, QR_G_L1, 6, 3)

int finish_group_class(int kind, int d, int n)
{
#define QR_X(C, K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return C;
    QR_GROUP_CLASSES(QR_X)
#undef QR_X
    return -1;
}

size_t finish_smem()
{
    size_t m = 16;
#define QR_X(C, K, DD, NNN) \
    m = std::max(m, sizeof(ProjSmem<float, DD, FullTree<DD, NNN, K>, kFinBS, kFinSC>));
    QR_BATCH_CLASSES(QR_X)
#undef QR_X
    return m;
}

// one (instance, row, chunk) per block; see the file comment
__global__ void __launch_bounds__(kFinBS) k_finish_batch(const FinishInst* __restrict__ fin,
                                                         const int4* __restrict__ items,
                                                         const FinishGroup* __restrict__ groups,
                                                         unsigned* __restrict__ row_done,
                                                         unsigned* __restrict__ grp_done,
                                                         unsigned long long* __restrict__ resid)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
    const int4 it = items[blockIdx.x];
    const FinishInst& F = fin[it.x];
    const QrParams& P = F.P;
    const int i = it.y, ch = it.z, tid = threadIdx.x;
    switch (F.cls) {
#define QR_X(C, K, DD, NNN)                                                                                       \
    case C:                                                                                                       \
        project_tree_item<float, DD, NNN, K, kFinBS, kFinSC>(P, F.S + (size_t)i * (size_t)P.M, F.perm,            \
                                                            F.partial + ((size_t)i * P.n_chunks + ch) * P.nGp, i, \
                                                            ch, smem);                                            \
        break;
        QR_BATCH_CLASSES(QR_X)
#undef QR_X
    default:
        break;
    }
    // the last chunk of row i to arrive reduces the row (partials of the
    // other blocks made visible by their fence before the count)
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(&row_done[F.row_base + i], 1u);
        s_last = prev == (unsigned)(P.n_chunks - 1);
        if (s_last) row_done[F.row_base + i] = 0u;  // ready for the next iteration
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double diff = 0.0;
    for (int e = tid; e < P.nGp; e += kFinBS) {
        double sx, sy, dv = 0.0;
        chunk_sum2(F.partial + (size_t)i * P.n_chunks * P.nGp + e, P.n_chunks, P.nGp, sx, sy);
        finish_coef<float>(P, sx, sy, e, i, F.nG, F.zero_idx, F.alpha, F.packed, F.row_stride, dv);
        diff = fmax(diff, dv);
    }
    reduce_residual(diff, &resid[it.x]);  // includes a block barrier: the master row is complete
    const double* a = reinterpret_cast<const double*>(F.alpha + (size_t)i * F.nG);
    for (int s = tid; s < F.tree_slots; s += kFinBS) F.tree[(size_t)i * F.tree_stride + s] = tree_slot<float>(a, F.tmap[s]);
    if (F.group < 0) return;
    // the last member of the group to finish row i repacks the group's row
    __threadfence();
    __syncthreads();
    const FinishGroup& G = groups[F.group];
    if (tid == 0) {
        const unsigned prev = atomicAdd(&grp_done[G.row_base + i], 1u);
        s_last = prev == (unsigned)(G.n_inst - 1);
        if (s_last) grp_done[G.row_base + i] = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int ntg = (G.n_inst + kGG - 1) / kGG;
    switch (G.gcls) {
#define QR_X(C, KD, DD, NNN)                                                                                   \
    case C: {                                                                                                 \
        constexpr int KK = GroupDims<FullTree<DD, NNN, KD>>::K;                                                \
        const int total = ntg * kGG * KK;                                                                     \
        for (int t = tid; t < total; t += kFinBS)                                                             \
            pack_group_elem<DD, NNN, KD>(G.inst, G.n_inst, G.nG, G.zero_idx, G.perm, G.Bpack, ntg, i,          \
                                        t / (kGG * KK), (t / KK) % kGG, t % KK);                              \
        break;                                                                                                \
    }
        QR_GROUP_CLASSES(QR_X)
#undef QR_X
    default:
        break;
    }
}

cudaError_t launch_finish_batch(const FinishInst* fin, const int4* items, long long n_items, const FinishGroup* groups,
                                unsigned* row_done, unsigned* grp_done, unsigned long long* resid, cudaStream_t st)
{
    const size_t sm = finish_smem();
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_finish_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    if (n_items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_finish_batch<<<(unsigned)n_items, kFinBS, sm, st>>>(fin, items, groups, row_done, grp_done, resid);
    return cudaGetLastError();
}

}  // namespace qr
