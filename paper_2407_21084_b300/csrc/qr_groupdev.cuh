// qr_groupdev.cuh -- layout of the shared-point group kernel's coefficient
// blocks (qr_group.cu) and the packing of one element, shared with the
// many-instance finishing kernel (qr_batch.cu), which repacks a group's rows
// as soon as every member's row is reduced.
#pragma once

#include <cuda_bf16.h>

#include "qr_group.h"
#include "qr_ptree.cuh"
#include "qr_tc.cuh"

namespace qr {

constexpr int kGBS = 128;  // threads = paths per tile = MMA M
constexpr int kGG = 32;    // instances per CTA = MMA N (32 TMEM columns)
constexpr int kGKC = 64;   // K-chunk: 32 complex basis values = one 128-byte row

template <class TR>
struct GroupDims {
    static constexpr int nchunks = (TR::n + 1 + 31) / 32;  // tree nodes + the alpha_0 column
    static constexpr int K = nchunks * kGKC;
    static constexpr uint32_t chunk_bytes = kGG * 128;              // 32 instance rows of one K-chunk
    static constexpr uint32_t block_bytes = nchunks * chunk_bytes;  // hi (or lo) of one row block
};

// element k of instance g of block gb, row r: A = (2 Re alpha_k, -2 Im alpha_k)
// over the tree nodes (canonical half-set entries through perm), then alpha_0,
// then zeros; split into BF16 hi and lo and stored at its swizzled position.
// The master rows are read from L2 (written by other CTAs of the same launch
// in the finishing kernel).
template <int D, int NN, int KIND>
__device__ __forceinline__ void pack_group_elem(const GroupInst* __restrict__ inst, int n_inst, int nG, int zero_idx,
                                                const int* __restrict__ perm, uint8_t* __restrict__ Bpack, int ntg,
                                                int r, int gb, int g, int k)
{
    using TR = FullTree<D, NN, KIND>;
    using GD = GroupDims<TR>;
    const int q = gb * kGG + g;
    double v = 0.0;
    if (q < n_inst && k < 2 * TR::n + 1) {
        const double2* row = inst[q].alpha + (size_t)r * nG;
        if (k == 2 * TR::n) {
            v = __ldcg(row + zero_idx).x;
        } else {
            const double2 a = __ldcg(row + zero_idx + perm[k >> 1]);
            v = (k & 1) ? -2.0 * a.y : 2.0 * a.x;
        }
    }
    const float vf = (float)v;
    const __nv_bfloat16 hi = __float2bfloat16_rn(vf);
    const __nv_bfloat16 lo = __float2bfloat16_rn(vf - __bfloat162float(hi));
    uint8_t* base = Bpack + ((size_t)r * ntg + gb) * 2 * (size_t)GD::block_bytes;
    const uint32_t o = (uint32_t)(k / kGKC) * GD::chunk_bytes + sw128_offset((uint32_t)g, (uint32_t)(k % kGKC));
    *reinterpret_cast<__nv_bfloat16*>(base + o) = hi;
    *reinterpret_cast<__nv_bfloat16*>(base + GD::block_bytes + o) = lo;
}

}  // namespace qr
