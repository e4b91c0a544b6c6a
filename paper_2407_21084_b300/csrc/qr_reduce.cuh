// qr_reduce.cuh -- the deterministic cross-chunk reduction of the projection
// (eq. Aqi:bar:M): device helpers shared by the single-problem reduction
// kernels (qr_kernels.cu) and the many-instance finishing kernel
// (qr_batch.cu), so that both take exactly the same operations in the same
// order (a batch instance's coefficients equal its single run's bit for bit).
#pragma once

#include "qr_device.cuh"
#include "qr_fast.h"

namespace qr {

// sum over the chunks of one coefficient entry: chunks in order within each
// of the kShardGroups groups, then the group sums in order; p points at the
// entry's partial of chunk 0, consecutive chunks nGp double2 apart. L2-only
// loads (partials written by other CTAs of the same launch).
__device__ __forceinline__ void chunk_sum2(const double2* p, int n_chunks, int nGp, double& sx, double& sy)
{
    sx = 0.0;
    sy = 0.0;
    for (int g = 0; g < kShardGroups; ++g) {
        double gx = 0.0, gy = 0.0;
        for (int c = group_chunk(g, n_chunks); c < group_chunk(g + 1, n_chunks); ++c) {
            const double2 v = __ldcg(p + (size_t)c * nGp);
            gx += v.x;
            gy += v.y;
        }
        sx += gx;
        sy += gy;
    }
}

// the end of a reduction for entry e of row i: 1/M, conjugate fill, the
// packed working row, and |alpha - alpha_old| for the residual
template <typename R>
__device__ __forceinline__ void finish_coef(const QrParams& P, double sx, double sy, int e, int i, int nG,
                                            int zero_idx, double2* alpha, V2<R>* packed, long long row_stride,
                                            double& diff)
{
    sx /= (double)P.M;
    sy /= (double)P.M;
    if (e == 0) sy = 0.0;
    diff = 0.0;
    if (!in_bounds(P, i >= 0 && i <= P.N && e >= 0 && e < P.nGp && zero_idx - e >= 0 && zero_idx + e < nG &&
                          e < row_stride))
        return;
    double2* row = alpha + (size_t)i * nG;
    const double2 old = row[zero_idx + e];
    diff = hypot(sx - old.x, sy - old.y);
    row[zero_idx + e] = make_double2(sx, sy);
    if (e > 0) row[zero_idx - e] = make_double2(sx, -sy);
    packed[(size_t)i * row_stride + e] = e == 0 ? mk2<R>((R)sx, (R)0) : mk2<R>((R)(2.0 * sx), (R)(2.0 * sy));
}

// block max of the residual, then one atomic into *out (max is order
// independent); every thread of the block calls it
__device__ __forceinline__ void reduce_residual(double diff, unsigned long long* out)
{
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_xor_sync(0xffffffffu, diff, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = diff;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        atomicMax(out, (unsigned long long)__double_as_longlong(mx));
    }
}

// one slot of a tree-layout coefficient row from the master row a (2 nG
// doubles, interleaved re/im): slot = (c00 a[i00] + c01 a[i01], c10 a[i10] + c11 a[i11])
template <typename R>
__device__ __forceinline__ V2<R> tree_slot(const double* a, const TreeMap& mp)
{
    double v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double t = 0.0;
#pragma unroll
        for (int u = 0; u < kTreeTerms; ++u)
            if (mp.c[h][u] != 0) t += mp.c[h][u] * a[mp.i[h][u]];
        v[h] = t;
    }
    return mk2<R>((R)v[0], (R)v[1]);
}

}  // namespace qr
