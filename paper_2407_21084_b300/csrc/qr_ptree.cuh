// qr_ptree.cuh -- compile-time tiles of the projection kernel (see
// qr_proj_tree.cu); included by every file that instantiates them.
#pragma once

#include "qr_device.cuh"
#include "qr_fast.h"

namespace qr {


template <int D, int NN, int KIND>
struct FullTree {
    static constexpr int kMax = 2048;
    struct Nodes {
        int n = 0;
        signed char dim[kMax] = {};
        signed char sgn[kMax] = {};
        short parent[kMax] = {};
    };
    static constexpr bool ext_ok(int S) { return KIND == QR_G_L1 ? S >= 1 : S < NN; }
    static constexpr int ext_S(int S) { return KIND == QR_G_L1 ? S - 1 : S + 1; }
    static constexpr bool new_ok(int S) { return KIND == QR_G_L1 ? S >= 1 : true; }
    static constexpr int new_S(int S) { return KIND == QR_G_L1 ? S - 1 : 1; }
    // node reached by multiplying its parent's basis by z_dim^sgn, in state S
    static constexpr void visit(Nodes& t, int L, int S, int parent, int sgn)
    {
        const int me = t.n++;
        t.dim[me] = (signed char)L;
        t.sgn[me] = (signed char)sgn;
        t.parent[me] = (short)parent;
        if (ext_ok(S)) visit(t, L, ext_S(S), me, sgn);
        if (new_ok(S))
            for (int l2 = L + 1; l2 < D; ++l2) {
                visit(t, l2, new_S(S), me, +1);
                visit(t, l2, new_S(S), me, -1);
            }
    }
    static constexpr Nodes build()
    {
        Nodes t{};
        const int S0 = KIND == QR_G_L1 ? NN - 1 : 1;
        for (int l = 0; l < D; ++l) visit(t, l, S0, -1, +1);
        return t;
    }
    static constexpr Nodes nodes = build();
    static constexpr int n = nodes.n;  // |Gamma_+| without k = 0
    static constexpr int tiles = (n + 31) / 32;
};

// basis value of node s (prefix products are shared by common subexpressions)
template <typename R, int D, class TR, int s>
__device__ __forceinline__ V2<R> bval(const V2<R> (&z)[D])
{
    constexpr int p = TR::nodes.parent[s];
    constexpr int dm = TR::nodes.dim[s];
    constexpr int sg = TR::nodes.sgn[s];
    V2<R> w = z[dm];
    if constexpr (sg < 0) w.y = -w.y;
    if constexpr (p < 0)
        return w;
    else
        return cmul<R>(bval<R, D, TR, p>(z), w);
}

template <typename R, int D, class TR, int T, int j>
struct TileSlots {
    static __device__ __forceinline__ void run(const V2<R> (&z)[D], R S, V2<R> (&acc)[32])
    {
        if constexpr (j < 32 && T * 32 + j < TR::n) {
            const V2<R> b = bval<R, D, TR, T * 32 + j>(z);
            acc[j].x = fma(S, b.x, acc[j].x);
            acc[j].y = fma(-S, b.y, acc[j].y);  // S conj(phi_k)
            TileSlots<R, D, TR, T, j + 1>::run(z, S, acc);
        }
    }
};

// reduce-scatter of 32 values over the warp: lane L returns the lane sum of v[L]
template <typename R>
__device__ __forceinline__ R fold32(R (&v)[32], int lane)
{
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const R send = up ? v[j] : v[j + h];
            const R keep = up ? v[j + h] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

template <typename R, int D, class TR, int BS, int SC>
struct ProjSmem {
    static constexpr int W = BS / 32;
    V2<R> z[D][SC];
    R S[SC];
    V2<R> acc[W][TR::tiles * 32];
};

template <typename R, int D, class TR, int BS, int SC, int T>
struct Tiles {
    static __device__ __forceinline__ void run(ProjSmem<R, D, TR, BS, SC>& sm, int warp, int lane)
    {
        if constexpr (T < TR::tiles) {
            V2<R> acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = mk2<R>((R)0, (R)0);
            constexpr int per_warp = SC / (BS / 32);
#pragma unroll 1
            for (int q = 0; q < per_warp; q += 32) {
                const int pth = warp * per_warp + q + lane;
                V2<R> z[D];
#pragma unroll
                for (int l = 0; l < D; ++l) z[l] = sm.z[l][pth];
                TileSlots<R, D, TR, T, 0>::run(z, sm.S[pth], acc);
            }
            R vr[32], vi[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                vr[j] = acc[j].x;
                vi[j] = acc[j].y;
            }
            const R sr = fold32<R>(vr, lane), si = fold32<R>(vi, lane);
            V2<R>& a = sm.acc[warp][T * 32 + lane];
            a.x += sr;
            a.y += si;
            Tiles<R, D, TR, BS, SC, T + 1>::run(sm, warp, lane);
        }
    }
};

// one (row i, chunk ch) of the projection: the FP64 partial sums of the
// chunk's paths into out[0 .. |Gamma_+|) (canonical half-set order through
// perm); S_row holds row i's responses (path m at S_row[m]); smem_raw is the
// block's dynamic shared memory (sizeof(ProjSmem) bytes). Every thread of
// the block calls it.
template <typename R, int D, int NN, int KIND, int BS, int SC>
__device__ __forceinline__ void project_tree_item(const QrParams& P, const R* __restrict__ S_row,
                                                  const int* __restrict__ perm, double2* __restrict__ out, int i,
                                                  int ch, unsigned char* smem_raw)
{
    using TR = FullTree<D, NN, KIND>;
    using SM = ProjSmem<R, D, TR, BS, SC>;
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    constexpr int W = BS / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long base = (long long)ch * P.chunk;
    const long long end = min((long long)P.M, base + P.chunk);
    for (int t = tid; t < W * TR::tiles * 32; t += BS) (&sm.acc[0][0])[t] = mk2<R>((R)0, (R)0);
    R s0 = 0;  // k = 0: sum of the responses (this thread's share)
    for (long long sub = base; sub < end; sub += SC) {
        __syncthreads();
        for (int r = tid; r < SC; r += BS) {
            const long long m = sub + r;
            const bool active = m < end;
            V2<R> ph[D];
            start_phases_dev<R, D>(P, i, active ? m : 0, ph);
#pragma unroll
            for (int l = 0; l < D; ++l) sm.z[l][r] = ph[l];
            const R Sv = active ? S_row[(size_t)m] : (R)0;
            sm.S[r] = Sv;
            s0 += Sv;
        }
        __syncthreads();
        Tiles<R, D, TR, BS, SC, 0>::run(sm, warp, lane);
    }
    __syncthreads();
    // k = 0 (slot 0 of the canonical half set): fixed-order block sum
    __shared__ double red[W];
    double d0 = (double)s0;
    for (int o = 16; o > 0; o >>= 1) d0 += __shfl_xor_sync(0xffffffffu, d0, o);
    if (lane == 0) red[warp] = d0;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < W; ++w) t += red[w];
        out[0] = make_double2(t, 0.0);
    }
    for (int s = tid; s < TR::n; s += BS) {
        double sx = 0.0, sy = 0.0;
        for (int w = 0; w < W; ++w) {
            sx += (double)sm.acc[w][s].x;
            sy += (double)sm.acc[w][s].y;
        }
        out[perm[s]] = make_double2(sx, sy);
    }
}

template <typename R, int D, int NN, int KIND, int BS, int SC>
__global__ void __launch_bounds__(BS) k_project_tree(const __grid_constant__ QrParams P, const R* __restrict__ S,
                                                     const int* __restrict__ perm, double2* __restrict__ partial,
                                                     int i_lo)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = P.c_hi - P.c_lo;  // the context's chunks
    const int i = i_lo + (int)(blockIdx.x / nc);
    const int ch = P.c_lo + (int)(blockIdx.x % nc);
    project_tree_item<R, D, NN, KIND, BS, SC>(P, S + (size_t)(i - i_lo) * (size_t)P.M, perm,
                                              partial + ((size_t)(i - i_lo) * P.n_chunks + ch) * P.nGp, i, ch,
                                              smem_raw);
}

template <typename R, int D, int NN, int KIND>
static cudaError_t project_tree_t(const QrParams& P, const void* S, const int* perm, double2* partial, int i_lo,
                                  int i_hi, cudaStream_t st)
{
#ifndef QR_PROJ_BS32
#define QR_PROJ_BS32 128
#endif
#ifndef QR_PROJ_SC32
#define QR_PROJ_SC32 1024
#endif
    constexpr int BS = sizeof(R) == 4 ? QR_PROJ_BS32 : 128;
    constexpr int SC = sizeof(R) == 4 ? QR_PROJ_SC32 : 512;
    using SM = ProjSmem<R, D, FullTree<D, NN, KIND>, BS, SC>;
    const size_t sm = sizeof(SM);
    // a chunk need not be a multiple of SC: its last block is partly empty
    // (zero responses, no contribution)
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    auto kern = k_project_tree<R, D, NN, KIND, BS, SC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)(P.c_hi - P.c_lo) * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, static_cast<const R*>(S), perm, partial, i_lo);
    return cudaGetLastError();
}

}  // namespace qr
