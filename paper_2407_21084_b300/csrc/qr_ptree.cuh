// qr_ptree.cuh -- compile-time tiles of the projection kernel (see
// qr_proj_tree.cu); included by every file that instantiates them.
#pragma once

#include "qr_device.cuh"
#include "qr_fast.h"

namespace qr {


template <int D, int NN, int KIND>
struct FullTree {
    static constexpr int kMax = 2048;
    // node s: basis value = basis of parent[s] times z_dim^sgn. A mirrored
    // pair s, s+1 (pairnext[s]) are k' + m e_dim and k' - m e_dim for the
    // frame node k' = frame[s] (-1: the root) and the power m = pw[s]: the
    // projection accumulates S conj(phi) of both from S conj(phi_frame) and
    // z_dim^m with 8 FMA.
    struct Nodes {
        int n = 0;
        signed char dim[kMax] = {};
        signed char sgn[kMax] = {};
        short parent[kMax] = {};
        short frame[kMax] = {};
        signed char pw[kMax] = {};
        bool pairnext[kMax] = {};
    };
    static constexpr bool ext_ok(int S) { return KIND == QR_G_L1 ? S >= 1 : S < NN; }
    static constexpr int ext_S(int S) { return KIND == QR_G_L1 ? S - 1 : S + 1; }
    static constexpr bool new_ok(int S) { return KIND == QR_G_L1 ? S >= 1 : true; }
    static constexpr int new_S(int S) { return KIND == QR_G_L1 ? S - 1 : 1; }
    // nodes of a last-dimension node in state S and its chain of extensions
    static constexpr int chain_len(int S) { return 1 + (ext_ok(S) ? chain_len(ext_S(S)) : 0); }
    static constexpr int add(Nodes& t, int L, int parent, int sgn)
    {
        const int me = t.n++;
        t.dim[me] = (signed char)L;
        t.sgn[me] = (signed char)sgn;
        t.parent[me] = (short)parent;
        t.frame[me] = -1;
        return me;
    }
    // node reached by multiplying its parent's basis by z_dim^sgn, in state S;
    // the +- chains of the last dimension are interleaved (+1, -1, +2, -2, ...)
    static constexpr void visit(Nodes& t, int L, int S, int parent, int sgn)
    {
        const int me = add(t, L, parent, sgn);
        if (ext_ok(S)) visit(t, L, ext_S(S), me, sgn);
        if (new_ok(S))
            for (int l2 = L + 1; l2 < D; ++l2) {
                const int S2 = new_S(S);
                if (l2 == D - 1) {
                    int pp = me, pm = me;
                    for (int m = 1; m <= chain_len(S2); ++m) {
                        pp = add(t, l2, pp, +1);
                        pm = add(t, l2, pm, -1);
                        t.frame[pp] = t.frame[pm] = (short)me;
                        t.pw[pp] = t.pw[pm] = (signed char)m;
                        t.pairnext[pp] = true;
                    }
                } else if (!ext_ok(S2) && !new_ok(S2)) {
                    // a +-1 pair of leaves in dimension l2
                    const int a = add(t, l2, me, +1), b = add(t, l2, me, -1);
                    t.frame[a] = t.frame[b] = (short)me;
                    t.pw[a] = t.pw[b] = 1;
                    t.pairnext[a] = true;
                } else {
                    visit(t, l2, S2, me, +1);
                    visit(t, l2, S2, me, -1);
                }
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
    // whether node s is the + member of a mirrored pair that tile layout keeps
    // together (both within one tile of 32)
    static constexpr bool pair_at(int s) { return nodes.pairnext[s] && (s % 32) != 31 && s + 1 < n; }
    // highest power of the last dimension's phase that tile T's pairs use
    static constexpr int tile_pow(int T)
    {
        int m = 1;
        for (int s = T * 32; s < T * 32 + 32 && s < n; ++s)
            if (pair_at(s) && nodes.dim[s] == D - 1 && nodes.pw[s] > m) m = nodes.pw[s];
        return m;
    }
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

template <typename R, int D, class TR, int T, int j, int NP>
struct TileSlots {
    // zl[m-1] = z[D-1]^m
    static __device__ __forceinline__ void run(const V2<R> (&z)[D], const V2<R> (&zl)[NP], R S, V2<R> (&acc)[32])
    {
        constexpr int s = T * 32 + j;
        if constexpr (j < 32 && s < TR::n) {
            if constexpr (TR::pair_at(s)) {
                // k' +- m e_l: with w = S conj(phi_k') = p + iq and z_l^m = a + ib,
                // S conj(phi_{k'+m e}) = w conj(z^m) = (pa + qb) + i(qa - pb) and
                // S conj(phi_{k'-m e}) = w z^m = (pa - qb) + i(qa + pb): the slots
                // gather the four sums (pa, qa) and (qb, pb), 4 FMA per path, and
                // PairForm turns them into the two coefficients per tile pass
                constexpr int f = TR::nodes.frame[s], dm = TR::nodes.dim[s], m = TR::nodes.pw[s];
                R p = S, q = (R)0;
                if constexpr (f >= 0) {
                    const V2<R> b = bval<R, D, TR, f>(z);
                    p = S * b.x;
                    q = -S * b.y;
                }
                V2<R> zm;
                if constexpr (m == 1)
                    zm = z[dm];
                else
                    zm = zl[m - 1];
                acc[j].x = fma(p, zm.x, acc[j].x);
                acc[j].y = fma(q, zm.x, acc[j].y);
                acc[j + 1].x = fma(q, zm.y, acc[j + 1].x);
                acc[j + 1].y = fma(p, zm.y, acc[j + 1].y);
                TileSlots<R, D, TR, T, j + 2, NP>::run(z, zl, S, acc);
            } else {
                const V2<R> b = bval<R, D, TR, s>(z);
                acc[j].x = fma(S, b.x, acc[j].x);
                acc[j].y = fma(-S, b.y, acc[j].y);  // S conj(phi_k)
                TileSlots<R, D, TR, T, j + 1, NP>::run(z, zl, S, acc);
            }
        }
    }
};

// the mirrored pairs of tile T: sums (pa, qa), (qb, pb) -> coefficients
// ((pa + qb, qa - pb), (pa - qb, qa + pb)) (linear, so it commutes with the
// sums over paths and lanes that follow)
template <typename R, class TR, int T, int j>
struct PairForm {
    static __device__ __forceinline__ void run(V2<R> (&acc)[32])
    {
        constexpr int s = T * 32 + j;
        if constexpr (j < 32 && s < TR::n) {
            if constexpr (TR::pair_at(s)) {
                const V2<R> u = acc[j], v = acc[j + 1];
                acc[j] = mk2<R>(u.x + v.x, u.y - v.y);
                acc[j + 1] = mk2<R>(u.x - v.x, u.y + v.y);
                PairForm<R, TR, T, j + 2>::run(acc);
            } else {
                PairForm<R, TR, T, j + 1>::run(acc);
            }
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

// per block of SC paths: their phases and responses; the block's running
// sums of every coefficient (one array per CTA: after each tile the warps'
// folded sums are added in warp order, staged in two buffers by tile parity)
template <typename R, int D, class TR, int BS, int SC>
struct ProjSmem {
    static constexpr int W = BS / 32;
    V2<R> z[D][SC];
    R S[SC];
    V2<R> acc[TR::tiles * 32];
    V2<R> stage[2][W][32];
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
                constexpr int NP = TR::tile_pow(T);
                V2<R> zl[NP];
                zl[0] = z[D - 1];
#pragma unroll
                for (int mm = 1; mm < NP; ++mm) zl[mm] = cmul<R>(zl[mm - 1], z[D - 1]);
                TileSlots<R, D, TR, T, 0, NP>::run(z, zl, sm.S[pth], acc);
            }
            PairForm<R, TR, T, 0>::run(acc);
            R vr[32], vi[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                vr[j] = acc[j].x;
                vi[j] = acc[j].y;
            }
            const R sr = fold32<R>(vr, lane), si = fold32<R>(vi, lane);
            sm.stage[T & 1][warp][lane] = mk2<R>(sr, si);
            // the staging buffer of this parity is free: warp 0 summed it
            // (tile T - 2) before it reached the barrier of tile T - 1
            __syncthreads();
            if (warp == 0) {
                V2<R> a = sm.acc[T * 32 + lane];
#pragma unroll
                for (int w = 0; w < BS / 32; ++w) {
                    a.x += sm.stage[T & 1][w][lane].x;
                    a.y += sm.stage[T & 1][w][lane].y;
                }
                sm.acc[T * 32 + lane] = a;
            }
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
    for (int t = tid; t < TR::tiles * 32; t += BS) sm.acc[t] = mk2<R>((R)0, (R)0);
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
        const double sx = (double)sm.acc[s].x, sy = (double)sm.acc[s].y;
        if (in_bounds(P, perm[s] > 0 && perm[s] < P.nGp)) out[perm[s]] = make_double2(sx, sy);
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
