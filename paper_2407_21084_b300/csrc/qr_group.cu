// qr_group.cu -- path-and-series kernel for instances that share their
// sample points: same d, N, M, sigma, b, index set, density, seed and Philox
// instance, so every instance sees the same Euler paths and the same basis
// values; only the coefficients (and the driver/terminal parameters a, s)
// differ. The series of G instances at a tile of 128 path points is then the
// dense product
//     Y[128 x G] = Phi[128 x K] A[K x G],   K = 2 |Gamma_+| - 1 (+ padding),
// Phi = (Re phi_k, Im phi_k) of the half set and A = (2 Re alpha_k,
// -2 Im alpha_k, alpha_0) of each instance. It runs on the tensor cores as
// BF16 with split operands: X = X_hi + X_lo (both BF16), Y ~= Phi_hi A_hi +
// Phi_hi A_lo + Phi_lo A_hi accumulated in FP32 (relative error ~2^-16 per
// product). Phi is built per step by the compile-time tree of the projection
// (qr_ptree.cuh), in K-chunks of 32 coefficients; A of the next row is
// staged by a bulk copy. A CTA handles one tile of paths for G = 32
// instances; the driver, truncation and response sums stay per instance in
// FP32 registers.
#include <cuda_bf16.h>

#include "qr_group.h"
#include "qr_ptree.cuh"
#include "qr_tree.cuh"

namespace qr {

constexpr int kGBS = 128;   // threads = paths per tile
constexpr int kGG = 32;     // instances per CTA
constexpr int kGKC = 64;    // K-chunk (32 complex coefficients)
constexpr int kGPadA = 8;   // bf16 padding of shared-memory rows (bank spread)

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// basis values (re, im) of the tree nodes of chunk C for one point, split to bf16 hi/lo into
// rows hi/lo (kGKC entries); entries past the tree hold the constant 1 (alpha_0) then 0
template <class TR, int D, int C, int j>
struct ChunkSlots {
    static __device__ __forceinline__ void run(const float2 (&z)[D], __nv_bfloat16* hi, __nv_bfloat16* lo)
    {
        if constexpr (j < 32) {
            constexpr int s = C * 32 + j;
            float re = 0.f, im = 0.f;
            if constexpr (s < TR::n) {
                const float2 b = bval<float, D, TR, s>(z);
                re = b.x;
                im = b.y;
            } else if constexpr (s == TR::n) {
                re = 1.f;  // alpha_0 column
            }
            const __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
            const __nv_bfloat16 rl = __float2bfloat16_rn(re - __bfloat162float(rh));
            const __nv_bfloat16 il = __float2bfloat16_rn(im - __bfloat162float(ih));
            reinterpret_cast<uint32_t*>(hi)[j] = pack_bf16(rh, ih);  // (re, im) at k = 2j, 2j + 1
            reinterpret_cast<uint32_t*>(lo)[j] = pack_bf16(rl, il);
            ChunkSlots<TR, D, C, j + 1>::run(z, hi, lo);
        }
    }
};

template <class TR, int D>
struct GroupSmem {
    static constexpr int nchunks = (TR::n + 1 + 31) / 32;  // tree nodes + alpha_0 column
    static constexpr int K = nchunks * kGKC;
    __nv_bfloat16 A_hi[kGG][K + kGPadA];  // coefficients, instance-major (B operand, col layout)
    __nv_bfloat16 A_lo[kGG][K + kGPadA];
    __nv_bfloat16 P_hi[kGBS][kGKC + kGPadA];  // basis chunk, point-major (A operand, row layout)
    __nv_bfloat16 P_lo[kGBS][kGKC + kGPadA];
    float Y[kGBS][kGG + 1];
    GroupInstParams ip[kGG];
    float fexp[kGG][kGroupNMax];
    uint64_t bar;
};

// one chunk of the GEMM: this warp's 32 rows x 32 instances, K-chunk of 64
template <class TR, int D>
__device__ __forceinline__ void gemm_chunk(GroupSmem<TR, D>& sm, int chunk, int warp, int lane, float (&acc)[2][4][4])
{
    const int r0 = warp * 32, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int kk = 0; kk < kGKC; kk += 16) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int row = r0 + mt * 16 + g;
            const uint32_t* ph0 = reinterpret_cast<const uint32_t*>(&sm.P_hi[row][kk + 2 * q]);
            const uint32_t* ph1 = reinterpret_cast<const uint32_t*>(&sm.P_hi[row + 8][kk + 2 * q]);
            const uint32_t* pl0 = reinterpret_cast<const uint32_t*>(&sm.P_lo[row][kk + 2 * q]);
            const uint32_t* pl1 = reinterpret_cast<const uint32_t*>(&sm.P_lo[row + 8][kk + 2 * q]);
            ah[mt][0] = ph0[0];
            ah[mt][1] = ph1[0];
            ah[mt][2] = ph0[4];  // k + 8
            ah[mt][3] = ph1[4];
            al[mt][0] = pl0[0];
            al[mt][1] = pl1[0];
            al[mt][2] = pl0[4];
            al[mt][3] = pl1[4];
        }
        const int kg = chunk * kGKC + kk;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int col = nt * 8 + g;
            const uint32_t* bh = reinterpret_cast<const uint32_t*>(&sm.A_hi[col][kg + 2 * q]);
            const uint32_t* bl = reinterpret_cast<const uint32_t*>(&sm.A_lo[col][kg + 2 * q]);
            const uint32_t bhi[2] = {bh[0], bh[4]};
            const uint32_t blo[2] = {bl[0], bl[4]};
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma_bf16(acc[mt][nt], ah[mt], bhi);
                mma_bf16(acc[mt][nt], ah[mt], blo);
                mma_bf16(acc[mt][nt], al[mt], bhi);
            }
        }
    }
}

// the K-chunks of one step: basis chunk into shared memory, then the GEMM
template <class TR, int D, int C>
struct GroupChunks {
    static __device__ __forceinline__ void run(GroupSmem<TR, D>& sm, const float2 (&z)[D], int tid, int warp,
                                               int lane, float (&acc)[2][4][4])
    {
        if constexpr (C < GroupSmem<TR, D>::nchunks) {
            ChunkSlots<TR, D, C, 0>::run(z, &sm.P_hi[tid][0], &sm.P_lo[tid][0]);
            __syncthreads();
            gemm_chunk<TR, D>(sm, C, warp, lane, acc);
            __syncthreads();
            GroupChunks<TR, D, C + 1>::run(sm, z, tid, warp, lane, acc);
        }
    }
};

template <int D, int NN, int KIND>
__global__ void __launch_bounds__(kGBS) k_paths_group(const __grid_constant__ QrParams P, const GroupInst* __restrict__ inst,
                                                     int n_inst, const __nv_bfloat16* __restrict__ Apack,
                                                     long long a_row_elems, int tiles_per_i,
                                                     unsigned* __restrict__ status)
{
    using TR = FullTree<D, NN, KIND>;
    using SM = GroupSmem<TR, D>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles_g = (n_inst + kGG - 1) / kGG;
    const int gblk = blockIdx.x % ntiles_g;  // which 32 instances
    const int rest = blockIdx.x / ntiles_g;
    const int i = rest / tiles_per_i;  // rows in ascending order: longest first
    const long long m = (long long)(rest % tiles_per_i) * kGBS + tid;
    const int g0 = gblk * kGG, ng = min(kGG, n_inst - g0);
    const int N = P.N;

    for (int g = tid; g < kGG; g += kGBS) sm.ip[g] = inst[min(g0 + g, n_inst - 1)].p;
    for (int t = tid; t < kGG * N; t += kGBS) {
        const int g = t / N, j = t % N;
        sm.fexp[g][j] = inst[min(g0 + g, n_inst - 1)].fexp[j];
    }
    if (tid == 0) {
        mbar_init(&sm.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    const StepConsts<float, D> KC(P);
    float x[D];
    {
        float2 unused[D];
        start_point<float, D>(P, i, m, x, unused, false);
    }
    float S[kGG];
#pragma unroll
    for (int g = 0; g < kGG; ++g) S[g] = 0.f;
    uint32_t phase = 0;
    const float dt = KC.dt;
    const uint32_t abytes = (uint32_t)(SM::K + kGPadA) * 2u * kGG;  // one of A_hi / A_lo

    for (int j = i; j < N; ++j) {
        const int row = j + 1;
        float z[D], x1[D];
        normals_fast<float, D>(P, i, (uint32_t)m, j, z);
        euler_fast<float, D>(KC, x, z, x1);
        if (row < N) {
            if (tid == 0) {
                fence_proxy_async_smem();
                const __nv_bfloat16* src = Apack + ((size_t)row * ntiles_g + gblk) * 2 * (size_t)a_row_elems;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&sm.bar)),
                             "r"(2 * abytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(&sm.A_hi[0][0])),
                    "l"(src), "r"(abytes), "r"(smem_u32(&sm.bar))
                    : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(&sm.A_lo[0][0])),
                    "l"(src + a_row_elems), "r"(abytes), "r"(smem_u32(&sm.bar))
                    : "memory");
            }
            float2 ph[D];
#pragma unroll
            for (int l = 0; l < D; ++l) ph[l] = nu_phase<float>(P, x1[l]);
            const bool ok = mbar_wait(&sm.bar, phase);
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {
                if (tid == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
            float acc[2][4][4];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
            GroupChunks<TR, D, 0>::run(sm, ph, tid, warp, lane, acc);
            // accumulators -> Y[point][instance]
            const int g = lane >> 2, q = lane & 3;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int r = warp * 32 + mt * 16 + g, c = nt * 8 + 2 * q;
                    sm.Y[r][c] = acc[mt][nt][0];
                    sm.Y[r][c + 1] = acc[mt][nt][1];
                    sm.Y[r + 8][c] = acc[mt][nt][2];
                    sm.Y[r + 8][c + 1] = acc[mt][nt][3];
                }
            __syncthreads();
        }
        // per instance: truncation T_L, driver f(t_j, X_j, y) and the response sum
#pragma unroll
        for (int g = 0; g < kGG; ++g) {
            const GroupInstParams& ip = sm.ip[g];
            float y;
            if (row < N) {
                y = sm.Y[tid][g];
                if (ip.clamp_L > 0.f) y = fminf(fmaxf(y, -ip.clamp_L), ip.clamp_L);
            } else {
                float sg = 0.f;
#pragma unroll
                for (int l = 0; l < D; ++l) sg += ip.gs[l] * x1[l];
                y = rcos<float>(sg);  // g(X_N) = cos(s.X_N)
            }
            float sf = 0.f;
#pragma unroll
            for (int l = 0; l < D; ++l) sf += ip.fs[l] * x[l];
            const float u = sm.fexp[g][j] * rcos<float>(sf);
            S[g] += (-y * y * y + (ip.f_c * u + u * u * u)) * dt;
            if (row == N) S[g] += y;
        }
#pragma unroll
        for (int l = 0; l < D; ++l) x[l] = x1[l];
        __syncthreads();
    }
    if (m < P.M) {
#pragma unroll
        for (int g = 0; g < kGG; ++g)
            if (g < ng) static_cast<float*>(inst[g0 + g].S)[(size_t)i * (size_t)P.M + (size_t)m] = S[g];
    }
}

// coefficient blocks of row r, instance block gb: [A_hi (32 x (K+pad))][A_lo (same)]
template <int D, int NN, int KIND>
__global__ void k_pack_group(const GroupInst* __restrict__ inst, int n_inst, int nG, int zero_idx,
                             const int* __restrict__ perm, __nv_bfloat16* __restrict__ Apack, int rows)
{
    using TR = FullTree<D, NN, KIND>;
    using SM = GroupSmem<TR, D>;
    constexpr int KP = SM::K + kGPadA;
    const int ntg = (n_inst + kGG - 1) / kGG;
    const long long total = (long long)rows * ntg * kGG * KP;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int k = (int)(t % KP);
    const int g = (int)((t / KP) % kGG);
    const int gb = (int)((t / ((long long)KP * kGG)) % ntg);
    const int r = (int)(t / ((long long)KP * kGG * ntg));
    const int q = gb * kGG + g;
    double v = 0.0;
    if (q < n_inst && k < 2 * TR::n + 1) {
        const double2* row = inst[q].alpha + (size_t)r * nG;
        if (k == 2 * TR::n) {
            v = row[zero_idx].x;
        } else {
            const double2 a = row[zero_idx + perm[k >> 1]];
            v = (k & 1) ? -2.0 * a.y : 2.0 * a.x;
        }
    }
    const float vf = (float)v;
    const __nv_bfloat16 hi = __float2bfloat16_rn(vf);
    const __nv_bfloat16 lo = __float2bfloat16_rn(vf - __bfloat162float(hi));
    __nv_bfloat16* base = Apack + ((size_t)r * ntg + gb) * 2 * (size_t)kGG * KP;
    base[(size_t)g * KP + k] = hi;
    base[(size_t)kGG * KP + (size_t)g * KP + k] = lo;
}

#define QR_GROUP_SETS(X) \
    X(QR_G_LINF, 2, 4)   \
    X(QR_G_L1, 6, 3)

bool group_supported(int kind, int d, int n)
{
#define QR_X(KD, DD, NNN) \
    if (kind == KD && d == DD && n == NNN) return true;
    QR_GROUP_SETS(QR_X)
#undef QR_X
    return false;
}

long long group_block_elems(int kind, int d, int n)
{
#define QR_X(KD, DD, NNN) \
    if (kind == KD && d == DD && n == NNN) return (long long)kGG * (GroupSmem<FullTree<DD, NNN, KD>, DD>::K + kGPadA);
    QR_GROUP_SETS(QR_X)
#undef QR_X
    return 0;
}

cudaError_t launch_pack_group(int kind, int d, int n, const GroupInst* inst, int n_inst, int nG, int zero_idx,
                              const int* perm, void* Apack, int rows, cudaStream_t st)
{
    const int ntg = (n_inst + kGG - 1) / kGG;
#define QR_X(KD, DD, NNN)                                                                                   \
    if (kind == KD && d == DD && n == NNN) {                                                                \
        const long long total = (long long)rows * ntg * group_block_elems(KD, DD, NNN);                    \
        k_pack_group<DD, NNN, KD><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(                         \
            inst, n_inst, nG, zero_idx, perm, static_cast<__nv_bfloat16*>(Apack), rows);                   \
        return cudaGetLastError();                                                                         \
    }
    QR_GROUP_SETS(QR_X)
#undef QR_X
    return cudaErrorInvalidValue;
}

cudaError_t launch_paths_group(int kind, int d, int n, const QrParams& P, const GroupInst* inst, int n_inst,
                               const void* Apack, unsigned* status, cudaStream_t st)
{
    if (P.N > kGroupNMax) return cudaErrorInvalidValue;
    const int ntg = (n_inst + kGG - 1) / kGG;
    const int tiles = (int)((P.M + kGBS - 1) / kGBS);
#define QR_X(KD, DD, NNN)                                                                                     \
    if (kind == KD && d == DD && n == NNN) {                                                                  \
        using SMT = GroupSmem<FullTree<DD, NNN, KD>, DD>;                                                     \
        auto kern = k_paths_group<DD, NNN, KD>;                                                               \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SMT)); \
        if (e != cudaSuccess) return e;                                                                      \
        const long long blocks = (long long)tiles * P.N * ntg;                                               \
        kern<<<(unsigned)blocks, kGBS, sizeof(SMT), st>>>(P, inst, n_inst,                                   \
                                                         static_cast<const __nv_bfloat16*>(Apack),           \
                                                         group_block_elems(KD, DD, NNN), tiles, status);      \
        return cudaGetLastError();                                                                           \
    }
    QR_GROUP_SETS(QR_X)
#undef QR_X
    return cudaErrorInvalidValue;
}

}  // namespace qr
