// qr_group.cu -- path-and-series kernel for instances that share their
// sample points: same d, N, M, sigma, b, index set, density, seed and Philox
// instance, so every instance sees the same Euler paths and the same basis
// values; only the coefficients (and the driver/terminal parameters a, s)
// differ. The series of G = 32 instances at a tile of 128 path points is then
// the dense product
//     Y[128 x G] = Phi[128 x K] A[K x G],   K = 2 |Gamma_+| - 1 (+ padding),
// Phi = (Re phi_k, Im phi_k) of the half set and A = (2 Re alpha_k,
// -2 Im alpha_k, alpha_0) of each instance. It runs on the 5th-generation
// tensor cores (tcgen05.mma, kind::f16) as BF16 with split operands:
// X = X_hi + X_lo (both BF16), Y ~= Phi_hi A_hi + Phi_hi A_lo + Phi_lo A_hi
// accumulated in FP32 in tensor memory (relative error ~2^-16 per product).
// Per step and K-chunk of 64 (32 complex basis values), every thread builds
// its point's row of Phi with the compile-time tree of the projection
// (qr_ptree.cuh) straight into the 128-byte swizzled shared-memory layout the
// tensor core reads (conflict-free 16-byte stores); one thread issues the 12
// MMAs of the chunk and commits them to an mbarrier, which releases the
// buffer for the next chunk. The coefficient blocks of the next row, packed
// in the same swizzled layout by k_pack_group, arrive by one bulk copy per
// step. After the last chunk each warp reads its 32 rows x 32 instances of
// the accumulator with tcgen05.ld; the driver, truncation and response sums
// stay per instance in FP32 registers. Every wait is bounded.
#include "qr_groupdev.cuh"
#include "qr_tree.cuh"

namespace qr {

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// basis values (re, im) of the tree nodes of chunk C for one point, split to
// BF16 hi/lo pairs; entries past the tree hold the constant 1 (alpha_0) then 0
template <class TR, int D, int C, int j>
struct ChunkSlots {
    static __device__ __forceinline__ void run(const float2 (&z)[D], uint32_t (&hi)[32], uint32_t (&lo)[32])
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
            hi[j] = pack_bf16(rh, ih);  // (re, im) at k = 2j, 2j + 1
            lo[j] = pack_bf16(rl, il);
            ChunkSlots<TR, D, C, j + 1>::run(z, hi, lo);
        }
    }
};

template <class TR, int D>
struct GroupSmem {
    using GD = GroupDims<TR>;
    uint8_t B_hi[GD::block_bytes];  // coefficient block (B operand, N x K), swizzled
    uint8_t B_lo[GD::block_bytes];
    uint8_t P_hi[kGBS * 128];  // basis chunk (A operand, M x 64), swizzled
    uint8_t P_lo[kGBS * 128];
    GroupInstParams ip[kGG];
    float fexp[kGG][kGroupNMax];
    float S[kGG][kGBS];  // response sums, one column per thread (conflict-free)
    uint64_t bar_b;    // coefficient block copy
    uint64_t bar_mma;  // tensor-core completion, one phase per commit
    uint32_t tslot;    // TMEM address of the accumulator
};

// one K-chunk of one step: the basis rows into shared memory, then (one
// thread) the 12 MMAs of the chunk and their commit. Returns false when a
// bounded wait ran out (block-uniform).
template <class TR, int D, int C>
struct GroupChunks {
    using SM = GroupSmem<TR, D>;
    using GD = GroupDims<TR>;
    static __device__ __forceinline__ bool run(SM& sm, const float2 (&z)[D], int tid, uint32_t tmem, uint32_t idesc,
                                               uint32_t& ph_b, uint32_t& ph_m)
    {
        if constexpr (C < GD::nchunks) {
            bool ok = true;
            if constexpr (C > 0) {
                // the previous chunk's MMAs read the basis buffer
                ok = mbar_wait(&sm.bar_mma, ph_m);
                ph_m ^= 1u;
            } else {
                // the coefficient block of this row
                ok = mbar_wait(&sm.bar_b, ph_b);
                ph_b ^= 1u;
            }
            uint32_t hi[32], lo[32];
            ChunkSlots<TR, D, C, 0>::run(z, hi, lo);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t o = (uint32_t)tid * 128u + ((uint32_t)((c ^ tid) & 7) << 4);
                *reinterpret_cast<uint4*>(sm.P_hi + o) = make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
                *reinterpret_cast<uint4*>(sm.P_lo + o) = make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
            }
            fence_proxy_async_smem();  // generic stores -> the tensor core's reads
            tc_fence_before();
            if (!__syncthreads_and(ok)) return false;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t pa = smem_u32(sm.P_hi), pl = smem_u32(sm.P_lo);
                const uint32_t bh = smem_u32(sm.B_hi) + C * GD::chunk_bytes, bl = smem_u32(sm.B_lo) + C * GD::chunk_bytes;
#pragma unroll
                for (int kk = 0; kk < kGKC / 16; ++kk) {
                    const uint32_t ko = 32u * kk;  // K-slice of 16 BF16 within the 128-byte rows
                    tc_mma_bf16(tmem, sw128_desc(pa + ko), sw128_desc(bh + ko), idesc, (C > 0 || kk > 0) ? 1u : 0u);
                    tc_mma_bf16(tmem, sw128_desc(pa + ko), sw128_desc(bl + ko), idesc, 1u);
                    tc_mma_bf16(tmem, sw128_desc(pl + ko), sw128_desc(bh + ko), idesc, 1u);
                }
                tc_commit(&sm.bar_mma);
            }
            return GroupChunks<TR, D, C + 1>::run(sm, z, tid, tmem, idesc, ph_b, ph_m);
        }
        return true;
    }
};

template <int D, int NN, int KIND>
__global__ void __launch_bounds__(kGBS) k_paths_group(const __grid_constant__ QrParams P, const GroupInst* __restrict__ inst,
                                                     int n_inst, const uint8_t* __restrict__ Bpack, int tiles_per_i,
                                                     unsigned* __restrict__ status)
{
    using TR = FullTree<D, NN, KIND>;
    using GD = GroupDims<TR>;
    using SM = GroupSmem<TR, D>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled tiles start on 1024-byte shared addresses (the launch adds the slack)
    const uint32_t raw = smem_u32(smem_raw);
    SM& sm = *reinterpret_cast<SM*>(smem_raw + (((raw + 1023u) & ~1023u) - raw));
    const int tid = threadIdx.x, warp = tid >> 5;
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
        mbar_init(&sm.bar_b, 1);
        mbar_init(&sm.bar_mma, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&sm.tslot, 32);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tslot;
    constexpr uint32_t idesc = idesc_bf16_f32(kGBS, kGG);

    const StepConsts<float, D> KC(P);
    float x[D];
    {
        float2 unused[D];
        start_point<float, D>(P, i, m, x, unused, false);
    }
    for (int g = 0; g < kGG; ++g) sm.S[g][tid] = 0.f;
    uint32_t ph_b = 0, ph_m = 0;
    const float dt = KC.dt;
    bool failed = false;

    for (int j = i; j < N; ++j) {
        const int row = j + 1;
        float z[D], x1[D];
        normals_fast<float, D>(P, i, (uint32_t)m, j, z);
        euler_fast<float, D>(KC, x, z, x1);
        if (row < N) {
            if (tid == 0) {
                fence_proxy_async_smem();
                const uint8_t* src = Bpack + ((size_t)row * ntiles_g + gblk) * 2 * (size_t)GD::block_bytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&sm.bar_b)),
                             "r"(2u * GD::block_bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sm.B_hi)),
                    "l"(src), "r"(GD::block_bytes), "r"(smem_u32(&sm.bar_b))
                    : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sm.B_lo)),
                    "l"(src + GD::block_bytes), "r"(GD::block_bytes), "r"(smem_u32(&sm.bar_b))
                    : "memory");
            }
            float2 ph[D];
#pragma unroll
            for (int l = 0; l < D; ++l) ph[l] = nu_phase_fast<float>(P, x1[l]);
            bool ok = GroupChunks<TR, D, 0>::run(sm, ph, tid, tmem, idesc, ph_b, ph_m);
            if (ok) {
                ok = __syncthreads_and(mbar_wait(&sm.bar_mma, ph_m));  // the last chunk's MMAs
                ph_m ^= 1u;
            }
            if (!ok) {
                if (tid == 0) atomicOr(status, ST_TIMEOUT);
                failed = true;
                break;
            }
            tc_fence_after();
        }
        // per instance: truncation T_L, driver f(t_j, X_j, y) and the response
        // sum; instances in groups of 8 (a rolled loop keeps the code short),
        // the series of 8 instances read from 8 accumulator columns at a time
#pragma unroll 1
        for (int g8 = 0; g8 < kGG; g8 += 8) {
            float y8[8];
            if (row < N) tmem_ld_32x8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)g8, y8);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int g = g8 + q;
                const GroupInstParams& ip = sm.ip[g];
                float yv;
                if (row < N) {
                    yv = y8[q];
                    if (ip.clamp_L > 0.f) yv = fminf(fmaxf(yv, -ip.clamp_L), ip.clamp_L);
                } else {
                    float sg = 0.f;
#pragma unroll
                    for (int l = 0; l < D; ++l) sg += ip.gs[l] * x1[l];
                    yv = rcos_fast<float>(sg);  // g(X_N) = cos(s.X_N)
                }
                float sf = 0.f;
#pragma unroll
                for (int l = 0; l < D; ++l) sf += ip.fs[l] * x[l];
                const float u = sm.fexp[g][j] * rcos_fast<float>(sf);
                float Sg = sm.S[g][tid] + (-yv * yv * yv + (ip.f_c * u + u * u * u)) * dt;
                if (row == N) Sg += yv;
                sm.S[g][tid] = Sg;
            }
        }
#pragma unroll
        for (int l = 0; l < D; ++l) x[l] = x1[l];
        tc_fence_before();
        __syncthreads();
    }
    if (!failed && m < P.M) {
        for (int g = 0; g < ng; ++g)
            static_cast<float*>(inst[g0 + g].S)[(size_t)i * (size_t)P.M + (size_t)m] = sm.S[g][tid];
    }
    // a timed-out wait may leave a copy or MMAs in flight: give them a bounded
    // chance to land before the tensor memory is released
    if (failed) {
        (void)mbar_wait(&sm.bar_b, ph_b);
        (void)mbar_wait(&sm.bar_mma, ph_m);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

// coefficient blocks of row r, instance block gb: [hi][lo], each nchunks K-chunks
// of 32 instance rows x 64 BF16 in the 128-byte swizzled layout
template <int D, int NN, int KIND>
__global__ void k_pack_group(const GroupInst* __restrict__ inst, int n_inst, int nG, int zero_idx,
                             const int* __restrict__ perm, uint8_t* __restrict__ Bpack, int rows)
{
    using GD = GroupDims<FullTree<D, NN, KIND>>;
    const int ntg = (n_inst + kGG - 1) / kGG;
    const long long total = (long long)rows * ntg * kGG * GD::K;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int k = (int)(t % GD::K);
    const int g = (int)((t / GD::K) % kGG);
    const int gb = (int)((t / ((long long)GD::K * kGG)) % ntg);
    const int r = (int)(t / ((long long)GD::K * kGG * ntg));
    pack_group_elem<D, NN, KIND>(inst, n_inst, nG, zero_idx, perm, Bpack, ntg, r, gb, g, k);
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
    if (kind == KD && d == DD && n == NNN) return (long long)GroupDims<FullTree<DD, NNN, KD>>::block_bytes / 2;
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
            inst, n_inst, nG, zero_idx, perm, static_cast<uint8_t*>(Apack), rows);                         \
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
        constexpr size_t smb = sizeof(GroupSmem<FullTree<DD, NNN, KD>, DD>) + 1024; /* + alignment slack */ \
        auto kern = k_paths_group<DD, NNN, KD>;                                                               \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);    \
        if (e != cudaSuccess) return e;                                                                      \
        const long long blocks = (long long)tiles * P.N * ntg;                                               \
        kern<<<(unsigned)blocks, kGBS, smb, st>>>(P, inst, n_inst, static_cast<const uint8_t*>(Apack), tiles,  \
                                                  status);                                                  \
        return cudaGetLastError();                                                                           \
    }
    QR_GROUP_SETS(QR_X)
#undef QR_X
    return cudaErrorInvalidValue;
}

}  // namespace qr
