// qr_cosine.cu -- direct kernels of the cosine basis (Sec. 2.2, Lemma
// ortho:dim1) on an N^d index set.
//
// phi_k(x) = prod_l C_{k_l}(F_nu(x_l)), C_0 = 1, C_a(u) = sqrt(2) cos(a pi u).
// Every lane keeps the real table C_a(u_l), a < K1p, of its point in shared
// memory (a column per lane, from the powers of z_l = e^{i pi u_l}, whose real
// parts are cos(a pi u_l)). Along the runs of Gamma (entries sharing
// k_1..k_{d-1}, with k_d = 0, 1, ...) the basis value is the run's prefix
// product times C_{k_d}(u_d), so
//   series      ybar(x) = sum_runs prefix(x) * sum_a c_{run,a} C_a(u_d)
//               (one FMA and one table read per coefficient, a prefix
//               product per run),
//   projection  a_k = (1/M) sum_m S^m phi_k(U^m), eq. (Aqi:bar:M), in tiles
//               of 32 packed positions whose lane values are reduced over the
//               warp by a 31-shuffle reduce-scatter.
// Coefficient rows are real (half the bytes of the complex Fourier rows) and
// Gamma is used as it is (no sign unfolding: 2^{d'} fewer entries). Responses
// (damping, truncation, driver, compensated sums), the bulk-copy staging of
// the next row and the bounded waits follow the generic path kernel.
#include "qr_cosine.h"
#include "qr_device.cuh"

#include <algorithm>

namespace qr {

namespace {

__host__ __device__ __forceinline__ size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

// four consecutive coefficients of a packed row (16-byte aligned groups)
template <typename R>
__device__ __forceinline__ void ld4(const R* p, R& a, R& b, R& c, R& d);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float& a, float& b, float& c, float& d)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x;
    b = v.y;
    c = v.z;
    d = v.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double& a, double& b, double& c, double& d)
{
    const double2 u = *reinterpret_cast<const double2*>(p), v = *reinterpret_cast<const double2*>(p + 2);
    a = u.x;
    b = u.y;
    c = v.x;
    d = v.y;
}

// C_a(u_l), a < K1p, into the lane's column t (stride BS) from z_l = e^{i pi u_l}
template <typename R, int D, int BS>
__device__ __forceinline__ void fill_cos(R* t, int K1p, const V2<R> (&z)[D])
{
    const R r2 = (R)1.4142135623730951;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        R* tl = t + (size_t)l * K1p * BS;
        V2<R> p = z[l];
        tl[0] = (R)1;
        for (int a = 1; a < K1p; ++a) {
            tl[(size_t)a * BS] = r2 * p.x;
            p = cmul<R>(p, z[l]);
        }
    }
}

// b[l] = b0 prod_{l' <= l} C_{k_l'}(u_l') for the prefix dimensions l = f .. d-2
// (the lower ones are unchanged); returns b[d-2] (b0 when d = 1)
template <typename R, int D, int BS>
__device__ __forceinline__ R prefix_update(R (&b)[D], R b0, int f, uint32_t kz, uint32_t kw, const R* t, int K1p)
{
    if constexpr (D == 1) {
        return b0;
    } else {
        if (f == D - 2) {  // the common case: only the last prefix coordinate changed
            constexpr int l = D - 2;
            const int kl = (int)(((l < 4 ? kz : kw) >> (8 * (l & 3))) & 0xffu);
            b[l] = (l == 0 ? b0 : b[l == 0 ? 0 : l - 1]) * t[((size_t)l * K1p + kl) * BS];
        } else {
#pragma unroll
            for (int l = 0; l < D - 1; ++l)
                if (l >= f) {
                    const int kl = (int)(((l < 4 ? kz : kw) >> (8 * (l & 3))) & 0xffu);
                    b[l] = (l == 0 ? b0 : b[l == 0 ? 0 : l - 1]) * t[((size_t)l * K1p + kl) * BS];
                }
        }
        return b[D - 2];
    }
}

// sum_k c_k phi_k at the lane's point; c: packed real row (groups of 4)
template <typename R, int D, int BS>
__device__ __forceinline__ R cos_series(const R* __restrict__ c, const CosGroup* __restrict__ G, int ng, const R* t,
                                        int K1p)
{
    R b[D];
    R p = (R)1, acc = (R)0, s0 = (R)0, s1 = (R)0;
    const R* tl = t + (size_t)(D - 1) * K1p * BS;
    for (int g = 0; g < ng; ++g) {
        const uint4 q = __ldg(G + g);
        const int a0 = (int)(q.x & 0xffffu), f = (int)(q.x >> 16);
        if (D > 1 && f < D - 1) {  // a new run: close the previous one, new prefix product
            acc = fma(p, s0 + s1, acc);
            s0 = (R)0;
            s1 = (R)0;
            p = prefix_update<R, D, BS>(b, (R)1, f, q.z, q.w, t, K1p);
        }
        R c0, c1, c2, c3;
        ld4<R>(c + 4 * (size_t)g, c0, c1, c2, c3);
        const R* ta = tl + (size_t)a0 * BS;
        s0 = fma(c0, ta[0], s0);
        s1 = fma(c1, ta[BS], s1);
        s0 = fma(c2, ta[2 * BS], s0);
        s1 = fma(c3, ta[3 * BS], s1);
    }
    return fma(p, s0 + s1, acc);
}

// reduce-scatter of 32 values over the warp: lane L returns the lane sum of v[L]
template <typename R>
__device__ __forceinline__ R cos_fold32(R (&v)[32], int lane)
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

template <typename R>
__host__ __device__ size_t cos_table_bytes(int d, int K1p, int BS)
{
    return al16((size_t)d * K1p * BS * sizeof(R));
}

// path kernel: tables, then (CG = false) two coefficient rows and two barriers
template <typename R>
size_t cos_paths_smem(int d, int K1p, long long row_stride, int BS, bool cg)
{
    return cos_table_bytes<R>(d, K1p, BS) + (cg ? 0 : 2 * al16((size_t)row_stride * sizeof(R)) + 16);
}

}  // namespace

// ------------------------------------------------------ path-and-series kernel
// CG: the coefficient rows are read from global memory (L1/L2-resident,
// warp-uniform) when two of them do not fit beside the tables
template <typename R, int D, int BS, bool CG>
__global__ void __launch_bounds__(BS) k_paths_cos(const __grid_constant__ QrParams P,
                                                  const CosGroup* __restrict__ G, int ng,
                                                  const R* __restrict__ packed, long long row_stride,
                                                  R* __restrict__ S, int i_lo, int tiles_per_i,
                                                  unsigned long long* __restrict__ counters,
                                                  unsigned* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int K1p = P.K1, N = P.N;
    const size_t tb = cos_table_bytes<R>(D, K1p, BS);
    const uint32_t rowbytes = (uint32_t)al16((size_t)row_stride * sizeof(R));
    R* tab = reinterpret_cast<R*>(smem);
    R* abuf[2] = {reinterpret_cast<R*>(smem + tb), reinterpret_cast<R*>(smem + tb + rowbytes)};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tb + 2 * (size_t)rowbytes);

    const int tid = threadIdx.x;
    const int i = i_lo + (int)(blockIdx.x / tiles_per_i);
    const long long m = (long long)(blockIdx.x % tiles_per_i) * BS + tid;
    const bool active = m < P.M;
    const bool trig = P.g_kind == QR_GT_TRIGPOLY;
    if (!CG) {
        if (tid == 0) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }

    // rows i+1 .. N are read as series (row N only for a polynomial g)
    bool inflight[2] = {false, false};
    uint32_t phase[2] = {0u, 0u};
    if (!CG && (i + 1 < N || (i + 1 == N && trig))) {
        if (tid == 0) bulk_load(abuf[0], packed + (size_t)(i + 1) * row_stride, rowbytes, &bars[0]);
        inflight[0] = true;
    }
    R x[D];
    {
        V2<R> unused[D];
        start_point<R, D>(P, i, m, x, unused, false);
    }
    const bool damp = P.q_damp != 0.0;
    const R qh = (R)(0.5 * P.q_damp);
    const R lw0 = damp ? damp_logw<R, D>(qh, x) : (R)0;  // log w(X_i^i)
    R sum = 0, comp = 0, gN = 0;
    unsigned long long hits = 0;
    R* mytab = tab + tid;
    const R dt = (R)P.dt;

    for (int j = i; j < N; ++j) {
        const int buf = (j - i) & 1, row = j + 1;
        const bool use_series = row < N || trig;
        const int nrow = row + 1;
        if (!CG && (nrow < N || (nrow == N && trig))) {
            // the other buffer was last read at the previous step, which
            // ended with a block barrier
            if (tid == 0) {
                fence_proxy_async_smem();
                bulk_load(abuf[buf ^ 1], packed + (size_t)nrow * row_stride, rowbytes, &bars[buf ^ 1]);
            }
            inflight[buf ^ 1] = true;
        }
        R z[D], x1[D];
        normals<R, D>(P, i, (uint32_t)m, j, z);
        euler<R, D>(P, x, z, x1);
        R y;
        if (use_series) {
            const R* crow = packed + (size_t)row * row_stride;
            if (!CG) {
                const bool ok = mbar_wait(&bars[buf], phase[buf]);
                phase[buf] ^= 1u;
                inflight[buf] = false;
                if (!__syncthreads_and(ok)) {
                    if (tid == 0) {
                        atomicOr(status, ST_TIMEOUT);
                        if (inflight[buf ^ 1]) (void)mbar_wait(&bars[buf ^ 1], phase[buf ^ 1]);
                    }
                    __syncthreads();
                    return;
                }
                crow = abuf[buf];
            }
            V2<R> zz[D];
#pragma unroll
            for (int l = 0; l < D; ++l) zz[l] = nu_phase<R>(P, x1[l]);  // e^{i pi F(x)} (half angle)
            fill_cos<R, D, BS>(mytab, K1p, zz);
            y = cos_series<R, D, BS>(crow, G, ng, mytab, K1p);
            if (damp && row < N) y = undamp<R>(y, damp_logw<R, D>(qh, x1));  // y = ybar^q w(X_{j+1})
            if (row < N && P.clamp_L > 0.0) {
                const R L = (R)P.clamp_L;
                if (y > L) {
                    y = L;
                    ++hits;
                } else if (y < -L) {
                    y = -L;
                    ++hits;
                }
            }
        } else {
            y = term_g<R, D>(P, x1);
        }
        if (row == N) gN = y;
        // S += f(t_j, X_j, y_{j+1}) dt, compensated
        const R term = drv_f<R, D>(P, j, x, y) * dt;
        const R yk = term - comp;
        const R tk = sum + yk;
        comp = (tk - sum) - yk;
        sum = tk;
#pragma unroll
        for (int l = 0; l < D; ++l) x[l] = x1[l];
        if (!CG) __syncthreads();
    }
    // S^q_i = [g(X_N) + sum_j f dt] / w(X_i^i), eq. (Sqi:bar:M)
    const R Sv = damp ? (gN + sum) * (R)exp((double)-lw0) : gN + sum;
    unsigned long long bad = 0;
    if (active) {
        S[(size_t)(i - i_lo) * (size_t)P.M + (size_t)m] = Sv;
        if (!isfinite(Sv)) bad = 1;
    } else {
        hits = 0;
    }
    hits = warp_sum_ull(hits);
    bad = warp_sum_ull(bad);
    if ((tid & 31) == 0) {
        if (hits) atomicAdd(&counters[CNT_CLAMP], hits);
        if (bad) atomicAdd(&counters[CNT_NONFINITE], bad);
    }
}

// --------------------------------------------------------- projection kernel
// One CTA: row i, a chunk of P.chunk paths, a pass of KT packed positions
// (a multiple of 32). Per round of BS paths every lane builds its table and
// walks the pass with the prefix chain started at S^m, so that the chain's
// last value is S^m phi_k(U^m); per tile of 32 positions the lane values are
// reduce-scattered over the warp and added to the warp's accumulators in
// shared memory, which are summed in fixed warp order at the end.
template <typename R, int D, int BS>
__global__ void __launch_bounds__(BS) k_project_cos(const __grid_constant__ QrParams P,
                                                    const CosGroup* __restrict__ G, int ngroups,
                                                    const R* __restrict__ S, double* __restrict__ partial,
                                                    long long row_stride, int i_lo, int KT, int passes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int W = BS / 32;
    const int K1p = P.K1;
    R* tab = reinterpret_cast<R*>(smem);
    R* wacc = reinterpret_cast<R*>(smem + cos_table_bytes<R>(D, K1p, BS));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int per_row = P.n_chunks * passes;
    const int ii = (int)(blockIdx.x / per_row), rem = (int)(blockIdx.x % per_row);
    const int ps = rem / P.n_chunks, ch = rem % P.n_chunks;
    const int i = i_lo + ii;
    const int gs = ps * (KT / 4);
    const int ge = min(ngroups, gs + KT / 4);  // both multiples of 8
    R* myacc = wacc + (size_t)warp * KT;
    for (int q = lane; q < KT; q += 32) myacc[q] = (R)0;
    __syncwarp();

    R* mytab = tab + tid;
    const R* tl = mytab + (size_t)(D - 1) * K1p * BS;
    const int rounds = P.chunk / BS;
    for (int r = 0; r < rounds; ++r) {
        const long long m = (long long)ch * P.chunk + (long long)r * BS + tid;
        const bool active = m < P.M;
        const R Sv = active ? S[(size_t)ii * (size_t)P.M + (size_t)m] : (R)0;
        V2<R> ph[D];
        start_phases_dev<R, D>(P, i, active ? m : 0, ph);  // e^{i pi U^m} (half angle)
        fill_cos<R, D, BS>(mytab, K1p, ph);
        R b[D];
        const uint4 q0 = __ldg(G + gs);
        R p = prefix_update<R, D, BS>(b, Sv, 0, q0.z, q0.w, mytab, K1p);
        for (int g0 = gs; g0 < ge; g0 += 8) {
            R v[32];
#pragma unroll
            for (int gg = 0; gg < 8; ++gg) {
                const uint4 q = __ldg(G + g0 + gg);
                const int a0 = (int)(q.x & 0xffffu), f = (int)(q.x >> 16);
                if (D > 1 && f < D - 1) p = prefix_update<R, D, BS>(b, Sv, f, q.z, q.w, mytab, K1p);
                const R* ta = tl + (size_t)a0 * BS;
                v[4 * gg + 0] = p * ta[0];
                v[4 * gg + 1] = p * ta[BS];
                v[4 * gg + 2] = p * ta[2 * BS];
                v[4 * gg + 3] = p * ta[3 * BS];
            }
            const R s = cos_fold32<R>(v, lane);
            myacc[(g0 - gs) * 4 + lane] += s;
        }
    }
    __syncthreads();
    const int npos = (ge - gs) * 4;
    double* out = partial + ((size_t)ii * P.n_chunks + ch) * (size_t)row_stride + (size_t)gs * 4;
    for (int q = tid; q < npos; q += BS) {
        double s = 0.0;
        for (int w = 0; w < W; ++w) s += (double)wacc[(size_t)w * KT + q];
        out[q] = s;
    }
}

// fixed-order sum over chunks, / M, into alpha (real part) and the packed row; residual
template <typename R>
__global__ void k_reduce_cos(const __grid_constant__ QrParams P, const double* __restrict__ partial,
                             const int* __restrict__ pos, double2* __restrict__ alpha, R* __restrict__ packed,
                             long long row_stride, int i_lo, int i_hi, unsigned long long* __restrict__ counters)
{
    const int nG = P.nGp;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)(i_hi - i_lo) * nG;
    double diff = 0.0;
    if (idx < total) {
        const int ii = (int)(idx / nG), e = (int)(idx % nG), i = i_lo + ii;
        const double* p = partial + (size_t)ii * P.n_chunks * (size_t)row_stride + pos[e];
        double s = 0.0;
        for (int c = 0; c < P.n_chunks; ++c) s += p[(size_t)c * row_stride];
        s /= (double)P.M;
        double2* a = alpha + (size_t)i * nG + e;
        diff = fabs(s - a->x);
        *a = make_double2(s, 0.0);
        packed[(size_t)i * row_stride + pos[e]] = (R)s;
    }
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_xor_sync(0xffffffffu, diff, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = diff;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        atomicMax(&counters[CNT_RESID], (unsigned long long)__double_as_longlong(mx));
    }
}

template <typename R>
__global__ void k_pack_cos(const double2* __restrict__ alpha, int nG, const int* __restrict__ pos,
                           R* __restrict__ packed, long long row_stride, int rows)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * nG) return;
    const int i = (int)(idx / nG), e = (int)(idx % nG);
    packed[(size_t)i * row_stride + pos[e]] = (R)alpha[(size_t)i * nG + e].x;
}

template <typename R, int D, int BS>
__global__ void __launch_bounds__(BS) k_eval_cos(const __grid_constant__ QrParams P, const CosGroup* __restrict__ G,
                                                 int ng, const R* __restrict__ crow, const double* __restrict__ xs,
                                                 long long n, double* __restrict__ ys, int use_g)
{
    extern __shared__ __align__(16) unsigned char smem[];
    R* tab = reinterpret_cast<R*>(smem);
    const long long p = (long long)blockIdx.x * BS + threadIdx.x;
    if (p >= n) return;
    R x[D];
#pragma unroll
    for (int l = 0; l < D; ++l) x[l] = (R)xs[p * D + l];
    if (use_g) {
        ys[p] = (double)term_g<R, D>(P, x);
        return;
    }
    V2<R> zz[D];
#pragma unroll
    for (int l = 0; l < D; ++l) zz[l] = nu_phase<R>(P, x[l]);
    R* mytab = tab + threadIdx.x;
    fill_cos<R, D, BS>(mytab, P.K1, zz);
    ys[p] = (double)cos_series<R, D, BS>(crow, G, ng, mytab, P.K1);
}

// ------------------------------------------------------------ launchers
namespace {

constexpr size_t kCap = 227 * 1024;

template <typename R, int D, int BS, bool CG>
cudaError_t paths_cos_bs(const QrParams& P, const CosGroup* G, int ng, const void* packed, long long row_stride,
                         void* S, int i_lo, int i_hi, unsigned long long* counters, unsigned* status, cudaStream_t st)
{
    const size_t sm = cos_paths_smem<R>(D, P.K1, row_stride, BS, CG);
    if (sm > kCap) return cudaErrorInvalidConfiguration;
    auto kern = k_paths_cos<R, D, BS, CG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int tiles = (int)((P.M + BS - 1) / BS);
    const long long blocks = (long long)tiles * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, G, ng, static_cast<const R*>(packed), row_stride, static_cast<R*>(S),
                                           i_lo, tiles, counters, status);
    return cudaGetLastError();
}

// 128-thread blocks with both coefficient rows in shared memory when they fit
// beside the tables, else rows from global memory; 64 threads when the
// tables alone do not fit 128 lanes
template <typename R, int D>
cudaError_t paths_cos_t(const QrParams& P, const CosGroup* G, int ng, const void* packed, long long row_stride,
                        void* S, int i_lo, int i_hi, unsigned long long* counters, unsigned* status, cudaStream_t st)
{
    if (cos_paths_smem<R>(D, P.K1, row_stride, 128, false) <= kCap)
        return paths_cos_bs<R, D, 128, false>(P, G, ng, packed, row_stride, S, i_lo, i_hi, counters, status, st);
    if (cos_paths_smem<R>(D, P.K1, row_stride, 128, true) <= kCap)
        return paths_cos_bs<R, D, 128, true>(P, G, ng, packed, row_stride, S, i_lo, i_hi, counters, status, st);
    return paths_cos_bs<R, D, 64, true>(P, G, ng, packed, row_stride, S, i_lo, i_hi, counters, status, st);
}

template <typename R, int D, int BS>
cudaError_t project_cos_bs(const QrParams& P, const CosGroup* G, int ngroups, const void* S, double* partial,
                           long long row_stride, int i_lo, int i_hi, cudaStream_t st)
{
    constexpr int W = BS / 32;
    const size_t tb = cos_table_bytes<R>(D, P.K1, BS);
    if (tb + (size_t)W * 32 * sizeof(R) > kCap) return cudaErrorInvalidConfiguration;
    // about 3 CTAs per SM where the tables allow it, else at least 1024
    // positions per pass (every pass rebuilds the tables of all its paths)
    const size_t budget = std::min(kCap, std::max((size_t)76 * 1024, tb + (size_t)W * 1024 * sizeof(R)));
    long long KT = (long long)((budget - tb) / (W * sizeof(R))) & ~31ll;
    if (KT > row_stride) KT = row_stride;
    const int passes = (int)((row_stride + KT - 1) / KT);
    const size_t sm = tb + (size_t)W * KT * sizeof(R);
    auto kern = k_project_cos<R, D, BS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)P.n_chunks * passes * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, G, ngroups, static_cast<const R*>(S), partial, row_stride, i_lo,
                                           (int)KT, passes);
    return cudaGetLastError();
}

template <typename R, int D>
cudaError_t project_cos_t(const QrParams& P, const CosGroup* G, int ngroups, const void* S, double* partial,
                          long long row_stride, int i_lo, int i_hi, cudaStream_t st)
{
    if (cos_table_bytes<R>(D, P.K1, 128) + 4 * 32 * sizeof(R) <= kCap)
        return project_cos_bs<R, D, 128>(P, G, ngroups, S, partial, row_stride, i_lo, i_hi, st);
    return project_cos_bs<R, D, 64>(P, G, ngroups, S, partial, row_stride, i_lo, i_hi, st);
}

template <typename R, int D, int BS>
cudaError_t eval_cos_bs(const QrParams& P, const CosGroup* G, int ng, const void* row, const double* x, long long n,
                        double* y, int use_g, cudaStream_t st)
{
    const size_t sm = cos_table_bytes<R>(D, P.K1, BS);
    if (sm > kCap) return cudaErrorInvalidConfiguration;
    auto kern = k_eval_cos<R, D, BS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    kern<<<(unsigned)((n + BS - 1) / BS), BS, sm, st>>>(P, G, ng, static_cast<const R*>(row), x, n, y, use_g);
    return cudaGetLastError();
}

template <typename R, int D>
cudaError_t eval_cos_t(const QrParams& P, const CosGroup* G, int ng, const void* row, const double* x, long long n,
                       double* y, int use_g, cudaStream_t st)
{
    if (cos_table_bytes<R>(D, P.K1, 128) <= kCap) return eval_cos_bs<R, D, 128>(P, G, ng, row, x, n, y, use_g, st);
    return eval_cos_bs<R, D, 64>(P, G, ng, row, x, n, y, use_g, st);
}

}  // namespace

#define QR_COS_DISPATCH(FN, R, ...)        \
    switch (P.d) {                         \
    case 1: return FN<R, 1>(__VA_ARGS__);  \
    case 2: return FN<R, 2>(__VA_ARGS__);  \
    case 3: return FN<R, 3>(__VA_ARGS__);  \
    case 4: return FN<R, 4>(__VA_ARGS__);  \
    case 5: return FN<R, 5>(__VA_ARGS__);  \
    case 6: return FN<R, 6>(__VA_ARGS__);  \
    case 7: return FN<R, 7>(__VA_ARGS__);  \
    case 8: return FN<R, 8>(__VA_ARGS__);  \
    default: return cudaErrorInvalidValue; \
    }

size_t cos_paths_smem_min(int prec, int d, int K1p)
{
    const size_t sm = prec == QR_FP32 ? cos_paths_smem<float>(d, K1p, 0, 64, true)
                                      : cos_paths_smem<double>(d, K1p, 0, 64, true);
    return sm <= kCap ? sm : 0;
}

cudaError_t launch_paths_cos(int prec, const QrParams& P, const CosGroup* groups, int ngroups, const void* packed,
                             long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                             unsigned* status, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_COS_DISPATCH(paths_cos_t, float, P, groups, ngroups, packed, row_stride, S, i_lo, i_hi, counters, status,
                        st)
    }
    QR_COS_DISPATCH(paths_cos_t, double, P, groups, ngroups, packed, row_stride, S, i_lo, i_hi, counters, status, st)
}

cudaError_t launch_project_cos(int prec, const QrParams& P, const CosGroup* groups, int ngroups, const void* S,
                               double* partial, long long row_stride, int i_lo, int i_hi, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_COS_DISPATCH(project_cos_t, float, P, groups, ngroups, S, partial, row_stride, i_lo, i_hi, st)
    }
    QR_COS_DISPATCH(project_cos_t, double, P, groups, ngroups, S, partial, row_stride, i_lo, i_hi, st)
}

cudaError_t launch_reduce_cos(int prec, const QrParams& P, const double* partial, const int* pos, double2* alpha,
                              void* packed, long long row_stride, int i_lo, int i_hi, unsigned long long* counters,
                              cudaStream_t st)
{
    const long long total = (long long)(i_hi - i_lo) * P.nGp;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (prec == QR_FP32)
        k_reduce_cos<float><<<blocks, 256, 0, st>>>(P, partial, pos, alpha, static_cast<float*>(packed), row_stride,
                                                    i_lo, i_hi, counters);
    else
        k_reduce_cos<double><<<blocks, 256, 0, st>>>(P, partial, pos, alpha, static_cast<double*>(packed), row_stride,
                                                     i_lo, i_hi, counters);
    return cudaGetLastError();
}

cudaError_t launch_pack_cos(int prec, const double2* alpha, int nG, const int* pos, void* packed,
                            long long row_stride, int rows, cudaStream_t st)
{
    const long long total = (long long)rows * nG;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (prec == QR_FP32)
        k_pack_cos<float><<<blocks, 256, 0, st>>>(alpha, nG, pos, static_cast<float*>(packed), row_stride, rows);
    else
        k_pack_cos<double><<<blocks, 256, 0, st>>>(alpha, nG, pos, static_cast<double*>(packed), row_stride, rows);
    return cudaGetLastError();
}

cudaError_t launch_eval_cos(int prec, const QrParams& P, const CosGroup* groups, int ngroups, const void* packed_row,
                            const double* x, long long n, double* y, int use_g, cudaStream_t st)
{
    if (prec == QR_FP32) {
        QR_COS_DISPATCH(eval_cos_t, float, P, groups, ngroups, packed_row, x, n, y, use_g, st)
    }
    QR_COS_DISPATCH(eval_cos_t, double, P, groups, ngroups, packed_row, x, n, y, use_g, st)
}

}  // namespace qr
