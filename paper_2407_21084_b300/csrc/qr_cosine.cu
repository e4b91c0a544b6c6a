// qr_cosine.cu -- direct kernels of the cosine basis (Sec. 2.2, Lemma
// ortho:dim1) on an N^d index set.
//
// phi_k(x) = prod_l C_{k_l}(F_nu(x_l)), C_0 = 1, C_a(u) = sqrt(2) cos(a pi u)
// = sqrt(2) Re z^a with z = e^{i pi u}. Along the runs of Gamma (entries
// sharing k_1..k_{d-1}, with k_d = 0, 1, ...) the basis value is the run's
// prefix product times C_{k_d}(u_d), and every factor is reached from the
// previous one by one complex product (see CosWalk), so
//   series      ybar(x) = sum_runs prefix(x) * sum_a c_{run,a} C_a(u_d):
//               per coefficient one FMA and Re(P z^j) (two FMAs), per group of
//               four one complex product, per run a prefix update;
//   projection  a_k = (1/M) sum_m S^m phi_k(U^m), eq. (Aqi:bar:M), in tiles
//               of 32 packed positions whose lane values are reduced over the
//               warp by a 31-shuffle reduce-scatter.
// Everything per lane lives in registers (no per-lane tables), coefficient
// rows are real (half the bytes of the complex Fourier rows) and Gamma is
// used as it is (no sign unfolding: 2^{d'} fewer entries). Responses
// (damping, truncation, driver, compensated sums), the bulk-copy staging of
// the next row and the bounded waits follow the generic path kernel.
#include "qr_cosine.h"
#include "qr_device.cuh"

#include <algorithm>

namespace qr {

constexpr int kCosBS = 128;

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

// Walk of one lane along Gamma in canonical order. For downward-closed sets
// listed lexicographically, the prefix of a new run differs from the previous
// one in one coordinate f, which grows by one, while the prefix coordinates
// after f go back to 0 (checked on the host). So every factor is a power of
// z_l = e^{i pi u_l} reached by one complex product from the previous one:
// C_k(u_l) = sqrt(2) Re z_l^k (k >= 1), C_0 = 1; no tables.
template <typename R, int D>
struct CosWalk {
    static constexpr int DP = D > 1 ? D - 1 : 1;
    V2<R> z[D];        // e^{i pi u_l}
    V2<R> w[DP];       // sqrt(2) z_l^{k_l} of the current prefix
    R b[DP];           // b0 prod_{l' <= l} C_{k_l'}(u_l')
    V2<R> z2, z3, z4;  // powers of the last coordinate's phase
    V2<R> P;           // sqrt(2) z_d^a for the next group of the current run
    R p;               // the current run's factor b0 prod_prefix C

    // the walk before the first run (all prefix coordinates 0)
    __device__ __forceinline__ void init(const V2<R> (&ph)[D], R b0)
    {
#pragma unroll
        for (int l = 0; l < D; ++l) z[l] = ph[l];
        const V2<R> zl = z[D - 1];
        z2 = cmul<R>(zl, zl);
        z3 = cmul<R>(z2, zl);
        z4 = cmul<R>(z2, z2);
#pragma unroll
        for (int l = 0; l < DP; ++l) {
            b[l] = b0;
            w[l] = mk2<R>((R)1.4142135623730951, (R)0);
        }
        P = z4;
        p = b0;
    }

    // prefix coordinate L one up, the later prefix coordinates back to 0
    template <int L>
    __device__ __forceinline__ void step(R b0)
    {
        w[L] = cmul<R>(w[L], z[L]);
        b[L] = (L == 0 ? b0 : b[L == 0 ? 0 : L - 1]) * w[L].x;
#pragma unroll
        for (int l = L + 1; l < D - 1; ++l) {
            w[l] = mk2<R>((R)1.4142135623730951, (R)0);
            b[l] = b[L];
        }
        p = b[D - 2];
    }

    __device__ __forceinline__ void new_run(int f, R b0)
    {
        if constexpr (D > 1) {
            if (f == D - 2) {  // the common case: the last prefix coordinate
                step<D - 2>(b0);
            } else {
                step_at<0>(f, b0);
            }
        }
    }
    template <int L>
    __device__ __forceinline__ void step_at(int f, R b0)
    {
        if constexpr (L < D - 2) {
            if (f == L)
                step<L>(b0);
            else
                step_at<L + 1>(f, b0);
        }
    }

    // prefix k_1..k_{d-1} from scratch (bytes of kz, kw) and the last
    // coordinate at a0: the state before the group that starts at a0
    __device__ __forceinline__ void seek(uint32_t kz, uint32_t kw, uint32_t ky, int a0, R b0)
    {
        const R r2 = (R)1.4142135623730951;
        if constexpr (D > 1) {
#pragma unroll
            for (int l = 0; l < D - 1; ++l) {
                const int k = (int)(((l < 4 ? kz : (l < 8 ? kw : ky)) >> (8 * (l & 3))) & 0xffu);
                V2<R> v = mk2<R>(r2, (R)0);
                for (int t = 0; t < k; ++t) v = cmul<R>(v, z[l]);
                w[l] = v;
                const R below = l == 0 ? b0 : b[l == 0 ? 0 : l - 1];
                b[l] = k == 0 ? below : below * v.x;
            }
            p = b[D - 2];
        } else {
            p = b0;
        }
        if (a0 > 0) {
            V2<R> v = mk2<R>(r2, (R)0);
            for (int t = 0; t < a0; ++t) v = cmul<R>(v, z[D - 1]);
            P = v;
        }
    }

    // C_{a+j}(u_d), j < 4, of the current run's next group (a = 0 when
    // start); P moves on to a + 4
    __device__ __forceinline__ void values(bool start, R& v0, R& v1, R& v2, R& v3)
    {
        const R r2 = (R)1.4142135623730951;
        const V2<R> zl = z[D - 1];
        if (start) {
            v0 = (R)1;
            v1 = r2 * zl.x;
            v2 = r2 * z2.x;
            v3 = r2 * z3.x;
            P = mk2<R>(r2 * z4.x, r2 * z4.y);
        } else {
            v0 = P.x;
            v1 = fma(P.x, zl.x, -P.y * zl.y);
            v2 = fma(P.x, z2.x, -P.y * z2.y);
            v3 = fma(P.x, z3.x, -P.y * z3.y);
            P = cmul<R>(P, z4);
        }
    }
};

template <typename R>
__device__ __forceinline__ uint32_t word_of(const uint4& v, int h)
{
    return h == 0 ? v.x : (h == 1 ? v.y : (h == 2 ? v.z : v.w));
}

// sum_k c_k phi_k at the walk's point; c: packed real row (groups of 4),
// flags: one byte per group (bit 7: a run starts, bits 0-3: its first
// changed prefix coordinate, d-1 for none), ng a multiple of 16
template <typename R, int D>
__device__ __forceinline__ R cos_series(const R* __restrict__ c, const uint4* __restrict__ flags, int ng,
                                        CosWalk<R, D>& W)
{
    R acc = (R)0, s0 = (R)0, s1 = (R)0;
    for (int g0 = 0; g0 < ng; g0 += 16) {
        const uint4 fl = __ldg(flags + g0 / 16);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            // the coefficients of four groups first, then their values
            R cc[16];
#pragma unroll
            for (int t = 0; t < 4; ++t)
                ld4<R>(c + 4 * (size_t)(g0 + 4 * h + t), cc[4 * t], cc[4 * t + 1], cc[4 * t + 2], cc[4 * t + 3]);
            const uint32_t fw = word_of<R>(fl, h);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t fb = (fw >> (8 * t)) & 0xffu;
                const bool start = (fb & 0x80u) != 0;
                if (start) {  // close the previous run
                    acc = fma(W.p, s0 + s1, acc);
                    s0 = (R)0;
                    s1 = (R)0;
                    if (D > 1 && (int)(fb & 15u) < D - 1) W.new_run((int)(fb & 15u), (R)1);
                }
                R v0, v1, v2, v3;
                W.values(start, v0, v1, v2, v3);
                s0 = fma(cc[4 * t], v0, s0);
                s1 = fma(cc[4 * t + 1], v1, s1);
                s0 = fma(cc[4 * t + 2], v2, s0);
                s1 = fma(cc[4 * t + 3], v3, s1);
            }
        }
    }
    return fma(W.p, s0 + s1, acc);
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

// path kernel: two coefficient rows and two barriers (none when CG)
template <typename R>
size_t cos_paths_smem(long long row_stride, bool cg)
{
    return cg ? 0 : 2 * al16((size_t)row_stride * sizeof(R)) + 16;
}

}  // namespace

// ------------------------------------------------------ path-and-series kernel
// CG: the coefficient rows are read from global memory (L1/L2-resident,
// warp-uniform loads) instead of being staged in shared memory, for rows too
// long to keep several blocks per SM
template <typename R, int D, bool CG>
__global__ void __launch_bounds__(kCosBS, sizeof(R) == 4 ? 4 : 2) k_paths_cos(const __grid_constant__ QrParams P,
                                                         const uint4* __restrict__ flags, int ng,
                                                         const R* __restrict__ packed, long long row_stride,
                                                         R* __restrict__ S, int i_lo, int tiles_per_i,
                                                         unsigned long long* __restrict__ counters,
                                                         unsigned* __restrict__ status)
{
    constexpr int BS = kCosBS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = P.N;
    const uint32_t rowbytes = (uint32_t)al16((size_t)row_stride * sizeof(R));
    R* abuf[2] = {reinterpret_cast<R*>(smem), reinterpret_cast<R*>(smem + rowbytes)};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * (size_t)rowbytes);

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
    // buffer state in registers, selected by the step parity (indexed arrays
    // would live in local memory)
    bool infl0 = false, infl1 = false;
    uint32_t par0 = 0u, par1 = 0u;
    if (!CG && (i + 1 < N || (i + 1 == N && trig))) {
        if (tid == 0) bulk_load(abuf[0], packed + (size_t)(i + 1) * row_stride, rowbytes, &bars[0]);
        infl0 = true;
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
                bulk_load((buf ? abuf[0] : abuf[1]), packed + (size_t)nrow * row_stride, rowbytes, &bars[buf ^ 1]);
            }
            if (buf) infl0 = true;
            else infl1 = true;
        }
        R z[D], x1[D];
        normals<R, D>(P, i, (uint32_t)m, j, z);
        euler<R, D>(P, x, z, x1);
        R y;
        if (use_series) {
            const R* crow = packed + (size_t)row * row_stride;
            if (!CG) {
                const bool ok = mbar_wait(&bars[buf], buf ? par1 : par0);
                if (buf) {
                    par1 ^= 1u;
                    infl1 = false;
                } else {
                    par0 ^= 1u;
                    infl0 = false;
                }
                if (!__syncthreads_and(ok)) {
                    if (tid == 0) {
                        atomicOr(status, ST_TIMEOUT);
                        if (buf ? infl0 : infl1) (void)mbar_wait(&bars[buf ^ 1], buf ? par0 : par1);
                    }
                    __syncthreads();
                    return;
                }
                crow = (buf ? abuf[1] : abuf[0]);
            }
            V2<R> zz[D];
#pragma unroll
            for (int l = 0; l < D; ++l) zz[l] = nu_phase<R>(P, x1[l]);  // e^{i pi F(x)} (half angle)
            CosWalk<R, D> W;
            W.init(zz, (R)1);
            y = cos_series<R, D>(crow, flags, ng, W);
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
        if (in_bounds(P, i - i_lo >= 0 && i - i_lo < P.N)) S[(size_t)(i - i_lo) * (size_t)P.M + (size_t)m] = Sv;
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
// (a multiple of 32). Per round of PPL*BS paths every lane walks the pass
// with PPL paths, their factors started at S^m, so that the walks' values
// are S^m phi_k(U^m); per tile of 32 positions the lane's sums over its
// paths are reduce-scattered over the warp (one 31-shuffle fold for PPL
// paths) and added to the warp's accumulators in shared memory, which are
// summed in fixed warp order at the end.
template <typename R, int D, int PPL>
__global__ void __launch_bounds__(kCosBS, PPL == 2 ? 3 : (sizeof(R) == 4 ? 4 : 2))
    k_project_cos(const __grid_constant__ QrParams P,
                                                           const CosGroup* __restrict__ G,
                                                           const uint4* __restrict__ flags, int ngroups,
                                                           const R* __restrict__ S, double* __restrict__ partial,
                                                           long long row_stride, int i_lo, int KT, int passes)
{
    constexpr int BS = kCosBS, W = BS / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    R* wacc = reinterpret_cast<R*>(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int per_row = P.n_chunks * passes;
    const int ii = (int)(blockIdx.x / per_row), rem = (int)(blockIdx.x % per_row);
    const int ps = rem / P.n_chunks, ch = rem % P.n_chunks;
    const int i = i_lo + ii;
    const int gs = ps * (KT / 4);
    const int ge = min(ngroups, gs + KT / 4);  // both multiples of 16
    R* myacc = wacc + (size_t)warp * KT;
    for (int q = lane; q < KT; q += 32) myacc[q] = (R)0;
    __syncwarp();

    const uint4 q0 = __ldg(G + gs);
    const int a00 = (int)(q0.x & 0xffffu);
    const int rounds = P.chunk / (PPL * BS);
    for (int r = 0; r < rounds; ++r) {
        CosWalk<R, D> Wk[PPL];
        R Sv[PPL];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const long long m = (long long)ch * P.chunk + (long long)(r * PPL + u) * BS + tid;
            const bool active = m < P.M;
            Sv[u] = active && in_bounds(P, ii >= 0 && ii < P.N) ? S[(size_t)ii * (size_t)P.M + (size_t)m] : (R)0;
            V2<R> ph[D];
            start_phases_dev<R, D>(P, i, active ? m : 0, ph);  // e^{i pi U^m} (half angle)
            Wk[u].init(ph, Sv[u]);
            Wk[u].seek(q0.z, q0.w, q0.y, a00, Sv[u]);
        }
        for (int g0 = gs; g0 < ge; g0 += 8) {
            const uint2 fl = __ldg(reinterpret_cast<const uint2*>(flags) + g0 / 8);
            R v[32];
#pragma unroll
            for (int gg = 0; gg < 8; ++gg) {
                const uint32_t fb = ((gg < 4 ? fl.x : fl.y) >> (8 * (gg & 3))) & 0xffu;
                const bool start = (fb & 0x80u) != 0;
#pragma unroll
                for (int u = 0; u < PPL; ++u) {
                    // (the pass's first group: seek placed the walk on its run already)
                    if (D > 1 && start && (int)(fb & 15u) < D - 1 && g0 + gg != gs)
                        Wk[u].new_run((int)(fb & 15u), Sv[u]);
                    R v0, v1, v2, v3;
                    Wk[u].values(start, v0, v1, v2, v3);
                    if (u == 0) {
                        v[4 * gg + 0] = Wk[u].p * v0;
                        v[4 * gg + 1] = Wk[u].p * v1;
                        v[4 * gg + 2] = Wk[u].p * v2;
                        v[4 * gg + 3] = Wk[u].p * v3;
                    } else {
                        v[4 * gg + 0] = fma(Wk[u].p, v0, v[4 * gg + 0]);
                        v[4 * gg + 1] = fma(Wk[u].p, v1, v[4 * gg + 1]);
                        v[4 * gg + 2] = fma(Wk[u].p, v2, v[4 * gg + 2]);
                        v[4 * gg + 3] = fma(Wk[u].p, v3, v[4 * gg + 3]);
                    }
                }
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
        if (in_bounds(P, ii >= 0 && ii < P.N && ch >= 0 && ch < P.n_chunks && gs * 4 + q < row_stride)) out[q] = s;
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

template <typename R, int D>
__global__ void __launch_bounds__(kCosBS) k_eval_cos(const __grid_constant__ QrParams P,
                                                     const uint4* __restrict__ flags, int ng,
                                                     const R* __restrict__ crow, const double* __restrict__ xs,
                                                     long long n, double* __restrict__ ys, int use_g)
{
    const long long p = (long long)blockIdx.x * kCosBS + threadIdx.x;
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
    CosWalk<R, D> W;
    W.init(zz, (R)1);
    ys[p] = (double)cos_series<R, D>(crow, flags, ng, W);
}

// ------------------------------------------------------------ launchers
namespace {

constexpr size_t kCap = 227 * 1024;
// rows staged in shared memory only while four blocks per SM still fit
constexpr size_t kRowsSmemMax = 52 * 1024;

template <typename R, int D, bool CG>
cudaError_t paths_cos_cg(const QrParams& P, const uint4* flags, int ng, const void* packed, long long row_stride,
                         void* S, int i_lo, int i_hi, unsigned long long* counters, unsigned* status, cudaStream_t st)
{
    constexpr int BS = kCosBS;
    const size_t sm = cos_paths_smem<R>(row_stride, CG);
    auto kern = k_paths_cos<R, D, CG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int tiles = (int)((P.M + BS - 1) / BS);
    const long long blocks = (long long)tiles * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, BS, sm, st>>>(P, flags, ng, static_cast<const R*>(packed), row_stride,
                                           static_cast<R*>(S), i_lo, tiles, counters, status);
    return cudaGetLastError();
}

template <typename R, int D>
cudaError_t paths_cos_t(const QrParams& P, const uint4* flags, int ng, const void* packed, long long row_stride,
                        void* S, int i_lo, int i_hi, unsigned long long* counters, unsigned* status, cudaStream_t st)
{
    if (cos_paths_smem<R>(row_stride, false) <= kRowsSmemMax)
        return paths_cos_cg<R, D, false>(P, flags, ng, packed, row_stride, S, i_lo, i_hi, counters, status, st);
    return paths_cos_cg<R, D, true>(P, flags, ng, packed, row_stride, S, i_lo, i_hi, counters, status, st);
}

template <typename R, int D, int PPL>
cudaError_t project_cos_ppl(const QrParams& P, const CosGroup* G, const uint4* flags, int ngroups, const void* S,
                            double* partial, long long row_stride, int i_lo, int i_hi, cudaStream_t st)
{
    constexpr int W = kCosBS / 32;
    // per-warp accumulators of up to 2048 positions (32 KB in FP32); every
    // pass walks its paths from their start points again (KT and the pass
    // starts are multiples of 64 positions: whole words of flags)
    long long KT = std::min<long long>(row_stride, 2048);
    const int passes = (int)((row_stride + KT - 1) / KT);
    const size_t sm = (size_t)W * KT * sizeof(R);
    if (sm > kCap) return cudaErrorInvalidConfiguration;
    auto kern = k_project_cos<R, D, PPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)P.n_chunks * passes * (i_hi - i_lo);
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, kCosBS, sm, st>>>(P, G, flags, ngroups, static_cast<const R*>(S), partial, row_stride,
                                               i_lo, (int)KT, passes);
    return cudaGetLastError();
}

// two paths per lane (one fold for both) in FP32, where the two walks fit
// the registers of 3 blocks per SM (at most 160 for d <= 8)
template <typename R, int D>
cudaError_t project_cos_t(const QrParams& P, const CosGroup* G, const uint4* flags, int ngroups, const void* S,
                          double* partial, long long row_stride, int i_lo, int i_hi, cudaStream_t st)
{
    if (sizeof(R) == 4 && D <= 8 && P.chunk % (2 * kCosBS) == 0)
        return project_cos_ppl<R, D, 2>(P, G, flags, ngroups, S, partial, row_stride, i_lo, i_hi, st);
    return project_cos_ppl<R, D, 1>(P, G, flags, ngroups, S, partial, row_stride, i_lo, i_hi, st);
}

template <typename R, int D>
cudaError_t eval_cos_t(const QrParams& P, const uint4* flags, int ng, const void* row, const double* x, long long n,
                       double* y, int use_g, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_eval_cos<R, D><<<(unsigned)((n + kCosBS - 1) / kCosBS), kCosBS, 0, st>>>(P, flags, ng,
                                                                              static_cast<const R*>(row), x, n, y,
                                                                              use_g);
    return cudaGetLastError();
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
    case 9: return FN<R, 9>(__VA_ARGS__);  \
    case 10: return FN<R, 10>(__VA_ARGS__); \
    case 11: return FN<R, 11>(__VA_ARGS__); \
    case 12: return FN<R, 12>(__VA_ARGS__); \
    default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_paths_cos(int prec, const QrParams& P, const uint8_t* flags, int ngroups, const void* packed,
                             long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                             unsigned* status, cudaStream_t st)
{
    const uint4* fl = reinterpret_cast<const uint4*>(flags);
    if (prec == QR_FP32) {
        QR_COS_DISPATCH(paths_cos_t, float, P, fl, ngroups, packed, row_stride, S, i_lo, i_hi, counters, status, st)
    }
    QR_COS_DISPATCH(paths_cos_t, double, P, fl, ngroups, packed, row_stride, S, i_lo, i_hi, counters, status, st)
}

cudaError_t launch_project_cos(int prec, const QrParams& P, const CosGroup* groups, const uint8_t* flags, int ngroups,
                               const void* S, double* partial, long long row_stride, int i_lo, int i_hi,
                               cudaStream_t st)
{
    const uint4* fl = reinterpret_cast<const uint4*>(flags);
    if (prec == QR_FP32) {
        QR_COS_DISPATCH(project_cos_t, float, P, groups, fl, ngroups, S, partial, row_stride, i_lo, i_hi, st)
    }
    QR_COS_DISPATCH(project_cos_t, double, P, groups, fl, ngroups, S, partial, row_stride, i_lo, i_hi, st)
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

cudaError_t launch_eval_cos(int prec, const QrParams& P, const uint8_t* flags, int ngroups, const void* packed_row,
                            const double* x, long long n, double* y, int use_g, cudaStream_t st)
{
    const uint4* fl = reinterpret_cast<const uint4*>(flags);
    if (prec == QR_FP32) {
        QR_COS_DISPATCH(eval_cos_t, float, P, fl, ngroups, packed_row, x, n, y, use_g, st)
    }
    QR_COS_DISPATCH(eval_cos_t, double, P, fl, ngroups, packed_row, x, n, y, use_g, st)
}

}  // namespace qr
