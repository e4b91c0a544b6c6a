// qr_internal.h -- types shared by the host side and the kernels of libqrmc.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qr.h"

namespace qr {

constexpr int kDMax = 12;       // dimensions (the direct cosine kernels)
constexpr int kDMaxFourier = 8; // dimensions of the Z^d sets (table entries hold 8 coordinates)
constexpr int kNMax = 256;  // time steps

enum { QR_TAG_START = 0, QR_TAG_INCR = 1, QR_TAG_TEST = 2 };

// device status bits
// status word bits: a bounded wait ran out; (checked builds) an index fell
// outside its buffer and the access was skipped
enum : unsigned { ST_TIMEOUT = 1u, ST_BOUNDS = 2u };

// counters[0] = clamp hits, counters[1] = non-finite responses,
// counters[2] = residual (bits of a non-negative double, atomicMax)
enum { CNT_CLAMP = 0, CNT_NONFINITE = 1, CNT_RESID = 2, CNT_SPARE = 3, CNT_N = 4 };

// One entry of the coefficient table: k, as int16 per dimension for d <= 4
// (|k_l| <= 32767: the long one-dimensional sets of Sec. 5) or int8 for
// d > 4 (|k_l| <= 127). The table is [k = 0, then Gamma_+ = {k : first
// nonzero k_l > 0}] in canonical order; first[e] is the first dimension in
// which entry e differs from entry e-1.
struct alignas(8) GEntry {
    union {
        signed char k8[8];
        short k16[4];
    };
    template <int D>
    __host__ __device__ __forceinline__ int kv(int l) const
    {
        return D <= 4 ? (int)k16[l] : (int)k8[l];
    }
    __host__ int get(int d, int l) const { return d <= 4 ? (int)k16[l] : (int)k8[l]; }
    __host__ void set(int d, int l, int v)
    {
        if (d <= 4)
            k16[l] = (short)v;
        else
            k8[l] = (signed char)v;
    }
};
constexpr int gentry_kmax(int d) { return d <= 4 ? 32767 : 127; }

struct QrParams {
    int d, N, nGp, K1;  // K1 = max|k_l| + 1
    long long M;
    int nu_kind, mu_is3;
    double mu, inv_mu;
    double T, dt, sqdt;
    double b[kDMax];
    double sig[kDMax * kDMax];  // row-major d x d, stored with row stride d
    int sig_diag;
    int f_kind;
    double f_lam, f_kap, f_c;
    double f_s[kDMax];
    int g_kind;  // QR_GT_*
    double g_s[kDMax], g_kap, g_lam;
    double fexp[kNMax];  // time factor of f at t_j
    float fexp32[kNMax]; // the same, rounded to FP32 (FP32 path kernels)
    uint32_t key0, key1;
    int instance;
    double clamp_L;  // <= 0: off
    int lattice_n;
    int chunk;     // projection: paths per CTA
    int n_chunks;  // ceil(M / chunk)
    int c_lo, c_hi;  // chunks this context simulates and projects (a shard of paths; all by default)
    int half_angle;  // cosine basis: phases e^{i pi F(x)} instead of e^{2 pi i F(x)}
    double q_damp;   // damping exponent q of eq. (yqi); 0: none
    unsigned* check; // the context's status word (bounds checks of checked builds)
};

// The cross-chunk sum of the projection is taken in two fixed levels: the
// chunks of each of kShardGroups groups in order, then the group sums in
// order. A shard of a problem over W ranks (W dividing kShardGroups) owns
// whole groups, so W ranks that exchange their group sums reproduce the
// one-GPU coefficients bit for bit.
constexpr int kShardGroups = 8;
__host__ __device__ inline int group_chunk(int g, int n_chunks)
{
    return (int)(((long long)g * n_chunks) / kShardGroups);
}
// kernel launchers (qr_kernels.cu); all asynchronous on `st`
cudaError_t launch_paths(int prec, const QrParams& P, const GEntry* tab, const uint8_t* first,
                         const void* packed, long long row_stride, void* S, int i_lo, int i_hi,
                         unsigned long long* counters, unsigned* status, cudaStream_t st);
cudaError_t launch_project(int prec, const QrParams& P, const GEntry* tab, const uint8_t* first,
                           const void* S, double2* partial, int i_lo, int i_hi, cudaStream_t st);
cudaError_t launch_reduce(int prec, const QrParams& P, const double2* partial, double2* alpha, int nG,
                          int zero_idx, void* packed, long long row_stride, int i_lo, int i_hi,
                          unsigned long long* counters, cudaStream_t st);
cudaError_t launch_pack(int prec, const QrParams& P, const double2* alpha, int nG, int zero_idx,
                        void* packed, long long row_stride, int rows, cudaStream_t st);
// a bounded wait that runs out on purpose (status |= ST_TIMEOUT after ~1 s)
cudaError_t launch_wait_selftest(unsigned* status, cudaStream_t st);
// cosine basis: symmetrise the raw projections of rows [i_lo, i_hi) over the
// sign orbits (CSR orb_off/orb_idx over the canonical Z^d order) into alpha
cudaError_t launch_sym_cos(const double2* raw, double2* alpha, int nG, const int* orb_off, const int* orb_idx,
                           int i_lo, int i_hi, unsigned long long* counters, cudaStream_t st);
cudaError_t launch_eval(int prec, const QrParams& P, const GEntry* tab, const uint8_t* first,
                        const void* packed_row, const double* x, long long n, double* y, int use_g,
                        cudaStream_t st);
cudaError_t launch_test_points(const QrParams& P, int i, long long n, double* x, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr_key, long long n, uint32_t* out, cudaStream_t st);
cudaError_t launch_sample(int prec, const QrParams& P, int i, long long m0, long long n, int j,
                          double* u, double* x, double* z, cudaStream_t st);
cudaError_t launch_normals_tree(const QrParams& P, int i, long long m0, long long n, int j, double* z,
                                cudaStream_t st);

// first path of the context's chunk range, and the end of that range
__host__ __device__ inline long long shard_m_lo(const QrParams& P) { return (long long)P.c_lo * P.chunk; }
__host__ __device__ inline long long shard_m_hi(const QrParams& P)
{
    const long long e = (long long)P.c_hi * P.chunk;
    return e < P.M ? e : P.M;
}

// group sums of the chunk partials: gsum[g][row][e] for the groups
// [g_lo, g_hi) (rows i_lo .. i_hi-1; partial rows relative to i_lo)
cudaError_t launch_group_sums(const QrParams& P, const double2* partial, double2* gsum, int g_lo, int g_hi, int i_lo,
                              int i_hi, cudaStream_t st);
// the reduction from all kShardGroups group sums (as launch_reduce does from
// the partials): alpha, packed rows, residual
cudaError_t launch_reduce_groups(int prec, const QrParams& P, const double2* gsum, double2* alpha, int nG, int zero_idx,
                                 void* packed, long long row_stride, int i_lo, int i_hi,
                                 unsigned long long* counters, cudaStream_t st);

// read-only view of a context's device problem description (qr_api.cu)
struct CtxView {
    int prec, N, nG, zero_idx;
    const QrParams* P;
    const GEntry* tab;
    const uint8_t* first;
    cudaStream_t stream;
    int device;      // the device the context's buffers and stream live on
    int proj_nodes;  // nonzero: a compiled tiled projection covers the index set
    int gkind, gn;   // its index-set kind and level
    const int* perm; // its slot -> canonical half-set order
    bool sharded;    // restricted to a chunk range by qr_shard
};
}  // namespace qr

struct qr_ctx;
namespace qr {
bool ctx_view(const qr_ctx* c, CtxView* v);
void ctx_set_error(qr_ctx* c, const char* msg);
}  // namespace qr
