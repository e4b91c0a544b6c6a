// qr_fast.cu -- path-and-series kernel specialised at compile time for the
// |k|_1 <= n and |k|_inf <= n index sets.
//
// The series ybar(x) = Re sum_{k in Gamma} alpha_k phi_k(x) is evaluated over
// the half set Gamma_+ = {0} u {k : first nonzero k_l > 0} (alpha_{-k} =
// conj(alpha_k)), walking the "chain tree" of Gamma_+: the parent of k is k
// with its last nonzero coordinate moved one step towards 0, so every node's
// basis value is its parent's times a single base phase z_l or conj(z_l),
// z_l = e^{2 pi i F_nu(x_l)}. Only the d base phases live in registers; no
// power table is needed. The tree is evaluated bottom-up (Horner): the value
// of a subtree in its root's frame is
//     V_c = coef_c + sum_{children ch} w_ch V_ch,
// and ybar = Re V_0, one complex FMA per tree edge. Children that are leaves in a new dimension
// come in +-1 pairs whose two coefficients are pre-combined on the host, so a
// pair costs 4 FMA. The + and - subtrees of a new dimension share code
// through a two-trip runtime loop (w = z or conj z), which keeps the unrolled
// code to a few hundred tree nodes for d = 6, n = 5.
//
// Coefficients are stored per time row in the traversal order ("tree
// layout", one float2/double2 slot per half-set coefficient) by k_pack_tree
// and staged in shared memory by bulk copies, double buffered.

#include "qr_reduce.cuh"
#include "qr_tree.cuh"

namespace qr {

template <typename R>
__global__ void k_pack_tree(const double* __restrict__ alpha, int nG, const TreeMap* __restrict__ map, int slots,
                            V2<R>* __restrict__ out, long long row_stride, int rows)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * slots) return;
    const int r = (int)(idx / slots), s = (int)(idx % slots);
    out[(size_t)r * row_stride + s] = tree_slot<R>(alpha + (size_t)r * 2 * nG, map[s]);
}

// ------------------------------------------------------------ dispatch
// (kind, d, n) sets with a compiled tree kernel
#define QR_TREE_SETS(X)   \
    X(QR_G_LINF, 1, 3)    \
    X(QR_G_LINF, 2, 2)    \
    X(QR_G_LINF, 2, 4)    \
    X(QR_G_L1, 3, 2)      \
    X(QR_G_L1, 4, 4)      \
    X(QR_G_L1, 6, 5)

int tree_slots(int kind, int d, int n)
{
#define QR_X(K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return tree_slots_t<DD, NNN, K>();
    QR_TREE_SETS(QR_X)
#undef QR_X
    return tree_slots_more(kind, d, n);
}

cudaError_t launch_paths_tree(int prec, int kind, int n, const QrParams& P, const void* tree, long long row_stride,
                              void* S, int i_lo, int i_hi, unsigned long long* counters, unsigned* status,
                              cudaStream_t st)
{
#define QR_X(K, DD, NNN)                                                                                      \
    if (kind == K && P.d == DD && n == NNN)                                                                   \
        return prec == QR_FP32                                                                                \
                   ? paths_tree_t<float, DD, NNN, K>(P, tree, row_stride, S, i_lo, i_hi, counters, status, st) \
                   : paths_tree_t<double, DD, NNN, K>(P, tree, row_stride, S, i_lo, i_hi, counters, status, st);
    QR_TREE_SETS(QR_X)
#undef QR_X
    return launch_paths_tree_more(prec, kind, n, P, tree, row_stride, S, i_lo, i_hi, counters, status, st);
}

cudaError_t launch_pack_tree(int prec, const double2* alpha, int nG, const TreeMap* map, int slots, void* out,
                             long long row_stride, int rows, cudaStream_t st)
{
    const long long total = (long long)rows * slots;
    if (total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    const double* a = reinterpret_cast<const double*>(alpha);
    if (prec == QR_FP32)
        k_pack_tree<float><<<blocks, 256, 0, st>>>(a, nG, map, slots, static_cast<float2*>(out), row_stride, rows);
    else
        k_pack_tree<double><<<blocks, 256, 0, st>>>(a, nG, map, slots, static_cast<double2*>(out), row_stride, rows);
    return cudaGetLastError();
}

// the Box-Muller normals of Euler step j exactly as the FP32 tree path kernels
// draw them (normals_fast), widened to double: z is n rows of d values
template <int D>
__global__ void k_normals_tree(const __grid_constant__ QrParams P, int i, long long m0, long long n, int j,
                               double* __restrict__ z)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float zz[D];
    normals_fast<float, D>(P, i, (uint32_t)(m0 + t), j, zz);
#pragma unroll
    for (int l = 0; l < D; ++l) z[t * D + l] = (double)zz[l];
}

cudaError_t launch_normals_tree(const QrParams& P, int i, long long m0, long long n, int j, double* z,
                                cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n + 127) / 128);
    switch (P.d) {
#define QR_X(DD) \
    case DD: k_normals_tree<DD><<<blocks, 128, 0, st>>>(P, i, m0, n, j, z); break;
        QR_X(1) QR_X(2) QR_X(3) QR_X(4) QR_X(5) QR_X(6) QR_X(7) QR_X(8)
#undef QR_X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}


}  // namespace qr
