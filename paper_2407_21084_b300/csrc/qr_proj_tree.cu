// qr_proj_tree.cu -- projection kernel (eq. Aqi:bar:M) specialised at
// compile time for the |k|_1 <= n and |k|_inf <= n index sets.
//
// alpha_{i,k} = (1/M) sum_m S_i^m conj(phi_k(U^m)) needs every basis value
// phi_k(U^m) once per path, accumulated over paths. The half set is walked
// in the chain-tree order (parent = last nonzero coordinate one step towards
// 0, so phi_k = phi_parent * z_l or conj(z_l)); the walk is cut into tiles of
// 32 coefficients whose code is unrolled at compile time. A warp keeps the 32
// accumulators of a tile in registers while its lanes run over many paths,
// then folds them across lanes with a reduce-scatter butterfly (31 shuffles
// per component per tile, lane L ending with slot L), so the cross-lane
// reduction is paid once per tile per 256 paths instead of once per
// coefficient per 32 paths. Phases e^{2 pi i U_l} and responses of a block
// of paths are computed once into shared memory and reused by every tile.
// Per-warp partial sums live in shared memory and are combined in a fixed
// warp order: the result is independent of scheduling.
#include "qr_ptree.cuh"

namespace qr {

#define QR_PROJ_SETS(X) \
    X(QR_G_LINF, 2, 4)  \
    X(QR_G_L1, 4, 4)    \
    X(QR_G_L1, 6, 5)

int proj_tree_nodes(int kind, int d, int n)
{
#define QR_X(K, DD, NNN) \
    if (kind == K && d == DD && n == NNN) return FullTree<DD, NNN, K>::n;
    QR_PROJ_SETS(QR_X)
#undef QR_X
    return proj_tree_nodes_more(kind, d, n);
}

cudaError_t launch_project_tree(int prec, int kind, int n, const QrParams& P, const void* S, const int* perm,
                                double2* partial, int i_lo, int i_hi, cudaStream_t st)
{
#define QR_X(K, DD, NNN)                                                                               \
    if (kind == K && P.d == DD && n == NNN)                                                            \
        return prec == QR_FP32 ? project_tree_t<float, DD, NNN, K>(P, S, perm, partial, i_lo, i_hi, st) \
                               : project_tree_t<double, DD, NNN, K>(P, S, perm, partial, i_lo, i_hi, st);
    QR_PROJ_SETS(QR_X)
#undef QR_X
    return launch_project_tree_more(prec, kind, n, P, S, perm, partial, i_lo, i_hi, st);
}

}  // namespace qr
