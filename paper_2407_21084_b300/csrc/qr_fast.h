// qr_fast.h -- tree-layout path-and-series kernels (qr_fast.cu).
#pragma once

#include "qr_internal.h"

namespace qr {

// The mirrored chains k +- m e_l of the dimensions l = d-2, d-3, ..., (this
// many, at most d-2 of them) are evaluated in pair form (one sum and one
// difference subtree per m against the powers of that dimension's phase)
// instead of two Horner chains; the device traversal (qr_tree.cuh) and the
// host layout (build_tree_map) both follow this setting.
#ifndef QR_TREE_PAIR_LEVELS
#define QR_TREE_PAIR_LEVELS 2
#endif

// One slot of the tree layout: slot.x = sum_t c[0][t] a[i[0][t]] (terms with
// c = 0 skipped), slot.y likewise with row 1, where a is a master coefficient
// row seen as 2|Gamma| doubles (re, im interleaved). Each pair level doubles
// the coefficients a slot can combine.
constexpr int kTreeTerms = 2 << QR_TREE_PAIR_LEVELS;
struct TreeMap {
    int i[2][kTreeTerms];
    double c[2][kTreeTerms];
};

// number of slots of the compiled tree for (kind, d, n); 0 if not compiled
int tree_slots(int kind, int d, int n);
cudaError_t launch_paths_tree(int prec, int kind, int n, const QrParams& P, const void* tree, long long row_stride,
                              void* S, int i_lo, int i_hi, unsigned long long* counters, unsigned* status,
                              cudaStream_t st);
cudaError_t launch_pack_tree(int prec, const double2* alpha, int nG, const TreeMap* map, int slots, void* out,
                             long long row_stride, int rows, cudaStream_t st);

// projection specialised for the same sets (qr_proj_tree.cu): partial sums
// are written in canonical half-set order through perm (tree slot -> e >= 1)
int proj_tree_nodes(int kind, int d, int n);
cudaError_t launch_project_tree(int prec, int kind, int n, const QrParams& P, const void* S, const int* perm,
                                double2* partial, int i_lo, int i_hi, cudaStream_t st);

// further sets (qr_fast_more.cu, qr_proj_more.cu), reached through the dispatchers above
int tree_slots_more(int kind, int d, int n);
cudaError_t launch_paths_tree_more(int prec, int kind, int n, const QrParams& P, const void* tree,
                                   long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                                   unsigned* status, cudaStream_t st);
int proj_tree_nodes_more(int kind, int d, int n);
cudaError_t launch_project_tree_more(int prec, int kind, int n, const QrParams& P, const void* S, const int* perm,
                                     double2* partial, int i_lo, int i_hi, cudaStream_t st);

// path kernels for the sets of the paper's own experiments (qr_fast_paper.cu),
// reached through the above; their projections use the table kernel (a
// compile-time projection of these long chains takes too long to build)
int tree_slots_paper(int kind, int d, int n);
cudaError_t launch_paths_tree_paper(int prec, int kind, int n, const QrParams& P, const void* tree,
                                    long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                                    unsigned* status, cudaStream_t st);

}  // namespace qr
