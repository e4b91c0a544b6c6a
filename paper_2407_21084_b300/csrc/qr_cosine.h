// qr_cosine.h -- direct kernels of the cosine basis on an N^d index set
// (Sec. 2.2, Lemma ortho:dim1): real coefficient rows, real per-lane tables.
#pragma once
#include "qr_internal.h"

namespace qr {

// Gamma in canonical order splits into runs that share k_1..k_{d-1} and have
// k_d = 0, 1, ..., len-1 (true of Gamma_F, Gamma_T and Gamma_H: all are
// downward closed). Each run is padded with zero coefficients to a multiple
// of 4 and cut into groups of 4 consecutive packed positions; group g covers
// positions 4g..4g+3 of a packed row. The group count is padded to a
// multiple of 16 (runs of zero coefficients).
//
// The prefix of a new run differs from the previous run's prefix in one
// coordinate f, which is one larger, and the prefix coordinates after f are
// 0 (lexicographic order of a downward-closed set; checked by qr_init): the
// kernels step every factor by one complex product. Per group they read one
// flag byte: bit 7 = a run starts here, bits 0-3 = f (d-1 for the first run
// and the padding, whose prefix is all zeros or unchanged).
//
// CosGroup (16 bytes, for starting a walk in the middle of Gamma):
//   x: a0 = k_d of the group's first position (bits 0-15)
//   z, w, y: k_1..k_4, k_5..k_8 and k_9..k_11 of the run's prefix, one byte each
using CosGroup = uint4;

constexpr int kCosPrefixMax = 255;  // prefix coordinates are stored in one byte

cudaError_t launch_paths_cos(int prec, const QrParams& P, const uint8_t* flags, int ngroups, const void* packed,
                             long long row_stride, void* S, int i_lo, int i_hi, unsigned long long* counters,
                             unsigned* status, cudaStream_t st);
// partial[(i - i_lo) * n_chunks + chunk][position], FP64
cudaError_t launch_project_cos(int prec, const QrParams& P, const CosGroup* groups, const uint8_t* flags, int ngroups,
                               const void* S, double* partial, long long row_stride, int i_lo, int i_hi,
                               cudaStream_t st);
// fixed-order chunk sums / M into alpha (real parts, rows i_lo..i_hi-1), the packed rows and the residual
cudaError_t launch_reduce_cos(int prec, const QrParams& P, const double* partial, const int* pos, double2* alpha,
                              void* packed, long long row_stride, int i_lo, int i_hi, unsigned long long* counters,
                              cudaStream_t st);
// packed rows [0, rows) from alpha (real parts); padding positions are left as they are (zero)
cudaError_t launch_pack_cos(int prec, const double2* alpha, int nG, const int* pos, void* packed,
                            long long row_stride, int rows, cudaStream_t st);
cudaError_t launch_eval_cos(int prec, const QrParams& P, const uint8_t* flags, int ngroups, const void* packed_row,
                            const double* x, long long n, double* y, int use_g, cudaStream_t st);

}  // namespace qr
