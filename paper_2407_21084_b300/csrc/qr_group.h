// qr_group.h -- tensor-core series for instances sharing sample points (qr_group.cu).
#pragma once

#include "qr_internal.h"

namespace qr {

constexpr int kGroupNMax = 64;  // time steps supported by the shared-point kernel

struct GroupInstParams {
    float fs[kDMax];  // wave vector of the manufactured solution in f
    float gs[kDMax];  // wave vector of g = cos(gs.x)
    float f_c;        // constant of the cubic driver
    float clamp_L;
};

struct GroupInst {
    GroupInstParams p;
    float fexp[kGroupNMax];  // e^{a (T - t_j)}
    void* S;                 // responses of the instance, N x M floats
    const double2* alpha;    // master coefficient rows of the instance
};

// compiled for (kind, d, n)?
bool group_supported(int kind, int d, int n);
// bf16 elements of one (hi or lo) coefficient block of 32 instances, and the
// whole packed array for rows 0..N-1
long long group_block_elems(int kind, int d, int n);
cudaError_t launch_pack_group(int kind, int d, int n, const GroupInst* inst, int n_inst, int nG, int zero_idx,
                              const int* perm, void* Apack, int rows, cudaStream_t st);
cudaError_t launch_paths_group(int kind, int d, int n, const QrParams& P, const GroupInst* inst, int n_inst,
                               const void* Apack, unsigned* status, cudaStream_t st);

}  // namespace qr
