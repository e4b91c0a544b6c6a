// qr_batch.h -- multi-instance persistent path kernel (qr_batch.cu).
#pragma once

#include "qr_fast.h"
#include "qr_group.h"
#include "qr_internal.h"

namespace qr {

// one instance as the persistent kernel sees it (FP32 precision form)
struct BatchInst {
    QrParams P;
    int cls;                       // compiled class (batch_class)
    const void* tree;              // (N+1) tree-layout coefficient rows
    long long tree_stride;         // slots per row
    void* S;                       // responses N x M
    unsigned long long* counters;  // CNT_* of the instance
    unsigned* status;
};

struct BatchItem {
    int inst, i, tile0, ntiles;
};

// one instance as the finishing kernel sees it: projection, reduction and
// repacks of its rows
struct FinishInst {
    QrParams P;
    int cls;                  // compiled class (batch_class)
    const float* S;           // responses N x M
    double2* partial;         // N x n_chunks x |Gamma_+|
    double2* alpha;           // (N+1) x |Gamma| master rows
    float2* packed;           // table-layout working rows
    long long row_stride;
    float2* tree;             // tree-layout working rows
    long long tree_stride;
    const TreeMap* tmap;
    int tree_slots;
    const int* perm;          // projection order (tree node -> half-set entry)
    int nG, zero_idx;
    int row_base;             // first of this instance's per-row arrival counters
    int group;                // shared-point group (FinishGroup index), -1 if none
};

// a shared-point group as the finishing kernel sees it
struct FinishGroup {
    int gcls;                 // group class: 0 = |k|_inf <= 4 in d = 2, 1 = |k|_1 <= 3 in d = 6
    const GroupInst* inst;    // members
    int n_inst, nG, zero_idx;
    const int* perm;
    uint8_t* Bpack;           // the group kernel's coefficient blocks
    int row_base;             // first of the group's per-row arrival counters
};

// items are (instance, row, chunk, 0)
size_t finish_smem();
int finish_group_class(int kind, int d, int n);  // -1 if the group kernel has no such class
cudaError_t launch_finish_batch(const FinishInst* fin, const int4* items, long long n_items, const FinishGroup* groups,
                                unsigned* row_done, unsigned* grp_done, unsigned long long* resid, cudaStream_t st);

int batch_class(int kind, int d, int n);  // -1 if not compiled
int batch_tile_paths();
int batch_blocks_per_sm(size_t max_rowbytes);
cudaError_t launch_paths_batch(const BatchInst* inst, const BatchItem* items, int n_items, unsigned* next_item,
                               size_t max_rowbytes, int grid, cudaStream_t st);

}  // namespace qr
