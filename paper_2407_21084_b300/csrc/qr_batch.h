// qr_batch.h -- multi-instance persistent path kernel (qr_batch.cu).
#pragma once

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

int batch_class(int kind, int d, int n);  // -1 if not compiled
int batch_tile_paths();
int batch_blocks_per_sm(size_t max_rowbytes);
cudaError_t launch_paths_batch(const BatchInst* inst, const BatchItem* items, int n_items, unsigned* next_item,
                               size_t max_rowbytes, int grid, cudaStream_t st);

}  // namespace qr
