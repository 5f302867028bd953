// Radix sort of template keys (processing order of the mixed path) and top-k
// selection of statistic values (survivors of an adaptive N_seg stage).
#pragma once

#include "tfs_internal.cuh"

namespace tfs {

size_t sort_scratch_bytes(int64_t n);
// perm[i] = index of the template processed i-th: ascending TplConst::key, stable.
cudaError_t sort_templates(const TplConst* tpl, int64_t n, int32_t* perm, void* scratch, int n_sm,
                           cudaStream_t s, int* launches);

size_t topk_scratch_bytes(int64_t n);
// out_idx[0..k) = indices of the k largest stat values, decreasing; ties by lower index.
cudaError_t select_top(const double* stat, int64_t n, int64_t k, int64_t* out_idx, void* scratch,
                       cudaStream_t s, int* launches);

}  // namespace tfs
