// Learned radius proposal: model storage, features, MLP kernels and the
// learned query path (not in the paper; results never change).
#pragma once

#include "kdt_internal.cuh"

namespace kdt {
// d_visits (optional): per-query processed nodes of the bounded pass plus,
// for re-run queries, of the fallback pass; results are not written if d_ids
// is NULL
int run_learned_query(kdt_tree *t, const float *d_q, int64_t Q, int k, float r2, int flags, int32_t *d_ids,
                      float *d_d2, int32_t *d_visits, cudaStream_t s);
int run_query(const kdt_tree *t, const float *d_q, int64_t Q, int k, float r2, int flags, int mode, int32_t *d_ids,
              float *d_d2, int32_t *d_visits, cudaStream_t s);
void free_model(kdt_tree *t);
// tensor-core inference (kdt_mlp_tc.cu): per-query cull radius of the learned
// pass (for the first *n_lim queries of perm when n_lim is given), and the
// model output for given normalised features
int tc_radius(const kdt_tree *t, const float *wts, const float *d_q, int64_t Q, const uint32_t *perm, float r2_user,
              float *r2q, cudaStream_t s, const unsigned long long *n_lim = nullptr);
int tc_forward(const float *wts, const float *d_x, int64_t n, float *d_y, int *d_err, cudaStream_t s);
// tensor-core loss and gradient over samples [begin, begin + count): one block
// per 128 samples, partial[block][KDT_MLP_PARAMS + 1]; *blocks receives their number
int tc_loss_grad(const float *wts, const float *d_x, const float *d_label, int64_t begin, int64_t count,
                 float *d_partial, int *d_err, cudaStream_t s, int *blocks);
void fill_inf(float *p, int64_t n, cudaStream_t s);
}  // namespace kdt
