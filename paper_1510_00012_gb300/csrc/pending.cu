// Entry points of the pruning MLP that this build does not provide yet:
// they report D2_ENOTSUP.
#include "d2_internal.cuh"

struct d2_prune { int dummy; };

extern "C" d2_prune* d2_prune_create(d2_ctx*, int32_t, int32_t, int32_t, const float*, uint64_t) { return nullptr; }
extern "C" void d2_prune_destroy(d2_prune*) {}
extern "C" int64_t d2_prune_param_count(const d2_prune*) { return 0; }
extern "C" int d2_prune_get_params(d2_ctx* c, const d2_prune*, float*) { return d2_fail(c, D2_ENOTSUP, "not built"); }
extern "C" int d2_prune_set_params(d2_ctx* c, d2_prune*, const float*) { return d2_fail(c, D2_ENOTSUP, "not built"); }
extern "C" int d2_prune_set_margin(d2_prune*, int32_t, float) { return D2_ENOTSUP; }
extern "C" int d2_prune_embed(d2_ctx* c, const d2_prune*, const d2_bags*, const int64_t*, int64_t, float*, float*, void*) { return d2_fail(c, D2_ENOTSUP, "not built"); }
extern "C" int d2_prune_loss_grad(d2_ctx* c, const d2_prune*, const d2_bags*, int32_t, int32_t, const float*, const float*, const int64_t*, const int32_t*, const float*, int64_t, double*, float*, void*) { return d2_fail(c, D2_ENOTSUP, "not built"); }
extern "C" int d2_prune_train(d2_ctx* c, d2_prune*, const d2_bags*, int32_t, int32_t, const float*, const float*, const int64_t*, const int32_t*, const float*, int64_t, int32_t, int32_t, float, uint64_t, float*) { return d2_fail(c, D2_ENOTSUP, "not built"); }
int d2_assign_pruned(d2_ctx* c, const d2_bags*, int, int, const float*, const float*, const d2_prune*, int32_t*, float*, int64_t*, cudaStream_t) { return d2_fail(c, D2_ENOTSUP, "pruned assignment not built"); }
