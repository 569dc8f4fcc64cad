// Placeholder entry points of the tensor-core chain, the adjoint and the proposer (replaced as those
// paths land).
#include "internal.h"
namespace leb {
}  // namespace leb
extern "C" {
leb_status leb_proposer_create(int, int, int, unsigned long long, leb_proposer* out) { if (out) *out = nullptr; return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_destroy(leb_proposer) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_set_norm(leb_proposer, const float*, const float*, const float*, const float*, void*) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_forward(leb_proposer, int, const float*, float*, void*, size_t, void*) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_train_step(leb_proposer, int, const float*, const float*, float, float*, void*, size_t, void*) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_workspace_size(leb_proposer, int, size_t*) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_get_layer(leb_proposer, int, float*, float*, void*) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_set_layer(leb_proposer, int, const float*, const float*, void*) { return LEB_ERR_UNSUPPORTED; }
leb_status leb_proposer_get_grad(leb_proposer, int, float*, float*, void*) { return LEB_ERR_UNSUPPORTED; }
}
