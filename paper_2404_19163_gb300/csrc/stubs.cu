// Entry points declared in zfact.h whose kernels are not built yet: they
// report ZFACT_ERR_UNSUPPORTED through the normal error channel.
#include "ctx.h"

#define ZF_STUB(name)                                                             \
  if (c) ctx_fail(c, ZFACT_ERR_UNSUPPORTED, "%s is not available in this build", name); \
  return ZFACT_ERR_UNSUPPORTED;

extern "C" int zfact_features(zfact_ctx* c, const double*, int64_t, float*) { ZF_STUB("zfact_features") }
extern "C" int zfact_mlp_forward(zfact_ctx* c, const float*, const float*, const float*, const float*, int, float*) {
  ZF_STUB("zfact_mlp_forward")
}
extern "C" int zfact_mlp_backward(zfact_ctx* c, const float*, const float*, const float*, const float*, const float*,
                                  const int*, int, float, float*, double*) {
  ZF_STUB("zfact_mlp_backward")
}
extern "C" int zfact_mlp_adam(zfact_ctx* c, float*, const float*, float*, float*, int, int, float, float, float,
                              float) {
  ZF_STUB("zfact_mlp_adam")
}
extern "C" int zfact_propose(zfact_ctx* c, const double*, int64_t, const float*, const float*, const float*, double*,
                             int*) {
  ZF_STUB("zfact_propose")
}
