// pending.cu -- entry points whose kernels are not in this build yet.
#include "internal.h"

extern "C" int pars3_spmm(const pars3_handle *, int32_t, double, int32_t, const void *, void *, void *) {
    return PARS3_EUNSUPPORTED;
}
extern "C" int pars3_spmm_batched(pars3_handle *const *, int32_t, int32_t, const double *, int32_t,
                                  const void *const *, void *const *, int32_t, void *) {
    return PARS3_EUNSUPPORTED;
}
extern "C" int pars3_autotune(int32_t, const int32_t *, const int32_t *, const double *, const int32_t *,
                              const pars3_split_params *, int32_t, int32_t, pars3_split_params *, double *) {
    return PARS3_EUNSUPPORTED;
}
