// pending.cu -- entry points whose kernels are not in this build yet.
#include "internal.h"

extern "C" int pars3_autotune(int32_t, const int32_t *, const int32_t *, const double *, const int32_t *,
                              const pars3_split_params *, int32_t, int32_t, pars3_split_params *, double *) {
    return PARS3_EUNSUPPORTED;
}
