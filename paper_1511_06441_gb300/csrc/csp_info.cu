// libcsp: facts about the build (no kernels here).
#include <cstdint>

#include "csp.h"
#include "csp_device.cuh"

#ifndef CSP_BATCH_MIN_CTAS_PER_SM
#define CSP_BATCH_MIN_CTAS_PER_SM 1  // (the batch kernel's default, csp_batch.cu)
#endif

extern "C" void csp_build_shape(int32_t *shape)
{
    if (!shape) return;
    shape[0] = csp::TPB;
    shape[1] = csp::IPT;
    shape[2] = csp::NSTAGE;
    shape[3] = CSP_MIN_CTAS_PER_SM;
    shape[4] = CSP_BATCH_MIN_CTAS_PER_SM;
}
