// The job table of a batch (gk_batch_fit), passed to kernels by value.
#pragma once

#include <stdint.h>

#include "../../include/gkm.h"

namespace gkm {

constexpr int MAX_BATCH_JOBS = GK_MAX_BATCH_JOBS;

struct BatchTable {
    int32_t njobs;
    int64_t first[MAX_BATCH_JOBS + 1];   // job j owns samples first[j] .. first[j + 1) - 1
    int32_t kfirst[MAX_BATCH_JOBS + 1];  // and clusters kfirst[j] .. kfirst[j + 1) - 1 of the fit
};

}  // namespace gkm
