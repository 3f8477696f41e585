// fp_batched.cu -- several resident forests and uneven batches in one call.
#include <cuda_runtime.h>

#include "../../include/forest_pack.h"
#include "fp_common.h"

extern "C" int fp_predict_batched(const fp_device_forest *const *forests, const fp_batch *batches, int32_t k,
                                  void *stream) {
    if (k < 0 || (k > 0 && (!forests || !batches))) {
        fp_set_error("fp_predict_batched: bad arguments");
        return FP_EINVAL;
    }
    for (int32_t i = 0; i < k; ++i) {
        if (!forests[i] || batches[i].n < 0 || (batches[i].n > 0 && !batches[i].X)) {
            fp_set_error("fp_predict_batched: bad batch %d", i);
            return FP_EINVAL;
        }
    }
    for (int32_t i = 0; i < k; ++i) {
        int rc = fp_predict(forests[i], batches[i].X, batches[i].n, batches[i].out_votes, batches[i].out_class,
                            stream);
        if (rc) return rc;
    }
    return FP_OK;
}
