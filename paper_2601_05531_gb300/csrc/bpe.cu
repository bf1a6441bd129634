// bpe.cu -- BPE merge application (placeholder until the BPE kernels land).
#include "handle.h"

namespace dnatok {
dnatok_status bpe_create(dnatok_handle *h, const int32_t *, int32_t) {
    return fail(h, DNATOK_ERR_STATE, "BPE mode not built yet");
}
void bpe_destroy(dnatok_handle *) {}
dnatok_status bpe_encode(dnatok_handle *h, const uint8_t *, int64_t, const int64_t *, int64_t,
                         int32_t *, int64_t, int64_t *, int64_t, int64_t *, cudaStream_t) {
    return fail(h, DNATOK_ERR_STATE, "BPE mode not built yet");
}
}  // namespace dnatok
