// stream.cu -- host-streamed pipeline (placeholder).
#include "handle.h"

namespace dnatok {
void stream_destroy(dnatok_handle *) {}
}  // namespace dnatok
