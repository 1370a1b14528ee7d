// Internal bridge between the library's translation units: the device, the
// stream and the error reporting of a context (defined in hh_host.cu).
#pragma once

#include <cuda_runtime.h>

#include "hh.h"

namespace hh {

int ctx_device(hh_ctx* h);
cudaStream_t ctx_stream(hh_ctx* h);
// Records msg as the context's last error and returns s.
hh_status ctx_fail(hh_ctx* h, hh_status s, const char* msg);
// Makes the context's device current and orders its stream after the caller's.
hh_status ctx_enter(hh_ctx* h);

}  // namespace hh
