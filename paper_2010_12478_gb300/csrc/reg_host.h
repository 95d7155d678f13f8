// Host-side helpers shared by the C-ABI translation units of libreg.
#pragma once

#include "reg_internal.h"

namespace reg {

reg_config_t host_config(reg_ctx_t *ctx);        // the context's configuration
int host_device(reg_ctx_t *ctx);                 // the context's CUDA device
int host_fail(int code, const char *fmt, ...);   // set the last-error message, return code
void stop_stream_service(reg_ctx_t *ctx);        // stop the streaming service of a context
int validate_config(const reg_config_t &c);      // REG_OK, or REG_EINVAL with the last-error message set

}  // namespace reg
