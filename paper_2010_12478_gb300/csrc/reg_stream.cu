// Streaming service of libreg (reg_stream_*).
#include "reg_internal.h"

extern "C" int reg_stream_open(reg_ctx_t *, int, int, reg_stream_t **out)
{
    if (out) *out = nullptr;
    return REG_ESTATE;
}
extern "C" int reg_stream_submit(reg_stream_t *, const float *, uint64_t) { return REG_ESTATE; }
extern "C" int reg_stream_poll(reg_stream_t *, reg_result_t *, int, int *n_out, int)
{
    if (n_out) *n_out = 0;
    return REG_ESTATE;
}
extern "C" int reg_stream_close(reg_stream_t *) { return REG_ESTATE; }
