// fp_common.h -- helpers shared by the translation units of the library.
#pragma once
#include <stdarg.h>
#include <stdint.h>

#include "../../include/forest_pack.h"
#include "fp_internal.h"

// Record a printf-style message for fp_last_error() on this thread.
void fp_set_error(const char *fmt, ...);

void fp_fill_info(const FpImageHeader *h, fp_packed_info *info);
const FpImageHeader *fp_packed_header(const fp_packed_forest *pf);
const uint8_t *fp_packed_bytes(const fp_packed_forest *pf);
