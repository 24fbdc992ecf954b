#include "ms2_host.h"
extern "C" ms2_status ms2_batch_create(const ms2_system *, int, ms2_batch *) { return ms2_fail(MS2_ESTATE, "batch: pending"); }
extern "C" ms2_status ms2_batch_step(ms2_batch, long long) { return ms2_fail(MS2_ESTATE, "batch: pending"); }
extern "C" ms2_status ms2_batch_destroy(ms2_batch) { return MS2_OK; }
