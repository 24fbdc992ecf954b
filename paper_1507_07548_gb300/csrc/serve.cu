#include "ms2_host.h"
extern "C" ms2_status ms2_serve_open(size_t, int, const ms2_options *, ms2_server *) { return ms2_fail(MS2_ESTATE, "serve: pending"); }
extern "C" ms2_status ms2_serve_submit(ms2_server, const ms2_job *, long long *) { return ms2_fail(MS2_ESTATE, "serve: pending"); }
extern "C" ms2_status ms2_serve_poll(ms2_server, ms2_job_result *, int, int *) { return ms2_fail(MS2_ESTATE, "serve: pending"); }
extern "C" ms2_status ms2_serve_drain(ms2_server, double) { return ms2_fail(MS2_ESTATE, "serve: pending"); }
extern "C" ms2_status ms2_serve_close(ms2_server) { return MS2_OK; }
