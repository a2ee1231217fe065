// Serving scheduler of a context (serve.cu): continuous batching of
// motion-compensation jobs; used by the C ABI in ecc_api.cu.
#pragma once
#include <cstdint>
#include <string>

#include "../../include/ecc.h"

struct ecc_serve;

namespace ecc {

// Device memory a job holds at admission (resident + precompute transient).
int serve_footprint(const ecc_job* job, size_t* bytes, std::string* why);
// Starts the admission and round threads on `device`; budget 0 = 80 % of the
// device memory free at this call.  NULL on failure (*why set).
ecc_serve* serve_create(int device, size_t budget, std::string* why);
// Stops the threads (unfinished jobs are dropped) and frees everything.
void serve_destroy(ecc_serve* s);
int serve_submit(ecc_serve* s, const ecc_job* job, uint64_t* ticket, std::string* why);
int serve_poll(ecc_serve* s, uint64_t ticket, ecc_result* out, std::string* why);
void serve_stats(ecc_serve* s, long long* rounds, long long* job_rounds, int* max_batch, long long* line_pairs);
void serve_times(ecc_serve* s, double* upload_ms, double* precompute_ms, double* round_ms);

}  // namespace ecc
