// Host-side helpers of libsad.so: status/error reporting and argument checks.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/sad.h"

namespace sad {

void set_error(const char* fmt, ...);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Returns SAD_OK after a launch, or SAD_ECUDA with the CUDA message recorded.
inline int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SAD_ECUDA;
  }
  return SAD_OK;
}

inline int einval(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_error("%s", buf);
  return SAD_EINVAL;
}

// Common validation of an image/list/site-count triple.
inline int check_problem(int32_t capacity, int32_t H, int32_t W, int32_t K, bool need_k) {
  if (capacity < 0) return einval("capacity must be >= 0 (got %d)", capacity);
  if (H <= 0 || W <= 0) return einval("image must be non-empty (H=%d, W=%d)", H, W);
  if (H > 32768 || W > 32768) return einval("image side above 32768 (H=%d, W=%d)", H, W);
  if (need_k && K != 4 && K != 8 && K != 16) return einval("K must be 4, 8 or 16 (got %d)", K);
  return SAD_OK;
}

struct AdamArgs;
AdamArgs adam_args(const sad_adam_hparams* hp);

// While tracing is on (sad_trace_enable), records a CUDA event on `s` when
// constructed and another when destroyed; the pair is one launch of stage
// `name` (a string literal).  Does nothing when tracing is off or the stream
// is being captured into a graph.
struct TraceScope {
  TraceScope(cudaStream_t st, const char* nm);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;
  cudaStream_t s;
  const char* name;
  cudaEvent_t e0, e1;
};

}  // namespace sad
