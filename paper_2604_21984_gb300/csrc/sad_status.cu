// Status strings and the thread-local error message of libsad.so.
#include "sad_host.h"

namespace sad {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

}  // namespace sad

extern "C" {

const char* sad_status_string(int status) {
  switch (status) {
    case SAD_OK: return "ok";
    case SAD_EINVAL: return "invalid argument";
    case SAD_ECUDA: return "CUDA error";
    case SAD_EWORKSPACE: return "workspace too small";
    case SAD_ETIMEOUT: return "device wait timed out";
    case SAD_EINTERNAL: return "internal error";
    default: return "unknown status";
  }
}

const char* sad_last_error(void) { return sad::g_last_error.c_str(); }

int sad_abi_version(void) { return 8; }

}  // extern "C"
