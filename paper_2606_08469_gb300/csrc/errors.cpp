// Thread-local error message of the last failing ABI call.
#include <cstdarg>
#include <cstdio>

#include "octa_internal.h"

namespace octa {
namespace {
thread_local char g_msg[512] = "";
}

void clear_error() { g_msg[0] = '\0'; }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

}  // namespace octa

extern "C" const char* octa_last_error(void) { return octa::g_msg; }
extern "C" int32_t octa_abi_version(void) { return 8; }
