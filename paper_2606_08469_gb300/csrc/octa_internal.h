// Internal declarations shared by the library's translation units (host side).
#pragma once
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "octaoctree.h"

namespace octa {

// Thread-local message of the last failing call (octa_last_error()).
void set_error(const char* fmt, ...);
void clear_error();

// Status code + message in one expression.
int fail(int code, const char* fmt, ...);

}  // namespace octa
