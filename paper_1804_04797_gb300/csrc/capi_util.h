// Error reporting shared by the C-ABI translation units.
#pragma once

#include <cstdio>
#include <string>

#include "../../include/sv.h"

namespace svc {

// Thread-local text of the last error (returned by sv_last_error).
std::string &last_error();

inline void clear_error() { last_error().clear(); }

inline sv_status fail(sv_status st, const char *msg) {
  last_error() = msg;
  return st;
}

// fmt takes exactly one %s (a) followed by one %lld (b)
inline sv_status failf(sv_status st, const char *fmt, const char *a, long long b) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), fmt, a, b);
  last_error() = buf;
  return st;
}

}  // namespace svc
