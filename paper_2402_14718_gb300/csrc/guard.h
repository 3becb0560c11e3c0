// Host exceptions stop at the C ABI.
#pragma once
#include <exception>
#include <new>
#include <string>

#include "../../include/sb.h"

namespace sbh {
void set_error(const std::string& msg);

// Runs the body of a C entry point. A C++ exception thrown on the host (a
// failed allocation above all) becomes SB_ERR_OOM and an error message
// instead of crossing the C interface.
template <typename F>
sb_status guarded(const char* name, F&& body) {
  try {
    return body();
  } catch (const std::exception& e) {
    try {
      set_error(std::string(name) + ": host error (" + e.what() + ")");
    } catch (...) {
    }
    return SB_ERR_OOM;
  } catch (...) {
    try {
      set_error(std::string(name) + ": host error");
    } catch (...) {
    }
    return SB_ERR_OOM;
  }
}
}  // namespace sbh
