// abi_guard.cuh -- no C++ exception crosses the C ABI or leaves a thread of
// the library: the only ones the host code can meet are the standard
// library's (host memory, a thread that cannot be started), reported as
// RBFFD_ENOMEM with their text.
#pragma once
#include <exception>

#include "common.cuh"

namespace rbffd {

template <typename F>
int guarded(F &&body) {
  try {
    return body();
  } catch (const std::exception &e) {
    set_error("host resources exhausted: %s", e.what());
  } catch (...) {
    set_error("host resources exhausted");
  }
  return RBFFD_ENOMEM;
}

}  // namespace rbffd
