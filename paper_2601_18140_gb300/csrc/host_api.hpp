// Shared by the library's host translation units: the export attribute of the
// C ABI, the status-code error type, and guarded(), which runs an entry point's
// body, turns any exception into a status code and keeps its message for
// rteaal_last_error() (one message per host thread).
#pragma once

#include <cstdint>
#include <new>
#include <stdexcept>
#include <string>

#include "lower.hpp"
#include "rteaal.h"

#define RT_EXPORT extern "C" __attribute__((visibility("default")))

namespace rteaal {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// This thread's last failure message (defined in inspect.cpp).
std::string& last_error();

template <typename F>
int guarded(F&& f) {
  try {
    f();
    return RTEAAL_OK;
  } catch (const Error& e) {
    last_error() = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    last_error() = "host allocation failed";
    return RTEAAL_E_NOMEM;
  } catch (const std::exception& e) {
    last_error() = e.what();
    return RTEAAL_E_INVALID;
  }
}

inline void require(bool c, const char* msg) {
  if (!c) throw Error(RTEAAL_E_INVALID, msg);
}

// Figures of a netlist (as the caller wrote it) and of its lowering.
void fill_stats(const Netlist& nl, const Lowered& L, uint64_t metadata_bytes, rteaal_design_stats* o);

}  // namespace rteaal
