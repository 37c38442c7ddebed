// Per-thread error text and other host-side odds and ends of libnsort.
#include <string>

#include "nsort.h"
#include "nsort_internal.h"

namespace nsort {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }
const char *last_error_cstr() { return g_last_error.c_str(); }

size_t segmented_temp_bytes(int kind, uint64_t n, uint64_t nseg) {
  (void)kind; (void)n; (void)nseg;
  return 0;
}

}  // namespace nsort
