// Error reporting of the C ABI.
#include <string>

#include "common.cuh"

namespace sg {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
}  // namespace sg

extern "C" const char* sg_last_error(void) { return sg::g_last_error.c_str(); }
