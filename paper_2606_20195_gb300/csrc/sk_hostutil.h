// Host-side helpers shared by the C-ABI translation units: thread-local error message.
#pragma once

#include "../../include/sk.h"

namespace sk {

// Record a formatted message for sk_last_error() on this thread and return `code`.
sk_status set_error(sk_status code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
void clear_error();
const char* last_error_message();

}  // namespace sk
