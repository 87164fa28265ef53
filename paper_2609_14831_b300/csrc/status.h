// status.h -- thread-local error reporting behind cut_last_error().
#pragma once
#include <string>

#include "cut.h"

namespace cut {
cut_status set_error(cut_status s, const std::string &msg);
cut_status set_ok();
}  // namespace cut
