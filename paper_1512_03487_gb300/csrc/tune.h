// The autotuner's table: one process-wide map from a text key (kernel, launch
// geometry, precision, ...) to the integer choice the tuner made for it (a
// grid size or a launch-shape index). Kept on the host, saved and loaded as
// text by lqcd_tune_save / lqcd_tune_load.
#pragma once

#include <string>

namespace lqcd {

// The stored choice for key, if any.
bool tune_lookup(const std::string& key, int* value);
// Records (or replaces) the choice for key.
void tune_store(const std::string& key, int value);

}  // namespace lqcd
