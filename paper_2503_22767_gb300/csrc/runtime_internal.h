// Declarations shared between the C-ABI translation units (not part of the ABI).
#pragma once

#include <string>

#include "mpm.h"

namespace mpm {
// Host-side validation of an mpm_config, the rules mpm_create applies;
// returns MPM_OK or MPM_ERR_ARG with the reason in *why.
int check_config(const mpm_config* cfg, std::string* why);
}  // namespace mpm
