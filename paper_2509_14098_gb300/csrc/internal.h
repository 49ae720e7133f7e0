// internal.h — helpers shared by the C-ABI translation units (internal).
#pragma once
#include <string>
#include <vector>

#include "planner.h"
#include "sv.h"

namespace svh {
// record msg as the calling thread's last error and return s
sv_status set_error(sv_status s, const char* msg);
// validate a C-ABI circuit and convert its gates; "" or the first error
std::string gates_from_circuit(const sv_circuit* c, std::vector<GateRec>* out);
}  // namespace svh
