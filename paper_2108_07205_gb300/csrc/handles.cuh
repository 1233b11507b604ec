// Definitions of the opaque C-ABI handles (include/rwsolve.h).
#pragma once
#include "refine.cuh"

struct rw_hbs_s {
  rw::Wall wall;
};
struct rw_ref_s {
  rw::Refinement ref;
  const rw_hbs_s* h = nullptr;
};

namespace rw {
// Error reporting shared by every extern "C" entry point (abi.cu).
int abi_fail(int code, const std::string& msg);
void abi_clear_error();
}  // namespace rw
