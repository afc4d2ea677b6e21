// Definitions of the opaque C-ABI handles (shared by the C-ABI translation units).
#pragma once
#include <memory>

#include "../../include/mfns.h"
#include "problem.hpp"

struct mfns_ctx {
  int device = 0;
  mfns::Budget budget;
};
struct mfns_mesh {
  mfns_ctx* ctx = nullptr;
  mfns::Forest forest;
};
struct mfns_problem {
  mfns_ctx* ctx = nullptr;
  std::unique_ptr<mfns::Problem> p;
};

namespace mfns {
// records the message returned by mfns_last_error and returns `code`
int capi_fail(int code, const char* msg);
}  // namespace mfns
