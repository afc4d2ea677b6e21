// Definitions of the opaque C-ABI handles (shared by the C-ABI translation units).
#pragma once
#include <memory>
#include <utility>
#include <vector>

#include "../../include/mfns.h"
#include "problem.hpp"

// The batched preconditioner of the last batched round and its stream; rebuilt when the set
// of batched problems (or one of their captured graphs) changes.
struct BatchRound {
  std::vector<std::pair<uint64_t, uint64_t>> key;  // (uid, graph epoch) of the members, in order
  mfns::BatchPrecondPtr plan;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  ~BatchRound() {
    plan.reset();
    if (done) cudaEventDestroy(done);
    if (stream) cudaStreamDestroy(stream);
  }
};

struct mfns_ctx {
  int device = 0;
  mfns::Budget budget;
  bool batching = true;  // mfns_batch_step batches eligible preconditioners
  std::unique_ptr<BatchRound> round;
};

// plan of a batched round over `ps` (cached in the context while the set is unchanged)
BatchRound* batch_round(mfns_ctx* ctx, const std::vector<mfns::Problem*>& ps);
struct mfns_mesh {
  mfns_ctx* ctx = nullptr;
  mfns::Forest forest;
};
// Staging of mfns_vmult_host: two device input and output sets of one (operator, precision),
// the two copy streams and the events that order the pipeline.
struct HostIO {
  int which = 0, prec = 0;
  int64_t n = 0;
  mfns::DevBuf in[2], out[2];
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr, ev_in[2] = {}, ev_ap[2] = {}, ev_out[2] = {};
  ~HostIO() {
    for (cudaEvent_t e : {ev_start, ev_done, ev_in[0], ev_in[1], ev_ap[0], ev_ap[1], ev_out[0], ev_out[1]})
      if (e) cudaEventDestroy(e);
    if (s_in) cudaStreamDestroy(s_in);
    if (s_out) cudaStreamDestroy(s_out);
  }
};

struct mfns_problem {
  mfns_ctx* ctx = nullptr;
  std::unique_ptr<HostIO> hio;  // declared before p: destroyed after it
  std::unique_ptr<mfns::Problem> p;
};

namespace mfns {
// records the message returned by mfns_last_error and returns `code`
int capi_fail(int code, const char* msg);
}  // namespace mfns
