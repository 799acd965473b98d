// Shared internal definitions of the gpnufft library (not part of the ABI).
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>

#include <cuda_runtime.h>

#include "gpnufft.h"

namespace gpn {

// Internal failure carrying a gp_status; converted to a return code at the ABI.
struct Error : std::runtime_error {
  int status;
  Error(int st, const std::string& msg) : std::runtime_error(msg), status(st) {}
};

[[noreturn]] void fail(int status, const std::string& msg);

#define GPN_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      ::gpn::fail(GP_ECUDA, std::string(#call " failed: ") + cudaGetErrorString(e_) + " at " + \
                                __FILE__ + ":" + std::to_string(__LINE__));                     \
  } while (0)

#define GPN_CHECK(cond, status, msg)  \
  do {                                \
    if (!(cond)) ::gpn::fail(status, msg); \
  } while (0)

constexpr int kMaxDim = 3;
constexpr int kMaxChannels = 32;   // N_sigma + 1 at most
constexpr int kMaxWidth = 16;      // spreading kernel width at most (cells)

}  // namespace gpn
