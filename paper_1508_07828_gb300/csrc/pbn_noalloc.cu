// pbn_skart_static: the Skart batch statistics without any device allocation.
//
// pbn_skart keeps its batch sums in a buffer that the library allocates with
// cudaMalloc the first time a stream needs one and grows later.  Some callers
// cannot let a library do that: a host program that hands out all device
// memory through its own allocator and forbids allocations behind its back,
// or a latency-critical loop in which cudaMalloc and cudaFree would stall the
// whole device.  For them this entry point keeps the batch sums in a
// fixed-size array that lives in the library's device image, so a call
// allocates nothing; the caller still passes the chains (inputs) and the
// result slot (output).
#include <stdio.h>

#include <mutex>

#include "pbn_internal.cuh"

namespace {

// One batch sum per (chain, batch); 2^18 entries = 1 MiB of device memory that
// every GPU which loads the library keeps until the process exits.
constexpr int64_t kStaticBatches = PBN_SKART_STATIC_MAX_BATCHES;
static __device__ __align__(256) int32_t g_static_batch_sums[kStaticBatches];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int32_t *g_static_ptr[kMaxDevices] = {};  // device address of the array, per device

thread_local char g_msg[256];

int reject(int code) {
  pbn::set_last_error(g_msg);
  return code;
}

}  // namespace

extern "C" int pbn_skart_static(const pbn_chains *ch, int64_t start, int64_t kappa, int64_t bpc, int64_t spacer,
                                double alpha_ci, double alpha_ran, pbn_skart_result *out, void *stream) {
  g_msg[0] = '\0';
  if (!ch || !ch->bits || !out) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: NULL chains, bitstream or result");
    return reject(PBN_ERR_INVALID);
  }
  if (kappa < 1 || bpc < 1 || spacer < 0) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: kappa %lld, batches %lld, spacer %lld out of range",
             (long long)kappa, (long long)bpc, (long long)spacer);
    return reject(PBN_ERR_INVALID);
  }
  if (kappa > (1ll << 30)) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: kappa %lld above 2^30", (long long)kappa);
    return reject(PBN_ERR_UNSUPPORTED);
  }
  if (ch->omega < 1) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: omega %lld below 1", (long long)ch->omega);
    return reject(PBN_ERR_INVALID);
  }
  // capacity before any product of the two sizes, so that the product below
  // cannot overflow
  if (ch->omega > kStaticBatches / bpc) {
    snprintf(g_msg, sizeof g_msg,
             "pbn_skart_static: %lld chains x %lld batches exceed the fixed capacity of %lld batch sums; "
             "use pbn_skart",
             (long long)ch->omega, (long long)bpc, (long long)kStaticBatches);
    return reject(PBN_ERR_UNSUPPORTED);
  }
  if (ch->omega * bpc < 2) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: needs at least 2 batches");
    return reject(PBN_ERR_INVALID);
  }
  const int64_t len = kappa * bpc;
  if (start < ch->bits_base || start + len - ch->bits_base > ch->bits_cap || start + len > ch->length) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: window [%lld, %lld) outside the recorded positions",
             (long long)start, (long long)(start + len));
    return reject(PBN_ERR_INVALID);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: no usable current device");
    return reject(PBN_ERR_CUDA);
  }
  int32_t *scratch;
  {
    // Set-up, once per device, with that device current: the host cannot use
    // the array's name as a device address, so ask the runtime for it.
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_static_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_batch_sums);
      if (e != cudaSuccess) {
        snprintf(g_msg, sizeof g_msg, "pbn_skart_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return reject(PBN_ERR_CUDA);
      }
      g_static_ptr[dev] = static_cast<int32_t *>(p);
    }
    scratch = g_static_ptr[dev];
  }
  // Every batch sum the statistics read is written by this call first, so the
  // array needs no clearing between calls.
  e = pbn::launch_skart_into(*ch, start - ch->bits_base, kappa, bpc, spacer, alpha_ci, alpha_ran, out, scratch,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "pbn_skart_static: launch failed: %s", cudaGetErrorString(e));
    return reject(PBN_ERR_CUDA);
  }
  return PBN_OK;
}
