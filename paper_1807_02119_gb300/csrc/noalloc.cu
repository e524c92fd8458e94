// pk_eval_noalloc: a whole evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: code embedded in a host application whose own
// allocator has reserved the device memory, or a service that forbids allocation once
// it is running.  For them the workspace of an evaluation (initial-tensor program,
// per-tensor bookkeeping, split-K partial sums and every intermediate tensor) lives in
// one file-scope device array of fixed size instead of caller- or library-allocated
// memory.  Every GPU that loads this library holds the array until the process exits.
//
// The array's name, used in host code, is only a host-side stand-in for the device
// symbol, not a device address: handing it to a kernel would fault or, where the GPU
// can reach host memory, silently use the wrong memory.  The device address is taken
// with cudaGetSymbolAddress once per device, with that device current, and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "handles.h"
#include "pk_internal.h"

namespace {

constexpr unsigned long long kNoallocScratchBytes = 64ull << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on device `dev`, which must be current.  The first
// call on a device looks it up; later calls reuse the cached address.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

pk_status noalloc_fail(pk_ctx* c, pk_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

}  // namespace

extern "C" pk_status pk_eval_noalloc(pk_ctx* ctx, const pk_plan* p, int32_t precision,
                                     pk_scaled* Z, pk_scaled* V) {
  if (!ctx || !p || !Z) return noalloc_fail(ctx, PK_EINVAL, "null argument");
  if (precision != PK_C128 && precision != PK_C64 && precision != PK_SPLIT)
    return noalloc_fail(ctx, PK_EINVAL, "bad precision");
  if (ctx->device < 0) return noalloc_fail(ctx, PK_ENODEVICE, "host-only context");
  if (ctx->device >= kMaxDevices) return noalloc_fail(ctx, PK_ENODEVICE, "device index too large");
  const pk::Plan& P = p->p;
  const uint64_t need = P.ws_bytes(precision);
  if (need > kNoallocScratchBytes)
    return noalloc_fail(ctx, PK_ENOMEM,
                        "plan needs " + std::to_string(need) +
                            " workspace bytes; pk_eval_noalloc's static scratch holds " +
                            std::to_string(kNoallocScratchBytes) + " (use pk_eval)");
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != ctx->device) e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess)   // the symbol lookup below must run with ctx->device current
    return noalloc_fail(ctx, PK_ECUDA, std::string("pk_eval_noalloc: cannot make device ") +
                                           std::to_string(ctx->device) + " current: " +
                                           cudaGetErrorString(e));
  pk_status status = PK_OK;
  void* ws = nullptr;
  e = scratch_address(ctx->device, &ws);
  if (e == cudaSuccess && !P.program.empty())
    e = cudaMemcpyAsync(ws, P.program.data(), P.program.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess)
    e = pk::launch_plan(P, precision, ws, (char*)ws + P.off_arena, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->pinned_result,
                        (const char*)ws + P.off_result + sizeof(pk::SliceResult) * P.n_slices,
                        sizeof(pk::SliceResult), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    status = noalloc_fail(ctx, PK_ECUDA, std::string("pk_eval_noalloc: ") + cudaGetErrorString(e));
  } else {
    std::string err;
    status = pk::decode_total(P, *ctx->pinned_result, Z, V, err);
    if (status != PK_OK) noalloc_fail(ctx, status, "pk_eval_noalloc: " + err);
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return status;
}
