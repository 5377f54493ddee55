// qfx_amplitudes_static: the amplitude computation for callers that cannot allocate
// device memory.  Some host applications own the whole device through their own memory
// manager and reject foreign allocations, some run under latency limits that
// cudaMalloc's implicit synchronisation would break, and some plugins are handed only
// their input and output buffers.  Such callers cannot provide the workspace that
// qfx_amplitudes needs, so this entry point uses a fixed scratch array compiled into the
// library instead.
//
// The array is a file-scope __device__ object of QFX_STATIC_SCRATCH_BYTES bytes.  Every
// GPU that loads this library holds it until the process exits.  In host code its name
// is only a host-side stand-in, so the device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.  The
// first call on a device does that set-up; make that first call before any stream
// capture.
//
// All calls share the array and it keeps the last call's contents: each call copies the
// plan's tables into it and clears the per-item header and the output before use, and
// every other byte a call reads it has written first.  Calls that overlap on the GPU
// (for example on two streams) race on the array.
//
// The tables are copied from the plan's own host image, which lives as long as the plan.
// This entry point does not page-lock that image; unless another call (qfx_plan_upload,
// qfx_amplitudes) has done so, the copy is from pageable memory and may make the host
// wait for work already queued on the stream.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "qfx_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[QFX_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

qfx_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qfx::cuda_fail(e, "qfx_amplitudes_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return qfx::fail(QFX_EUNSUPPORTED, "qfx_amplitudes_static: device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return qfx::cuda_fail(e, "qfx_amplitudes_static: cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return QFX_OK;
}

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

}  // namespace

extern "C" qfx_status qfx_amplitudes_static(const qfx_plan* p, const uint64_t* x1,
                                            int64_t n_batch, int64_t slice_begin,
                                            int64_t slice_end, double* out, void* stream) {
  qfx_status s = qfx::check_amplitudes_args(p, x1, n_batch, slice_begin, slice_end, out);
  if (s != QFX_OK) return s;
  const uint64_t tables = qfx::table_bytes(p);
  const uint64_t need = qfx_workspace_bytes(p, 1);   // the tables plus one work item
  if (need > (uint64_t)QFX_STATIC_SCRATCH_BYTES)
    return qfx::fail(QFX_ENOMEM, "qfx_amplitudes_static: plan needs " + std::to_string(need) +
                                     " bytes of scratch, the static array holds " +
                                     std::to_string((uint64_t)QFX_STATIC_SCRATCH_BYTES) +
                                     " (use qfx_amplitudes with a caller workspace)");
  void* base = nullptr;
  s = scratch_address(&base);
  if (s != QFX_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // the source is the plan's own host image, which lives as long as the plan
  cudaError_t e = cudaMemcpyAsync(base, p->timg, tables, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return qfx::cuda_fail(e, "qfx_amplitudes_static: table copy");
  const qfx::DeviceTables t = qfx::tables_at(base, p->toffs);
  char* ws = (char*)base + tables;
  const int64_t G = qfx::items_in_flight(p, (size_t)(QFX_STATIC_SCRATCH_BYTES - tables));
  return qfx::exec_amplitudes(p, t, x1, n_batch, slice_begin, slice_end, ws, G, out, stream);
}
