// mm_fine_propagate_noalloc: the fine propagator with its scratch memory
// taken from a fixed device array that the library defines, so that the
// call itself never allocates.
//
// Who needs it: callers that may not allocate device memory at the moment
// they run F -- a host application that has handed the whole GPU to its own
// memory pool, a real-time loop that must not hit the allocator's slow
// path or an out-of-memory failure halfway through a run, or code that runs
// where the allocator is not available to it.  They create the context once
// at start-up and then call this entry point as often as they like.
//
// The scratch is one file-scope __device__ array of MM_NOALLOC_SCRATCH_BYTES.
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current.  That
// look-up is done by mm_create (noalloc_setup below), for the device the
// context is created on: it loads this file's module, which reserves the
// array on that device until the process exits, and it also loads the
// kernels of the context's launch choice, so that under lazy module loading
// no call of the entry point has to load (and allocate for) anything.  All
// calls share the array: calls that overlap on the GPU (different streams,
// no ordering between them) race on it.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>

#include "mm_internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[MM_NOALLOC_SCRATCH_BYTES];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Device address of the scratch array on `dev` (looked up once per device).
mm_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return mm_fail(MM_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return mm_cuda_fail(e, "cudaGetDevice");
    if (cur != dev) return mm_fail(MM_ERR_INVALID, "the context's device is not current");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return mm_cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MM_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         (uintptr_t)p % 16 == 0;
}

}  // namespace

namespace mmk {

cudaError_t fine_preload(const FinePlan& f) {
  if (f.kernel == 2) {  // planning a launch configures (and so loads) the instance
    resident_plan(f.args.nx, f.args.nv, 1, 1, f.res_C, f.res_smem);
    return cudaGetLastError();
  }
  return fine_stream_preload(f.args, f.vpt, f.fp32);
}

mm_status noalloc_setup(mm_ctx* c) {
  void* base;
  mm_status st = scratch_address(ctx_device(c), &base);
  if (st != MM_OK) return st;
  FinePlan f;
  if ((st = fine_plan(c, 1, 1.0, &f, false)) != MM_OK) return st;
  const cudaError_t e = fine_preload(f);
  if (e != cudaSuccess) return mm_cuda_fail(e, "mm_create: loading the fine kernel");
  return MM_OK;
}

}  // namespace mmk

extern "C" mm_status mm_fine_propagate_noalloc(mm_ctx* ctx, int32_t batch, double t_span,
                                               const double* rho_in, const void* g_in,
                                               double* rho_out, void* g_out, uint8_t* mask_out,
                                               mm_fine_stats* stats, void* stream) {
  mmk::FinePlan f;
  mm_status st = mmk::fine_plan(ctx, batch, t_span, &f);
  if (st != MM_OK) return st;
  if (batch == 0) {
    if (stats) memset(stats, 0, sizeof(*stats));
    return MM_OK;
  }
  if (!rho_in || !g_in || !rho_out || !g_out) return mm_fail(MM_ERR_INVALID, "NULL array");

  // Scratch: status word and kinetic counter; for the streaming kernel also
  // the second step buffer of g, a copy of g_in when it aliases g_out and the
  // step count is odd (the first step would overwrite it), and the column
  // arrays when they do not fit shared memory.  The resident kernel keeps g
  // in shared memory and carries a state from round to round in the
  // caller's output arrays, so it needs only the status word.
  const bool resident = f.kernel == 2;
  const bool alias = !resident && g_in == g_out && (f.n_steps & 1);
  const size_t o_buf1 = kAlign;
  const size_t o_copy = o_buf1 + (resident ? 0 : up(f.g_bytes));
  const size_t o_cols = o_copy + (alias ? up(f.g_bytes) : 0);
  const size_t need = o_cols + (resident || f.col_in_smem ? 0 : up(f.col_bytes * (size_t)batch));
  if (need > MM_NOALLOC_SCRATCH_BYTES)
    return mm_fail(MM_ERR_INVALID,
                   "mm_fine_propagate_noalloc: this batch needs " + std::to_string(need) +
                       " bytes of scratch, more than the fixed " +
                       std::to_string((size_t)MM_NOALLOC_SCRATCH_BYTES) +
                       "; use a smaller batch or mm_fine_propagate");

  cudaError_t e = cudaSetDevice(f.device);
  if (e != cudaSuccess) return mm_cuda_fail(e, "cudaSetDevice");
  if (!on_device(rho_in) || !on_device(g_in) || !on_device(rho_out) || !on_device(g_out) ||
      (mask_out && !on_device(mask_out)))
    return mm_fail(MM_ERR_INVALID,
                   "mm_fine_propagate_noalloc takes 16-byte aligned device arrays only "
                   "(host arrays would need staging buffers)");
  unsigned char* base;
  if ((st = scratch_address(f.device, (void**)&base)) != MM_OK) return st;

  cudaStream_t s = (cudaStream_t)stream;
  mmk::FineArgs& a = f.args;
  a.rho_in = rho_in;
  a.rho_out = rho_out;
  a.g_in = g_in;
  a.g_buf0 = g_out;
  a.g_buf1 = resident ? nullptr : base + o_buf1;
  a.mask_out = mask_out;
  a.col_ws = resident || f.col_in_smem ? nullptr : base + o_cols;
  a.status = (int*)base;
  a.kin_count = (unsigned long long*)(base + 16);
  // the status word and the counter must start at zero on every call
  e = cudaMemsetAsync(base, 0, 24, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "clear scratch status");
  if (alias) {
    e = cudaMemcpyAsync(base + o_copy, g_in, f.g_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "alias copy");
    a.g_in = base + o_copy;
  }
  int launches = 1;
  e = resident ? mmk::launch_fine_resident(a, f.res_C, f.res_smem, s, &launches)
               : mmk::launch_fine(a, f.vpt, f.fp32, f.smem, s);
  if (e != cudaSuccess) return mm_cuda_fail(e, "fine kernel launch");
  if (stats) {
    int hs[6] = {0};
    e = cudaMemcpyAsync(hs, base, 24, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mm_cuda_fail(e, "read scratch status");
    unsigned long long kc;
    memcpy(&kc, (char*)hs + 16, 8);
    stats->steps = f.n_steps;
    stats->kinetic_updates = (int64_t)kc;
    stats->full_updates = f.n_steps * (int64_t)batch * a.nx * a.nv;
    stats->device_status = hs[0];
    stats->elapsed_ms = 0.0;
    stats->launches = launches;
    if (hs[0] != 0) return mm_fail((mm_status)hs[0], "fine: non-finite density");
  }
  return MM_OK;
}
