// qt_noalloc.cu -- qt_mesolve_dev_noalloc: the master-equation solve of
// qt_mesolve_dev for callers that cannot allocate device memory.
//
// qt_mesolve_dev obtains its solver workspace (the density matrix, the seven
// Dormand-Prince stage derivatives, two stage inputs, the candidate step and
// the per-CTA reduction slots) with cudaMalloc on its first use.  Some callers
// cannot do that: code that runs while another component owns the device's
// memory budget (a serving process that reserved all free memory up front),
// code whose allocator must never be entered on the solve path, or a caller
// that has to keep cudaMalloc/cudaFree, which can synchronise the device, out
// of a latency-critical loop.  This entry point takes its workspace from the
// file-scope array below instead and calls no cudaMalloc, cudaFree or
// allocating library routine.
//
// The array is a __device__ object of this translation unit.  CUDA loads a
// unit's device code lazily (the default since CUDA 12.2): the array is
// committed on a device when this unit's module is first loaded there, which
// is the cudaGetSymbolAddress below.  qt_system_create runs that look-up for
// the current device, so the 16 MiB are committed when a system is created,
// before the caller hands its free memory to another allocator, and not in
// the middle of a solve; from then on the device holds them until the
// process exits.
#include <mutex>
#include <string>

#include "qt_internal.h"

namespace {

// 16 MiB: enough for dim <= 307 in FP64 and dim <= 431 in mixed precision
// (11 d^2 complex elements plus 64 FP64 reduction slots for each of the
// ceil(d^2 / 256) CTAs the cooperative launch may use on any device).
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];  // device address of the array, per device

// Device address of the scratch array on the current device.  The first
// look-up on a device resolves it with cudaGetSymbolAddress (with that device
// current); later calls reuse it, so a device reset after the first look-up
// (cudaDeviceReset) is not supported.  In host code the array's name is only
// a host-side stand-in, never a device address, so it is not passed to
// kernels.  Returns QT_OK, or an error code with its text in *why.
int scratch_address(void **out, std::string *why) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return QT_ENODEV;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *why = "device index out of range";
    return QT_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *why = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
      return QT_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QT_OK;
}

}  // namespace

namespace qt {

// Loads the scratch array on the current device (see above); failures are
// left for qt_mesolve_dev_noalloc to report.
void noalloc_prepare() {
  void *p = nullptr;
  std::string why;
  (void)scratch_address(&p, &why);
}

}  // namespace qt

extern "C" int qt_mesolve_dev_noalloc(qt_system s, const qt_c128 *state0_dev, int state_is_ket,
                                      const double *tlist_dev, int n_t, const qt_opts *o,
                                      qt_c128 *expect_dev, qt_c128 *states_dev,
                                      qt_stats *stats_dev, void *stream) {
  void *ws = nullptr;
  std::string why;
  int rc = scratch_address(&ws, &why);
  if (rc != QT_OK) return qt::set_error(rc, why.c_str());
  // The solver writes every workspace element before reading it, so stale
  // contents from an earlier call need no clearing; the counters and status
  // word that must start at zero live in the system and are reset by the call.
  return qt::mesolve_dev_ws(s, state0_dev, state_is_ket, tlist_dev, n_t, o, expect_dev,
                            states_dev, stats_dev, stream, ws, kNoAllocScratchBytes);
}
