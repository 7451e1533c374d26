// spk_sketch_apply_static: the sketch application S X of spk_sketch_apply,
// for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a process that carved
// the whole device heap into its own pool at start-up (any further driver
// allocation fails or breaks its accounting), a framework whose allocator
// must stay the only owner of device memory, or a service with a fixed
// memory budget that has to be proven before it runs.  This entry point
// therefore takes its working memory from one file-scope device array of
// fixed size, reserved when the library is loaded on a device and kept until
// the process exits.  The caller still provides the input X and the output SX.
//
// Limits (checked before any device work; larger inputs get SPK_ERR_ARG):
//   n <= 2^20 rows, 1 <= r <= 4 columns, n' * r <= 2^20 where
//   n' = 2^ceil(log2 n), 1 <= s <= min(n', 32768).
// The array holds 10.1 MiB: the two-level transform's intermediate (8 MiB),
// the selected rows, the signs and the row-selection work space.
//
// Set-up: the first call on a device, with that device current, resolves
// the array's device address with cudaGetSymbolAddress (a host-side name of
// a __device__ variable is not a device address) and creates one event;
// later calls on that device reuse both.  Every call waits on the host for
// its stream (the row selection reads a count back, and the call returns
// only when S X is written), so no call may be made while its stream is
// being captured into a CUDA graph.
//
// Sharing: every call on a device uses the same array and leaves its
// contents behind.  The selection counter is cleared by each call; every
// other byte a call reads it has written earlier in the same call.  Calls
// whose device work overlaps (different streams, or different host threads
// without ordering) race on the array and give wrong results: order them.
// A call that returns SPK_ERR_TIMEOUT may leave kernels queued that still
// write the array; the event recorded at the end of each call's device work
// makes the next call on that device wait for them first (bounded: that
// call returns SPK_ERR_TIMEOUT too while they have not finished).
#include "spk_internal.cuh"

#include <cstdio>
#include <cstring>
#include <mutex>

namespace {

constexpr int64_t kMaxN = int64_t(1) << 20;
constexpr int64_t kMaxPadTimesR = int64_t(1) << 20;
constexpr int32_t kMaxS = 32768;
constexpr size_t kTransformBytes = size_t(kMaxPadTimesR) * sizeof(double);      // 8 MiB
constexpr size_t kRowsBytes = size_t(kMaxS) * sizeof(int32_t);                   // 128 KiB
constexpr size_t kSignsBytes = size_t(kMaxN);                                    // 1 MiB
constexpr size_t kDrawBytes = 1024 * 1024;                                       // selection
constexpr size_t kScratchBytes = kTransformBytes + kRowsBytes + kSignsBytes + kDrawBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
// recorded after each call's last kernel: the array is free once it completes
cudaEvent_t g_done[kMaxDevices] = {nullptr};

int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

void set_err(char* err, size_t errlen, const char* msg) {
  if (err && errlen > 0) {
    strncpy(err, msg, errlen - 1);
    err[errlen - 1] = '\0';
  }
}

}  // namespace

extern "C" int spk_sketch_apply_static(int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                                       const double* X_dev, int32_t r, double* SX_dev,
                                       void* stream, char* err, size_t errlen) {
  char msg[256];
  if (!X_dev || !SX_dev || n < 1 || r < 1 || r > spk::kMaxR) {
    set_err(err, errlen, "spk_sketch_apply_static: null pointer, n < 1 or r outside [1, 4]");
    return SPK_ERR_ARG;
  }
  const int64_t npad = next_pow2(n);
  if (n > kMaxN || npad * r > kMaxPadTimesR || s < 1 || s > kMaxS || s > npad) {
    snprintf(msg, sizeof msg,
             "spk_sketch_apply_static: size beyond the static scratch (n=%lld <= 2^20, "
             "n'*r=%lld <= 2^20, 1 <= s=%d <= min(n', 32768))",
             (long long)n, (long long)(npad * r), s);
    set_err(err, errlen, msg);
    return SPK_ERR_ARG;
  }
  if (spk::sketch_draws_scratch_bytes(n, s) > kDrawBytes) {
    set_err(err, errlen, "spk_sketch_apply_static: row-selection space exceeded");
    return SPK_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_err(err, errlen, "spk_sketch_apply_static: no usable current device");
    return SPK_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  cudaEvent_t done = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        snprintf(msg, sizeof msg, "spk_sketch_apply_static: cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString(e));
        set_err(err, errlen, msg);
        return SPK_ERR_CUDA;
      }
      g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    if (!g_done[dev]) {
      cudaError_t e = cudaEventCreateWithFlags(&g_done[dev], cudaEventDisableTiming);
      if (e != cudaSuccess) {
        cudaGetLastError();
        g_done[dev] = nullptr;
        set_err(err, errlen, "spk_sketch_apply_static: cudaEventCreate failed");
        return SPK_ERR_CUDA;
      }
    }
    base = g_scratch_addr[dev];
    done = g_done[dev];
  }
  // kernels of an earlier call that timed out may still use the array
  {
    const int w0 = spk::bounded_event_wait(done, spk::kHostWaitSeconds);
    if (w0 == 1) {
      set_err(err, errlen, "spk_sketch_apply_static: an earlier call's device work is still "
                           "running on the shared array");
      return SPK_ERR_TIMEOUT;
    }
    if (w0 != 0) {
      cudaGetLastError();
      set_err(err, errlen, "spk_sketch_apply_static: earlier device work failed");
      return SPK_ERR_CUDA;
    }
  }
  double* transform = reinterpret_cast<double*>(base);
  int32_t* rows = reinterpret_cast<int32_t*>(base + kTransformBytes);
  int8_t* signs = reinterpret_cast<int8_t*>(base + kTransformBytes + kRowsBytes);
  void* draw = base + kTransformBytes + kRowsBytes + kSignsBytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char derr[256] = {0};
  int rc = spk::sketch_draws_launch(n, s, seed, sketch_id, rows, signs, draw, kDrawBytes, st,
                                    derr, sizeof derr);
  if (rc != SPK_OK) {
    // the draws may have queued kernels before failing: mark their end
    cudaEventRecord(done, st);
    cudaGetLastError();
    set_err(err, errlen, derr);
    return rc;
  }
  spk::SketchDev sk;
  spk::sketch_geometry(sk, n, s, 0, (int)sizeof(double), r);
  sk.rows = rows;
  sk.signs = signs;
  spk::sketch_apply_launch<double, double>(sk, X_dev, r, SX_dev, transform, st);
  if (cudaEventRecord(done, st) != cudaSuccess) {
    cudaGetLastError();
    set_err(err, errlen, "spk_sketch_apply_static: cudaEventRecord failed");
    return SPK_ERR_CUDA;
  }
  const int w = spk::bounded_stream_wait(st, spk::kHostWaitSeconds);
  if (w == 1) {
    set_err(err, errlen, "spk_sketch_apply_static: device work did not finish");
    return SPK_ERR_TIMEOUT;
  }
  if (w != 0 || cudaGetLastError() != cudaSuccess) {
    set_err(err, errlen, "spk_sketch_apply_static: kernel failed");
    return SPK_ERR_CUDA;
  }
  set_err(err, errlen, "");
  return SPK_OK;
}
