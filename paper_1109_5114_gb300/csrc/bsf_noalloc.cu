// bsf_filter_noalloc: the whole forward filter without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a host
// application that has handed its entire device-memory budget to its own pool
// at start-up, or a latency-critical loop in which cudaMalloc / cudaFree are
// not acceptable because they can synchronise the whole device.  For them
// this entry point runs the same kernels as bsf_filter on scratch memory that
// lives in one file-scope device array, so a call allocates nothing.
//
// The array (kScratchBytes, 24 MiB) is part of the library image: every GPU
// that loads the library holds it until the process exits.  All calls share
// it and it keeps the contents of the last call, so two calls that overlap on
// the GPU (different streams, or different host threads) race and corrupt
// each other's results; serialise them.
//
// Host code cannot use the array's name as a device address (on the host it
// is a stand-in symbol).  The first call on each device looks its device
// address up with cudaGetSymbolAddress while that device is current; that
// first call should therefore happen before any stream capture begins.
// Under CUDA's lazy module loading (the default since CUDA 12.2) this file's
// module, and with it the 24 MiB array, is loaded by that first lookup, which
// can also synchronise the device: a caller that will hand all remaining
// device memory to its own pool should make one small warm-up call on each
// device at start-up, before reserving the pool (or run with
// CUDA_MODULE_LOADING=EAGER, which loads every module at context creation).
#include <cstring>
#include <mutex>

#include "bsf_internal.h"

// rows per chunk of the vertical sums here (the static array is sized for it)
constexpr int kNoallocChunk = 64;

namespace {

constexpr size_t kScratchBytes = 24u << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {nullptr};

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device address of the scratch array on the current device (looked up once
// per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int bsf_filter_noalloc(const void* img, int dtype, long long ld, int H, int W, int n,
                                  int boundary, int reach, int frac_bits, const float* cov,
                                  void* out, int out_dtype, long long ldo, void* stream) {
  // argument checks (nothing touches the device before they pass)
  if (!img || !cov || !out) return BSF_EINVAL;
  if (H <= 0 || W <= 0 || n < 1 || n > 3 || boundary < BSF_ZERO || boundary > BSF_SYMMETRIC)
    return BSF_EINVAL;
  if (dtype != BSF_U8 && dtype != BSF_F32 && dtype != BSF_F64) return BSF_EINVAL;
  if (out_dtype != BSF_F32 && out_dtype != BSF_F64) return BSF_EINVAL;
  if (ld < W || ldo < W || reach < 3 * n || frac_bits < 0 || frac_bits > 62) return BSF_EINVAL;

  // carve the scratch: status | S [Hp][pitch] | chunk aggregates of the vertical sums
  const long long Hp = (long long)H + 2LL * reach, Wp = (long long)W + 2LL * reach;
  const long long pitch = round_up((size_t)Wp, 32);
  const long long nchunks = (Hp + kNoallocChunk - 1) / kNoallocChunk;
  const size_t off_S = round_up(sizeof(DevStatus), 256);
  const size_t scan_bytes = (size_t)nchunks * n * (size_t)(Wp + Hp - 1) * 8;
  const size_t off_agg = off_S + round_up((size_t)pitch * Hp * 8, 256);
  const size_t need = off_agg + scan_bytes;
  if ((long long)H * W > (1LL << 24) || Hp * pitch > (1LL << 24) || need > kScratchBytes)
    return BSF_ERANGE;  // larger than the static workspace (24 MiB)

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return BSF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = static_cast<unsigned char*>(base);
  DevStatus* st = reinterpret_cast<DevStatus*>(b);
  void* S = b + off_S;
  void* agg = b + off_agg;

  // once anything is queued, a failure still waits for the queued work, so
  // that no kernel of this call touches the shared array after the return
  auto fail_after_queue = [s]() {
    (void)cudaStreamSynchronize(s);
    return BSF_ECUDA;
  };
  // the status word must start from zero; everything else is fully written
  // before it is read
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return fail_after_queue();
  if (bsf_launch_scan_rows(BSF_FIX64, n, img, dtype, ld, H, W, reach, 0, boundary, frac_bits, S, pitch,
                           (int)Hp, (int)Wp, st, s) != cudaSuccess)
    return fail_after_queue();
  const int skews[3] = {0, 1, -1};
  for (int i = 0; i < 3; ++i)
    if (bsf_launch_vscan(BSF_FIX64, n, skews[i], false, S, pitch, (int)Hp, (int)Wp, kNoallocChunk, agg, nullptr,
                         s) != cudaSuccess)
      return fail_after_queue();
  if (bsf_launch_stencil_d1(BSF_FIX64, n, S, pitch, reach, cov, BSF_COV_C, BSF_STEP_D1, H, W, 0, H, frac_bits, out,
                            out_dtype, ldo, st, s) != cudaSuccess)
    return fail_after_queue();

  // synchronous: report the device-side status of this call
  DevStatus host{};
  if (cudaMemcpyAsync(&host, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return fail_after_queue();
  if (cudaStreamSynchronize(s) != cudaSuccess) return BSF_ECUDA;
  return host.err;
}
