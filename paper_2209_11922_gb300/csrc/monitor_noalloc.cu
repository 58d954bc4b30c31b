// monitor_noalloc.cu - field monitors (mass, energy, max|u|, non-finite count) for callers that
// cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns every
// allocation (a framework's memory pool or a fixed memory budget), real-time loops where an
// allocation (and the device synchronisation it may imply) is not allowed, or a check that must be
// usable before any plan exists. etd_monitor_noalloc computes the same reductions as etd_monitor
// without a plan and without allocating: its per-CTA partial sums live in the file-scope array
// g_monitor_scratch below, which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/etd.h"
#include "monitor.cuh"

void etd_internal_set_error(const char* msg);   // etd_api.cu

namespace {

// One partial record per CTA: four doubles (mass, quadratic energy, potential energy, max|u|)
// followed, after all records, by one int64 non-finite count per CTA.
constexpr int kMaxRecords = ETD_MONITOR_NOALLOC_MAX_UNKNOWNS / 2048;   // one CTA per 2048 unknowns
constexpr size_t kScratchBytes = (size_t)kMaxRecords * (4 * sizeof(double) + sizeof(long long));

static __device__ __align__(256) unsigned char g_monitor_scratch[kScratchBytes];

// Device address of g_monitor_scratch per device, resolved once per device (cudaGetSymbolAddress
// gives the address in the current device's context; the host-side symbol itself is not it).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

etd_status noalloc_fail(etd_status s, const char* fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  etd_internal_set_error(buf);   // reported by etd_last_error()
  return s;
}

}  // namespace

extern "C" etd_status etd_monitor_noalloc(int ndim, const int64_t* N, const double* h, double D, etd_dtype dtype,
                                          const void* u, etd_monitors* out_dev, void* stream) {
  etd_internal_set_error("");
  if (ndim != 2 && ndim != 3) return noalloc_fail(ETD_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (!N || !h || !u || !out_dev) return noalloc_fail(ETD_ERR_INVALID_ARG, "N, h, u and out must be non-NULL");
  if (dtype != ETD_F32 && dtype != ETD_F64) return noalloc_fail(ETD_ERR_INVALID_ARG, "dtype must be ETD_F32 or ETD_F64");
  if (!(std::isfinite(D) && D > 0)) return noalloc_fail(ETD_ERR_INVALID_ARG, "D must be finite and > 0");
  long long n = 1;
  etd::MonitorGeom g;
  g.ndim = ndim;
  for (int a = 0; a < 3; ++a) {
    if (a < ndim) {
      if (N[a] < 2 || N[a] > (1LL << 30)) return noalloc_fail(ETD_ERR_INVALID_ARG, "N[%d] out of range", a);
      if (!(std::isfinite(h[a]) && h[a] > 0)) return noalloc_fail(ETD_ERR_INVALID_ARG, "h[%d] must be finite and > 0", a);
      g.m[a] = (int)(N[a] - 1);
      g.h[a] = h[a];
      // reject before multiplying: n * (N[a] - 1) never exceeds the maximum, so it cannot overflow
      if (N[a] - 1 > (long long)ETD_MONITOR_NOALLOC_MAX_UNKNOWNS / n)
        return noalloc_fail(ETD_ERR_INVALID_ARG,
                            "more than the maximum of %d unknowns for etd_monitor_noalloc (its fixed scratch "
                            "holds %d partial records); use etd_monitor with a plan",
                            ETD_MONITOR_NOALLOC_MAX_UNKNOWNS, kMaxRecords);
      n *= (N[a] - 1);
    } else {
      g.m[a] = 1;
      g.h[a] = 1.0;
    }
  }
  g.D = D;
  g.periodic = 0;   // homogeneous Dirichlet and the Allen-Cahn double well
  g.flin = 1.0;
  g.fcub = -1.0;
  g.flog = 0.0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(ETD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(ETD_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_monitor_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(ETD_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  const int blocks = (int)((n + 2047) / 2048);   // <= kMaxRecords by the per-axis checks above
  double* part = static_cast<double*>(base);
  long long* bad = reinterpret_cast<long long*>(part + 4 * (size_t)kMaxRecords);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every record the final kernel reads is written by this call's first kernel, so nothing left
  // in the scratch by an earlier call is read and nothing needs clearing.
  if (dtype == ETD_F32)
    etd::monitor_partial_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(u), g, part, bad);
  else
    etd::monitor_partial_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(u), g, part, bad);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(ETD_ERR_CUDA, "monitor launch: %s", cudaGetErrorString(e));
  double* o = reinterpret_cast<double*>(out_dev);
  etd::monitor_final_kernel<<<1, 256, 0, s>>>(part, bad, blocks, o, reinterpret_cast<long long*>(o + 3));
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(ETD_ERR_CUDA, "monitor launch: %s", cudaGetErrorString(e));
  return ETD_OK;
}
