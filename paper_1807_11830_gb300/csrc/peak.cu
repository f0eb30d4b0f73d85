// FP32 FMA throughput of the device (the ALU roofline's denominator for the
// transform-bound kernels).  Every thread runs independent chains of fused
// multiply-adds, a = a * m + c, enough of them per warp and enough warps per
// SM that the FMA pipes never wait on a result; the launch covers every SM
// at full occupancy.  Flops = 2 per FMA.
#include <cuda_runtime.h>

#include <string>

#include "sense.h"

namespace sense {
void record_error(const std::string& msg);
}

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;   // independent chains per thread
constexpr int kUnroll = 16;  // FMAs per chain per loop trip

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float* sink, int trips) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + 7 * k);
  const float m = 0.99999994f, c = 1e-7f;  // |a| stays bounded: a fixed point at c / (1 - m)
#pragma unroll 1
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true; keeps every chain live
}

sense_status peak_fail(sense_status st, const std::string& msg) {
  sense::record_error(msg);
  return st;
}

}  // namespace

extern "C" sense_status sense_fp32_peak(int device, double* tflops_out) {
  if (!tflops_out) return peak_fail(SENSE_EINVAL, "tflops_out is NULL");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return peak_fail(SENSE_EINVAL, "device index out of range");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0);
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  const int trips = 2048;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(float) * (size_t)blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(e0, 0);
    k_fma_peak<<<blocks, kPeakThreads>>>(sink, trips);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return peak_fail(SENSE_ECUDA, std::string("FMA peak: ") + cudaGetErrorString(e));
  const double fmas = (double)blocks * kPeakThreads * trips * kUnroll * kChains;
  *tflops_out = 2.0 * fmas / (best * 1e-3) / 1e12;
  return SENSE_OK;
}
