// Arithmetic peaks of the current device, measured: FP64 and FP32 fused multiply-add
// throughput and FP64 exp() throughput. They are the denominators an ALU-bound kernel is
// judged against; the FP64 Newton residual (carrier statistics with FP64 exponentials at
// every Gauss point, then the FP64 stiffness) is bound by the FP64 pipe on this part.
//
// Each thread runs eight independent dependency chains (enough to cover the pipe latency
// with the warps an SM holds), on a grid of 8 blocks of 256 threads per SM. The chains'
// results are kept live by a store guarded by a comparison with a sentinel the chains never
// reach, so the compiler keeps every operation and nothing is written.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/qcad.h"
#include "mesh.h"
#include "qcad_host.h"

namespace qcad {
namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

// a <- a * b + c on every chain; with 0 < b < 1 and c > 0 the chains approach c / (1 - b).
template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_peak_kernel(T* out, int iters, T b, T c, T sentinel) {
  T a[PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = T(1e-3) * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) s += a[i];
  if (s == sentinel) out[blockIdx.x] = s;
}

// a <- exp(-a) on every chain: values stay in (0, 1] and approach the root of a = exp(-a).
__global__ void __launch_bounds__(PEAK_THREADS) exp_peak_kernel(double* out, int iters, double sentinel) {
  double a[PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = exp(-a[i]);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) s += a[i];
  if (s == sentinel) out[blockIdx.x] = s;
}

// Best of three timed launches (after one untimed) in seconds.
template <class L>
double best_time(cudaStream_t s, L&& launch) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  launch();
  CK(cudaGetLastError());
  double best = 1e30;
  for (int r = 0; r < 3; ++r) {
    CK(cudaEventRecord(e0, s));
    launch();
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, 1e-3 * ms);
  }
  CK(cudaGetLastError());
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return best;
}

}  // namespace

qcad_status alu_peaks(double* fp64_tflops, double* fp32_tflops, double* fp64_exp_per_s) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * PEAK_BLOCKS_PER_SM;
  const double threads = (double)blocks * PEAK_THREADS;
  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  DevBuf out;
  out.ensure((size_t)blocks * sizeof(double) + 64);
  // iteration counts sized for about 10 ms per launch at this part's rates
  const int it64 = 2500, it32 = 160000, itexp = 200;
  const double t64 = best_time(s, [&] {
    note_launch(), fma_peak_kernel<double><<<blocks, PEAK_THREADS, 0, s>>>(out.as<double>(), it64, 0.999, 1e-3, -1.0);
  });
  const double t32 = best_time(s, [&] {
    note_launch(), fma_peak_kernel<float><<<blocks, PEAK_THREADS, 0, s>>>(reinterpret_cast<float*>(out.p), it32,
                                                                            0.999f, 1e-3f, -1.0f);
  });
  const double texp = best_time(s, [&] {
    note_launch(), exp_peak_kernel<<<blocks, PEAK_THREADS, 0, s>>>(out.as<double>(), itexp, -1.0);
  });
  CK(cudaStreamSynchronize(s));
  CK(cudaStreamDestroy(s));
  if (fp64_tflops) *fp64_tflops = 2.0 * PEAK_CHAINS * it64 * threads / t64 * 1e-12;
  if (fp32_tflops) *fp32_tflops = 2.0 * PEAK_CHAINS * it32 * threads / t32 * 1e-12;
  if (fp64_exp_per_s) *fp64_exp_per_s = (double)PEAK_CHAINS * itexp * threads / texp;
  return QCAD_OK;
}

}  // namespace qcad
